"""Host-side argument checks of sph_sort_keys_static's Python wrapper: a short
output or a tensor on another device is rejected before any launch (no GPU
needed; 'meta' tensors stand in for a second device)."""
import pytest
import torch

from paper_2003_10850_gb300 import _check_sort_static


def _t(n, dtype, device="cpu"):
    return torch.empty(n, dtype=dtype, device=device)


def test_accepts_matching_sizes_and_device():
    _check_sort_static(_t(10, torch.int64), _t(10, torch.int64), _t(10, torch.int32), torch.device("cpu"))


@pytest.mark.parametrize("ns,np_", [(9, 10), (10, 9), (11, 10), (10, 11)])
def test_rejects_output_size_mismatch(ns, np_):
    with pytest.raises(ValueError):
        _check_sort_static(_t(10, torch.int64), _t(ns, torch.int64), _t(np_, torch.int32), torch.device("cpu"))


@pytest.mark.parametrize("which", [0, 1, 2])
def test_rejects_tensor_on_other_device(which):
    ts = [_t(10, torch.int64), _t(10, torch.int64), _t(10, torch.int32)]
    ts[which] = torch.empty(10, dtype=ts[which].dtype, device="meta")
    with pytest.raises(ValueError):
        _check_sort_static(*ts, torch.device("cpu"))


def test_rejects_non_tensor():
    with pytest.raises(TypeError):
        _check_sort_static([0] * 10, _t(10, torch.int64), _t(10, torch.int32), torch.device("cpu"))
