"""sph_sort_keys_static: the key sort that allocates nothing, for callers that
cannot call cudaMalloc (inside another framework's memory budget, on a
time-critical loop, or without a sph_ctx). Its output must equal the existing
sort inside sph_build_grid -- sorted keys and permutation bit-exact, the
tolerance these tests use for integer work -- on two calls in a row, whose
second call reuses the static scratch the first one left behind.

Collected last (file name) so that a run stopping at the first failure has
already run every other test.
"""
import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu


def _reference_sort(S, ctx, p):
    """Sorted keys and permutation from the existing entry points, plus the
    unsorted keys rebuilt from them (keys[perm[k]] = sorted_keys[k])."""
    pos = torch.from_numpy(np.asarray(p.pos, np.float32)).cuda()
    mass = torch.from_numpy(np.asarray(p.mass, np.float32)).cuda()
    grid = S.sph_build_grid(ctx, pos, mass, S.default_params(box=p.box))
    n = p.n
    perm = torch.empty(n, dtype=torch.int32, device="cuda")
    skeys = torch.empty(n, dtype=torch.int64, device="cuda")
    S.sph_grid_export(grid, perm, skeys)
    keys = torch.empty_like(skeys)
    keys[perm.long()] = skeys
    grid.free()
    return keys, skeys, perm


def test_static_sort_matches_grid_sort_twice():
    from paper_2003_10850_gb300 import build
    build.build()
    import paper_2003_10850_gb300 as S
    ctx = S.Context(0)
    cases = [W.clustered(300_000, 60, seed=41), W.lattice(32, 0.3, seed=42)]
    for p in cases:                      # two calls in a row, different sizes
        keys, skeys_ref, perm_ref = _reference_sort(S, ctx, p)
        out_keys = torch.full_like(keys, -1)
        out_perm = torch.full_like(perm_ref, -1)
        S.sph_sort_keys_static(keys, out_keys, out_perm)
        torch.cuda.synchronize()
        assert torch.equal(out_keys, skeys_ref)
        assert torch.equal(out_perm, perm_ref)
    ctx.close()


def test_static_sort_full_width_keys_with_duplicates():
    """Keys over all 64 bits (bit 63 set in about half of them) drawn from
    1000 values, so that most keys repeat: sorted keys and permutation must
    equal numpy's stable argsort of the unsigned keys, on two calls in a row
    (the second reuses the scratch the first left behind)."""
    import paper_2003_10850_gb300 as S
    rng = np.random.default_rng(43)
    for n in (100_003, 65_536):
        vals = rng.integers(0, 2**64, size=1000, dtype=np.uint64)
        keys_u = vals[rng.integers(0, 1000, size=n)]
        assert (keys_u >> np.uint64(63)).any() and not (keys_u >> np.uint64(63)).all()
        order = np.argsort(keys_u, kind="stable")
        keys = torch.from_numpy(keys_u.view(np.int64)).cuda()
        out_keys = torch.full_like(keys, -1)
        out_perm = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        S.sph_sort_keys_static(keys, out_keys, out_perm)
        torch.cuda.synchronize()
        assert np.array_equal(out_keys.cpu().numpy().view(np.uint64), keys_u[order])
        assert np.array_equal(out_perm.cpu().numpy(), order.astype(np.int32))


def test_static_sort_rejects_oversize():
    import paper_2003_10850_gb300 as S
    from paper_2003_10850_gb300 import abi
    n = abi.SPH_SORT_STATIC_MAX_KEYS + 1
    keys = torch.zeros(n, dtype=torch.int64, device="cuda")
    out = torch.empty_like(keys)
    perm = torch.empty(n, dtype=torch.int32, device="cuda")
    with pytest.raises(S.SPHError) as e:
        S.sph_sort_keys_static(keys, out, perm)
    assert e.value.status == abi.SPH_ERR_INVALID
