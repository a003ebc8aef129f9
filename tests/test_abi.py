"""The C-ABI library builds, loads and exports every symbol include/sph.h
declares; host-side validation works without a GPU (no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2003_10850_gb300 import abi, build
    build.build()
    return abi.load()


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(sph_[a-z_0-9]+)\s*\(", txt))
    return sorted(names)


def test_every_declared_symbol_is_exported(lib):
    declared = _declared()
    assert len(declared) >= 12
    for name in declared:
        assert hasattr(lib, name), name


def test_binding_covers_the_abi():
    from paper_2003_10850_gb300 import abi
    assert set(_declared()) <= set(abi.EXPORTED)


def test_default_params_and_struct_layout(lib):
    from paper_2003_10850_gb300 import abi
    p = abi.default_params()
    assert (p.box, p.n_target, p.max_iter, p.alpha_visc) == (1.0, 64.0, 64, 1.0)
    assert abs(p.n_tol - 64e-6) < 1e-18 and abs(p.gamma - 5.0 / 3.0) < 1e-15
    assert p.walk_radius == 0.0 and p.blocks_per_sm == 0
    assert ctypes.sizeof(abi.sph_params) == 72
    assert ctypes.sizeof(abi.sph_stats) == 96
    assert ctypes.sizeof(abi.sph_gravity_params) == 40


def test_host_validation_without_gpu(lib):
    from paper_2003_10850_gb300 import abi
    out = ctypes.c_void_p()
    assert lib.sph_create(None, 0) == abi.SPH_ERR_INVALID
    # NULL context is rejected before any CUDA call
    p = abi.default_params()
    assert lib.sph_build_grid(None, None, 0, None, 10, ctypes.byref(p), None, ctypes.byref(out)) \
        == abi.SPH_ERR_INVALID
    assert lib.sph_sync_status(None, None, None) == abi.SPH_ERR_INVALID
    assert lib.sph_last_error(None) == b"context is NULL"


def test_later_entry_points_reject_a_null_context_without_gpu(lib):
    """The time-integration, viscosity and gravity entry points check their
    context before any CUDA call."""
    from paper_2003_10850_gb300 import abi
    gp = abi.sph_gravity_params(1.0, 0.5, 0.0, 0.1, 0.0)
    dts = (ctypes.c_double * 1)(0.1)
    assert lib.sph_gravity(None, None, None, 0, ctypes.byref(gp), None, None, None, None) == abi.SPH_ERR_INVALID
    assert lib.sph_visc_rate(None, None, 0, None, None, None, None, 5 / 3, 0.1, 1.0, 0.2, None, None) \
        == abi.SPH_ERR_INVALID
    assert lib.sph_kick_scalar(None, None, 0, None, dts, 1, None, None, None, None) == abi.SPH_ERR_INVALID
    assert lib.sph_predict_scalar(None, 1, 0.1, None, None, None) == abi.SPH_ERR_INVALID
    assert lib.sph_timebins(None, None, None, None, 0, 1, 0, 0.3, 1.0, 2, None, None) == abi.SPH_ERR_INVALID
    assert lib.sph_drift(None, None, None, 1, 0.1, 1.0, None, None, None, None, None) == abi.SPH_ERR_INVALID
    p = abi.default_params()
    assert lib.sph_hydro_force_visc(None, None, None, None, None, None, None, None, None, None, None, 0, None,
                                    None, None, None, ctypes.byref(p), None) == abi.SPH_ERR_INVALID
