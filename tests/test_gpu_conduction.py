"""GPU parity of the thermal conduction term (sph_hydro_force_conduction)
against the FP64 oracle, through the C ABI: the conduction heating rate
within 1e-4 of its per-particle scale (sum of the pair terms' magnitudes),
the hydrodynamic outputs as for sph_hydro_force, from the recorded neighbour
lists and from the walk; energy conservation of the GPU result.
"""
import numpy as np
import pytest
import torch

import oracle
import workloads as W
from sph_cases import as_f32, check_force, dev, gpu_grid, host, oracle_all

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    from paper_2003_10850_gb300 import build
    build.build()
    import paper_2003_10850_gb300 as S
    return S


@pytest.fixture(scope="module")
def ctx(S):
    return S.Context(0)


def _case(kind):
    if kind == "clustered":
        p = as_f32(W.clustered(50_000, 40, seed=202))
    else:   # jittered lattice with a periodic temperature profile
        q = W.config1(32)
        u = 1.0 + 0.5 * np.sin(2 * np.pi * q.pos[:, 0]) * np.cos(2 * np.pi * q.pos[:, 2])
        p = as_f32(W.Particles(q.pos, q.vel, q.mass, u, q.box))
    kappa = np.random.default_rng(11).uniform(0.1, 2.0, p.n).astype(np.float32).astype(np.float64)
    return p, kappa


@pytest.mark.parametrize("switch", [False, True])
@pytest.mark.parametrize("kind", ["lattice", "clustered"])
def test_conduction_parity(S, ctx, kind, switch):
    p, kappa = _case(kind)
    X, d, _ = oracle_all(p)
    h, rho, om = (d[k].astype(np.float32) for k in ("h", "rho", "omega"))
    sw = {}
    if switch:
        dv, cv = oracle.divcurl(X, p.vel, p.mass, h, rho, box=p.box)
        sw = {"divv": dv.astype(np.float32), "curlv": cv.astype(np.float32)}
    params = S.default_params(box=p.box)
    grid = gpu_grid(S, ctx, p, params)
    S.density(ctx, grid, dev(h), None, S.default_params(box=p.box, flags=S.SPH_FIXED_H))
    S.sph_sync_status(ctx)
    n = p.n
    m = p.mass
    for hh, lists in ((h, True), ((h * np.float32(1.001)).astype(np.float32), False)):
        fo = oracle.force(X, p.vel, p.mass, p.u, hh, rho, om, box=p.box, **sw)
        co, cs = oracle.conduction(X, p.mass, p.u, hh, rho, kappa, box=p.box)
        acc, du, vs = torch.zeros(n, 3, device="cuda"), torch.zeros(n, device="cuda"), torch.zeros(n, device="cuda")
        dc = torch.zeros(n, device="cuda")
        hs = torch.zeros(n, dtype=torch.int64, device="cuda")
        S.sph_hydro_force_conduction(ctx, grid, dev(p.vel), dev(p.u), dev(hh), dev(rho), dev(om),
                                     dev(sw["divv"]) if switch else None, dev(sw["curlv"]) if switch else None,
                                     dev(kappa), None, acc, du, vs, dc, hs, params)
        rc, st = S.sph_sync_status(ctx, raise_on_error=False)
        assert rc == 0 and (st["pair_tests"] == 0) == lists
        g = {"acc": host(acc), "dudt": host(du), "vsig": host(vs), "hash": host(hs).view(np.uint64)}
        check_force(g, fo, np.arange(n), 1e-4)
        dcg = host(dc).astype(np.float64)
        assert np.all(np.abs(dcg - co) <= 1e-4 * cs + 1e-30), (np.abs(dcg - co) / cs).max()
        assert abs((m * dcg).sum()) <= 1e-5 * (m * cs).sum()
    assert np.abs(co).max() > 1e-3 * cs.max()   # the profile conducts


def test_conduction_requires_kappa_and_default_path(S, ctx):
    p, kappa = _case("lattice")
    grid = gpu_grid(S, ctx, p, S.default_params(box=p.box))
    n = p.n
    z = lambda *s: torch.zeros(*s, device="cuda")
    with pytest.raises(S.SPHError):
        S.sph_hydro_force_conduction(ctx, grid, dev(p.vel), dev(p.u), z(n) + 0.1, z(n) + 1, z(n) + 1, None, None,
                                     dev(kappa), None, z(n, 3), z(n), z(n), z(n), None,
                                     S.default_params(box=p.box, flags=S.SPH_PER_THREAD_WALK))
