"""GPU parity of the time-dependent artificial viscosity against the FP64
oracle, through the C ABI: the force pass with a viscosity parameter per
particle (sph_hydro_force_visc; alpha_ij = (alpha_i + alpha_j)/2, with and
without Balsara's switch, from the recorded lists and from the walk), the
Morris & Monaghan rate (sph_visc_rate), and a KDK cycle that integrates the
parameters (sph_kick_scalar, sph_predict_scalar).

Tolerances: the force as for the plain force (1e-4 of the per-particle
pair-term scale, pair sets exact); the rate elementwise in FP32 (1e-6 of its
terms' magnitudes); in the KDK cycle the first rates within what the
divergence's tolerance (1e-4 of its scale) lets through, and the integrated
alpha within 2e-3 of the largest change of alpha over the cycle.
"""
import numpy as np
import pytest
import torch

import oracle
import workloads as W
from oracle import kdk as OK
from sph_cases import as_f32, check_force, dev, gpu_grid, host, oracle_all

pytestmark = pytest.mark.gpu

GAMMA = 5.0 / 3.0


@pytest.fixture(scope="module")
def S():
    from paper_2003_10850_gb300 import build
    build.build()
    import paper_2003_10850_gb300 as S
    return S


@pytest.fixture(scope="module")
def ctx(S):
    return S.Context(0)


@pytest.fixture(scope="module")
def clustered():
    p = as_f32(W.clustered(40_000, 30, seed=303))
    return p, oracle_all(p)


@pytest.mark.parametrize("switch", [False, True])
def test_force_per_particle_alpha(S, ctx, clustered, switch):
    p, (X, d, _) = clustered
    h, rho, om = (d[k].astype(np.float32) for k in ("h", "rho", "omega"))
    rng = np.random.default_rng(9)
    alpha = rng.uniform(0.02, 1.5, p.n).astype(np.float32)
    sw = {}
    if switch:
        div_o, curl_o = oracle.divcurl(X, p.vel, p.mass, h, rho, box=p.box)
        sw = {"divv": div_o.astype(np.float32), "curlv": curl_o.astype(np.float32)}
    params = S.default_params(box=p.box)
    grid = gpu_grid(S, ctx, p, params)
    S.density(ctx, grid, dev(h), None, S.default_params(box=p.box, flags=S.SPH_FIXED_H))
    S.sph_sync_status(ctx)
    f_mean = oracle.force(X, p.vel, p.mass, p.u, h, rho, om, box=p.box, alpha=float(alpha.mean()), **sw)
    for hh, lists in ((h, True), ((h * np.float32(1.001)).astype(np.float32), False)):
        fo = oracle.force(X, p.vel, p.mass, p.u, hh, rho, om, box=p.box, alpha=alpha.astype(np.float64), **sw)
        n = p.n
        acc, du, vs = torch.zeros(n, 3, device="cuda"), torch.zeros(n, device="cuda"), torch.zeros(n, device="cuda")
        hs = torch.zeros(n, dtype=torch.int64, device="cuda")
        dsw = (dev(sw["divv"]), dev(sw["curlv"])) if switch else (None, None)
        S.sph_hydro_force_visc(ctx, grid, dev(p.vel), dev(p.u), dev(hh), dev(rho), dev(om), dev(alpha), *dsw, None,
                               acc, du, vs, hs, params)
        rc, st = S.sph_sync_status(ctx, raise_on_error=False)
        assert rc == 0 and (st["pair_tests"] == 0) == lists
        g = {"acc": host(acc), "dudt": host(du), "vsig": host(vs), "hash": host(hs).view(np.uint64)}
        check_force(g, fo, np.arange(n), 1e-4)
    # the per-particle alphas matter: the force differs from the one at their mean
    da = np.linalg.norm(f_mean["acc"] - fo["acc"], axis=1) / fo["scale_a"]
    assert da.max() > 1e-3


def test_visc_rate_elementwise(S, ctx):
    rng = np.random.default_rng(4)
    n = 100_000
    h = rng.uniform(1e-3, 0.1, n).astype(np.float32)
    u = (10.0 ** rng.uniform(-2, 2, n)).astype(np.float32)
    divv = rng.normal(0.0, 50.0, n).astype(np.float32)
    divv[:1000] = 0.0
    alpha = rng.uniform(0.0, 1.2, n).astype(np.float32)
    amin, amax, ell = 0.0625, 1.0, 0.25   # exact in FP32
    ref = oracle.visc_rate(h, u, divv, alpha, amin, amax, ell, GAMMA)
    c = np.sqrt(GAMMA * (GAMMA - 1.0) * u.astype(np.float64))
    scale = np.abs(alpha - amin) * ell * c / h + np.maximum(-divv, 0) * np.abs(amax - alpha)
    out = torch.zeros(n, device="cuda")
    act = np.sort(rng.choice(n, n // 3, replace=False)).astype(np.int32)
    S.sph_visc_rate(ctx, dev(act, torch.int32), dev(h), dev(u), dev(divv), dev(alpha), out, GAMMA, amin, amax, ell)
    S.sph_visc_rate(ctx, None, dev(h), dev(u), dev(divv), dev(alpha), out, GAMMA, amin, amax, ell)
    S.sph_sync_status(ctx)
    g = host(out).astype(np.float64)
    assert np.all(np.abs(g - ref) <= 1e-6 * scale + 1e-30)
    with pytest.raises(S.SPHError):
        S.sph_visc_rate(ctx, None, dev(h), dev(u), dev(divv), dev(alpha), out, GAMMA, 1.0, 0.5, ell)


def test_kdk_cycle_with_time_dependent_viscosity(S, ctx):
    from paper_2003_10850_gb300.kdk import KDK
    p = as_f32(W.clustered(4096, 6, seed=23))
    max_bin = 2
    visc = {"alpha0": 0.5, "alpha_min": 0.1, "alpha_max": 1.0, "ell": 0.2}
    probe = OK.KDK(p.pos, p.vel, p.mass, p.u, np.zeros(p.n, np.uint8), 1e-3, max_bin)
    dt = np.float32(0.3) * probe.h.astype(np.float32) / probe.vsig.astype(np.float32)
    dt_max = float(2 ** max_bin * dt.min()) * 0.999
    bins = OK.timebins(probe.h, probe.vsig, 0.3, dt_max, max_bin)
    ref = OK.KDK(p.pos, p.vel, p.mass, p.u, bins, dt_max, max_bin, balsara=True, visc=visc)
    g = KDK(ctx, dev(p.pos, torch.float64), dev(p.mass), dev(p.vel), dev(p.u), dt_max, max_bin,
            bins=dev(bins, torch.uint8), balsara=True, visc=visc)
    # the first rates (all particles, at t = 0) agree elementwise, within what
    # the divergence's tolerance (1e-4 of its scale) lets through
    _, _, sd, _ = oracle.divcurl(oracle.quantize(p.pos), p.vel, p.mass, ref.h, ref.rho, scales=True)
    bound = 1e-4 * sd * abs(visc["alpha_max"] - visc["alpha0"]) + 1e-5 * np.abs(ref.dav) + 1e-6
    assert np.all(np.abs(host(g.dalpha) - ref.dav) <= bound)
    for _ in range(1 << max_bin):
        assert g.step() == ref.step()
    a_g = host(g.synchronized_alpha()).astype(np.float64)
    a_o = ref.synchronized_alpha()
    moved = np.abs(a_o - visc["alpha0"])
    assert moved.max() > 0.02                              # alpha evolved
    assert np.all(np.abs(a_g - a_o) <= 2e-3 * moved.max() + 1e-6)
    v_g, u_g = (host(t).astype(np.float64) for t in g.synchronized_velocity())
    v_o, u_o = ref.synchronized_velocity()
    dv = np.linalg.norm(v_g - v_o, axis=1)
    assert np.all(dv <= 2e-3 * ref.scale_a + 1e-6 * (np.linalg.norm(v_o, axis=1) + 0.1))
