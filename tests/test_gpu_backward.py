"""GPU adjoint (sph_backward) against the FP64 reference gradient.

Both sides take the same seeded random seeds (dL/da, dL/drho) -- a linear
loss L = sum abar.a + sum rhobar.rho -- so the comparison isolates the
reverse pass; nothing the GPU computes is fed to the reference.

Tolerance, per particle, relative to the reference magnitude plus the median
magnitude: the 99th percentile <= 5e-5 and the maximum <= 3e-3. The GPU sums
FP32 pair terms with compensation (median error ~3e-7), but the position
gradient through rho is the difference of two near-equal parts -- the direct
d rho/dx at fixed h and the implicit-h correction, which cancel exactly at
leading order for equal masses -- so a few particles lose three to four more
digits.
"""
import numpy as np
import pytest
import torch

import oracle
import workloads as W
from oracle import adjoint
from sph_cases import as_f32, dev, host

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


def _errs(g, ref):
    ref = np.asarray(ref, np.float64)
    err = np.abs(np.asarray(g, np.float64) - ref)
    scale = np.abs(ref) + np.median(np.abs(ref))
    if not np.any(scale > 0):
        return err.reshape(len(ref), -1).max(1)       # an identically zero gradient must come out zero
    return (err / scale).reshape(len(ref), -1).max(1)


def _check(g, ref, q99, qmax):
    e = _errs(g, ref)
    assert np.quantile(e, 0.99) <= q99 and e.max() <= qmax, (np.quantile(e, 0.99), e.max())


def _close(g, ref, tol):
    return float(_errs(g, ref).max())


def _gpu_forward(S, ctx, p, params):
    grid = S.sph_build_grid(ctx, dev(p.pos), dev(p.mass), params)
    h = torch.zeros(p.n, device="cuda")
    d = S.density(ctx, grid, h, None, params)
    f = S.hydro_force(ctx, grid, dev(p.vel), dev(p.u), h, d["rho"], d["omega"], None, params)
    S.sph_sync_status(ctx)
    return grid, h, d, f


@pytest.mark.parametrize("alpha", [0.0, 1.0])
def test_vjp_matches_reference(S, ctx, alpha):
    p = as_f32(W.clustered(20_000, 30, seed=505))
    params = S.default_params(alpha_visc=alpha)
    grid, h, d, f = _gpu_forward(S, ctx, p, params)
    rng = np.random.default_rng(9)
    abar = rng.normal(size=(p.n, 3))
    rbar = rng.normal(size=p.n)
    g_pos = torch.empty(p.n, 3, device="cuda")
    g_u = torch.empty(p.n, device="cuda")
    g_m = torch.empty(p.n, device="cuda")
    S.sph_backward(ctx, grid, dev(p.vel), dev(p.u), h, d["rho"], d["omega"], dev(abar), dev(rbar),
                   g_pos, g_u, g_m, params)
    rc, _ = S.sph_sync_status(ctx)
    assert rc == 0
    # reference: FP64 autograd of the same linear loss
    X = oracle.quantize(p.pos)
    h_star = oracle.density(X, p.mass, None, tol=1e-12)["h"]
    pairs = oracle.pair_list(X, h_star)
    x, m, ut, acc, rho = adjoint.forward_torch(X, p.mass, p.u, p.vel, 1.0, h_star, pairs, alpha=alpha)
    L = (acc * torch.as_tensor(abar)).sum() + (rho * torch.as_tensor(rbar)).sum()
    L.backward()
    _check(host(g_pos), x.grad.numpy(), 5e-5, 3e-3)
    _check(host(g_u), ut.grad.numpy(), 5e-5, 3e-3)
    _check(host(g_m), m.grad.numpy(), 5e-5, 3e-3)


def test_autograd_function_config5_loss(S, ctx):
    """The differentiation workload's loss through SPHDensityForce at 262,144
    particles: translation invariance of dL/dx (holds at any size), and on a
    20k instance the gradient of the quadratic loss against the reference."""
    from paper_2003_10850_gb300.autograd import SPHDensityForce
    for n, check_ref in ((262_144, False), (20_000, True)):
        p = as_f32(W.config5(n) if n == 262_144 else W.clustered(n, 30, seed=606))
        X = oracle.quantize(p.pos)
        pos = dev(p.pos).requires_grad_(True)
        mass = dev(p.mass).requires_grad_(True)
        u = dev(p.u).requires_grad_(True)
        rng = np.random.default_rng(5)
        if check_ref:
            d0 = oracle.density(X, p.mass, None, tol=1e-12)
            f0 = oracle.force(X, p.vel, p.mass, p.u, d0["h"], d0["rho"], d0["omega"])
            a_star = f0["acc"] * (1 + 0.01 * rng.normal(size=(n, 1)))
            r_star = d0["rho"] * (1 + 0.01 * rng.normal(size=n))
        acc, rho = SPHDensityForce.apply(pos, dev(p.vel), mass, u, torch.zeros(n, device="cuda"), ctx)
        if not check_ref:
            a_star = host(acc).astype(np.float64) * (1 + 0.01 * rng.normal(size=(n, 1)))
            r_star = host(rho).astype(np.float64) * (1 + 0.01 * rng.normal(size=n))
        loss = ((acc - dev(a_star)) ** 2).sum() + ((rho - dev(r_star)) ** 2).sum()
        loss.backward()
        gp = host(pos.grad).astype(np.float64)
        assert np.all(np.abs(gp.sum(0)) <= 1e-4 * np.abs(gp).sum(0))
        if check_ref:
            ref = adjoint.reference_gradient(X, p.mass, p.u, p.vel, 1.0, a_star, r_star, h_star=d0["h"])
            # The seeds 2(a - a*) carry the FP32 forward error (up to 1e-4 of the
            # pair-term scale, which exceeds |a| where forces cancel) against 1%
            # target offsets, so single particles are ill-conditioned; the
            # gradient is checked in aggregate (relative L2 error) and at the
            # 99th percentile. The seed-free comparison above is per particle.
            for g, r in ((gp, ref["g_pos"]), (host(u.grad), ref["g_u"]), (host(mass.grad), ref["g_mass"])):
                r = np.asarray(r, np.float64)
                assert np.linalg.norm(g - r) <= 5e-3 * np.linalg.norm(r)
                assert np.quantile(_errs(g, r), 0.99) <= 2e-3
