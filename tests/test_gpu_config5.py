"""Config 5 at its stated size: 262,144 clustered particles (seed 5). The GPU
adjoint of the density and force passes (sph_backward) against central finite
differences of the FP64 oracle, step 1e-6 on continuous FP64 positions, on
1,026 sampled coordinates (342 particles x 3 axes, seeded).

The loss is linear in the passes' outputs, L = sum abar.a + sum rbar.rho, with
seeded seeds: the workload's quadratic loss is this one with the seeds
2(a - a*) and 2(rho - rho*), which would carry the FP32 forward error into the
comparison; fixed seeds isolate the reverse pass.

Local re-evaluation: moving x_k changes h, rho and Omega only of the set A1 of
particles whose sphere holds k (|x_i - x_k| < h_i, with a margin for the step),
and a only of the set A2 of particles that have k or a member of A1 as a force
partner (|x_i - x_j| < max(h_i, h_j)); both lie within 2 h_max of k (h_max: the
largest converged h of the system). Each difference is therefore evaluated by
the oracle on the particles within 3 h_max (plus a margin) of k: the density
of A1 (solved again from the converged h), then the force of A2, with the
converged h, rho and Omega of the full system for every particle outside A1.
The local sum L_k = sum_{A2} abar_i.a_i + sum_{A1} rbar_i rho_i then differs
from L by terms that do not depend on x_k. The artificial
viscosity has a kink where w_ij changes sign; a coordinate whose central
differences at the step and at half of it disagree (a step across the kink) is
excluded and counted.

Tolerance as the 20k reference comparison: per coordinate, relative to the
reference magnitude plus its median, the 99th percentile <= 5e-5 and the
maximum <= 3e-3.
"""
import numpy as np
import pytest
import torch

import oracle
import workloads as W
from sph_cases import as_f32, dev, host

pytestmark = pytest.mark.gpu

N_PART = 342
EPS = 1e-6


@pytest.fixture(scope="module")
def S():
    from paper_2003_10850_gb300 import build
    build.build()
    import paper_2003_10850_gb300 as S
    return S


@pytest.fixture(scope="module")
def ctx(S):
    return S.Context(0)


def _wrap(d):
    return d - np.round(d)


def test_config5_gradient_against_finite_differences(S, ctx):
    spatial = pytest.importorskip("scipy.spatial")
    p = as_f32(W.config5())
    n = p.n
    assert n == 262_144
    rng = np.random.default_rng(55)
    abar = rng.normal(size=(n, 3))
    rbar = rng.normal(size=n)
    # GPU: forward passes, then the adjoint with the seeds
    params = S.default_params()
    grid = S.sph_build_grid(ctx, dev(p.pos), dev(p.mass), params)
    h = torch.zeros(n, device="cuda")
    d = S.density(ctx, grid, h, None, params)
    S.hydro_force(ctx, grid, dev(p.vel), dev(p.u), h, d["rho"], d["omega"], None, params)
    g_pos = torch.empty(n, 3, device="cuda")
    g_u = torch.empty(n, device="cuda")
    g_m = torch.empty(n, device="cuda")
    S.sph_backward(ctx, grid, dev(p.vel), dev(p.u), h, d["rho"], d["omega"], dev(abar), dev(rbar),
                   g_pos, g_u, g_m, params)
    rc, _ = S.sph_sync_status(ctx)
    assert rc == 0
    gp = host(g_pos).astype(np.float64)
    grid.free()
    # oracle: the converged state of the whole system (continuous positions)
    full = oracle.density(None, p.mass, None, tol=1e-12, xc=p.pos)
    hmax = float(full["h"].max())
    tree = spatial.cKDTree(p.pos, boxsize=1.0 + 1e-12)
    ks = W.sample_indices(n, N_PART, seed=56)
    ref = np.zeros((N_PART, 3))
    jump = np.zeros((N_PART, 3))
    for t, k in enumerate(ks):
        patch = np.asarray(tree.query_ball_point(p.pos[k], 3.0 * hmax * 1.05), np.int64)
        dk = np.linalg.norm(_wrap(p.pos[patch] - p.pos[k]), axis=1)
        hp = full["h"][patch]
        # densities that may change: k inside the particle's sphere (with a margin
        # for the step and the h that moves with it)
        a1 = np.nonzero(dk < hp * 1.001 + 4 * EPS)[0]
        # accelerations that may change: k or a member of a1 is a force partner
        near = np.nonzero(dk < 2.0 * hmax * 1.02)[0]
        dij = np.linalg.norm(_wrap(p.pos[patch[near]][:, None, :] - p.pos[patch[a1]][None, :, :]), axis=2)
        reach = np.maximum(hp[near][:, None], hp[a1][None, :]) * 1.001 + 4 * EPS
        a2 = near[(dij < reach).any(axis=1)]
        # the particles that enter: within h_max of a member of a2
        keep = dk < dk[a2].max() + hmax * 1.02
        kl = int(np.nonzero(patch == k)[0][0])
        remap = np.cumsum(keep) - 1
        patch, a1, a2, kl = patch[keep], remap[a1], remap[a2], int(remap[kl])
        pos0 = p.pos[patch].copy()
        sub = lambda a: np.ascontiguousarray(a[patch])
        m, v, u = sub(p.mass), sub(p.vel), sub(p.u)
        h0, rho0, om0 = sub(full["h"]), sub(full["rho"]), sub(full["omega"])

        def loss(pos):
            dd = oracle.density(None, m, h0, tol=1e-12, active=a1, xc=pos)
            hh, rr, oo = h0.copy(), rho0.copy(), om0.copy()
            hh[a1], rr[a1], oo[a1] = dd["h"][a1], dd["rho"][a1], dd["omega"][a1]
            ff = oracle.force(None, v, m, u, hh, rr, oo, active=a2, xc=pos)
            return (abar[patch[a2]] * ff["acc"][a2]).sum() + (rbar[patch[a1]] * rr[a1]).sum()

        def central(ax, eps):
            lp_pos, lm_pos = pos0.copy(), pos0.copy()
            lp_pos[kl, ax] += eps
            lm_pos[kl, ax] -= eps
            return (loss(np.mod(lp_pos, 1.0)) - loss(np.mod(lm_pos, 1.0))) / (2 * eps)

        for ax in range(3):
            ref[t, ax] = central(ax, EPS)
            jump[t, ax] = abs(ref[t, ax] - central(ax, EPS / 2))
    # On a smooth stretch the central differences at eps and eps/2 agree to
    # O(eps^2 / h^2) (below 1e-5 of the gradient here); a step that crosses the
    # viscosity kink (w_ij = 0) moves them apart by a share of one pair's term.
    # Such coordinates are excluded.
    med = np.median(np.abs(ref))
    kink = jump > 1e-4 * (np.abs(ref) + med)
    excluded = int(kink.sum())
    ok = ~kink
    assert excluded <= 0.05 * ref.size, (excluded, np.quantile(jump / (np.abs(ref) + med), [0.5, 0.9, 0.99]))
    g = gp[ks][ok]
    r = ref[ok]
    err = np.abs(g - r) / (np.abs(r) + np.median(np.abs(r)))
    print(f"config 5: {ok.sum()} coordinates ({excluded} excluded), error q99 {np.quantile(err, 0.99):.2e} "
          f"max {err.max():.2e}")
    assert np.quantile(err, 0.99) <= 5e-5 and err.max() <= 3e-3, (np.quantile(err, 0.99), err.max())
