"""Pins for the FP64 reference gradient (oracle/adjoint.py): its forward
values equal the C oracle's; its gradient equals central finite differences
of the C oracle's loss (positions moved continuously, every h re-solved);
the position gradient sums to zero (translation invariance). CPU only."""
import numpy as np
import pytest

import oracle
import workloads as W
from oracle import adjoint

torch = pytest.importorskip("torch")


def _setup(n=1200, seed=7, alpha=1.0):
    p = W.clustered(n, 3, seed=seed)
    X = oracle.quantize(p.pos)
    xc = X.astype(np.float64) / 2.0**32          # the quantised positions, as reals
    d = oracle.density(None, p.mass, None, tol=1e-12, xc=xc)
    f = oracle.force(None, p.vel, p.mass, p.u, d["h"], d["rho"], d["omega"], alpha=alpha, xc=xc)
    rng = np.random.default_rng(seed)
    a_star = f["acc"] * (1 + 0.01 * rng.normal(size=(n, 1)))
    rho_star = d["rho"] * (1 + 0.01 * rng.normal(size=n))
    return p, X, xc, d, f, a_star, rho_star


def _loss_c(p, xc, mass, u, a_star, rho_star, alpha):
    d = oracle.density(None, mass, None, tol=1e-13, xc=np.mod(xc, 1.0))
    f = oracle.force(None, p.vel, mass, u, d["h"], d["rho"], d["omega"], alpha=alpha, xc=np.mod(xc, 1.0))
    return ((f["acc"] - a_star) ** 2).sum() + ((d["rho"] - rho_star) ** 2).sum()


def test_reference_forward_matches_oracle():
    p, X, xc, d, f, a_star, rho_star = _setup(alpha=1.0)
    pairs = oracle.pair_list(X, d["h"])
    _, _, _, acc, rho = adjoint.forward_torch(X, p.mass, p.u, p.vel, 1.0, d["h"], pairs, requires_grad=False)
    np.testing.assert_allclose(rho.numpy(), d["rho"], rtol=1e-11)
    da = np.linalg.norm(acc.numpy() - f["acc"], axis=1)
    assert np.all(da <= 1e-10 * f["scale_a"])


@pytest.mark.parametrize("alpha", [0.0, 1.0])
def test_reference_gradient_matches_finite_differences(alpha):
    p, X, xc, d, f, a_star, rho_star = _setup(alpha=alpha)
    g = adjoint.reference_gradient(X, p.mass, p.u, p.vel, 1.0, a_star, rho_star, alpha=alpha, h_star=d["h"])
    rng = np.random.default_rng(3)
    L0 = _loss_c(p, xc, p.mass, p.u, a_star, rho_star, alpha)
    checked = 0
    for k in rng.choice(p.n, 12, replace=False):
        for ax in (0, 1, 2):
            e = 2e-7
            xp = xc.copy(); xp[k, ax] += e
            xm = xc.copy(); xm[k, ax] -= e
            Lp = _loss_c(p, xp, p.mass, p.u, a_star, rho_star, alpha)
            Lm = _loss_c(p, xm, p.mass, p.u, a_star, rho_star, alpha)
            fd = (Lp - Lm) / (2 * e)
            if alpha > 0:
                # a step that straddles a viscosity kink (w_ij = 0) makes the central
                # difference depend on the step: compare with a doubled step
                xp[k, ax] += e
                xm[k, ax] -= e
                fd2 = (_loss_c(p, xp, p.mass, p.u, a_star, rho_star, alpha) -
                       _loss_c(p, xm, p.mass, p.u, a_star, rho_star, alpha)) / (4 * e)
                if abs(fd2 - fd) > 1e-5 * abs(fd) + 1e-8 * L0:
                    continue
            assert abs(g["g_pos"][k, ax] - fd) <= 2e-5 * abs(fd) + 1e-7 * L0, (k, ax, g["g_pos"][k, ax], fd)
            checked += 1
        for name, arr in (("g_u", p.u), ("g_mass", p.mass)):
            e = 1e-6 * arr[k]
            ap = arr.copy(); ap[k] += e
            am = arr.copy(); am[k] -= e
            if name == "g_u":
                fd = (_loss_c(p, xc, p.mass, ap, a_star, rho_star, alpha) -
                      _loss_c(p, xc, p.mass, am, a_star, rho_star, alpha)) / (2 * e)
            else:
                fd = (_loss_c(p, xc, ap, p.u, a_star, rho_star, alpha) -
                      _loss_c(p, xc, am, p.u, a_star, rho_star, alpha)) / (2 * e)
            assert abs(g[name][k] - fd) <= 2e-5 * abs(fd) + 1e-7 * L0 / arr[k], (name, k, g[name][k], fd)
    assert checked >= 24


def test_reference_gradient_translation_invariant():
    p, X, xc, d, f, a_star, rho_star = _setup(alpha=1.0)
    g = adjoint.reference_gradient(X, p.mass, p.u, p.vel, 1.0, a_star, rho_star, h_star=d["h"])
    s = np.abs(g["g_pos"]).sum(0)
    assert np.all(np.abs(g["g_pos"].sum(0)) <= 1e-10 * s)
