"""Pins for the oracle's time-dependent artificial viscosity: a viscosity
parameter alpha_i per particle, the pair taking (alpha_i + alpha_j)/2, and
the rate of Morris & Monaghan (1997),
  d alpha/dt = -(alpha - alpha_min) ell c / h + max(-div v, 0) (alpha_max - alpha),
integrated by the KDK integrator like u (the paper's code carries the
"improved SPH" viscosity, Sec. 1). CPU only.

What pins them, beyond restating the formulas:
* equal alpha_i reduce to the scalar-alpha force, bit for bit;
* two approaching particles: the viscous force depends on the pair only
  through the mean (alpha_1 + alpha_2)/2 (not alpha_i, the max, or any other
  mean), and is linear in it;
* any alpha_i conserve momentum and energy exactly (a non-symmetric alpha_ij
  breaks both);
* the rate's fixed point and slope are those of the linear ODE, and on a
  lattice at rest (a = 0, div v = 0) the integrated alpha follows the closed
  form alpha_min + (alpha_0 - alpha_min) exp(-t ell c / h), with the error
  falling as dt^2.
"""
import math

import numpy as np

import oracle
import workloads as W
from oracle import kdk as K

GAMMA = 5.0 / 3.0


def _gas(n_side=9, seed=3):
    p = W.lattice(n_side, 0.3, seed=seed, vel_sigma=0.3, u_range=(0.5, 1.5))
    X = oracle.quantize(p.pos)
    d = oracle.density(X, p.mass, None, n_target=64.0)
    return p, X, d


def test_equal_alphas_are_the_scalar_force():
    p, X, d = _gas()
    a = oracle.force(X, p.vel, p.mass, p.u, d["h"], d["rho"], d["omega"], alpha=0.7)
    b = oracle.force(X, p.vel, p.mass, p.u, d["h"], d["rho"], d["omega"], alpha=np.full(p.n, 0.7))
    for k in ("acc", "dudt", "vsig", "hash"):
        assert np.array_equal(a[k], b[k])


def test_pair_takes_the_mean_of_its_alphas():
    pos = np.array([[0.45, 0.5, 0.5], [0.55, 0.52, 0.5]])
    X = oracle.quantize(pos)
    vel = np.array([[1.0, 0.2, 0.0], [-1.0, 0.0, 0.1]])   # approaching: w_ij < 0
    m = np.array([0.6, 1.4])
    u = np.array([1.0, 2.0])
    h = np.array([0.3, 0.25])
    rho = np.array([1.1, 0.9])
    om = np.array([1.0, 1.05])

    def visc(alpha):
        f = oracle.force(X, vel, m, u, h, rho, om, alpha=alpha, brute=True)
        f0 = oracle.force(X, vel, m, u, h, rho, om, alpha=0.0, brute=True)
        return np.concatenate([(f["acc"] - f0["acc"]).ravel(), f["dudt"] - f0["dudt"]])

    ref = visc(0.6)
    assert np.abs(ref).max() > 1e-3
    for pair in ((0.2, 1.0), (1.0, 0.2), (0.6, 0.6), (0.0, 1.2)):
        np.testing.assert_allclose(visc(np.array(pair)), ref, rtol=1e-13, atol=1e-15 * np.abs(ref).max())
    np.testing.assert_allclose(visc(np.array([0.1, 0.5])), 0.5 * ref, rtol=1e-13, atol=1e-15 * np.abs(ref).max())


def test_any_alphas_conserve_momentum_and_energy():
    p, X, d = _gas(seed=4)
    rng = np.random.default_rng(11)
    alpha = rng.uniform(0.05, 1.5, p.n)
    f = oracle.force(X, p.vel, p.mass, p.u, d["h"], d["rho"], d["omega"], alpha=alpha)
    ma = p.mass[:, None] * f["acc"]
    scale = (p.mass * f["scale_a"]).sum()
    assert np.abs(ma.sum(0)).max() <= 1e-12 * scale
    de = (ma * p.vel).sum() + (p.mass * f["dudt"]).sum()
    assert abs(de) <= 1e-12 * (p.mass * (f["scale_a"] * np.linalg.norm(p.vel, axis=1) + f["scale_u"])).sum()
    # the viscosity does work here: a different alpha field changes the result
    g = oracle.force(X, p.vel, p.mass, p.u, d["h"], d["rho"], d["omega"], alpha=alpha[::-1].copy())
    assert np.abs(g["dudt"] - f["dudt"]).max() > 1e-6 * np.abs(f["dudt"]).max()


def test_rate_fixed_point_and_slope():
    rng = np.random.default_rng(2)
    n = 1000
    h = rng.uniform(0.01, 0.1, n)
    u = rng.uniform(0.1, 10.0, n)
    divv = rng.normal(0.0, 30.0, n)
    amin, amax, ell = 0.05, 1.5, 0.3
    c = np.sqrt(GAMMA * (GAMMA - 1.0) * u)
    inv_tau = ell * c / h
    D = np.maximum(-divv, 0.0)
    fixed = (amin * inv_tau + D * amax) / (inv_tau + D)
    r = oracle.visc_rate(h, u, divv, fixed, amin, amax, ell, GAMMA)
    assert np.all(np.abs(r) <= 1e-13 * (inv_tau + D) * amax)
    np.testing.assert_allclose(fixed[divv >= 0], amin, rtol=1e-15)
    assert np.all((fixed >= amin * (1 - 1e-15)) & (fixed <= amax))
    a1, a2 = 0.2, 0.9
    slope = (oracle.visc_rate(h, u, divv, np.full(n, a2), amin, amax, ell, GAMMA)
             - oracle.visc_rate(h, u, divv, np.full(n, a1), amin, amax, ell, GAMMA)) / (a2 - a1)
    np.testing.assert_allclose(slope, -(inv_tau + D), rtol=1e-12)


def test_alpha_decays_on_a_lattice_at_rest():
    p = W.lattice(8, 0.0, seed=0, vel_sigma=0.0, u_range=(1.0, 1.0))
    visc = {"alpha0": 1.0, "alpha_min": 0.1, "alpha_max": 1.0, "ell": 0.5}
    T = 1.5
    errs = []
    for k in (8, 16):
        r = K.KDK(p.pos, p.vel, p.mass, p.u, np.zeros(p.n, np.uint8), T / k, 0, visc=visc)
        h = r.h[0]
        assert np.allclose(r.h, h, rtol=1e-12)
        for _ in range(k):
            r.step()
        a = r.synchronized_alpha()
        tau = h / (visc["ell"] * math.sqrt(GAMMA * (GAMMA - 1.0) * 1.0))
        exact = visc["alpha_min"] + (visc["alpha0"] - visc["alpha_min"]) * math.exp(-T / tau)
        assert T / tau > 1.0                          # alpha decays by a large factor
        errs.append(np.abs(a - exact).max())
        assert np.abs(a - a.mean()).max() <= 1e-12   # uniform state stays uniform
    assert errs[0] < 0.05 * (visc["alpha0"] - visc["alpha_min"])
    assert 3.0 < errs[0] / errs[1] < 5.0
