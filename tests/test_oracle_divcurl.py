"""Pins for the oracle's velocity divergence / curl and Balsara's viscosity
switch (the "improved SPH" direction of the paper's code, Sec. 1; the forms
are Gadget-2's). CPU only.

What pins them, beyond restating the sums:
* cubic-lattice symmetry: for a linear velocity field v = A x seen by a
  particle whose neighbourhood does not wrap, sum_n n_a n_b f(|n|) =
  delta_ab / 3 sum_n |n|^2 f(|n|) over the lattice, so the SPH estimates are
  exactly  div = tr(A) k  and  curl = |2 omega| k  (omega the axial vector of
  A's antisymmetric part; the symmetric part has no curl), with one lattice
  constant k = -(m / (3 rho)) sum_n |r_n| W'(|r_n|), enumerated here;
* the continuum limit: k = 1 to within a few per cent on a resolved lattice;
* Galilean invariance and cell list = brute force;
* the switch: in a pure shear (div = 0 exactly) it turns the viscosity off,
  so the switched force equals the alpha = 0 force; conservation of momentum
  and energy holds for any per-particle factor.
"""
import math

import numpy as np

import oracle
import workloads as W

GAMMA = 5.0 / 3.0


def _lattice_k(a, h, m, rho):
    """-(m/(3 rho)) sum_{0 < |n| a < h} |r_n| W'(|r_n|, h), W' = 8/(pi h^4) w'(q)."""
    k = int(math.ceil(h / a)) + 1
    g = np.arange(-k, k + 1)
    nx, ny, nz = np.meshgrid(g, g, g, indexing="ij")
    r = a * np.sqrt(nx**2 + ny**2 + nz**2).ravel()
    r = r[(r > 0) & (r < h)]
    _, dw = oracle.kernel(r / h)
    dWdr = 8.0 / (math.pi * h**4) * dw
    return -(m / (3.0 * rho)) * np.sum(r * dWdr)


def _lattice_setup(n_side=16):
    p = W.lattice(n_side, 0.0, seed=0, vel_sigma=0.0, u_range=(1.0, 1.0))
    X = oracle.quantize(p.pos)
    d = oracle.density(X, p.mass, None, n_target=64.0)
    h = d["h"][0]
    inner = np.all((p.pos > h) & (p.pos < 1.0 - h), axis=1)   # neighbourhoods that do not wrap
    return p, X, d, h, inner


def test_linear_field_on_lattice_gives_trace_and_axial_vector():
    p, X, d, h, inner = _lattice_setup()
    assert inner.sum() > 500
    rng = np.random.default_rng(7)
    A = rng.normal(size=(3, 3))
    vel = p.pos @ A.T
    div, curl = oracle.divcurl(X, vel, p.mass, d["h"], d["rho"])
    kap = _lattice_k(1.0 / 16, h, p.mass[0], d["rho"][0])
    np.testing.assert_allclose(div[inner], np.trace(A) * kap, rtol=1e-11)
    omega = 0.5 * np.array([A[2, 1] - A[1, 2], A[0, 2] - A[2, 0], A[1, 0] - A[0, 1]])
    np.testing.assert_allclose(curl[inner], 2.0 * np.linalg.norm(omega) * kap, rtol=1e-11)
    # a symmetric field has no curl, an antisymmetric one no divergence
    S = 0.5 * (A + A.T)
    div_s, curl_s = oracle.divcurl(X, p.pos @ S.T, p.mass, d["h"], d["rho"])
    assert np.abs(curl_s[inner]).max() <= 1e-12 * np.abs(div_s[inner]).max()
    R = 0.5 * (A - A.T)
    div_r, curl_r = oracle.divcurl(X, p.pos @ R.T, p.mass, d["h"], d["rho"])
    assert np.abs(div_r[inner]).max() <= 1e-12 * curl_r[inner].max()
    # continuum limit: the SPH derivative of a linear field is the derivative
    assert abs(kap - 1.0) < 0.05


def test_divcurl_galilean_and_cell_list_equals_brute():
    p = W.clustered(3000, 5, seed=61)
    X = oracle.quantize(p.pos)
    d = oracle.density(X, p.mass, None)
    a = oracle.divcurl(X, p.vel, p.mass, d["h"], d["rho"])
    b = oracle.divcurl(X, p.vel + np.array([0.3, -1.2, 2.0]), p.mass, d["h"], d["rho"])
    c = oracle.divcurl(X, p.vel, p.mass, d["h"], d["rho"], brute=True)
    for x, y in zip(a, b):
        np.testing.assert_allclose(x, y, rtol=1e-9, atol=1e-12 * np.abs(x).max())
    for x, y in zip(a, c):
        np.testing.assert_allclose(x, y, rtol=1e-12, atol=1e-14 * np.abs(x).max())
    assert np.all(a[1] >= 0)


def test_switch_off_in_pure_shear():
    """Simple shear v = (s y, 0, 0) on the perfect lattice: div = 0 exactly
    where the neighbourhood does not wrap (tr A = 0) while curl and the
    approaching pairs (w_ij < 0) are not, so the Balsara factor is 0 there and,
    for a particle whose partners all have factor 0, the switched force equals
    the alpha = 0 (pressure only) force although the plain viscosity acts."""
    p, X, d, h, inner = _lattice_setup()
    vel = np.zeros_like(p.pos)
    vel[:, 0] = 0.8 * (p.pos[:, 1] - 0.5)
    div, curl = oracle.divcurl(X, vel, p.mass, d["h"], d["rho"])
    u = np.full(p.n, 1.0)
    f_sw = oracle.force(X, vel, p.mass, u, d["h"], d["rho"], d["omega"], alpha=1.0, divv=div, curlv=curl)
    f_0 = oracle.force(X, vel, p.mass, u, d["h"], d["rho"], d["omega"], alpha=0.0)
    f_1 = oracle.force(X, vel, p.mass, u, d["h"], d["rho"], d["omega"], alpha=1.0)
    deep = np.all((p.pos > 2.2 * h) & (p.pos < 1.0 - 2.2 * h), axis=1)   # partners all inner too
    assert deep.sum() > 20
    sc = f_1["scale_a"][deep][:, None]
    np.testing.assert_allclose(f_sw["acc"][deep] / sc, f_0["acc"][deep] / sc, rtol=0, atol=1e-12)
    assert curl[deep].min() > 0.1
    # and the unswitched viscosity is not zero there (shear has approaching pairs)
    assert np.abs(f_1["dudt"][deep] - f_0["dudt"][deep]).max() > 1e-6 * np.abs(f_1["scale_u"][deep]).max()


def test_switch_keeps_conservation_and_only_scales_viscosity():
    p = W.clustered(4000, 6, seed=71)
    X = oracle.quantize(p.pos)
    d = oracle.density(X, p.mass, None)
    div, curl = oracle.divcurl(X, p.vel, p.mass, d["h"], d["rho"])
    f = oracle.force(X, p.vel, p.mass, p.u, d["h"], d["rho"], d["omega"], divv=div, curlv=curl)
    m = p.mass
    mom = (m[:, None] * f["acc"]).sum(0)
    assert np.linalg.norm(mom) <= 1e-12 * (m * np.linalg.norm(f["acc"], axis=1)).sum()
    e = m * ((p.vel * f["acc"]).sum(1) + f["dudt"])
    assert abs(e.sum()) <= 1e-12 * (m * (np.abs((p.vel * f["acc"]).sum(1)) + np.abs(f["dudt"]))).sum()
    # the switch only rescales Pi: between the alpha = 0 and alpha = 1 forces pair by
    # pair, so the dissipation sum_i m_i du_i (viscous part) shrinks but keeps its sign
    f0 = oracle.force(X, p.vel, p.mass, p.u, d["h"], d["rho"], d["omega"], alpha=0.0)
    f1 = oracle.force(X, p.vel, p.mass, p.u, d["h"], d["rho"], d["omega"], alpha=1.0)
    visc_sw = (m * (f["dudt"] - f0["dudt"])).sum()
    visc_1 = (m * (f1["dudt"] - f0["dudt"])).sum()
    assert 0.0 <= visc_sw <= visc_1
    # factors within [0, 1): a huge divergence makes the switch transparent
    big = np.full(p.n, 1e30)
    fb = oracle.force(X, p.vel, p.mass, p.u, d["h"], d["rho"], d["omega"], divv=big, curlv=np.zeros(p.n))
    np.testing.assert_allclose(fb["acc"], f1["acc"], rtol=0, atol=1e-12 * f1["scale_a"].max())
