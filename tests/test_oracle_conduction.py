"""Pins for the oracle's thermal conduction pass (NEXT-2; the paper's code
has a conduction module, Sec. 1; the form is Cleary & Monaghan's 1999 SPH
conduction, as Jubelgas, Springel & Dolag 2004 used it in Gadget). CPU only.

What pins it, beyond restating the sum:
* energy conservation: the pair terms are antisymmetric, sum_i m_i du_i = 0;
* the second law: sum_i m_i u_i du_i <= 0 (heat flows down the gradient);
* a uniform u conducts nothing; a linear u on a perfect lattice conducts
  nothing either (symmetric neighbour shells), away from the periodic seam;
* a quadratic u = |x|^2 on the perfect lattice gives, for every particle whose
  neighbourhood does not wrap, du = -(2 kappa m / rho^2) sum_n |r_n| W'(|r_n|),
  a lattice sum enumerated here, and that is (kappa / rho) Laplacian(u) =
  6 kappa / rho to within a few per cent (continuum limit);
* linear in kappa; the harmonic mean insulates where a neighbour has kappa 0;
  cell list = brute force.
"""
import math

import numpy as np

import oracle
import workloads as W


def _lattice_setup(n_side=16):
    p = W.lattice(n_side, 0.0, seed=0, vel_sigma=0.0, u_range=(1.0, 1.0))
    X = oracle.quantize(p.pos)
    d = oracle.density(X, p.mass, None, n_target=64.0)
    h = d["h"][0]
    inner = np.all((p.pos > h) & (p.pos < 1.0 - h), axis=1)
    return p, X, d, h, inner


def test_conservation_and_second_law():
    p = W.clustered(4000, 6, seed=81)
    X = oracle.quantize(p.pos)
    d = oracle.density(X, p.mass, None)
    kappa = np.random.default_rng(3).uniform(0.1, 2.0, p.n)
    du, sc = oracle.conduction(X, p.mass, p.u, d["h"], d["rho"], kappa)
    m = p.mass
    assert abs((m * du).sum()) <= 1e-12 * (m * sc).sum()
    assert (m * p.u * du).sum() < 0.0
    # brute force gives the same sums
    du_b, _ = oracle.conduction(X, p.mass, p.u, d["h"], d["rho"], kappa, brute=True)
    np.testing.assert_allclose(du, du_b, rtol=1e-11, atol=1e-13 * sc.max())
    # linear in kappa
    du2, _ = oracle.conduction(X, p.mass, p.u, d["h"], d["rho"], 3.0 * kappa)
    np.testing.assert_allclose(du2, 3.0 * du, rtol=1e-12, atol=1e-14 * sc.max())
    # uniform u conducts nothing
    du0, _ = oracle.conduction(X, p.mass, np.full(p.n, 2.5), d["h"], d["rho"], kappa)
    assert np.all(du0 == 0.0)


def test_insulating_neighbours():
    p = W.clustered(3000, 5, seed=83)
    X = oracle.quantize(p.pos)
    d = oracle.density(X, p.mass, None)
    kappa = np.zeros(p.n)
    kappa[7] = 5.0                       # one conductor among insulators
    du, _ = oracle.conduction(X, p.mass, p.u, d["h"], d["rho"], kappa)
    assert np.all(du == 0.0)


def test_linear_and_quadratic_profiles_on_lattice():
    p, X, d, h, inner = _lattice_setup()
    kap = np.full(p.n, 0.7)
    m, rho = p.mass[0], d["rho"][0]
    # linear profile: symmetric shells cancel
    g = np.array([0.3, -1.1, 0.8])
    du_lin, sc = oracle.conduction(X, p.mass, 5.0 + p.pos @ g, d["h"], d["rho"], kap)
    assert np.abs(du_lin[inner]).max() <= 1e-12 * sc[inner].max()
    # quadratic profile: a lattice sum
    u = (p.pos ** 2).sum(1)
    du_q, _ = oracle.conduction(X, p.mass, u, d["h"], d["rho"], kap)
    a = 1.0 / 16
    k = int(math.ceil(h / a)) + 1
    gg = np.arange(-k, k + 1)
    nx, ny, nz = np.meshgrid(gg, gg, gg, indexing="ij")
    r = a * np.sqrt(nx**2 + ny**2 + nz**2).ravel()
    r = r[(r > 0) & (r < h)]
    _, dw = oracle.kernel(r / h)
    dWdr = 8.0 / (math.pi * h**4) * dw
    expect = -(2.0 * 0.7 * m / rho**2) * np.sum(r * dWdr)
    np.testing.assert_allclose(du_q[inner], expect, rtol=1e-11)
    # continuum: (kappa / rho) * Laplacian(|x|^2) = 6 kappa / rho
    assert abs(expect / (6.0 * 0.7 / rho) - 1.0) < 0.05
