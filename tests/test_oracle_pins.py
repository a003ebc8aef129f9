"""Pins for the FP64 oracle: facts fixed by mathematics, by textbook forms of
the kernel, or by brute force -- none of them re-derives the oracle's own
formulas. Every mistake class that matters (a dropped term, a wrong sign, a
transposed index, a wrong normalisation) breaks at least one of these.

CPU only (no GPU marker).
"""
import math
import os

import numpy as np
import pytest

import oracle
import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden")
GAMMA = 5.0 / 3.0


# --------------------------------------------------------------------------
# Kernel (cubic spline, support h)
# --------------------------------------------------------------------------

def test_kernel_golden_values():
    """Textbook values of the M4 spline (tests/golden/kernel_m4.txt)."""
    tab = np.loadtxt(os.path.join(GOLD, "kernel_m4.txt"))
    w, dw = oracle.kernel(tab[:, 0])
    np.testing.assert_allclose(w, tab[:, 1], rtol=0, atol=1e-15)
    np.testing.assert_allclose(dw, tab[:, 2], rtol=0, atol=1e-15)


def test_kernel_normalisation_quadrature():
    """int W dV = 1:  (8/pi) * 4 pi * int_0^1 w(q) q^2 dq = 1 (Gauss-Legendre)."""
    xg, wg = np.polynomial.legendre.leggauss(40)
    total = 0.0
    for a, b in ((0.0, 0.5), (0.5, 1.0)):   # split at the kink so quadrature is exact
        q = 0.5 * (b - a) * xg + 0.5 * (a + b)
        w, _ = oracle.kernel(q)
        total += 0.5 * (b - a) * np.sum(wg * w * q * q)
    assert abs(8.0 / math.pi * 4.0 * math.pi * total - 1.0) < 1e-14


def test_kernel_matches_monaghan_form():
    """Same kernel as Monaghan's form in the half-support convention h_M = h/2:
    W = 1/(pi h_M^3) {1 - 3/2 s^2 + 3/4 s^3 (s<1); (2-s)^3/4 (1<=s<2)}, s = r/h_M."""
    q = np.linspace(0.0, 1.2, 1201)
    s = 2.0 * q
    ref = np.where(s < 1, 1 - 1.5 * s**2 + 0.75 * s**3, np.where(s < 2, 0.25 * (2 - s) ** 3, 0.0))
    # W(r,h) = 8/(pi h^3) w(q) must equal 1/(pi (h/2)^3) ref(s): so w == ref.
    w, _ = oracle.kernel(q)
    np.testing.assert_allclose(w, ref, rtol=0, atol=1e-15)


def test_kernel_derivative_and_continuity():
    q = np.linspace(1e-3, 0.999, 997)
    e = 1e-6
    wp, _ = oracle.kernel(q + e)
    wm, _ = oracle.kernel(q - e)
    _, dw = oracle.kernel(q)
    np.testing.assert_allclose(dw, (wp - wm) / (2 * e), rtol=0, atol=1e-8)
    for q0 in (0.5, 1.0):
        a, da = oracle.kernel(np.array([q0 - 1e-12, q0 + 1e-12]))
        assert abs(a[0] - a[1]) < 1e-10 and abs(da[0] - da[1]) < 1e-10
    w0, dw0 = oracle.kernel(np.array([0.0]))
    assert w0[0] == 1.0 and dw0[0] == 0.0


# --------------------------------------------------------------------------
# Quantisation, Morton keys, sort
# --------------------------------------------------------------------------

def test_quantize_known_values():
    pos = np.array([[0.0, 0.5, 0.25], [-0.25, 1.0, 1.25], [2.0**-33, 1.0 - 2.0**-34, 3 * 2.0**-33]])
    X = oracle.quantize(pos, 1.0)
    # 2^-33 * 2^32 = 0.5 ties to even (0); 1 - 2^-34 rounds to 2^32 and wraps to 0;
    # 3*2^-33 -> 1.5 ties to even (2)
    assert X.tolist() == [[0, 2**31, 2**30], [3 * 2**30, 0, 2**30], [0, 0, 2]]
    X2 = oracle.quantize(pos * 3.0, 3.0)
    assert np.array_equal(X, X2) or np.abs(X.astype(np.int64) - X2.astype(np.int64)).max() <= 1


def _morton_brute(x, y, z):
    k = 0
    for b in range(21):
        k |= ((x >> (11 + b)) & 1) << (3 * b + 2)
        k |= ((y >> (11 + b)) & 1) << (3 * b + 1)
        k |= ((z >> (11 + b)) & 1) << (3 * b)
    return k


def test_morton_keys_brute():
    rng = np.random.default_rng(7)
    X = rng.integers(0, 2**32, size=(500, 3), dtype=np.uint64).astype(np.uint32)
    k = oracle.morton_keys(X)
    ref = [_morton_brute(int(a), int(b), int(c)) for a, b, c in X]
    assert [int(v) for v in k] == ref
    assert int(oracle.morton_keys(np.array([[2**11, 0, 0]], np.uint32))[0]) == 4
    assert int(oracle.morton_keys(np.array([[0, 0, 2**31]], np.uint32))[0]) == 1 << 60
    kb = oracle.morton_keys(X, box_index=5, box_bits=3)
    assert all(int(a) == (5 << 60) | (int(b) >> 3) for a, b in zip(kb, k))


def test_sort_perm_matches_lexsort():
    rng = np.random.default_rng(3)
    keys = rng.integers(0, 50, size=2000).astype(np.uint64)  # many ties
    perm = oracle.sort_perm(keys)
    assert np.array_equal(perm, np.lexsort((np.arange(2000), keys)))


# --------------------------------------------------------------------------
# Neighbour predicate and search
# --------------------------------------------------------------------------

def _brute_set(X, i, h, box=1.0):
    d = (X.astype(np.int64) - X[i].astype(np.int64))
    d = (d + 2**31) % 2**32 - 2**31                # two's-complement minimum image
    D2 = [int(a) * int(a) + int(b) * int(b) + int(c) * int(c) for a, b, c in d]
    H = h * 2.0**32 / box
    return sorted(j for j in range(len(X)) if j != i and float(D2[j]) < H * H)


@pytest.mark.parametrize("kind", ["lattice", "clustered"])
def test_neighbour_sets_cell_list_vs_brute(kind):
    p = W.lattice(10, 0.3, seed=11) if kind == "lattice" else W.clustered(3000, 5, seed=12)
    X = oracle.quantize(p.pos)
    rng = np.random.default_rng(1)
    for i in rng.choice(p.n, 25, replace=False):
        for h in (0.01, 0.07, 0.2, 0.49):
            a = oracle.neighbours(X, i, h, brute=False)
            b = oracle.neighbours(X, i, h, brute=True)
            assert np.array_equal(a, b)
    for i in rng.choice(p.n, 5, replace=False):
        assert oracle.neighbours(X, i, 0.13, brute=True).tolist() == _brute_set(X, i, 0.13)


def test_predicate_boundary_is_strict():
    # j exactly at distance h (integer units) is not a neighbour; one unit closer is.
    X = np.array([[0, 0, 0], [2**28, 0, 0], [2**28 - 1, 0, 0]], dtype=np.uint32)
    h = 2.0**28 / 2.0**32
    assert oracle.neighbours(X, 0, h).tolist() == [2]
    X[1, 0] = (2**32 - 2**28) & 0xFFFFFFFF     # across the periodic boundary
    assert oracle.neighbours(X, 0, h).tolist() == [2]


# --------------------------------------------------------------------------
# Density and the smoothing-length solve
# --------------------------------------------------------------------------

def _lattice_sum(a, h, fn):
    """sum over lattice vectors n with |n| a < h of fn(|n| a / h)."""
    k = int(math.ceil(h / a)) + 1
    g = np.arange(-k, k + 1)
    nx, ny, nz = np.meshgrid(g, g, g, indexing="ij")
    r = a * np.sqrt(nx**2 + ny**2 + nz**2).ravel()
    q = r[r < h] / h
    return fn(q)


def test_perfect_lattice_density_closed_form():
    n_side = 16   # (i + 1/2)/16 * 2^32 is an integer: the quantised lattice is exact
    p = W.lattice(n_side, 0.0, seed=0, vel_sigma=0.0, u_range=(1.0, 1.0))
    X = oracle.quantize(p.pos)
    d = oracle.density(X, p.mass, None, n_target=64.0)
    a = 1.0 / n_side
    h = d["h"]
    assert np.ptp(h) <= 1e-12 * h[0]
    h0 = h[0]
    w_sum = _lattice_sum(a, h0, lambda q: oracle.kernel(q)[0].sum())
    # N_eff(h) = (32/3) sum w  must hit the target
    assert abs(32.0 / 3.0 * w_sum - 64.0) < 1e-9
    rho_ref = p.mass[0] * 8.0 / (math.pi * h0**3) * w_sum
    np.testing.assert_allclose(d["rho"], rho_ref, rtol=1e-12)
    # neighbour count: lattice points strictly inside the sphere, minus self
    n_in = _lattice_sum(a, h0, lambda q: q.size) - 1
    assert np.all(d["n_ngb"] == n_in)
    # continuum limit: rho ~ mass * number density within a few per cent
    assert abs(rho_ref / 1.0 - 1.0) < 0.05


def test_h_root_hits_target_and_is_unique():
    p = W.clustered(4000, 6, seed=21)
    X = oracle.quantize(p.pos)
    d = oracle.density(X, p.mass, None, n_target=64.0, tol=1e-10)
    assert d["any_status"] == 0
    assert np.abs(d["neff"] - 64.0).max() <= 1e-10
    # a different starting guess converges to the same root
    d2 = oracle.density(X, p.mass, d["h"] * 3.0, n_target=64.0, tol=1e-10)
    np.testing.assert_allclose(d2["h"], d["h"], rtol=1e-9)
    # N_eff is the number-weighted sum: independent of the masses
    d3 = oracle.density(X, p.mass * np.random.default_rng(0).uniform(0.5, 2, p.n), None,
                        n_target=64.0, tol=1e-10)
    np.testing.assert_allclose(d3["h"], d["h"], rtol=1e-12)


def test_drho_dh_matches_finite_difference():
    p = W.clustered(3000, 4, seed=31)
    X = oracle.quantize(p.pos)
    d = oracle.density(X, p.mass, None, n_target=64.0)
    eps = 1e-7
    dp = oracle.density(X, p.mass, d["h"] * (1 + eps), fixed_h=True)
    dm = oracle.density(X, p.mass, d["h"] * (1 - eps), fixed_h=True)
    fd = (dp["rho"] - dm["rho"]) / (2 * eps * d["h"])
    np.testing.assert_allclose(d["drho_dh"], fd, rtol=1e-5, atol=1e-6 * np.abs(fd).max())
    fdn = (dp["neff"] - dm["neff"]) / (2 * eps * d["h"])
    # dN/dh > 0 at the root; Omega is finite and positive
    assert np.all(fdn > 0) and np.all(d["omega"] > 0)


def test_density_brute_equals_cell_list():
    p = W.clustered(2500, 5, seed=41)
    X = oracle.quantize(p.pos)
    a = oracle.density(X, p.mass, None)
    b = oracle.density(X, p.mass, None, brute=True)
    assert np.array_equal(a["n_ngb"], b["n_ngb"]) and np.array_equal(a["hash"], b["hash"])
    np.testing.assert_allclose(a["rho"], b["rho"], rtol=1e-13)
    np.testing.assert_allclose(a["h"], b["h"], rtol=1e-13)


def test_h_too_large_is_reported():
    p = W.lattice(3, 0.2, seed=5)          # 27 particles cannot reach 64 neighbours
    X = oracle.quantize(p.pos)
    d = oracle.density(X, p.mass, None, n_target=64.0)
    assert np.all(d["status"] & oracle.H_TOO_LARGE)


# --------------------------------------------------------------------------
# Force
# --------------------------------------------------------------------------

def _dens_force(p, alpha=1.0, brute=False, **kw):
    X = oracle.quantize(p.pos, p.box)
    d = oracle.density(X, p.mass, None, box=p.box, brute=brute)
    f = oracle.force(X, p.vel, p.mass, p.u, d["h"], d["rho"], d["omega"], box=p.box,
                     alpha=alpha, brute=brute, **kw)
    return X, d, f


def test_perfect_lattice_force_vanishes():
    p = W.lattice(16, 0.0, seed=0, vel_sigma=0.0, u_range=(1.0, 1.0))
    _, d, f = _dens_force(p)
    scale = f["scale_a"].max()
    assert np.abs(f["acc"]).max() <= 1e-12 * scale
    assert np.abs(f["dudt"]).max() <= 1e-12 * max(f["scale_u"].max(), 1e-300) + 1e-300
    c = math.sqrt(GAMMA * (GAMMA - 1.0) * 1.0)
    np.testing.assert_allclose(f["vsig"], 2 * c, rtol=1e-14)     # static: v_sig = c_i + c_j


@pytest.mark.parametrize("kind", ["lattice", "clustered"])
def test_conservation(kind):
    p = W.config1(12) if kind == "lattice" else W.clustered(5000, 8, seed=51)
    _, d, f = _dens_force(p)
    m = p.mass
    mom = (m[:, None] * f["acc"]).sum(0)
    assert np.linalg.norm(mom) <= 1e-12 * (m * np.linalg.norm(f["acc"], axis=1)).sum()
    e_terms = m * ((p.vel * f["acc"]).sum(1) + f["dudt"])
    scale = (m * (np.abs((p.vel * f["acc"]).sum(1)) + np.abs(f["dudt"]))).sum()
    assert abs(e_terms.sum()) <= 1e-12 * scale


def test_symmetric_pair_set_brute_vs_cell_list():
    p = W.clustered(3000, 5, seed=61)
    _, d, fa = _dens_force(p)
    X = oracle.quantize(p.pos)
    fb = oracle.force(X, p.vel, p.mass, p.u, d["h"], d["rho"], d["omega"], brute=True)
    assert np.array_equal(fa["n_pairs"], fb["n_pairs"]) and np.array_equal(fa["hash"], fb["hash"])
    np.testing.assert_allclose(fa["acc"], fb["acc"], rtol=0, atol=1e-12 * fb["scale_a"].max())
    # pair set is symmetric: total count is even, and each density neighbour is a force pair
    assert fa["n_pairs"].sum() % 2 == 0
    assert np.all(fa["n_pairs"] >= d["n_ngb"])


def test_galilean_invariance():
    p = W.clustered(3000, 5, seed=71)
    _, d, f = _dens_force(p)
    q = W.Particles(p.pos, p.vel + np.array([0.7, -0.3, 1.1]), p.mass, p.u, p.box)
    X = oracle.quantize(q.pos)
    g = oracle.force(X, q.vel, q.mass, q.u, d["h"], d["rho"], d["omega"])
    np.testing.assert_allclose(g["acc"], f["acc"], rtol=0, atol=1e-12 * f["scale_a"].max())
    np.testing.assert_allclose(g["dudt"], f["dudt"], rtol=0, atol=1e-12 * f["scale_u"].max())


def test_shift_and_permutation():
    p = W.clustered(2000, 4, seed=81)
    X = oracle.quantize(p.pos)
    d = oracle.density(X, p.mass, None, brute=True)
    f = oracle.force(X, p.vel, p.mass, p.u, d["h"], d["rho"], d["omega"], brute=True)
    Xs = (X.astype(np.uint64) + np.array([12345, 2**31 + 7, 2**32 - 99], np.uint64)) % 2**32
    Xs = Xs.astype(np.uint32)
    ds = oracle.density(Xs, p.mass, None, brute=True)
    fs = oracle.force(Xs, p.vel, p.mass, p.u, ds["h"], ds["rho"], ds["omega"], brute=True)
    for k in ("h", "rho", "omega", "n_ngb", "hash"):
        assert np.array_equal(d[k], ds[k]), k
    for k in ("acc", "dudt", "vsig", "n_pairs"):
        assert np.array_equal(f[k], fs[k]), k
    perm = np.random.default_rng(0).permutation(p.n)
    dp = oracle.density(X[perm], p.mass[perm], None, brute=True)
    np.testing.assert_allclose(dp["h"], d["h"][perm], rtol=1e-13)
    np.testing.assert_allclose(dp["rho"], d["rho"][perm], rtol=1e-13)
    assert np.array_equal(dp["n_ngb"], d["n_ngb"][perm])


def test_mass_scaling():
    p = W.clustered(2000, 4, seed=91)
    _, d, f = _dens_force(p)
    q = W.Particles(p.pos, p.vel, p.mass * 7.0, p.u, p.box)
    _, d2, f2 = _dens_force(q)
    np.testing.assert_allclose(d2["h"], d["h"], rtol=1e-14)
    np.testing.assert_allclose(d2["rho"], 7.0 * d["rho"], rtol=1e-13)
    np.testing.assert_allclose(f2["acc"], f["acc"], rtol=0, atol=1e-12 * f["scale_a"].max())
    np.testing.assert_allclose(f2["dudt"], f["dudt"], rtol=0, atol=1e-12 * f["scale_u"].max())


def _adiabatic_energy(xc, p, K, n_target=64.0):
    d = oracle.density(None, p.mass, None, n_target=n_target, tol=1e-12, xc=xc)
    u = K * d["rho"] ** (GAMMA - 1.0) / (GAMMA - 1.0)
    return (p.mass * u).sum(), d, u


def test_pressure_force_is_energy_gradient():
    """Equal masses, alpha = 0: the grad-h force is exactly -grad E / m_i with
    E = sum_j m_j u_j(rho_j) at fixed entropy (Springel & Hernquist 2002), with
    every h_j re-solved as x moves. Central differences on continuous positions."""
    p = W.lattice(10, 0.3, seed=3, vel_sigma=0.0)
    E0, d0, _ = _adiabatic_energy(p.pos, p, 1.0)
    K = p.u / d0["rho"] ** (GAMMA - 1.0)         # entropy fixed from u at the start
    u0 = K * d0["rho"] ** (GAMMA - 1.0) / (GAMMA - 1.0)
    f = oracle.force(None, p.vel, p.mass, u0, d0["h"], d0["rho"], d0["omega"], alpha=0.0, xc=p.pos)
    eps = 1e-6
    for i in (0, 137, 555):
        for ax in range(3):
            xp = p.pos.copy(); xp[i, ax] += eps
            xm = p.pos.copy(); xm[i, ax] -= eps
            g = (_adiabatic_energy(xp, p, K)[0] - _adiabatic_energy(xm, p, K)[0]) / (2 * eps)
            assert abs(-g / p.mass[i] - f["acc"][i, ax]) <= 2e-6 * f["scale_a"][i], (i, ax)


def test_dudt_is_adiabatic_rate():
    """alpha = 0: du_i/dt equals d/dt u_i(rho_i(x + v t)) at fixed entropy."""
    p = W.lattice(10, 0.3, seed=4, vel_sigma=0.1)
    _, d0, _ = _adiabatic_energy(p.pos, p, 1.0)
    K = p.u / d0["rho"] ** (GAMMA - 1.0)
    u0 = K * d0["rho"] ** (GAMMA - 1.0) / (GAMMA - 1.0)
    f = oracle.force(None, p.vel, p.mass, u0, d0["h"], d0["rho"], d0["omega"], alpha=0.0, xc=p.pos)
    dt = 1e-6
    up = _adiabatic_energy(np.mod(p.pos + dt * p.vel, 1.0), p, K)[2]
    um = _adiabatic_energy(np.mod(p.pos - dt * p.vel, 1.0), p, K)[2]
    fd = (up - um) / (2 * dt)
    np.testing.assert_allclose(f["dudt"], fd, rtol=0, atol=2e-6 * f["scale_u"].max())


def test_viscosity_dissipates_linearly():
    """The viscous part conserves energy by itself, heats every particle
    (du_AV >= 0 when signal velocities are positive) and is linear in alpha."""
    p = W.config1(10)
    X, d, f0 = _dens_force(p, alpha=0.0)
    f1 = oracle.force(X, p.vel, p.mass, p.u, d["h"], d["rho"], d["omega"], alpha=1.0)
    f2 = oracle.force(X, p.vel, p.mass, p.u, d["h"], d["rho"], d["omega"], alpha=2.0)
    du_av = f1["dudt"] - f0["dudt"]
    da_av = f1["acc"] - f0["acc"]
    assert np.all(du_av >= -1e-12 * f1["scale_u"])
    assert du_av.sum() > 0
    e = (p.mass * ((p.vel * da_av).sum(1) + du_av)).sum()
    assert abs(e) <= 1e-11 * (p.mass * np.abs(du_av)).sum()
    np.testing.assert_allclose(f2["dudt"] - f0["dudt"], 2 * du_av, rtol=0, atol=1e-12 * f1["scale_u"].max())
    np.testing.assert_allclose(f2["acc"] - f0["acc"], 2 * da_av, rtol=0, atol=1e-12 * f1["scale_a"].max())


def test_active_subset_matches_full():
    p = W.clustered(3000, 5, seed=101)
    X, d, f = _dens_force(p)
    act = np.sort(np.random.default_rng(2).choice(p.n, 300, replace=False))
    da = oracle.density(X, p.mass, None, active=act)
    np.testing.assert_allclose(da["h"][act], d["h"][act], rtol=1e-13)
    assert np.all(np.isnan(np.delete(da["h"], act)))
    fa = oracle.force(X, p.vel, p.mass, p.u, d["h"], d["rho"], d["omega"], active=act)
    np.testing.assert_array_equal(fa["acc"][act], f["acc"][act])


def _golden_visc():
    rows = {}
    path = os.path.join(os.path.dirname(__file__), "golden", "viscosity_pair.txt")
    with open(path) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                c, *v = line.split()
                rows[c] = [float(x) for x in v]
    return rows


@pytest.mark.parametrize("case", ["A", "B", "C"])
def test_viscosity_pair_hand_values(case):
    """Magnitude of the artificial viscosity: two isolated particles whose a,
    du/dt and v_sig are worked by hand from the published Gadget-2 / Monaghan
    (1997) forms (tests/golden/viscosity_pair.txt). A wrong factor (alpha in
    place of alpha/2, a 2 in place of the 3 in v_sig, the mean density in the
    wrong place) changes these values."""
    want = _golden_visc()[case]
    pos = np.array([[7 / 16, 0.5, 0.5], [9 / 16, 0.5, 0.5]])
    if case == "A":
        m, h, rho, om, u, al = [1, 1], [0.25, 0.25], [1, 1], [1, 1], [0.6, 0.6], 1.0
        v = [[1, 0, 0], [-1, 0, 0]]
    else:
        m, h, rho, om, u, al = [1, 2], [0.25, 0.2], [1, 3], [0.9, 1.1], [0.6, 0.2], 0.8
        v = [[0.5, 0.3, 0], [-1, 0.3, 0.2]] if case == "B" else [[-0.5, 0.3, 0], [1, 0.3, 0.2]]
    X = oracle.quantize(pos)
    arr = lambda a: np.asarray(a, np.float64)
    for brute in (True, False):
        f = oracle.force(X, arr(v), arr(m), arr(u), arr(h), arr(rho), arr(om), alpha=al, brute=brute)
        got = [f["acc"][0, 0], f["acc"][1, 0], f["dudt"][0], f["dudt"][1], f["vsig"][0], f["vsig"][1]]
        np.testing.assert_allclose(got, want, rtol=1e-13, atol=1e-12)
        np.testing.assert_array_equal(f["acc"][:, 1:], 0.0)
        np.testing.assert_array_equal(f["n_pairs"], [1, 1])
