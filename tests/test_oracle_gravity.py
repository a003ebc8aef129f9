"""Pins for the oracle's short-range gravity (the Barnes-Hut part of the
paper's TreePM gravity, Sec. 1 and Sec. 3; the split is Gadget's). CPU only.

What pins it, beyond restating its formulas:
* two bodies beyond the softening: the acceleration is minus the derivative
  of the short-range potential -G m erfc(r / 2 r_s) / r, by central finite
  differences;
* two bodies inside the softening, no split: G m M(r) / r^2 with M the mass
  of the (separately pinned) cubic-spline kernel inside r, by quadrature;
* theta = 0 (nothing accepted): the walk is the direct sum over the pairs
  inside the cutoff, summed here by brute force; momentum is conserved;
* a perfect lattice feels no force;
* a compact clump seen from afar acts as its monopole;
* the Barnes-Hut error falls with the opening angle, while the node
  interactions grow and the particle interactions shrink.
"""
import math

import numpy as np
import pytest

import oracle
import workloads as W

SPLIT = dict(r_split=0.04, r_cut=0.18, h_soft=0.002)


def _two(r, axis=(1.0, 0.0, 0.0), m2=0.7):
    e = np.asarray(axis) / np.linalg.norm(axis)
    pos = np.array([[0.4, 0.45, 0.5], [0.4, 0.45, 0.5]]) + np.outer([0.0, 1.0], e) * r
    X = oracle.quantize(pos)
    d = (X[1].astype(np.int64) - X[0].astype(np.int64)) / 2.0**32   # the quantized separation
    rr = np.linalg.norm(d)
    return X, np.array([1.3, m2]), rr, d / rr


def test_two_bodies_follow_the_split_potential():
    rs, G = 0.03, 2.5
    phi = lambda r: -math.erfc(r / (2 * rs)) / r
    for r in (0.01, 0.03, 0.07, 0.12):
        X, m, rr, e = _two(r, axis=(1.0, 2.0, -0.5))
        g = oracle.gravity(X, m, G=G, theta=0.5, r_split=rs, r_cut=0.2, h_soft=0.001)
        step = 1e-6 * rr
        dphi = (phi(rr + step) - phi(rr - step)) / (2 * step)
        expect = G * m[1] * dphi          # a_1 = -grad_1 G m_2 phi(|x_2 - x_1|) = G m_2 phi'(r) e
        a = g["acc"][0]
        np.testing.assert_allclose(a @ e, expect, rtol=1e-7)
        assert np.linalg.norm(a - (a @ e) * e) <= 1e-12 * abs(expect)
        np.testing.assert_allclose(g["acc"][1] * m[1], -a * m[0], rtol=1e-12)
        assert g["n_pairs"][0] == 1 and g["n_nodes"][0] == 0


def test_softened_two_bodies_follow_the_kernel_mass():
    hs = 0.05
    q = np.linspace(0.0, 1.0, 20001)
    w, _ = oracle.kernel(q)
    integrand = 4 * math.pi * 8 / math.pi * w * q**2      # 4 pi W(s, 1) s^2, W = 8/pi w(q)
    cum = np.concatenate([[0.0], np.cumsum(0.5 * (integrand[1:] + integrand[:-1]) * np.diff(q))])
    for r in (0.004, 0.02, 0.025, 0.04, 0.049, 0.06):
        X, m, rr, e = _two(r)
        g = oracle.gravity(X, m, G=1.0, theta=0.0, r_split=0.0, r_cut=0.2, h_soft=hs)
        Mq = np.interp(rr / hs, q, cum) if rr < hs else 1.0
        np.testing.assert_allclose(g["acc"][0] @ e, m[1] * Mq / rr**2, rtol=2e-6)
    assert oracle.soft_mass(1.0) == pytest.approx(1.0, abs=1e-15)
    assert oracle.soft_mass(0.5 - 1e-12) == pytest.approx(oracle.soft_mass(0.5 + 1e-12), abs=1e-10)


def _coarse_d2(X, i):
    d = (X.astype(np.int64) - X[i].astype(np.int64) + 2**31) % 2**32 - 2**31
    return ((np.abs(d) >> 8) ** 2).sum(1), d


def test_theta_zero_is_the_direct_sum():
    p = W.clustered(1500, 4, seed=7)
    X = oracle.quantize(p.pos)
    G, rs, rc, hs = 1.7, SPLIT["r_split"], SPLIT["r_cut"], SPLIT["h_soft"]
    g = oracle.gravity(X, p.mass, G=G, theta=0.0, **SPLIT)
    RC2 = (rc * 2.0**24) ** 2
    u = 2.0**-32
    assert np.all(g["n_nodes"] == 0)
    for i in range(0, p.n, 37):
        D2, d = _coarse_d2(X, i)
        sel = (D2 < RC2) & (np.arange(p.n) != i)
        assert g["n_pairs"][i] == sel.sum()
        rv = d[sel] * u
        r = np.linalg.norm(rv, axis=1)
        nz = r > 0
        rv, r, mj = rv[nz], r[nz], p.mass[sel][nz]
        Mq = np.array([oracle.soft_mass(x / hs) for x in r])
        gf = np.array([math.erfc(x / (2 * rs)) + x / (rs * math.sqrt(math.pi)) * math.exp(-x * x / (4 * rs * rs))
                       for x in r])
        a = (G * mj * Mq / r**3 * gf)[:, None] * rv
        np.testing.assert_allclose(g["acc"][i], a.sum(0), rtol=0, atol=1e-12 * g["scale"][i])
    mom = (p.mass[:, None] * g["acc"]).sum(0)
    assert np.abs(mom).max() <= 1e-13 * (p.mass * g["scale"]).sum()


def test_lattice_feels_no_force():
    p = W.lattice(10, 0.0, seed=0, vel_sigma=0.0)
    X = oracle.quantize(p.pos)
    g = oracle.gravity(X, p.mass, theta=0.0, r_split=0.05, r_cut=0.2345, h_soft=0.01)
    assert g["n_pairs"].min() > 40
    assert np.all(np.linalg.norm(g["acc"], axis=1) <= 1e-7 * g["scale"])


def test_far_clump_acts_as_its_monopole():
    rng = np.random.default_rng(3)
    clump = 0.3 + 2e-4 * rng.standard_normal((64, 3))
    probe = np.array([[0.3, 0.38, 0.33]])
    pos = np.concatenate([clump, probe])
    X = oracle.quantize(pos)
    m = rng.uniform(0.5, 1.5, 65)
    rs = 0.05
    g = oracle.gravity(X, m, G=1.0, theta=0.5, r_split=rs, r_cut=0.2, h_soft=1e-5)
    i = 64
    assert g["n_nodes"][i] >= 1 and g["n_pairs"][i] < 64
    xu = X.astype(np.float64) * 2.0**-32
    com = (m[:64, None] * xu[:64]).sum(0) / m[:64].sum()
    rv = com - xu[i]
    r = np.linalg.norm(rv)
    gf = math.erfc(r / (2 * rs)) + r / (rs * math.sqrt(math.pi)) * math.exp(-r * r / (4 * rs * rs))
    expect = m[:64].sum() * gf / r**3 * rv
    np.testing.assert_allclose(g["acc"][i], expect, rtol=1e-5)


def test_barnes_hut_error_falls_with_theta():
    p = W.clustered(20000, 20, seed=1)
    X = oracle.quantize(p.pos)
    ex = oracle.gravity(X, p.mass, theta=0.0, **SPLIT)
    an = np.linalg.norm(ex["acc"], axis=1)
    q99, nodes, pairs = [], [], []
    for th in (0.3, 0.5, 0.8):
        g = oracle.gravity(X, p.mass, theta=th, **SPLIT)
        err = np.linalg.norm(g["acc"] - ex["acc"], axis=1)
        q99.append(np.percentile(err / ex["scale"], 99))
        nodes.append(g["n_nodes"].mean())
        pairs.append(g["n_pairs"].mean())
        if th == 0.5:
            assert np.median(err / an) < 3e-3
    assert q99[0] < q99[1] < q99[2] and q99[0] < 0.02
    assert nodes[0] < nodes[1] < nodes[2] and pairs[0] > pairs[1] > pairs[2]


def test_relabelling_the_particles_changes_nothing():
    """The tree is built from the positions (ties of equal keys by index), so a
    relabelling of particles with distinct keys gives the same walk for every
    particle: results equal, bit for bit, after undoing the relabelling.
    Catches index mix-ups between sorted and caller order."""
    p = W.clustered(5000, 6, seed=21)
    X = oracle.quantize(p.pos)
    assert len(np.unique(oracle.morton_keys(X))) == p.n
    g = oracle.gravity(X, p.mass, theta=0.6, **SPLIT)
    perm = np.random.default_rng(4).permutation(p.n)
    gp = oracle.gravity(X[perm], p.mass[perm], theta=0.6, **SPLIT)
    inv = np.argsort(perm)
    for k in ("acc", "scale", "n_nodes", "n_pairs"):
        assert np.array_equal(gp[k][inv], g[k])


def _real_criterion_counts(X, theta, r_cut):
    """Per-particle node and particle interaction counts of the Barnes-Hut walk
    with the opening criterion in real-valued form, decided in exact rational
    arithmetic (no 2^16 fixed point, no ceil of the cutoff): in coarse units
    (integer coordinates / 2^8, gaps rounded down, far distances up) a child of
    an opened node is skipped if D^2 >= rc^2, taken as its monopole if
    theta > 0, D > 0, F^2 < rc^2, l <= D and l <= theta D, else opened; a
    particle of an opened leaf interacts if its coarse distance is below rc.
    rc = r_cut 2^24 / L. The tree is the one the definition fixes, built here
    independently: Morton order of the top 21 bits per axis (x most
    significant), ties by index; leaves of 8; nodes of 8 children; boxes the
    min/max integer coordinates."""
    from fractions import Fraction
    n = X.shape[0]
    top = (X >> 11).astype(np.uint64)
    key = np.zeros(n, np.uint64)
    for b in range(21):
        for a in range(3):
            key |= ((top[:, a] >> np.uint64(b)) & np.uint64(1)) << np.uint64(3 * b + 2 - a)
    order = np.lexsort((np.arange(n), key))
    levels = []                                   # per level: list of (lo, hi) integer boxes
    Xs = X[order].astype(np.int64)
    leaves = [(Xs[p:p + 8].min(0), Xs[p:p + 8].max(0)) for p in range(0, n, 8)]
    levels.append(leaves)
    while len(levels[-1]) > 1:
        prev = levels[-1]
        levels.append([(np.min([b[0] for b in prev[c:c + 8]], 0), np.max([b[1] for b in prev[c:c + 8]], 0))
                       for c in range(0, len(prev), 8)])
    th2 = Fraction(theta) ** 2
    rc2 = (Fraction(r_cut) * 2**24) ** 2
    two32 = 1 << 32
    nodes = np.zeros(n, np.int64)
    pairs = np.zeros(n, np.int64)
    for i in range(n):
        xi = X[i].astype(np.int64)
        stack = [(len(levels) - 1, 0)]
        while stack:
            k, t = stack.pop()
            if k == 0:
                for p in range(8 * t, min(8 * t + 8, n)):
                    j = order[p]
                    if j == i:
                        continue
                    d = (X[j].astype(np.int64) - xi + two32 // 2) % two32 - two32 // 2
                    if sum((abs(int(c)) >> 8) ** 2 for c in d) < rc2:
                        pairs[i] += 1
                continue
            for c in range(8 * t, min(8 * t + 8, len(levels[k - 1]))):
                lo, hi = levels[k - 1][c]
                D2 = F2 = 0
                l = 0
                for a in range(3):
                    x, lo_a, hi_a = int(xi[a]), int(lo[a]), int(hi[a])
                    if x < lo_a or x > hi_a:
                        gap = min((lo_a - x) % two32, (x - hi_a) % two32)
                        far = gap + (hi_a - lo_a)
                    else:
                        gap, far = 0, max(x - lo_a, hi_a - x)
                    D2 += (gap >> 8) ** 2
                    F2 += (-(-far // 256)) ** 2
                    l = max(l, (hi_a - lo_a) >> 8)
                if D2 >= rc2:
                    continue
                if theta > 0 and D2 > 0 and F2 < rc2 and l * l <= D2 and l * l <= th2 * D2:
                    nodes[i] += 1
                    continue
                stack.append((k - 1, c))
    return nodes, pairs


@pytest.mark.parametrize("theta", [0.25, 0.5, 0.75, 1.0])
def test_integer_criterion_is_the_real_one(theta):
    """Whenever theta^2 2^16 is an integer (theta = 1/4, 1/2, 3/4, 1) the
    oracle's fixed-point decisions (2^16 l^2 <= rint(theta^2 2^16) D^2 and
    D^2 < ceil(rc^2)) are the real-valued Barnes-Hut criterion l <= theta D and
    the cutoff D < rc: node and particle interaction counts of every particle
    match a walk that decides in exact rational arithmetic."""
    p = W.clustered(700, 4, seed=77)
    X = oracle.quantize(np.asarray(p.pos, np.float32).astype(np.float64))
    r_cut = 0.23
    g = oracle.gravity(X, p.mass, theta=theta, r_cut=r_cut)
    nodes, pairs = _real_criterion_counts(X, theta, r_cut)
    assert nodes.sum() > 0 and pairs.sum() > 0
    np.testing.assert_array_equal(g["n_nodes"], nodes)
    np.testing.assert_array_equal(g["n_pairs"], pairs)
