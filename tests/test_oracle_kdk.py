"""Pins for the oracle's kick-drift-kick integrator on power-of-two time bins
(NEXT-3; the paper's adaptive time steps, Sec. 2.2). CPU only.

* conservation: total energy (kinetic + thermal) to second order in dt,
  total momentum exactly when all particles share one step;
* second order: halving dt cuts the error of the final state by ~4;
* bookkeeping: every particle in the finest bin of a 3-bin hierarchy is the
  single-bin integration with that step, bit for bit; particles in a coarser
  bin are active every 2^k ticks;
* the Courant bin rule on hand-made steps, including exact powers of two.
"""
import numpy as np

import workloads as W
from oracle import kdk as K


def _gas(n_side=11, seed=1):
    p = W.lattice(n_side, 0.3, seed=seed, vel_sigma=0.1, u_range=(0.9, 1.1))
    return p


def _min_image(d, L=1.0):
    return d - L * np.round(d / L)


def _energy(r):
    v, u = r.synchronized_velocity()
    return (r.mass * (0.5 * (v * v).sum(1) + u)).sum(), (r.mass[:, None] * v).sum(0)


def test_energy_second_order_and_momentum():
    """Total energy (kinetic + thermal; the viscosity only converts one into
    the other) is conserved to second order in dt, and total momentum exactly
    when every particle kicks with the same step (sum_i m_i a_i = 0)."""
    p = _gas()
    n = p.n
    bins = np.zeros(n, np.uint8)
    T = 0.04
    e0 = (p.mass * (0.5 * (p.vel * p.vel).sum(1) + p.u)).sum()
    mom0 = (p.mass[:, None] * p.vel).sum(0)
    errs = []
    for k in (4, 8):
        r = K.KDK(p.pos, p.vel, p.mass, p.u, bins, T / k, 0)
        for _ in range(k):
            r.step()
        e, mom = _energy(r)
        errs.append(abs(e - e0))
        assert np.abs(mom - mom0).max() <= 1e-14 * np.abs(p.mass[:, None] * p.vel).sum()
    assert errs[1] < errs[0] and 2.5 < errs[0] / errs[1] < 6.0
    assert errs[0] < 1e-3 * e0


def test_second_order_in_dt():
    p = _gas(seed=2)
    n = p.n
    bins = np.zeros(n, np.uint8)
    T = 0.04
    finals = []
    for k in (4, 8, 16):
        r = K.KDK(p.pos, p.vel, p.mass, p.u, bins, T / k, 0)
        for _ in range(k):
            r.step()
        finals.append(r.pos.copy())
    e1 = np.abs(_min_image(finals[0] - finals[1])).max()
    e2 = np.abs(_min_image(finals[1] - finals[2])).max()
    assert 3.0 < e1 / e2 < 5.0


def test_bins_bookkeeping():
    p = _gas(n_side=8, seed=3)
    n = p.n
    fine = K.KDK(p.pos, p.vel, p.mass, p.u, np.full(n, 2, np.uint8), 0.02, 2)
    single = K.KDK(p.pos, p.vel, p.mass, p.u, np.zeros(n, np.uint8), 0.005, 0)
    for _ in range(4):
        assert fine.step() == n
        single.step()
    assert np.array_equal(fine.pos, single.pos) and np.array_equal(fine.vel, single.vel)
    # coarse particles are active at ticks 2 and 4 (bin 1) or 4 (bin 0)
    bins = np.repeat(np.arange(3, dtype=np.uint8), n // 3 + 1)[:n]
    mixed = K.KDK(p.pos, p.vel, p.mass, p.u, bins, 0.02, 2)
    counts = [mixed.step() for _ in range(4)]
    nb = np.bincount(bins, minlength=3)
    assert counts == [nb[2], nb[2] + nb[1], nb[2], n]


def test_courant_bin_rule():
    h = np.array([0.1, 0.1, 0.1, 0.1, 0.2, 0.05], np.float32)
    vs = np.array([3.0, 0.0, 1.5, 0.375, 1.0, 1.0], np.float32)
    # dt = 0.3 h / vs (FP32); dt_max = 0.08: bins so that dt_max / 2^b <= dt
    b = K.timebins(h, vs, 0.3, 0.08, 4)
    with np.errstate(divide="ignore"):
        dt = np.float32(0.3) * h / vs
    for i in range(h.size):
        if vs[i] <= 0:
            assert b[i] == 0
        elif b[i] < 4:
            assert np.float32(0.08) <= np.ldexp(dt[i], int(b[i]))
            assert b[i] == 0 or not (np.float32(0.08) <= np.ldexp(dt[i], int(b[i]) - 1))
    # a tick off a bin's boundary raises the bin
    b5 = K.timebins(h, vs, 0.3, 0.08, 4, tick=2)
    assert np.all(b5 >= 3) and np.all((2 % (1 << (4 - b5.astype(int)))) == 0)


def test_energy_second_order_with_time_dependent_viscosity_and_switch():
    """With per-particle alpha (integrated like u) and Balsara's switch the pair
    terms stay symmetric, so total energy is still conserved to second order in
    dt and momentum exactly on one shared step."""
    p = _gas(seed=5)
    n = p.n
    bins = np.zeros(n, np.uint8)
    visc = {"alpha0": 0.6, "alpha_min": 0.1, "alpha_max": 1.0, "ell": 0.2}
    T = 0.04
    e0 = (p.mass * (0.5 * (p.vel * p.vel).sum(1) + p.u)).sum()
    mom0 = (p.mass[:, None] * p.vel).sum(0)
    errs = []
    for k in (4, 8):
        r = K.KDK(p.pos, p.vel, p.mass, p.u, bins, T / k, 0, balsara=True, visc=visc)
        for _ in range(k):
            r.step()
        e, mom = _energy(r)
        errs.append(abs(e - e0))
        assert np.abs(mom - mom0).max() <= 1e-14 * np.abs(p.mass[:, None] * p.vel).sum()
        assert np.ptp(r.synchronized_alpha()) > 1e-3          # the alphas evolved apart
    assert errs[1] < errs[0] and 2.5 < errs[0] / errs[1] < 6.0
