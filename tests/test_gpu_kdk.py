"""GPU kick-drift-kick integration on power-of-two time bins (NEXT-3): the
device bookkeeping bit for bit against the oracle's rules, and a dt_max cycle
of the integrator against the FP64 oracle integrator on the same bins.

Tolerances: bins and active sets exact (integer decisions, both sides in
FP32 from the same inputs). Velocities within 1e-4 of the accumulated scale
sum_steps scale * |dt| of their kicks (the force tolerance of 1e-4 of the
pair-term scale; measured up to 4e-6 over three seeds), positions within
dt_max times that. Energies within 5e-4 of their accumulated scale (measured
up to 2e-4): du/dt sums v_ij . grad W with v_ij = v_i - v_j formed in FP32 from
velocities that carry the blobs' bulk flow, so each difference keeps the
rounding of |v_i| (6e-8 of it), which is up to 1e-4 of a small |v_ij|; the
accelerations are dominated by the pressure terms, which take no velocity.
"""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import kdk as OK
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


def _dt_max(h, vsig, max_bin, courant=0.3):
    """dt_max a little below 2^max_bin times the smallest FP32 Courant step."""
    dt = np.float32(courant) * np.asarray(h, np.float32) / np.asarray(vsig, np.float32)
    return float(2 ** max_bin * dt.min()) * 0.999


def test_timebins_and_active_sets_exact(S, ctx):
    rng = np.random.default_rng(5)
    n = 20_000
    h = (10.0 ** rng.uniform(-3, -1, n)).astype(np.float32)
    vs = (10.0 ** rng.uniform(-1, 1, n)).astype(np.float32)
    vs[:50] = 0.0
    h[50:60] = (0.08 / 0.3 * vs[50:60] / 2.0 ** np.arange(10)).astype(np.float32)   # near exact boundaries
    bins = torch.zeros(n, dtype=torch.uint8, device="cuda")
    S.sph_timebins(ctx, dev(h), dev(vs), None, 0, 0.3, 0.08, 6, bins)
    assert np.array_equal(host(bins), OK.timebins(h, vs, 0.3, 0.08, 6))
    act = np.sort(rng.choice(n, 3000, replace=False)).astype(np.int32)
    S.sph_timebins(ctx, dev(h), dev(vs), dev(act, torch.int32), 12, 0.3, 0.08, 6, bins)
    ref = OK.timebins(h, vs, 0.3, 0.08, 6)
    ref[act] = OK.timebins(h[act], vs[act], 0.3, 0.08, 6, tick=12)
    assert np.array_equal(host(bins), ref)
    # active sets of ticks 0..16 for the bins above
    p = as_f32(W.clustered(n, 10, seed=9))
    grid = S.sph_build_grid(ctx, dev(p.pos), dev(p.mass), S.default_params())
    b = host(bins).astype(np.int64)
    out = torch.zeros(n, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    for tick in range(17):
        S.sph_active_from_bins(ctx, grid, bins, tick, 6, out, cnt)
        k = int(cnt.item())
        expect = np.nonzero(tick % (1 << (6 - b)) == 0)[0]
        assert k == expect.size and np.array_equal(host(out)[:k], expect)


def test_kdk_cycle_against_oracle(S, ctx):
    from paper_2003_10850_gb300.kdk import KDK
    p = as_f32(W.clustered(4096, 6, seed=17))
    max_bin = 2
    # the bins: the oracle's Courant rule on the oracle's first force pass, with
    # dt_max such that the finest bin holds the smallest Courant step (a coarser
    # dt_max clamps particles at max_bin with steps above their Courant limit,
    # and the cold, strongly compressed gas of the clumps then reaches u < 0)
    probe = OK.KDK(p.pos, p.vel, p.mass, p.u, np.zeros(p.n, np.uint8), 1e-3, max_bin)
    dt_max = _dt_max(probe.h, probe.vsig, max_bin)
    bins = OK.timebins(probe.h, probe.vsig, 0.3, dt_max, max_bin)
    assert np.all(np.bincount(bins, minlength=max_bin + 1) > 0)
    ref = OK.KDK(p.pos, p.vel, p.mass, p.u, bins, dt_max, max_bin)
    g = KDK(ctx, dev(p.pos, torch.float64), dev(p.mass), dev(p.vel), dev(p.u), dt_max, max_bin,
            bins=dev(bins, torch.uint8))
    for _ in range(1 << max_bin):
        assert g.step() == ref.step()
    v_g, u_g = (host(t).astype(np.float64) for t in g.synchronized_velocity())
    v_o, u_o = ref.synchronized_velocity()
    dv = np.linalg.norm(v_g - v_o, axis=1)
    assert np.all(dv <= 1e-4 * ref.scale_a + 1e-6 * (np.linalg.norm(v_o, axis=1) + 0.1)), \
        (dv / (ref.scale_a + 1e-30)).max()
    du = np.abs(u_g - u_o)
    assert np.all(du <= 5e-4 * ref.scale_u + 1e-6 * np.abs(u_o)), (du / (ref.scale_u + 1e-30)).max()
    dx = host(g.pos) - ref.pos
    dx -= np.round(dx)
    assert np.all(np.linalg.norm(dx, axis=1) <= dt_max * (1e-4 * ref.scale_a + 1e-6) + 1e-9)
    # the cycle moved the gas and changed its energy
    assert np.abs(v_o - p.vel).max() > 100 * dv.max()
    assert np.all(u_o > 0)


def test_kdk_rebinning_follows_the_rule(S, ctx):
    """With re-binning, the bins the device assigns to the particles of a
    tick are the Courant rule (with the boundary condition of the tick) on
    their own h and v_sig."""
    from paper_2003_10850_gb300.kdk import KDK
    p = as_f32(W.clustered(8192, 8, seed=19))
    state = (ctx, dev(p.pos, torch.float64), dev(p.mass), dev(p.vel), dev(p.u))
    probe = KDK(*state, 1e-3, 3)
    dt_max = _dt_max(host(probe.h), host(probe.vsig), 3)
    g = KDK(*state, dt_max, 3)
    assert np.array_equal(host(g.bins), OK.timebins(host(g.h), host(g.vsig), 0.3, dt_max, 3))
    assert len(np.unique(host(g.bins))) == 4
    for _ in range(8):
        na = g.step()
        act = host(g.active)[:na]
        expect = OK.timebins(host(g.h)[act], host(g.vsig)[act], 0.3, dt_max, 3, tick=g.tick)
        assert np.array_equal(host(g.bins)[act], expect)
    assert torch.isfinite(g.u).all() and bool((g.u > 0).all())


def test_kdk_cycle_graph_replays_eager(S, ctx):
    """A dt_max cycle captured as one CUDA graph (nothing read back per tick:
    the active list is padded with -1 up to its capacity and every call takes
    the whole list) ends in bit for bit the state of the same cycle run
    eagerly, tick by tick, and records the same active counts."""
    from paper_2003_10850_gb300.kdk import KDK
    p = as_f32(W.clustered(8192, 8, seed=23))
    state = (ctx, dev(p.pos, torch.float64), dev(p.mass), dev(p.vel), dev(p.u))
    probe = KDK(*state, 1e-3, 2)
    dt_max = _dt_max(host(probe.h), host(probe.vsig), 2)
    a = KDK(*state, dt_max, 2)
    b = KDK(*state, dt_max, 2)
    counts = [a.step() for _ in range(4)]
    assert counts[3] == p.n and 0 < min(counts)
    b.capture_cycle()
    b.run_cycle()
    torch.cuda.synchronize()
    for k in ("pos", "vel", "u", "vel_pred", "u_pred", "h", "rho", "omega", "acc", "dudt", "vsig", "bins"):
        assert torch.equal(getattr(a, k), getattr(b, k)), k
    assert host(b.tick_counts).tolist() == [counts[3], counts[0], counts[1], counts[2]]
    # the graph replays at every later cycle boundary
    for _ in range(4):
        a.step(sync=False)
    b.run_cycle()
    torch.cuda.synchronize()
    assert torch.equal(a.pos, b.pos) and torch.equal(a.vel, b.vel)


def test_active_from_bins_pads_with_minus_one(S, ctx):
    n = 5000
    p = as_f32(W.clustered(n, 4, seed=29))
    grid = S.sph_build_grid(ctx, dev(p.pos), dev(p.mass), S.default_params())
    b = np.random.default_rng(3).integers(0, 4, n).astype(np.uint8)
    out = torch.full((n,), 7, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    S.sph_active_from_bins(ctx, grid, dev(b, torch.uint8), 2, 3, out, cnt)
    k = int(cnt.item())
    expect = np.nonzero(2 % (1 << (3 - b.astype(np.int64))) == 0)[0]
    o = host(out)
    assert k == expect.size and np.array_equal(o[:k], expect) and np.all(o[k:] == -1)
