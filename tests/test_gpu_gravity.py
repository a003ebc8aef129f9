"""GPU parity of the short-range gravity pass (sph_gravity) against the FP64
oracle, through the C ABI.

Every decision of the walk (skip, monopole, open; pair inside the cutoff) is
exact integer arithmetic on both sides, so the per-particle node and pair
counts must agree exactly. The accelerations differ by FP32 rounding (pair
terms, node centres of mass, sums) and by the kernel's erfc approximation
(Abramowitz & Stegun 7.1.26: at most 1.2e-5 of a term's split factor, in
FP32): within 2e-5 of the per-particle scale sum |G m K(r) r|.
"""
import numpy as np
import pytest
import torch

import oracle
import workloads as W
from sph_cases import as_f32, dev, host

pytestmark = pytest.mark.gpu

TOL = 2e-5


@pytest.fixture(scope="module")
def S():
    from paper_2003_10850_gb300 import build
    build.build()
    import paper_2003_10850_gb300 as S
    return S


@pytest.fixture(scope="module")
def ctx(S):
    return S.Context(0)


def _split(n, box=1.0):
    """TreePM split of a mesh with 1 cell per particle spacing: r_s = 1.25 cells,
    r_cut = 4.5 r_s, spline softening 1/30 of a spacing times 2.8."""
    cell = box / round(n ** (1 / 3))
    return dict(r_split=1.25 * cell, r_cut=min(4.5 * 1.25 * cell, 0.25 * box), h_soft=2.8 * cell / 30)


def _gpu(S, ctx, p, gp, active=None, params=None):
    grid = S.sph_build_grid(ctx, dev(p.pos), dev(p.mass), params or S.default_params(box=p.box))
    n = p.n
    acc = torch.zeros(n, 3, device="cuda")
    nn = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    npr = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    act = None if active is None else dev(active, torch.int32)
    S.sph_gravity(ctx, grid, act, gp, acc, nn, npr)
    _, st = S.sph_sync_status(ctx)
    grid.free()
    return host(acc), host(nn), host(npr), st


def _check(g_acc, g_nn, g_np, o, idx):
    assert np.array_equal(g_nn[idx], o["n_nodes"][idx])
    assert np.array_equal(g_np[idx], o["n_pairs"][idx])
    err = np.linalg.norm(g_acc[idx] - o["acc"][idx], axis=1)
    assert np.all(err <= TOL * o["scale"][idx]), (err / o["scale"][idx]).max()


@pytest.mark.parametrize("theta", [0.0, 0.5, 0.8])
def test_gravity_parity_clustered(S, ctx, theta):
    p = as_f32(W.clustered(30_000, 20, seed=401))
    sp = _split(p.n)
    X = oracle.quantize(p.pos)
    o = oracle.gravity(X, p.mass, G=1.0, theta=theta, **sp)
    acc, nn, npr, st = _gpu(S, ctx, p, S.gravity_params(G=1.0, theta=theta, **sp))
    _check(acc, nn, npr, o, np.arange(p.n))
    assert st["grav_nodes"] == o["n_nodes"].sum() and st["grav_pairs"] == o["n_pairs"].sum()
    if theta > 0:
        assert o["n_nodes"].sum() > p.n   # nodes are accepted: the walk is not a direct sum


def test_gravity_subset_matches_full_pass(S, ctx):
    p = as_f32(W.clustered(20_000, 12, seed=402))
    sp = _split(p.n)
    gp = S.gravity_params(G=2.0, theta=0.6, **sp)
    full = _gpu(S, ctx, p, gp)
    act = np.arange(0, p.n, 3, dtype=np.int32)
    sub = _gpu(S, ctx, p, gp, active=act)
    # every decision is the same exact rule: identical counts; the full pass
    # shares walks among groups of particles and the sparse subset walks one
    # particle at a time, so the sums differ in rounding order only
    assert np.array_equal(full[1][act], sub[1][act]) and np.array_equal(full[2][act], sub[2][act])
    o = oracle.gravity(oracle.quantize(p.pos), p.mass, G=2.0, theta=0.6, **sp)
    err = np.linalg.norm(full[0][act] - sub[0][act], axis=1)
    assert np.all(err <= TOL * o["scale"][act]), (err / o["scale"][act]).max()
    rest = np.setdiff1d(np.arange(p.n), act)
    assert np.all(sub[1][rest] == -1)


def test_gravity_lattice_and_tiny_boxes(S, ctx):
    p = as_f32(W.lattice(16, 0.0, seed=0, vel_sigma=0.0))
    gp = S.gravity_params(theta=0.0, r_split=0.05, r_cut=0.2345, h_soft=0.01)
    acc, nn, npr, _ = _gpu(S, ctx, p, gp)
    o = oracle.gravity(oracle.quantize(p.pos), p.mass, theta=0.0, r_split=0.05, r_cut=0.2345, h_soft=0.01)
    _check(acc, nn, npr, o, np.arange(p.n))
    assert np.all(np.linalg.norm(acc, axis=1) <= 1e-5 * o["scale"])
    # a box of 1..9 particles: a single leaf, or a root over two leaves
    for n in (1, 2, 8, 9):
        q = as_f32(W.clustered(n, 1, seed=n))
        acc, nn, npr, _ = _gpu(S, ctx, q, gp)
        oq = oracle.gravity(oracle.quantize(q.pos), q.mass, theta=0.0, r_split=0.05, r_cut=0.2345, h_soft=0.01)
        _check(acc, nn, npr, oq, np.arange(n))


def test_gravity_batched_boxes(S, ctx):
    boxes = [as_f32(W.clustered(3000 + 1000 * b, 3, seed=410 + b, box=L)) for b, L in enumerate((1.0, 2.0, 0.5))]
    offs = np.cumsum([0] + [b.n for b in boxes])
    cat = lambda k: np.concatenate([getattr(b, k) for b in boxes])
    grid = S.sph_build_grid_batched(ctx, dev(cat("pos")), dev(cat("mass")), offs, [b.box for b in boxes],
                                    S.default_params())
    gp = S.gravity_params(theta=0.5, r_split=0.02, r_cut=0.1, h_soft=0.003)
    n = int(offs[-1])
    acc = torch.zeros(n, 3, device="cuda")
    nn = torch.zeros(n, dtype=torch.int32, device="cuda")
    npr = torch.zeros(n, dtype=torch.int32, device="cuda")
    S.sph_gravity(ctx, grid, None, gp, acc, nn, npr)
    S.sph_sync_status(ctx)
    for b, q in enumerate(boxes):
        sl = slice(offs[b], offs[b + 1])
        o = oracle.gravity(oracle.quantize(q.pos, q.box), q.mass, box=q.box, theta=0.5, r_split=0.02, r_cut=0.1,
                           h_soft=0.003)
        _check(host(acc)[sl], host(nn)[sl], host(npr)[sl], o, np.arange(q.n))
    grid.free()


def test_gravity_rejects_bad_parameters(S, ctx):
    p = as_f32(W.clustered(1000, 2, seed=3))
    grid = S.sph_build_grid(ctx, dev(p.pos), dev(p.mass), S.default_params())
    acc = torch.zeros(p.n, 3, device="cuda")
    for bad in (dict(r_cut=0.3), dict(theta=1.5), dict(r_cut=0.0), dict(h_soft=-1.0)):
        with pytest.raises(S.SPHError):
            S.sph_gravity(ctx, grid, None, S.gravity_params(**bad), acc)
    grid.free()


def test_gravity_2m_sampled(S, ctx):
    """2M clustered particles (blobs ~ sqrt N), the launch shape of the bench:
    sampled particles against the oracle's walk for them."""
    p = as_f32(W.clustered(2_000_000, 224, seed=404))
    sp = _split(p.n)
    acc, nn, npr, _ = _gpu(S, ctx, p, S.gravity_params(theta=0.5, **sp))
    idx = np.sort(np.random.default_rng(1).choice(p.n, 300, replace=False))
    o = oracle.gravity(oracle.quantize(p.pos), p.mass, theta=0.5, active=idx, **sp)
    _check(acc, nn, npr, o, idx)
