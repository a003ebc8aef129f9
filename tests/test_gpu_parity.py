"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on
the same seeded inputs, element by element.

Tolerances (stated per output): rho and h relative <= 1e-5; acc and du/dt
<= 1e-4 of the per-particle absolute scale (sum of the pair terms'
magnitudes); neighbour and pair sets bit-exact (checksums of the sets) at the
same h; integer keys and the sort permutation bit-exact.
"""
import numpy as np
import pytest
import torch

import oracle
import workloads as W
from sph_cases import as_f32, check_force, dev, gpu_density, gpu_force, gpu_grid, host, oracle_all, rel

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


@pytest.fixture(scope="module")
def lattice32():
    p = as_f32(W.config1(32))
    return p, oracle_all(p)


@pytest.fixture(scope="module")
def clustered50k():
    p = as_f32(W.clustered(50_000, 40, seed=202))
    return p, oracle_all(p)


# ---- a1/a2: quantise, key, sort -------------------------------------------

@pytest.mark.parametrize("kind", ["lattice", "clustered"])
def test_keys_and_sort_exact(S, ctx, kind, lattice32, clustered50k):
    p = (lattice32 if kind == "lattice" else clustered50k)[0]
    grid = gpu_grid(S, ctx, p, S.default_params(box=p.box))
    n = p.n
    perm = torch.empty(n, dtype=torch.int32, device="cuda")
    keys = torch.empty(n, dtype=torch.int64, device="cuda")
    X = torch.empty(n, 3, dtype=torch.int32, device="cuda")
    S.sph_grid_export(grid, perm, keys, X)
    X_o = oracle.quantize(p.pos, p.box)
    k_o = oracle.morton_keys(X_o)
    perm_o = oracle.sort_perm(k_o)
    assert np.array_equal(host(X).view(np.uint32), X_o)
    assert np.array_equal(host(perm), perm_o)
    assert np.array_equal(host(keys).view(np.uint64), k_o[perm_o])


def test_batched_keys_and_sort_exact(S, ctx):
    boxes = [as_f32(W.clustered(n, 3, seed=300 + i)) for i, n in enumerate((1000, 4097, 2500))]
    pos = np.concatenate([b.pos for b in boxes])
    mass = np.concatenate([b.mass for b in boxes])
    offs = np.cumsum([0] + [b.n for b in boxes])
    grid = S.sph_build_grid_batched(ctx, dev(pos), dev(mass), offs, [1.0] * 3, S.default_params())
    perm = torch.empty(offs[-1], dtype=torch.int32, device="cuda")
    keys = torch.empty(offs[-1], dtype=torch.int64, device="cuda")
    S.sph_grid_export(grid, perm, keys, None)
    k_o = np.concatenate([oracle.morton_keys(oracle.quantize(b.pos), i, 2) for i, b in enumerate(boxes)])
    perm_o = oracle.sort_perm(k_o)
    assert np.array_equal(host(perm), perm_o)
    assert np.array_equal(host(keys).view(np.uint64), k_o[perm_o])


# ---- a4: density ------------------------------------------------------------

PATHS = ["wpp", "thread"]


def _flags(S, path, fp64):
    if path == "wpp" and fp64:
        pytest.skip("the warp-per-particle path is FP32 only (FP64 runs the per-thread walks)")
    extra = {"wpp": S.SPH_WARP_WALK, "thread": S.SPH_PER_THREAD_WALK}[path]
    return (S.SPH_FP64 if fp64 else 0) | extra


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("fp64", [False, True])
@pytest.mark.parametrize("kind", ["lattice", "clustered"])
def test_density_fixed_h_sets_exact(S, ctx, kind, fp64, path, lattice32, clustered50k):
    p, (X, d, _) = lattice32 if kind == "lattice" else clustered50k
    h32 = d["h"].astype(np.float32)
    params = S.default_params(box=p.box, flags=S.SPH_FIXED_H | _flags(S, path, fp64))
    grid = gpu_grid(S, ctx, p, params)
    g = gpu_density(S, ctx, grid, h32, params)
    assert g["rc"] == 0
    o = oracle.density(X, p.mass, h32.astype(np.float64), box=p.box, fixed_h=True)
    assert np.array_equal(g["n_ngb"], o["n_ngb"])
    assert np.array_equal(g["hash"], o["hash"])
    tol = 2e-7 if fp64 else 1e-5
    assert rel(g["rho"], o["rho"]).max() <= tol
    assert rel(g["omega"], o["omega"]).max() <= (1e-6 if fp64 else 1e-4)
    assert g["stats"]["density_pairs"] == int(o["n_ngb"].sum())


def _density_converged_checks(g, p, X, d, fp64):
    assert g["rc"] == 0 and not g["flags"].any()
    assert rel(g["h"], d["h"]).max() <= 1e-5
    assert rel(g["rho"], d["rho"]).max() <= 1e-5
    assert rel(g["omega"], d["omega"]).max() <= 1e-4
    # n_ngb at the converged h: between the oracle's counts at h (1 -/+ 1e-5)
    lo = oracle.density(X, p.mass, d["h"] * (1 - 1e-5), box=p.box, fixed_h=True)["n_ngb"]
    hi = oracle.density(X, p.mass, d["h"] * (1 + 1e-5), box=p.box, fixed_h=True)["n_ngb"]
    assert np.all((g["n_ngb"] >= lo) & (g["n_ngb"] <= hi))


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("fp64", [False, True])
@pytest.mark.parametrize("kind", ["lattice", "clustered"])
def test_density_converged(S, ctx, kind, fp64, path, lattice32, clustered50k):
    p, (X, d, _) = lattice32 if kind == "lattice" else clustered50k
    params = S.default_params(box=p.box, flags=_flags(S, path, fp64))
    grid = gpu_grid(S, ctx, p, params)
    g = gpu_density(S, ctx, grid, np.zeros(p.n, np.float32), params)   # h <= 0: local guess
    _density_converged_checks(g, p, X, d, fp64)
    # a perturbed start converges to the same root
    g2 = gpu_density(S, ctx, grid, W.perturb(d["h"], 0.3, seed=9).astype(np.float32), params)
    assert rel(g2["h"], d["h"]).max() <= 1e-5


@pytest.mark.parametrize("bps", [4, 5, 6, 8])
def test_register_budgets_agree(S, ctx, bps, clustered50k):
    """The default path's kernels at each register budget the autotuner can
    pick (blocks per SM: density 4 or 5, force 6 or 8): converged density
    against the oracle; then, at the oracle's h (a fixed-h density call that
    records the lists), the force from the recorded lists against the oracle,
    pair sets exact."""
    p, (X, d, _) = clustered50k
    params = S.default_params(box=p.box, blocks_per_sm=bps)
    grid = gpu_grid(S, ctx, p, params)
    g = gpu_density(S, ctx, grid, W.perturb(d["h"], 0.02, seed=4).astype(np.float32), params)
    _density_converged_checks(g, p, X, d, False)
    h, rho, om = _oracle_inputs32(d)
    gd = gpu_density(S, ctx, grid, h, S.default_params(box=p.box, blocks_per_sm=bps, flags=S.SPH_FIXED_H))
    assert gd["rc"] == 0
    f = oracle.force(X, p.vel, p.mass, p.u, h, rho, om, box=p.box)
    gf = gpu_force(S, ctx, grid, p, h, rho, om, params)
    assert gf["rc"] == 0 and gf["stats"]["pair_tests"] == 0
    check_force(gf, f, np.arange(p.n), 1e-4)


def test_density_plain_fp32(S, ctx, clustered50k):
    p, (X, d, _) = clustered50k
    params = S.default_params(box=p.box, flags=S.SPH_PLAIN_FP32)
    grid = gpu_grid(S, ctx, p, params)
    g = gpu_density(S, ctx, grid, np.zeros(p.n, np.float32), params)
    assert rel(g["h"], d["h"]).max() <= 1e-4
    assert rel(g["rho"], d["rho"]).max() <= 1e-4


# ---- a5: force --------------------------------------------------------------

def _oracle_inputs32(d):
    return [d[k].astype(np.float32) for k in ("h", "rho", "omega")]


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("fp64", [False, True])
@pytest.mark.parametrize("kind", ["lattice", "clustered"])
def test_force_parity(S, ctx, kind, fp64, path, lattice32, clustered50k):
    p, (X, d, _) = lattice32 if kind == "lattice" else clustered50k
    h, rho, om = _oracle_inputs32(d)
    f = oracle.force(X, p.vel, p.mass, p.u, h, rho, om, box=p.box)
    params = S.default_params(box=p.box, flags=_flags(S, path, fp64))
    grid = gpu_grid(S, ctx, p, params)
    g = gpu_force(S, ctx, grid, p, h, rho, om, params)
    assert g["rc"] == 0
    check_force(g, f, np.arange(p.n), 1e-6 if fp64 else 1e-4)
    assert g["stats"]["force_pairs"] == int(f["n_pairs"].sum())
    # momentum conservation of the GPU result
    mom = np.linalg.norm((p.mass[:, None] * g["acc"]).sum(0))
    assert mom <= 1e-5 * (p.mass * np.linalg.norm(g["acc"], axis=1)).sum()


@pytest.mark.parametrize("kind", ["lattice", "clustered"])
def test_force_reuses_density_lists(S, ctx, kind, lattice32, clustered50k):
    """An all-active density pass on the default path records each particle's
    neighbour list; the force pass then takes its pairs from those lists (and
    their transpose) instead of walking: no candidate is tested, and the
    results and pair sets equal the oracle's. Changing h invalidates the lists
    and the walk serves the call, with the same results."""
    p, (X, d, _) = lattice32 if kind == "lattice" else clustered50k
    h, rho, om = _oracle_inputs32(d)
    params = S.default_params(box=p.box)
    grid = gpu_grid(S, ctx, p, params)
    gd = gpu_density(S, ctx, grid, h, S.default_params(box=p.box, flags=S.SPH_FIXED_H))
    assert gd["rc"] == 0
    f = oracle.force(X, p.vel, p.mass, p.u, h, rho, om, box=p.box)
    g = gpu_force(S, ctx, grid, p, h, rho, om, params)
    assert g["rc"] == 0
    assert g["stats"]["pair_tests"] == 0
    check_force(g, f, np.arange(p.n), 1e-4)
    assert g["stats"]["force_pairs"] == int(f["n_pairs"].sum())
    h2 = (h * np.float32(1.001)).astype(np.float32)
    f2 = oracle.force(X, p.vel, p.mass, p.u, h2, rho, om, box=p.box)
    g2 = gpu_force(S, ctx, grid, p, h2, rho, om, params)
    assert g2["rc"] == 0 and g2["stats"]["pair_tests"] > 0
    check_force(g2, f2, np.arange(p.n), 1e-4)
    # an active subset of the force pass still reads the lists
    act = W.sample_indices(p.n, p.n // 7, seed=31).astype(np.int32)
    g3 = gpu_force(S, ctx, grid, p, h, rho, om, params, active=act)
    assert g3["stats"]["pair_tests"] == 0
    check_force(g3, f, act, 1e-4)


def _partial_selection(p, d, sel):
    """Active sets of the shapes a time-bin hierarchy gives: the densest 20%
    (small h: short time steps, spatially clumped), a ball around the densest
    particle, and a scattered 15% (mostly lone members of their leaves)."""
    if sel == "dense":
        return np.nonzero(d["h"] <= np.quantile(d["h"], 0.2))[0].astype(np.int32)
    if sel == "ball":
        c = p.pos[int(np.argmin(d["h"]))]
        r = np.linalg.norm((p.pos - c + 0.5 * p.box) % p.box - 0.5 * p.box, axis=1)
        return np.nonzero(r <= np.quantile(r, 0.1))[0].astype(np.int32)
    return W.sample_indices(p.n, int(0.15 * p.n), seed=33).astype(np.int32)


@pytest.mark.parametrize("sel", ["dense", "ball", "scattered"])
def test_force_reuses_partial_density_lists(S, ctx, sel, clustered50k):
    """With SPH_PARTIAL_LISTS a density call on an active list records the
    active particles' lists and their extra partners: the active ones through
    the transpose, the
    inactive ones (fixed h) found by the member-parallel sweep. The force pass
    on that list reads them (members the sweep left to the one-particle kernel
    walk), with the oracle's results and pair sets. Also: the list padded with
    -1 up to n (its count on the device), and a force set larger than the
    density set (the particles without a list of this call walk)."""
    p, (X, d, _) = clustered50k
    h, rho, om = _oracle_inputs32(d)
    act = _partial_selection(p, d, sel)
    params = S.default_params(box=p.box)
    pf = S.default_params(box=p.box, flags=S.SPH_FIXED_H | S.SPH_PARTIAL_LISTS)
    grid = gpu_grid(S, ctx, p, params)
    f = oracle.force(X, p.vel, p.mass, p.u, h, rho, om, box=p.box)
    # walked: without SPH_PARTIAL_LISTS a density call on an active list records no lists
    gd = gpu_density(S, ctx, grid, h, S.default_params(box=p.box, flags=S.SPH_FIXED_H), active=act)
    assert gd["rc"] == 0
    g0 = gpu_force(S, ctx, grid, p, h, rho, om, params, active=act)
    assert g0["rc"] == 0 and g0["stats"]["list_force"] == 0
    check_force(g0, f, act, 1e-4)
    # walked: a density call on the per-thread path records no lists
    gd = gpu_density(S, ctx, grid, h, S.default_params(box=p.box, flags=S.SPH_FIXED_H | S.SPH_PER_THREAD_WALK),
                     active=act)
    assert gd["rc"] == 0
    gw = gpu_force(S, ctx, grid, p, h, rho, om, params, active=act)
    assert gw["rc"] == 0
    check_force(gw, f, act, 1e-4)
    walked = gw["stats"]["pair_tests"]
    assert walked > 0
    # recorded by the partial density call
    gd = gpu_density(S, ctx, grid, h, pf, active=act)
    assert gd["rc"] == 0
    g = gpu_force(S, ctx, grid, p, h, rho, om, params, active=act)
    assert g["rc"] == 0
    check_force(g, f, act, 1e-4)
    assert g["stats"]["force_pairs"] == int(f["n_pairs"][act].sum())
    if sel != "scattered":   # clumped sets: nearly every active particle reads its lists
        assert g["stats"]["pair_tests"] < walked / 4, (g["stats"]["pair_tests"], walked)
        assert g["stats"]["list_force"] >= 0.9 * act.size
    # padded to n, count on the device
    pad = np.concatenate([act, np.full(p.n - act.size, -1, np.int32)])
    gd = gpu_density(S, ctx, grid, h, pf, active=pad)
    assert gd["rc"] == 0
    g2 = gpu_force(S, ctx, grid, p, h, rho, om, params, active=pad)
    assert g2["rc"] == 0
    check_force(g2, f, act, 1e-4)
    if sel != "scattered":
        assert g2["stats"]["pair_tests"] < walked / 4
    # a larger force set: the particles outside the density set walk
    more = np.union1d(act, W.sample_indices(p.n, p.n // 20, seed=34)).astype(np.int32)
    g3 = gpu_force(S, ctx, grid, p, h, rho, om, params, active=more)
    assert g3["rc"] == 0
    check_force(g3, f, more, 1e-4)


def test_lists_from_an_explicit_list_of_all_particles(S, ctx, clustered50k):
    """An active list that names every particle (shuffled) records the full
    lists like a call without a list; the same list padded with -1 in place of
    a tenth of its entries (count below n on the device) records lists that
    cannot serve, and the force pass walks, with the oracle's results."""
    p, (X, d, _) = clustered50k
    h, rho, om = _oracle_inputs32(d)
    params = S.default_params(box=p.box)
    pf = S.default_params(box=p.box, flags=S.SPH_FIXED_H)
    grid = gpu_grid(S, ctx, p, params)
    f = oracle.force(X, p.vel, p.mass, p.u, h, rho, om, box=p.box)
    every = np.random.default_rng(35).permutation(p.n).astype(np.int32)
    assert gpu_density(S, ctx, grid, h, pf, active=every)["rc"] == 0
    g = gpu_force(S, ctx, grid, p, h, rho, om, params, active=every)
    assert g["rc"] == 0 and g["stats"]["list_force"] == p.n and g["stats"]["pair_tests"] == 0
    check_force(g, f, np.arange(p.n), 1e-4)
    pad = every.copy()
    pad[: p.n // 10] = -1
    act = np.sort(pad[pad >= 0])
    assert gpu_density(S, ctx, grid, h, pf, active=pad)["rc"] == 0
    g2 = gpu_force(S, ctx, grid, p, h, rho, om, params, active=pad)
    assert g2["rc"] == 0 and g2["stats"]["list_force"] == 0 and g2["stats"]["pair_tests"] > 0
    check_force(g2, f, act, 1e-4)


def test_force_lists_that_do_not_fit(S, ctx):
    """With N_t = 200 every neighbour list overflows its 128 slots: the force
    pass hands every particle to the walk, with unchanged results."""
    p = as_f32(W.config1(16))
    X, d, f0 = oracle_all(p, n_target=200.0)
    h, rho, om = _oracle_inputs32(d)
    params = S.default_params(box=p.box, n_target=200.0, n_tol=200e-6)
    grid = gpu_grid(S, ctx, p, params)
    gd = gpu_density(S, ctx, grid, h, S.default_params(box=p.box, n_target=200.0, flags=S.SPH_FIXED_H))
    assert gd["rc"] == 0 and gd["n_ngb"].min() > 128
    f = oracle.force(X, p.vel, p.mass, p.u, h, rho, om, box=p.box)
    g = gpu_force(S, ctx, grid, p, h, rho, om, params)
    assert g["rc"] == 0 and g["stats"]["pair_tests"] > 0
    check_force(g, f, np.arange(p.n), 1e-4)


def _sparse_shell_around_clump(seed=12):
    """64 particles within ~0.001 of the centre, 160 in a sparse shell at
    0.05-0.15 around them, a uniform background beyond 0.3: every shell
    particle's h reaches the clump, so clump particles have more than 128
    extra partners (j with h_i <= r_ij < h_j)."""
    rng = np.random.default_rng(seed)
    c = np.array([0.5, 0.5, 0.5])
    clump = c + 0.001 * rng.standard_normal((64, 3))
    v = rng.standard_normal((160, 3))
    v /= np.linalg.norm(v, axis=1)[:, None]
    shell = c + v * rng.uniform(0.05, 0.15, (160, 1))
    bg = rng.uniform(0, 1, (20000, 3))
    bg = bg[np.linalg.norm(bg - c, axis=1) > 0.3]
    pos = np.concatenate([clump, shell, bg])
    n = len(pos)
    return as_f32(W.Particles(pos, rng.normal(0, 0.1, (n, 3)), np.full(n, 1.0 / n), rng.uniform(0.5, 1.5, n), 1.0))


def test_extra_partner_segments_that_overflow(S, ctx):
    """Particles with more than 128 extra partners overflow their fixed
    segments: the force pass walks for them and reads the lists for the
    rest, with the oracle's results."""
    p = _sparse_shell_around_clump()
    X, d, _ = oracle_all(p)
    h, rho, om = _oracle_inputs32(d)
    oi, oj = oracle.pair_list(X, h.astype(np.float64))
    xu = X.astype(np.int64)
    dd = (xu[oj] - xu[oi] + 2**31) % 2**32 - 2**31
    r = np.sqrt((dd.astype(np.float64) ** 2).sum(1)) / 2**32
    n_ext = np.bincount(oi[r >= h[oi]], minlength=p.n)
    assert (n_ext > 128).sum() >= 8            # the input overflows some segments
    params = S.default_params(box=p.box)
    grid = gpu_grid(S, ctx, p, params)
    gd = gpu_density(S, ctx, grid, h, S.default_params(box=p.box, flags=S.SPH_FIXED_H))
    assert gd["rc"] == 0
    f = oracle.force(X, p.vel, p.mass, p.u, h, rho, om, box=p.box)
    g = gpu_force(S, ctx, grid, p, h, rho, om, params)
    # a changed h makes every particle walk: the candidate tests of a full walk
    walk = gpu_force(S, ctx, grid, p, (h * np.float32(1.0001)).astype(np.float32), rho, om, params)
    assert g["rc"] == 0 and 0 < g["stats"]["pair_tests"] < walk["stats"]["pair_tests"] // 10
    check_force(g, f, np.arange(p.n), 1e-4)


def test_no_lists_grid(S, ctx, clustered50k):
    """A grid built with SPH_NO_LISTS records nothing; the force pass walks."""
    p, (X, d, _) = clustered50k
    h, rho, om = _oracle_inputs32(d)
    grid = gpu_grid(S, ctx, p, S.default_params(box=p.box, flags=S.SPH_NO_LISTS))
    params = S.default_params(box=p.box)
    gpu_density(S, ctx, grid, h, S.default_params(box=p.box, flags=S.SPH_FIXED_H))
    f = oracle.force(X, p.vel, p.mass, p.u, h, rho, om, box=p.box)
    g = gpu_force(S, ctx, grid, p, h, rho, om, params)
    assert g["stats"]["pair_tests"] > 0
    check_force(g, f, np.arange(p.n), 1e-4)


def test_force_plain_fp32(S, ctx, clustered50k):
    p, (X, d, _) = clustered50k
    h, rho, om = _oracle_inputs32(d)
    f = oracle.force(X, p.vel, p.mass, p.u, h, rho, om, box=p.box)
    params = S.default_params(box=p.box, flags=S.SPH_PLAIN_FP32)
    grid = gpu_grid(S, ctx, p, params)
    g = gpu_force(S, ctx, grid, p, h, rho, om, params)
    da = np.linalg.norm(g["acc"] - f["acc"], axis=1)
    assert np.quantile(da / f["scale_a"], 0.999) <= 1e-3


# ---- a6: active subsets and batched boxes ------------------------------------

@pytest.mark.parametrize("path", PATHS)
def test_active_subset(S, ctx, path, clustered50k):
    p, (X, d, _) = clustered50k
    act = W.sample_indices(p.n, p.n // 10, seed=17).astype(np.int32)
    params = S.default_params(box=p.box, flags=_flags(S, path, False))
    grid = gpu_grid(S, ctx, p, params)
    h0 = np.full(p.n, -7.0, np.float32)
    h0[act] = 0.0
    g = gpu_density(S, ctx, grid, h0, params, active=act)
    assert g["rc"] == 0
    assert rel(g["h"][act], d["h"][act]).max() <= 1e-5
    assert rel(g["rho"][act], d["rho"][act]).max() <= 1e-5
    inact = np.setdiff1d(np.arange(p.n), act)
    assert np.all(g["h"][inact] == -7.0) and np.all(g["n_ngb"][inact] == -1)
    h, rho, om = _oracle_inputs32(d)
    f = oracle.force(X, p.vel, p.mass, p.u, h, rho, om, box=p.box, active=act.astype(np.int64))
    gf = gpu_force(S, ctx, grid, p, h, rho, om, params, active=act)
    check_force(gf, f, act, 1e-4)
    assert np.all(gf["acc"][inact] == 0)
    # duplicates in the active list are ignored
    dup = np.concatenate([act, act[:100]])
    g2 = gpu_density(S, ctx, grid, h0, params, active=dup)
    assert np.array_equal(g2["n_ngb"][act], g["n_ngb"][act])
    # so are negative entries: the list padded with -1 to capacity n (the
    # launch shape then follows the capacity, so the sums may round
    # differently; the results meet the same bounds)
    pad = np.full(p.n, -1, np.int32)
    pad[:act.size] = act
    g3 = gpu_density(S, ctx, grid, h0, params, active=pad)
    assert g3["rc"] == 0
    assert rel(g3["h"][act], d["h"][act]).max() <= 1e-5
    assert rel(g3["rho"][act], d["rho"][act]).max() <= 1e-5
    assert np.all(g3["h"][inact] == -7.0) and np.all(g3["n_ngb"][inact] == -1)
    gf3 = gpu_force(S, ctx, grid, p, h, rho, om, params, active=pad)
    check_force(gf3, f, act, 1e-4)
    assert np.all(gf3["acc"][inact] == 0)


@pytest.mark.parametrize("span", [8, 512, 4096])
def test_group_span(S, ctx, span, clustered50k):
    """The member-parallel kernels with groups confined to aligned runs of 8,
    512 or 4096 sorted particles (params.group_size) on half the particles
    active: the same results as the oracle (a group only changes which walk
    a particle shares)."""
    p, (X, d, _) = clustered50k
    act = W.sample_indices(p.n, p.n // 2, seed=29).astype(np.int32)
    params = S.default_params(box=p.box, group_size=span)
    grid = gpu_grid(S, ctx, p, params)
    h0 = np.full(p.n, -7.0, np.float32)
    h0[act] = (d["h"][act] * 1.02).astype(np.float32)
    g = gpu_density(S, ctx, grid, h0, params, active=act)
    assert g["rc"] == 0
    assert rel(g["h"][act], d["h"][act]).max() <= 1e-5
    assert rel(g["rho"][act], d["rho"][act]).max() <= 1e-5
    h, rho, om = _oracle_inputs32(d)
    f = oracle.force(X, p.vel, p.mass, p.u, h, rho, om, box=p.box, active=act.astype(np.int64))
    gf = gpu_force(S, ctx, grid, p, h, rho, om, params, active=act)
    check_force(gf, f, act, 1e-4)


@pytest.mark.parametrize("path", PATHS)
def test_batched_boxes(S, ctx, path):
    sizes = (4096, 9000, 30000, 2000)
    Ls = (1.0, 2.0, 0.5, 1.0)
    boxes = []
    for i, (n, L) in enumerate(zip(sizes, Ls)):
        b = W.clustered(n, W.blobs_for(n), seed=100 + i)
        boxes.append(as_f32(W.Particles(b.pos * L, b.vel, b.mass, b.u, L)))
    pos = np.concatenate([b.pos for b in boxes])
    offs = np.cumsum([0] + [b.n for b in boxes])
    cat = lambda k: np.concatenate([getattr(b, k) for b in boxes])
    params = S.default_params(flags=_flags(S, path, False))
    grid = S.sph_build_grid_batched(ctx, dev(pos), dev(cat("mass")), offs, Ls, params)
    g = gpu_density(S, ctx, grid, np.zeros(offs[-1], np.float32), params)
    assert g["rc"] == 0
    hs, rhos, oms = [], [], []
    for i, b in enumerate(boxes):
        X, d, _ = oracle_all(b)
        sl = slice(offs[i], offs[i + 1])
        assert rel(g["h"][sl], d["h"]).max() <= 1e-5, i
        assert rel(g["rho"][sl], d["rho"]).max() <= 1e-5, i
        hs.append(d["h"]); rhos.append(d["rho"]); oms.append(d["omega"])
    h, rho, om = (np.concatenate(a).astype(np.float32) for a in (hs, rhos, oms))
    pall = W.Particles(pos, cat("vel"), cat("mass"), cat("u"), 1.0)
    gf = gpu_force(S, ctx, grid, pall, h, rho, om, params)
    n_pairs = 0
    for i, b in enumerate(boxes):
        sl = slice(offs[i], offs[i + 1])
        X = oracle.quantize(b.pos, b.box)
        f = oracle.force(X, b.vel, b.mass, b.u, h[sl], rho[sl], om[sl], box=b.box)
        gi = {k: gf[k][sl] for k in ("acc", "dudt", "vsig", "hash")}
        # the library hashes caller indices of the whole batch, the oracle its
        # box-local ones: exact sets are compared for box 0 (offset 0) and via
        # the total pair count for all boxes
        check_force(gi, f, np.arange(b.n), 1e-4, check_hash=(i == 0))
        n_pairs += int(f["n_pairs"].sum())
    assert gf["stats"]["force_pairs"] == n_pairs


# ---- edge cases ----------------------------------------------------------------

@pytest.mark.parametrize("path", PATHS)
def test_small_box_wide_groups(S, ctx, path):
    p = as_f32(W.clustered(600, 2, seed=77))          # h near L/4: groups wider than L/4
    X, d, f = oracle_all(p, n_target=32.0)
    params = S.default_params(n_target=32.0, n_tol=32e-6, flags=_flags(S, path, False))
    grid = gpu_grid(S, ctx, p, params)
    g = gpu_density(S, ctx, grid, np.zeros(p.n, np.float32), params)
    assert g["rc"] == 0
    assert rel(g["h"], d["h"]).max() <= 1e-5
    h, rho, om = _oracle_inputs32(d)
    fo = oracle.force(X, p.vel, p.mass, p.u, h, rho, om)
    gf = gpu_force(S, ctx, grid, p, h, rho, om, params)
    check_force(gf, fo, np.arange(p.n), 1e-4)


def test_error_statuses(S, ctx):
    from paper_2003_10850_gb300 import abi
    p = as_f32(W.lattice(3, 0.2, seed=5))               # 27 particles cannot reach 64 neighbours
    params = S.default_params()
    grid = gpu_grid(S, ctx, p, params)
    g = gpu_density(S, ctx, grid, np.zeros(p.n, np.float32), params)
    assert g["rc"] == abi.SPH_ERR_H_TOO_LARGE and np.all(g["flags"] & abi.SPH_ST_H_TOO_LARGE)
    q = as_f32(W.config1(16))
    grid = gpu_grid(S, ctx, q, S.default_params(max_iter=0))
    g = gpu_density(S, ctx, grid, np.full(q.n, 0.01, np.float32), S.default_params(max_iter=0))
    assert g["rc"] == abi.SPH_ERR_NOT_CONVERGED and np.all(g["flags"] & abi.SPH_ST_NOT_CONVERGED)
    bad = q.pos.copy()
    bad[5, 1] = np.nan
    grid = S.sph_build_grid(ctx, dev(bad), dev(q.mass), params)
    rc, _ = S.sph_sync_status(ctx, raise_on_error=False)
    assert rc == abi.SPH_ERR_INVALID
    with pytest.raises(S.SPHError):
        S.sph_build_grid(ctx, dev(q.pos), dev(q.mass), S.default_params(box=-1.0))
    with pytest.raises(TypeError):
        S.sph_build_grid(ctx, dev(q.pos).double().cpu(), dev(q.mass), params)
    # a group span must be a power of two in [8, 4096]
    for gs in (12, 4, 8192):
        with pytest.raises(S.SPHError) as e:
            gpu_density(S, ctx, grid, np.full(q.n, 0.01, np.float32), S.default_params(group_size=gs))
        assert e.value.status == abi.SPH_ERR_INVALID
    # the warp-group and cooperative paths are no longer built: their flags are rejected
    for fl in (S.SPH_WARP_GROUP, S.SPH_COOP_WALK):
        with pytest.raises(S.SPHError) as e:
            gpu_grid(S, ctx, q, S.default_params(flags=fl))
        assert e.value.status == abi.SPH_ERR_INVALID


def test_grid_freed_after_its_context(S):
    """A garbage collector may finalise a grid after the context that built
    it: freeing it then must not touch the destroyed context, nor leave a CUDA
    error pending for the caller's next call."""
    p = as_f32(W.lattice(8, 0.2, seed=3))
    c2 = S.Context(0)
    grid = gpu_grid(S, c2, p, S.default_params())
    c2.close()
    grid.free()
    x = torch.zeros(16, device="cuda")   # raises if an error were left pending
    torch.cuda.synchronize()
    assert float(x.sum()) == 0.0


def test_single_particle_and_tiny(S, ctx):
    from paper_2003_10850_gb300 import abi
    p = as_f32(W.lattice(1, 0.0, seed=0))
    params = S.default_params(n_target=16.0)
    grid = gpu_grid(S, ctx, p, params)
    g = gpu_density(S, ctx, grid, np.zeros(1, np.float32), params)
    assert g["rc"] == abi.SPH_ERR_H_TOO_LARGE          # N_eff = 32/3 < 16 for every h
    assert g["n_ngb"][0] == 0
    # a target at or below the self term 32/3 has no root: rejected on the host
    with pytest.raises(S.SPHError):
        gpu_density(S, ctx, grid, np.zeros(1, np.float32), S.default_params(n_target=10.0))


# ---- a6: the step captured as a CUDA graph ------------------------------------

@pytest.mark.parametrize("which", ["subset", "all"])
def test_graph_capture_replays_eager_results(S, ctx, clustered50k, which):
    """Grid rebuild + density + force over an active subset (walks) or over all
    particles (the force pass reads the density pass's neighbour lists),
    captured once and replayed: the outputs equal those of the eager calls bit
    for bit."""
    p, (X, d, _) = clustered50k
    params = S.default_params(box=p.box)
    idx = W.sample_indices(p.n, p.n // 5, seed=23) if which == "subset" else np.arange(p.n)
    act = dev(idx.astype(np.int32), torch.int32)
    pos, mass, vel, u = dev(p.pos), dev(p.mass), dev(p.vel), dev(p.u)
    grid = S.sph_build_grid(ctx, pos, mass, params)
    h0 = dev(d["h"].astype(np.float32) * 1.01)
    outs = {}
    for mode in ("eager", "graph"):
        h = h0.clone()
        # inactive neighbours keep a valid state (the oracle's, rounded to FP32)
        rho, om = dev(d["rho"].astype(np.float32)), dev(d["omega"].astype(np.float32))
        nn, fl = torch.zeros(p.n, dtype=torch.int32, device="cuda"), torch.zeros(p.n, dtype=torch.uint8, device="cuda")
        acc, du, vs = torch.zeros(p.n, 3, device="cuda"), torch.zeros(p.n, device="cuda"), torch.zeros(p.n, device="cuda")

        def body():
            h.copy_(h0)
            S.sph_grid_update(ctx, grid, pos, mass)
            S.sph_density(ctx, grid, h, act, rho, om, nn, fl, None, params)
            S.sph_hydro_force(ctx, grid, vel, u, h, rho, om, act, acc, du, vs, None, params)

        if mode == "eager":
            body()
        else:
            side = torch.cuda.Stream()
            side.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(side):
                body()
            torch.cuda.current_stream().wait_stream(side)
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g):
                body()
            for t in (acc, du, vs):
                t.zero_()
            rho.copy_(dev(d["rho"].astype(np.float32)))
            om.copy_(dev(d["omega"].astype(np.float32)))
            g.replay()
            g.replay()
        rc, _ = S.sph_sync_status(ctx, raise_on_error=False)
        assert rc == 0
        outs[mode] = [host(t) for t in (h, rho, om, nn, acc, du, vs)]
    for a, b in zip(outs["eager"], outs["graph"]):
        assert np.all(np.isfinite(a.astype(np.float64))) and np.array_equal(a, b)
