"""Launch-shape autotuner for the density and force passes.

Times a small set of configurations of each pass on the caller's own grid and
state (CUDA events on the current stream, best of `reps`), picks the fastest
per pass, and caches the choice per (GPU name, particle count, workload tag)
in paper_2003_10850_gb300/_build/autotune.json. The knobs are those of
sph_params: persistent blocks per SM (a register budget) and the walk radius
of the density pass (the radius of its near lists, as a multiple of h: larger
radii mean longer lists but fewer walks again when h grows), against the
per-thread walks as the other kernel family; and, on a partial active set
(`tune_group_span`), the group span of the member-parallel kernels (how far
apart in sorted order the up to 8 particles sharing a walk may lie: wider
spans make fuller groups of sparse sets, with larger boxes).
"""
from __future__ import annotations

import json
import os

import torch

from . import SPH_PER_THREAD_WALK, default_params, sph_density, sph_hydro_force, sph_sync_status

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "autotune.json")

# default path (flags 0) at two register budgets and three walk radii, and the
# per-thread walks
DENSITY_CANDIDATES = ([dict(flags=0, blocks_per_sm=b, walk_radius=r) for b in (4, 5) for r in (1.03, 1.04, 1.06)] +
                      [dict(flags=SPH_PER_THREAD_WALK, blocks_per_sm=16)])
FORCE_CANDIDATES = ([dict(flags=0, blocks_per_sm=b) for b in (6, 8)] +
                    [dict(flags=SPH_PER_THREAD_WALK, blocks_per_sm=16)])


def _load():
    try:
        with open(CACHE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _save(c):
    os.makedirs(os.path.dirname(CACHE), exist_ok=True)
    tmp = CACHE + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(c, f, indent=1, sort_keys=True)
    os.replace(tmp, CACHE)


def _time(fn, reps):
    best = float("inf")
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        b.synchronize()
        best = min(best, a.elapsed_time(b))
    return best


def tune(ctx, grid, st, vel, u, h, h_guess, active=None, tag="default", reps=2, use_cache=True):
    """Returns (density_params, force_params, report). `st` holds the output
    buffers rho, omega, n_ngb, flags, acc, dudt, vsig; h is overwritten with
    h_guess before every density trial."""
    key = f"{torch.cuda.get_device_name()}|n={grid.n}|{tag}"
    cache = _load() if use_cache else {}
    if key in cache:
        e = cache[key]
        return default_params(**e["density"]), default_params(**e["force"]), e
    dens = list(DENSITY_CANDIDATES)
    rep = {"density": {}, "force": {}}

    def run_d(kw):
        h.copy_(h_guess)
        sph_density(ctx, grid, h, active, st["rho"], st["omega"], st["n_ngb"], st["flags"], None,
                    default_params(**kw))

    best_d, best_dt = None, float("inf")
    for kw in dens:
        t = _time(lambda: run_d(kw), reps)
        sph_sync_status(ctx, raise_on_error=False)
        rep["density"][json.dumps(kw, sort_keys=True)] = t
        if t < best_dt:
            best_d, best_dt = kw, t
    run_d(best_d)   # leave the converged state of the winner in place

    def run_f(kw):
        sph_hydro_force(ctx, grid, vel, u, h, st["rho"], st["omega"], active, st["acc"], st["dudt"], st["vsig"],
                        None, default_params(**kw))

    best_f, best_ft = None, float("inf")
    for kw in FORCE_CANDIDATES:
        t = _time(lambda: run_f(kw), reps)
        rep["force"][json.dumps(kw, sort_keys=True)] = t
        if t < best_ft:
            best_f, best_ft = kw, t
    sph_sync_status(ctx, raise_on_error=False)
    entry = {"density": best_d, "force": best_f, "density_ms": best_dt, "force_ms": best_ft, "trials": rep}
    cache[key] = entry
    _save(cache)
    return default_params(**best_d), default_params(**best_f), entry


GROUP_SPANS = (64, 512, 4096)


def tune_group_span(ctx, grid, st, vel, u, h, h_guess, active, dparams, fparams, tag="default", reps=2,
                    use_cache=True):
    """Times density + force on `active` (a partial active set, where groups
    form from sparse particles) for each group span of GROUP_SPANS with the
    other knobs of dparams/fparams, and returns the fastest span (cached like
    tune())."""
    key = f"{torch.cuda.get_device_name()}|n={grid.n}|{tag}|group_span"
    cache = _load() if use_cache else {}
    if key in cache:
        return cache[key]["group_size"], cache[key]
    rep = {}
    best, best_t = GROUP_SPANS[0], float("inf")
    for gs in GROUP_SPANS:
        dp = default_params(flags=dparams.flags, blocks_per_sm=dparams.blocks_per_sm,
                            walk_radius=dparams.walk_radius, group_size=gs)
        fp = default_params(flags=fparams.flags, blocks_per_sm=fparams.blocks_per_sm, group_size=gs)

        def run():
            h.copy_(h_guess)
            sph_density(ctx, grid, h, active, st["rho"], st["omega"], st["n_ngb"], st["flags"], None, dp)
            sph_hydro_force(ctx, grid, vel, u, h, st["rho"], st["omega"], active, st["acc"], st["dudt"], st["vsig"],
                            None, fp)

        t = _time(run, reps)
        sph_sync_status(ctx, raise_on_error=False)
        rep[str(gs)] = t
        if t < best_t:
            best, best_t = gs, t
    entry = {"group_size": best, "ms": best_t, "trials": rep}
    cache[key] = entry
    _save(cache)
    return best, entry
