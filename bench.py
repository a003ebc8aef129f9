#!/usr/bin/env python
"""Benchmark: SPH pair-interactions/s (density + force) at 10M particles.

Workload (one "step" = one pass of the whole hot path): 10,000,000 clustered
gas particles (500 Gaussian blobs on a uniform background, seed 3) whose
adaptive time bins give sub-steps with 100 %, 10 %, 1 % and 0.1 % active
particles. A step rebuilds the neighbour grid in place (quantise, key, sort,
bound) and then runs, per sub-step, the density pass (smoothing-length
iteration on the device) and the hydro-force pass over that sub-step's
active set. Pairs = sum over active i of n_ngb,i (density, at the converged
h) + |{j : r_ij < max(h_i, h_j)}| (force), counted by the kernels.

Inputs (positions, state) total > 1 GB, far larger than the 129 MB L2.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun with N > 1 every rank runs an independent replica on its own
GPU (the path has no exchange step on one box); value = all ranks' pairs / max
time over ranks. --impl reference times the FP64 CPU oracle on the host.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SPH pair-interactions/s (density+force) at 10M particles, vs plain FP32 path"
UNIT = "pairs/s"
FLOPS_DENSITY_PAIR = 30.0   # FP32 flops per density pair (FMA = 2), one pass at the converged h
FLOPS_FORCE_PAIR = 90.0     # FP32 flops per force pair
FLOPS_GRAV_INTERACTION = 40.0   # FP32 flops per gravity interaction (softened, split pair or node term)
FP32_LANES_PER_SM = 128
# ncu figures of the density pass (k_density_mp, then k_density_wpp for the particles it
# leaves) on the 2,000,000-particle 100 % sub-step of this benchmark's workload (one launch of
# each, --set full, --clock-control none): DRAM bytes (dram__bytes_read.sum +
# dram__bytes_write.sum), warp instructions (smsp__inst_executed.sum), serialised durations,
# and the member-parallel kernel's pipe utilisation; the call counted 118,572,011 density pairs
DENSITY_NCU_2M = {"kernels": "k_density_mp + k_density_wpp", "launch": "2M clustered, 100 % sub-step",
                  "dram_bytes": (129.718016e6 + 458.693888e6) + (72.817152e6 + 42.396928e6),
                  "warp_inst": 3.403872364e9 + 9.68670724e8,
                  "ms": 4.384064 + 1.612096, "density_pairs": 118_572_011,
                  "fma_pipe_pct": 26.62, "alu_pipe_pct": 39.68, "issue_active_pct": 62.85}
# DRAM bytes of one density launch per active particle, scaled by the active particles of a launch
DENSITY_DRAM_BYTES_PER_ACTIVE = DENSITY_NCU_2M["dram_bytes"] / 2_000_000
H_PERTURB = 0.02            # per-step log-normal scatter of the h guesses: the density change between steps


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=10_000_000)
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the batched-boxes and adjoint lines")
    ap.add_argument("--cpu-n", type=int, default=1 << 20, help="particles of the CPU-baseline sample")
    ap.add_argument("--gravity-only", action="store_true",
                    help="only the short-range gravity pass on the workload (one JSON line with that figure)")
    return ap.parse_args(argv)


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


# ---------------------------------------------------------------------------
# CPU side: the FP64 oracle on a bounded sample (cpu_baseline, --impl reference)
# ---------------------------------------------------------------------------

def oracle_sample(n_s: int, seed: int = 3):
    """A bounded sample of the workload: the same generator at n_s particles
    (blob count scaled with sqrt(N)), all particles active, h guesses perturbed
    from the converged h exactly as in the GPU step."""
    import oracle
    import workloads as W
    p = W.clustered(n_s, W.blobs_for(n_s), seed=seed)
    p32 = lambda a: np.asarray(a, np.float32).astype(np.float64)
    X = oracle.quantize(p32(p.pos))
    m, v, u = p32(p.mass), p32(p.vel), p32(p.u)
    d0 = oracle.density(X, m, None, tol=64e-6)
    h_in = W.perturb(d0["h"], H_PERTURB, seed=11)
    return dict(X=X, m=m, v=v, u=u, h_in=h_in)


def oracle_step(s):
    import oracle
    t0 = time.perf_counter()
    d = oracle.density(s["X"], s["m"], s["h_in"], tol=64e-6)
    f = oracle.force(s["X"], s["v"], s["m"], s["u"], d["h"], d["rho"], d["omega"])
    dt = time.perf_counter() - t0
    pairs = int(d["n_ngb"].sum() + f["n_pairs"].sum())
    return pairs, dt


def host_cores():
    """The host's logical CPUs and those this process may run on (a cgroup or
    affinity mask can hold fewer than the machine has)."""
    total = os.cpu_count() or 0
    try:
        usable = len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        usable = total
    return {"host_cpus": total, "usable_cpus": usable}


def run_reference(args, rank):
    if rank != 0:
        return
    import oracle
    oracle.build()
    s = oracle_sample(args.cpu_n)
    for _ in range(args.warmup):
        oracle_step(s)
    pairs = secs = 0.0
    for _ in range(args.steps):
        pr, dt = oracle_step(s)
        pairs += pr
        secs += dt
    v = pairs / secs
    line = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": f"10M clustered time-binned SPH step; CPU sample: same generator at "
                                   f"N={args.cpu_n}, all active, density (from perturbed h) + force"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": f"clustered N={args.cpu_n}, all active, density+force", **host_cores()},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU side
# ---------------------------------------------------------------------------

class Clocks:
    """nvidia-smi sampling in the background during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(device), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].strip() == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def setup_workload(S, ctx, n, dev):
    import torch
    import workloads as W
    t0 = time.time()
    p = W.config3(n) if n == 10_000_000 else W.clustered(n, W.blobs_for(n), seed=3)
    f32 = lambda a: torch.from_numpy(np.asarray(a, np.float32)).to(dev)
    pos, mass, vel, u = f32(p.pos), f32(p.mass), f32(p.vel), f32(p.u)
    params = S.default_params()
    # Store the particles in the grid's Morton order (as the paper's code keeps
    # its particles in Hilbert order), then build the grid used by the steps.
    g0 = S.sph_build_grid(ctx, pos, mass, params)
    perm = torch.empty(n, dtype=torch.int32, device=dev)
    S.sph_grid_export(g0, perm)
    g0.free()
    order = perm.long()
    pos, mass, vel, u = (t[order].contiguous() for t in (pos, mass, vel, u))
    grid = S.sph_build_grid(ctx, pos, mass, params)
    # converge h once (all active), then a force pass for the Courant estimate
    h = torch.zeros(n, device=dev)
    st = {"rho": torch.zeros(n, device=dev), "omega": torch.zeros(n, device=dev),
          "n_ngb": torch.zeros(n, dtype=torch.int32, device=dev), "flags": torch.zeros(n, dtype=torch.uint8, device=dev),
          "acc": torch.zeros(n, 3, device=dev), "dudt": torch.zeros(n, device=dev), "vsig": torch.zeros(n, device=dev)}
    S.sph_density(ctx, grid, h, None, st["rho"], st["omega"], st["n_ngb"], st["flags"], None, params)
    S.sph_hydro_force(ctx, grid, vel, u, h, st["rho"], st["omega"], None, st["acc"], st["dudt"], st["vsig"],
                      None, params)
    S.sph_sync_status(ctx)
    dt_c = (0.3 * h / st["vsig"].clamp_min(1e-30)).cpu().numpy()
    bins = W.timebins(dt_c)
    acts = [torch.from_numpy(a).to(dev) for a in W.active_sets(bins)]
    # per sub-step h guesses: the converged h, scattered log-normally on that
    # sub-step's active particles only (inactive neighbours keep their h)
    h_conv = h.cpu().numpy().astype(np.float64)
    h_ins = []
    for k, a in enumerate(W.active_sets(bins)):
        hk = h_conv.copy()
        hk[a] = W.perturb(h_conv[a], H_PERTURB, seed=20 + k)
        h_ins.append(torch.from_numpy(hk.astype(np.float32)).to(dev))
    return dict(pos=pos, mass=mass, vel=vel, u=u, h=h, st=st, grid=grid, acts=acts, h_ins=h_ins,
                setup_s=time.time() - t0, n=n)


def step_body(S, ctx, wl, dparams, fparams, spans=None):
    """One step: grid rebuild, then density + force for each sub-step's active
    set. With `spans`, CUDA events bracket the grid rebuild and each sub-step
    (the h copy that loads a sub-step's guesses stays outside)."""
    import torch
    st = wl["st"]

    def ev():
        e = torch.cuda.Event(enable_timing=True)
        e.record()
        return e

    a = ev() if spans is not None else None
    S.sph_grid_update(ctx, wl["grid"], wl["pos"], wl["mass"])
    if spans is not None:
        spans.append((a, ev()))
    for act, h_in in zip(wl["acts"], wl["h_ins"]):
        wl["h"].copy_(h_in)
        a = ev() if spans is not None else None
        S.sph_density(ctx, wl["grid"], wl["h"], act, st["rho"], st["omega"], st["n_ngb"], st["flags"], None, dparams)
        S.sph_hydro_force(ctx, wl["grid"], wl["vel"], wl["u"], wl["h"], st["rho"], st["omega"], act, st["acc"],
                          st["dudt"], st["vsig"], None, fparams)
        if spans is not None:
            spans.append((a, ev()))


def kernel_names(S, dflags, fflags):
    """Names of the density and force kernels that the given path flags select."""
    def pick(fl, names):
        if fl & S.SPH_PLAIN_FP32:
            return names[0]
        if fl & (S.SPH_PER_THREAD_WALK | S.SPH_DENSITY_BUFFERED | S.SPH_FP64):
            return names[1] if not (fl & S.SPH_DENSITY_BUFFERED) else "k_density_buf"
        return names[2]
    return (pick(dflags, ("k_density_plain", "k_density_tpp<float>", "k_density_mp + k_density_wpp")),
            pick(fflags, ("k_force_plain", "k_force_mask", "k_force_list + k_force_mp + k_force_wpp")))


def timed_steps(S, ctx, wl, dparams, fparams, steps, warmup, dist=None):
    """Eager steps, each timed as the sum of its event-bracketed parts."""
    import torch
    for _ in range(warmup):
        step_body(S, ctx, wl, dparams, fparams)
    S.sph_sync_status(ctx)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    ms, launches, dk, fk, dl, fl = 0.0, 0, 0.0, 0.0, 0, 0
    dpairs = fpairs = 0
    for _ in range(steps):
        spans = []
        step_body(S, ctx, wl, dparams, fparams, spans)
        rc, stt = S.sph_sync_status(ctx)
        ms += sum(a.elapsed_time(b) for a, b in spans)
        dpairs += stt["density_pairs"]
        fpairs += stt["force_pairs"]
        launches += stt["launches"]
        dk += stt["density_kernel_ms"]
        fk += stt["force_kernel_ms"]
        dl += stt["density_launches"]
        fl += stt["force_launches"]
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    return dict(ms=ms, pairs=dpairs + fpairs, dpairs=dpairs, fpairs=fpairs, launches=launches,
                dens_ms=dk, force_ms=fk, dens_launches=dl, force_launches=fl)


def graph_steps(S, ctx, wl, dparams, fparams, steps, warmup, dist=None):
    """The whole step captured once as a CUDA graph and replayed: one event
    pair around each replay (the sub-steps' h copies are inside the graph)."""
    import torch
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        step_body(S, ctx, wl, dparams, fparams)
    torch.cuda.current_stream().wait_stream(side)
    S.sph_sync_status(ctx)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        step_body(S, ctx, wl, dparams, fparams)
    _, cap = S.sph_sync_status(ctx)          # host count of the kernels put in the graph
    for _ in range(warmup):
        graph.replay()
    S.sph_sync_status(ctx)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    ms, pairs = 0.0, 0
    for _ in range(steps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        graph.replay()
        b.record()
        _, stt = S.sph_sync_status(ctx)
        ms += a.elapsed_time(b)
        pairs += stt["density_pairs"] + stt["force_pairs"]
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    return dict(ms=ms, pairs=pairs, launches=cap["launches"])


def e2e_steps(S, ctx, wl, dparams, fparams, steps):
    """Same step through the public API from pinned HOST buffers: H2D of the
    step's inputs and D2H of its results inside the timed region. The inputs
    travel on a copy stream in the order the step needs them (positions and
    masses, the first h guesses, then velocities, energies and the later
    guesses), so that only the first ones delay the grid rebuild; each
    sub-step waits for its own h guesses, the first force pass for v and u."""
    import torch
    n = wl["n"]
    hst = {k: wl[k].cpu().pin_memory() for k in ("pos", "mass", "vel", "u")}
    h_ins = [h.cpu().pin_memory() for h in wl["h_ins"]]
    h_dev = [torch.empty_like(wl["h"]) for _ in h_ins]
    outs = {k: torch.empty(wl["st"][k].shape, dtype=wl["st"][k].dtype).pin_memory()
            for k in ("rho", "omega", "acc", "dudt", "vsig")}
    h_out = torch.empty(n).pin_memory()
    st = wl["st"]
    h2d = sum(t.numel() * t.element_size() for t in hst.values()) + sum(t.numel() * 4 for t in h_ins)
    d2h = sum(t.numel() * t.element_size() for t in outs.values()) + n * 4
    main = torch.cuda.current_stream()
    cs = torch.cuda.Stream()
    pairs = 0
    torch.cuda.synchronize()
    t_ms = 0.0
    for _ in range(steps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        cs.wait_stream(main)   # the previous step is done with the input buffers
        with torch.cuda.stream(cs):
            wl["pos"].copy_(hst["pos"], non_blocking=True)
            wl["mass"].copy_(hst["mass"], non_blocking=True)
            e_pos = torch.cuda.Event()
            e_pos.record()
            e_h = []
            h_dev[0].copy_(h_ins[0], non_blocking=True)
            e_h.append(torch.cuda.Event())
            e_h[-1].record()
            wl["vel"].copy_(hst["vel"], non_blocking=True)
            wl["u"].copy_(hst["u"], non_blocking=True)
            e_vu = torch.cuda.Event()
            e_vu.record()
            for k in range(1, len(h_ins)):
                h_dev[k].copy_(h_ins[k], non_blocking=True)
                e_h.append(torch.cuda.Event())
                e_h[-1].record()
        main.wait_event(e_pos)
        S.sph_grid_update(ctx, wl["grid"], wl["pos"], wl["mass"])
        for k, act in enumerate(wl["acts"]):
            main.wait_event(e_h[k])
            S.sph_density(ctx, wl["grid"], h_dev[k], act, st["rho"], st["omega"], st["n_ngb"], st["flags"], None,
                          dparams)
            if k == 0:
                main.wait_event(e_vu)
            S.sph_hydro_force(ctx, wl["grid"], wl["vel"], wl["u"], h_dev[k], st["rho"], st["omega"], act,
                              st["acc"], st["dudt"], st["vsig"], None, fparams)
        for k in outs:
            outs[k].copy_(st[k], non_blocking=True)
        h_out.copy_(h_dev[-1], non_blocking=True)
        b.record()
        _, stt = S.sph_sync_status(ctx)
        t_ms += a.elapsed_time(b)
        pairs += stt["density_pairs"] + stt["force_pairs"]
    return dict(value=pairs / (t_ms / 1e3), unit=UNIT, h2d_bytes_per_step=int(h2d), d2h_bytes_per_step=int(d2h),
                ms_per_step=t_ms / steps)


def balsara_line(S, ctx, wl, dparams, fparams, reps=3):
    """Secondary line: the 100 % sub-step of the 10M clustered step with
    Balsara's switch (density + velocity divergence and curl, then the
    switched force), next to the same sub-step without it and with the
    time-dependent viscosity (per-particle alpha, seeded uniform in [0.1, 1],
    with the switch, plus the alpha rate)."""
    import torch
    st, n, dev = wl["st"], wl["n"], wl["h"].device
    act, h_in = wl["acts"][0], wl["h_ins"][0]
    dv, cv = torch.zeros(n, device=dev), torch.zeros(n, device=dev)
    gen = torch.Generator(device=dev).manual_seed(41)
    alpha = 0.1 + 0.9 * torch.rand(n, device=dev, generator=gen)
    dalpha = torch.zeros(n, device=dev)

    def switched():
        S.sph_density_divcurl(ctx, wl["grid"], wl["h"], act, st["rho"], st["omega"], st["n_ngb"], st["flags"], None,
                              wl["vel"], dv, cv, dparams)
        S.sph_hydro_force_balsara(ctx, wl["grid"], wl["vel"], wl["u"], wl["h"], st["rho"], st["omega"], dv, cv, act,
                                  st["acc"], st["dudt"], st["vsig"], None, fparams)

    def plain():
        S.sph_density(ctx, wl["grid"], wl["h"], act, st["rho"], st["omega"], st["n_ngb"], st["flags"], None, dparams)
        S.sph_hydro_force(ctx, wl["grid"], wl["vel"], wl["u"], wl["h"], st["rho"], st["omega"], act, st["acc"],
                          st["dudt"], st["vsig"], None, fparams)

    def visc():
        S.sph_density_divcurl(ctx, wl["grid"], wl["h"], act, st["rho"], st["omega"], st["n_ngb"], st["flags"], None,
                              wl["vel"], dv, cv, dparams)
        S.sph_hydro_force_visc(ctx, wl["grid"], wl["vel"], wl["u"], wl["h"], st["rho"], st["omega"], alpha, dv, cv,
                               act, st["acc"], st["dudt"], st["vsig"], None, fparams)
        S.sph_visc_rate(ctx, act, wl["h"], wl["u"], dv, alpha, dalpha)

    out = {}
    for name, fn in (("switched", switched), ("plain", plain), ("visc", visc)):
        wl["h"].copy_(h_in)
        fn()
        S.sph_sync_status(ctx)
        ms, pairs = 0.0, 0
        for _ in range(reps):
            wl["h"].copy_(h_in)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            _, stt = S.sph_sync_status(ctx)
            ms += a.elapsed_time(b)
            pairs += stt["density_pairs"] + stt["force_pairs"]
        out[name] = (pairs / (ms / 1e3), ms / reps)
    return {"workload": "10M clustered, 100 % active sub-step: density + velocity divergence and curl, "
                        "then the force with Balsara's switch",
            "value": out["switched"][0], "unit": UNIT, "ms_per_pass": out["switched"][1],
            "without_switch_ms_per_pass": out["plain"][1],
            "time_dependent_alpha_ms_per_pass": out["visc"][1]}


def conduction_line(S, ctx, wl, dparams, fparams, reps=3):
    """Secondary line: the 100 % sub-step of the 10M clustered step with
    thermal conduction in the force pass (conductivities log-uniform over a
    decade, seeded), next to the same force pass without it."""
    import torch
    st, n, dev = wl["st"], wl["n"], wl["h"].device
    act, h_in = wl["acts"][0], wl["h_ins"][0]
    kappa = torch.from_numpy((10.0 ** np.random.default_rng(9).uniform(-1, 0, n)).astype(np.float32)).to(dev)
    dc = torch.zeros(n, device=dev)
    wl["h"].copy_(h_in)
    S.sph_density(ctx, wl["grid"], wl["h"], act, st["rho"], st["omega"], st["n_ngb"], st["flags"], None, dparams)
    S.sph_sync_status(ctx)

    def cond():
        S.sph_hydro_force_conduction(ctx, wl["grid"], wl["vel"], wl["u"], wl["h"], st["rho"], st["omega"], None,
                                     None, kappa, act, st["acc"], st["dudt"], st["vsig"], dc, None, fparams)

    def plain():
        S.sph_hydro_force(ctx, wl["grid"], wl["vel"], wl["u"], wl["h"], st["rho"], st["omega"], act, st["acc"],
                          st["dudt"], st["vsig"], None, fparams)

    out = {}
    for name, fn in (("cond", cond), ("plain", plain)):
        fn()
        S.sph_sync_status(ctx)
        ms, pairs = 0.0, 0
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            _, stt = S.sph_sync_status(ctx)
            ms += a.elapsed_time(b)
            pairs += stt["force_pairs"]
        out[name] = (pairs / (ms / 1e3), ms / reps)
    return {"workload": "10M clustered, 100 % active sub-step: the force pass with thermal conduction "
                        "(from the density pass's neighbour lists)",
            "value": out["cond"][0], "unit": "force pairs/s", "ms_per_pass": out["cond"][1],
            "without_conduction_ms_per_pass": out["plain"][1]}


def kdk_line(S, ctx, wl, max_ticks=64):
    """Secondary line: one dt_max cycle of kick-drift-kick integration of the
    10M clustered gas on Courant time bins: drift and prediction of every
    particle, grid rebuild, density and force of the tick's active particles,
    kicks and re-binning, all on the device, with nothing read back per tick
    (the active list is padded to its capacity). The finest bin holds the
    smallest Courant step (no particle steps above its Courant limit);
    max_bin is the number of halvings from the median Courant step down to
    it, at most log2(max_ticks). The cycle runs once eagerly, then is
    captured as one CUDA graph and replayed."""
    import math
    import torch
    from paper_2003_10850_gb300.kdk import KDK
    st = wl["st"]
    dt_c = 0.3 * wl["h"] / st["vsig"].clamp_min(1e-30)
    dt_min = float(dt_c.min())
    dt_med = float(torch.quantile(dt_c[torch.randperm(wl["n"], device=dt_c.device)[:1_000_000]], 0.5))
    max_bin = max(1, min(int(math.log2(max_ticks)), math.ceil(math.log2(dt_med / dt_min))))
    dt_max = 2 ** max_bin * dt_min * 0.999
    g = KDK(ctx, wl["pos"].double(), wl["mass"], wl["vel"], wl["u"], dt_max, max_bin)
    ticks = 1 << max_bin
    # both timed cycles start from the state after the opening kick (one cycle
    # keeps every particle within its Courant limit; later ones need finer bins)
    names = ("pos", "vel", "u", "vel_pred", "u_pred", "h", "rho", "omega", "acc", "dudt", "vsig", "bins", "n_ngb",
             "flags")
    saved = {k: getattr(g, k).clone() for k in names}

    def restore():
        for k in names:
            getattr(g, k).copy_(saved[k])
        g.tick = 0

    def timed(fn):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        pairs0 = g.pairs
        a.record()
        fn()
        b.record()
        b.synchronize()
        g.collect()
        return a.elapsed_time(b), g.pairs - pairs0

    def eager():
        for _ in range(ticks):
            g.step(sync=False)

    eager_ms, _ = timed(eager)
    tc = g.tick_counts.cpu().tolist()
    counts = [tc[k % ticks] for k in range(1, ticks + 1)]
    restore()
    g.capture_cycle()
    timed(g.run_cycle)                      # warm-up replay
    restore()
    ms, pairs = timed(g.run_cycle)
    g.grid.free()
    return {"workload": f"10M clustered, kick-drift-kick on {max_bin + 1} Courant time bins, one dt_max cycle "
                        f"({ticks} ticks): drift + prediction, grid rebuild, density and force of the "
                        "active particles, kicks, re-binning; the cycle replayed as one CUDA graph",
            "value": pairs / (ms / 1e3), "unit": UNIT, "ms_per_cycle": ms, "eager_ms_per_cycle": eager_ms,
            "max_bin": max_bin, "dt_max": dt_max, "active_per_tick": counts}


def batched_line(S, ctx, dev, reps=3):
    """Secondary line: 64 independent boxes (N log-uniform in [4096, 524288])
    in one grid, density (from 2%-scattered converged h) + force, one launch
    per pass for all boxes."""
    import torch
    import workloads as W
    boxes = W.config4()
    offs = np.cumsum([0] + [b.n for b in boxes])
    cat = lambda k: torch.from_numpy(np.concatenate([getattr(b, k) for b in boxes]).astype(np.float32)).to(dev)
    pos, mass, vel, u = cat("pos"), cat("mass"), cat("vel"), cat("u")
    params = S.default_params()
    grid = S.sph_build_grid_batched(ctx, pos, mass, offs, [1.0] * len(boxes), params)
    n = int(offs[-1])
    h = torch.zeros(n, device=dev)
    d = S.density(ctx, grid, h, None, params)
    S.sph_sync_status(ctx)
    h_in = torch.from_numpy(W.perturb(h.cpu().numpy().astype(np.float64), H_PERTURB, 31).astype(np.float32)).to(dev)
    f = S.hydro_force(ctx, grid, vel, u, h, d["rho"], d["omega"], None, params)
    S.sph_sync_status(ctx)
    ms = 0.0
    pairs = 0
    for _ in range(reps):
        h.copy_(h_in)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        S.sph_density(ctx, grid, h, None, d["rho"], d["omega"], d["n_ngb"], d["flags"], None, params)
        S.sph_hydro_force(ctx, grid, vel, u, h, d["rho"], d["omega"], None, f["acc"], f["dudt"], f["vsig"], None, params)
        b.record()
        _, stt = S.sph_sync_status(ctx)
        ms += a.elapsed_time(b)
        pairs += stt["density_pairs"] + stt["force_pairs"]
    grid.free()
    return {"workload": "64 periodic boxes, N log-uniform in [4096, 524288] (seed 100+b), one grid, "
                        "all active, density + force", "n_total": n, "boxes": len(boxes),
            "value": pairs / (ms / 1e3), "unit": UNIT, "ms_per_pass": ms / reps}


def gravity_line(S, ctx, wl, reps=3):
    """Secondary line: the short-range gravity pass (Barnes-Hut walk,
    theta = 0.5) over the 10M clustered particles, all active, with the TreePM
    split of a mesh of one cell per mean particle spacing: r_s = 1.25 cells,
    r_cut = 4.5 r_s, spline softening 2.8 / 30 cells."""
    import torch
    n = wl["n"]
    cell = 1.0 / round(n ** (1.0 / 3.0))
    gp = S.gravity_params(G=1.0, theta=0.5, r_split=1.25 * cell, r_cut=4.5 * 1.25 * cell, h_soft=2.8 * cell / 30)
    acc = torch.zeros(n, 3, device=wl["h"].device)
    S.sph_gravity(ctx, wl["grid"], None, gp, acc)
    S.sph_sync_status(ctx)
    ms, nodes, pairs = 0.0, 0, 0
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        S.sph_gravity(ctx, wl["grid"], None, gp, acc)
        b.record()
        _, st = S.sph_sync_status(ctx)
        ms += a.elapsed_time(b)
        nodes += st["grav_nodes"]
        pairs += st["grav_pairs"]
    return {"workload": f"{n / 1e6:g}M clustered, all active: short-range gravity (TreePM split, r_s = 1.25 mean "
                        "spacings, r_cut = 4.5 r_s), Barnes-Hut walk at theta = 0.5, node moments included",
            "value": (nodes + pairs) / (ms / 1e3), "unit": "interactions/s", "ms_per_pass": ms / reps,
            "achieved_tflops": FLOPS_GRAV_INTERACTION * (nodes + pairs) / (ms / 1e3) / 1e12,
            "node_interactions_per_particle": nodes / reps / n, "pair_interactions_per_particle": pairs / reps / n}


def adjoint_line(S, ctx, dev, reps=3):
    """Secondary line: the differentiation workload (262,144 clustered
    particles): forward density + force, then sph_backward for the loss
    sum |a - a*|^2 + sum (rho - rho*)^2 with 1% scattered targets."""
    import torch
    import workloads as W
    p = W.config5()
    f32 = lambda a: torch.from_numpy(np.asarray(a, np.float32)).to(dev)
    pos, mass, vel, u = f32(p.pos), f32(p.mass), f32(p.vel), f32(p.u)
    params = S.default_params()
    grid = S.sph_build_grid(ctx, pos, mass, params)
    h = torch.zeros(p.n, device=dev)
    d = S.density(ctx, grid, h, None, params)
    f = S.hydro_force(ctx, grid, vel, u, h, d["rho"], d["omega"], None, params)
    _, stt = S.sph_sync_status(ctx)
    rng = np.random.default_rng(5)
    g_acc = 2 * (f["acc"] - f["acc"] * (1 + 0.01 * torch.from_numpy(rng.normal(size=(p.n, 1))).float().to(dev)))
    g_rho = 2 * (d["rho"] - d["rho"] * (1 + 0.01 * torch.from_numpy(rng.normal(size=p.n)).float().to(dev)))
    g_pos = torch.empty(p.n, 3, device=dev)
    g_u = torch.empty(p.n, device=dev)
    g_m = torch.empty(p.n, device=dev)
    S.sph_backward(ctx, grid, vel, u, h, d["rho"], d["omega"], g_acc, g_rho, g_pos, g_u, g_m, params)
    S.sph_sync_status(ctx)
    ms = 0.0
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        S.sph_backward(ctx, grid, vel, u, h, d["rho"], d["omega"], g_acc, g_rho, g_pos, g_u, g_m, params)
        b.record()
        S.sph_sync_status(ctx)
        ms += a.elapsed_time(b)
    grid.free()
    return {"workload": "262,144 clustered (seed 5), loss |a-a*|^2 + (rho-rho*)^2, all active",
            "backward_ms": ms / reps, "force_pairs": stt["force_pairs"],
            "pair_visits_per_s": 3 * stt["force_pairs"] / (ms / reps / 1e3)}


def over_ranks(ms_step, pairs_step, dist, device):
    """Whole-job figures of a run of independent replicas, one per rank: the
    slowest rank's time per step and the pairs of all ranks (no data moves
    between ranks but these two numbers)."""
    if dist is None:
        return ms_step, pairs_step
    import torch
    t = torch.tensor([ms_step, pairs_step], dtype=torch.float64, device=device)
    mx = t.clone()
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    sm = t.clone()
    dist.all_reduce(sm, op=dist.ReduceOp.SUM)
    return float(mx[0]), float(sm[1])


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    import torch
    dist = None
    if world > 1:
        import torch.distributed as tdist
        tdist.init_process_group("nccl", device_id=torch.device("cuda", local))
        dist = tdist
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2003_10850_gb300 import build as B
    if rank == 0 or world == 1:
        B.build()
    if dist is not None:
        dist.barrier()
    import paper_2003_10850_gb300 as S
    from paper_2003_10850_gb300 import autotune
    ctx = S.Context(local)
    wl = setup_workload(S, ctx, args.n, dev)
    if args.gravity_only:
        if rank == 0:
            print(json.dumps({"gravity": gravity_line(S, ctx, wl)}), flush=True)
        return
    # launch shapes per pass, tuned on the 100 % sub-step
    setup_s = wl["setup_s"]
    dpar, fpar, tuned = autotune.tune(ctx, wl["grid"], wl["st"], wl["vel"], wl["u"], wl["h"], wl["h_ins"][0],
                                      tag="clustered-100pct")
    # the group span of the member-parallel kernels, tuned on the 10 % sub-step
    span, span_rep = autotune.tune_group_span(ctx, wl["grid"], wl["st"], wl["vel"], wl["u"], wl["h"], wl["h_ins"][1],
                                              wl["acts"][1], dpar, fpar, tag="clustered-10pct")
    dpar.group_size = span
    fpar.group_size = span
    tuned["group_span"] = span_rep
    dtime = S.default_params(flags=dpar.flags | S.SPH_TIME_KERNELS, blocks_per_sm=dpar.blocks_per_sm,
                             walk_radius=dpar.walk_radius, group_size=span)
    ftime = S.default_params(flags=fpar.flags | S.SPH_TIME_KERNELS, blocks_per_sm=fpar.blocks_per_sm,
                             walk_radius=fpar.walk_radius, group_size=span)

    clocks = Clocks(local)
    res_g = graph_steps(S, ctx, wl, dpar, fpar, args.steps, args.warmup, dist)
    clk = clocks.stop()
    res = timed_steps(S, ctx, wl, dtime, ftime, args.steps, max(1, args.warmup // 3), dist)

    ms_step = res_g["ms"] / args.steps
    pairs_step = res_g["pairs"] / args.steps
    active_per_launch = sum(int(a.numel()) for a in wl["acts"]) / len(wl["acts"])
    ms_step, pairs_total = over_ranks(ms_step, pairs_step, dist, dev)
    value = pairs_total / (ms_step / 1e3)

    plain = None
    if not args.no_plain and rank == 0:
        pp = S.default_params(flags=S.SPH_PLAIN_FP32)
        k2 = max(1, min(2, args.steps))
        r2 = timed_steps(S, ctx, wl, pp, pp, k2, 1)
        plain = {"value": r2["pairs"] / (r2["ms"] / 1e3), "ms_per_step": r2["ms"] / k2, "unit": UNIT,
                 "kind": "thread per particle, FP32 sums, h iterated by the host, eager launches"}
    e2e = None
    if not args.no_e2e:
        e2e = e2e_steps(S, ctx, wl, dpar, fpar, max(1, min(3, args.steps)))
    extra = {}
    if not args.no_extra and rank == 0:
        extra["balsara"] = balsara_line(S, ctx, wl, dpar, fpar)
        extra["conduction"] = conduction_line(S, ctx, wl, dpar, fpar)
        extra["gravity"] = gravity_line(S, ctx, wl)
        extra["kdk"] = kdk_line(S, ctx, wl)
        del wl
        torch.cuda.empty_cache()
        extra["batched_boxes"] = batched_line(S, ctx, dev)
        extra["adjoint"] = adjoint_line(S, ctx, dev)

    pk, src = peaks()
    props = torch.cuda.get_device_properties(dev)
    sm_count = props.multi_processor_count
    peak_tf = sm_count * FP32_LANES_PER_SM * 2 * pk.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    dens_f = res["dpairs"] * FLOPS_DENSITY_PAIR
    force_f = res["fpairs"] * FLOPS_FORCE_PAIR
    dname, fname = kernel_names(S, dpar.flags, fpar.flags)
    if res["dens_ms"] >= res["force_ms"]:
        kern, flops, kms, kl = dname, dens_f, res["dens_ms"], res["dens_launches"]
    else:
        kern, flops, kms, kl = fname, force_f, res["force_ms"], res["force_launches"]
    achieved = (flops / max(kl, 1)) / (kms / max(kl, 1) / 1e3) / 1e12 if kms > 0 else None
    traffic = DENSITY_DRAM_BYTES_PER_ACTIVE * active_per_launch if kern == dname else None
    roofline = {"bound": "alu", "kernel": kern, "achieved": achieved, "peak": peak_tf, "unit": "TFLOP/s",
                "frac": achieved / peak_tf if achieved else None, "traffic": traffic,
                "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of the 2M 100 % density "
                                  "launches (both kernels), per active particle, times the mean active particles "
                                  "of a timed launch"
                                  if traffic else None,
                "peak_source": f"{sm_count} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 x "
                               f"{pk.get('sm_max_mhz', 2070.0)} MHz ({src} max SM clock)",
                "dram_gbs": (traffic / (kms / max(kl, 1) / 1e3) / 1e9) if traffic and kms > 0 else None,
                "dram_gbs_source": "traffic / the launch's CUDA-event time" if traffic else None,
                "fma_pipe_pct": DENSITY_NCU_2M["fma_pipe_pct"] if kern == dname else None,
                "alu_pipe_pct": DENSITY_NCU_2M["alu_pipe_pct"] if kern == dname else None,
                "warp_inst_per_pair": (DENSITY_NCU_2M["warp_inst"] / DENSITY_NCU_2M["density_pairs"]
                                       if kern == dname else None),
                "ncu_2M": {**DENSITY_NCU_2M, "dram_gbs": DENSITY_NCU_2M["dram_bytes"] / (DENSITY_NCU_2M["ms"] / 1e3) / 1e9,
                           "note": "pipe percentages of k_density_mp (sm__pipe_fma/alu_cycles_active, pct of "
                                   "peak sustained active); durations serialised under ncu"}
                if kern == dname else None,
                "density_kernel_ms_per_step": res["dens_ms"] / args.steps,
                "force_kernel_ms_per_step": res["force_ms"] / args.steps,
                "density_tflops": dens_f / (res["dens_ms"] / 1e3) / 1e12 if res["dens_ms"] else None,
                "force_tflops": force_f / (res["force_ms"] / 1e3) / 1e12 if res["force_ms"] else None}

    cpu = None
    if not args.no_cpu and rank == 0 and world == 1:
        import oracle
        oracle.build()
        s = oracle_sample(args.cpu_n)
        pr, dt = oracle_step(s)
        cpu = {"value": pr / dt, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle", **host_cores(),
               "sample": f"same generator at N={args.cpu_n} (blobs ~ sqrt N), all active, density from "
                         f"perturbed converged h + force, one step, {dt:.1f} s"}
        # the same step on one core, on a sixteenth of the sample
        n1 = max(4096, args.cpu_n // 16)
        s1 = oracle_sample(n1)
        prev = oracle.set_threads(1)
        pr1, dt1 = oracle_step(s1)
        oracle.set_threads(prev)
        cpu["one_core"] = {"value": pr1 / dt1, "unit": UNIT, "cores": 1,
                           "sample": f"same generator at N={n1}, one step, {dt1:.1f} s"}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": "10M clustered gas particles (500 blobs, seed 3), time bins giving "
                                       "100/10/1/0.1% active sub-steps; grid rebuild + density (h iteration) "
                                       "+ hydro force per sub-step; whole step replayed as one CUDA graph",
                           "n": args.n, "pairs_per_step": pairs_step, "l2": "inputs exceed L2 (>1 GB)",
                           "parallelism": f"replicas x{world}" if world > 1 else "1 GPU",
                           "h_guess_scatter": H_PERTURB,
                           "tuned": {"density": tuned["density"], "force": tuned["force"],
                                     "group_span": tuned["group_span"]["group_size"]},
                           "eager_ms_per_step": res["ms"] / args.steps,
                           "eager_value": res["pairs"] / (res["ms"] / 1e3)},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": int(res_g["launches"]), "clocks": clk,
                "plain_fp32": plain, "speedup_vs_plain": (value / plain["value"]) if plain else None,
                "setup_s": setup_s}
        line.update(extra)
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
