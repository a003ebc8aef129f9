"""Kick-drift-kick integration on power-of-two time bins.

The paper's code advances each particle on its own power-of-two time step
(Sec. 2.2, adaptive time steps): at every tick of the smallest step only the
particles whose step ends are active; every particle, inactive neighbours
included, is drifted to the current time. `KDK` sequences the library calls
of one tick; all arithmetic runs in the library's kernels:

  drift and prediction (sph_drift) -> grid rebuild (sph_grid_update) ->
  active set of the tick (sph_active_from_bins) -> density and force of that
  set at the predicted velocities and energies -> closing half kick, which
  resets the predictions to the synchronized values (sph_kick) -> new bins
  (sph_timebins) -> opening half kick.

Inactive particles keep the h, rho, Omega, a, du/dt of their last active
step; their velocities and energies are predicted to the current time with
those. Nothing is read back per tick: sph_active_from_bins pads the active
list with -1 to its capacity n, and every call takes the whole list
(n_active = n), skipping the padding on the device. So a whole dt_max cycle
can be captured as one CUDA graph (capture_cycle) and replayed (run_cycle).

Options: balsara=True limits the viscosity with Balsara's switch (div v and
curl v from sph_density_divcurl); visc=dict(alpha0, alpha_min, alpha_max,
ell) gives each particle its own viscosity parameter (sph_hydro_force_visc),
whose rate (sph_visc_rate, Morris & Monaghan) is kicked and predicted like
du/dt (sph_kick_scalar, sph_predict_scalar).
"""
from __future__ import annotations

import torch

from . import (default_params, sph_active_from_bins, sph_build_grid, sph_density, sph_density_divcurl, sph_drift,
               sph_grid_update, sph_hydro_force, sph_hydro_force_balsara, sph_hydro_force_visc, sph_kick,
               sph_kick_scalar, sph_predict_scalar, sph_sync_status, sph_timebins, sph_visc_rate)


class KDK:
    """State of one periodic box: pos (n, 3) float64, vel (n, 3) float32,
    mass, u float32 device tensors (copied). The time step of bin b is
    dt_max / 2^b, b in [0, max_bin]. `bins` (uint8, n) fixes the bins (no
    re-binning) if given; otherwise they come from the Courant step
    courant * h / v_sig and are re-assigned at the end of every step. A
    particle whose Courant step is below dt_max / 2^max_bin is held at
    max_bin, above its Courant limit: choose dt_max and max_bin so that the
    finest bin holds the smallest step."""

    def __init__(self, ctx, pos, mass, vel, u, dt_max, max_bin, params=None, courant=0.3, bins=None, balsara=False,
                 visc=None):
        self.ctx = ctx
        self.params = params or default_params()
        self.box = float(self.params.box)
        self.dt_max = float(dt_max)
        self.max_bin = int(max_bin)
        self.courant = float(courant)
        self.rebin = bins is None
        dev = pos.device
        self.pos = pos.to(torch.float64).contiguous().clone()
        self.mass = mass.to(torch.float32).contiguous().clone()
        self.vel = vel.to(torch.float32).contiguous().clone()
        self.u = u.to(torch.float32).contiguous().clone()
        self.vel_pred = self.vel.clone()
        self.u_pred = self.u.clone()
        n = self.n = self.pos.shape[0]
        f = lambda: torch.zeros(n, device=dev)
        self.h, self.rho, self.omega, self.dudt, self.vsig = f(), f(), f(), f(), f()
        self.acc = torch.zeros(n, 3, device=dev)
        self.n_ngb = torch.zeros(n, dtype=torch.int32, device=dev)
        self.balsara, self.visc = bool(balsara), visc
        if self.balsara or visc is not None:
            self.divv, self.curlv = f(), f()
        if visc is not None:
            self.alpha = torch.full((n,), float(visc["alpha0"]), device=dev)
            self.alpha_pred = self.alpha.clone()
            self.dalpha = f()
        self.flags = torch.zeros(n, dtype=torch.uint8, device=dev)
        self.active = torch.zeros(n, dtype=torch.int32, device=dev)
        self.count = torch.zeros(1, dtype=torch.int32, device=dev)
        # active count of each tick of a cycle (device; tick k at k mod 2^max_bin)
        self.tick_counts = torch.zeros(1 << self.max_bin, dtype=torch.int32, device=dev)
        self.grid = sph_build_grid(ctx, self.pos, self.mass, self.params)
        self.tick = 0
        self.pairs = 0
        self.graph = None
        everyone = torch.arange(n, dtype=torch.int32, device=dev)
        self._forces(everyone)
        self.collect()
        if bins is None:
            self.bins = torch.zeros(n, dtype=torch.uint8, device=dev)
            sph_timebins(ctx, self.h, self.vsig, None, 0, self.courant, self.dt_max, self.max_bin, self.bins)
        else:
            self.bins = bins.to(torch.uint8).contiguous().clone()
        self._kick(everyone, 0.5)          # opening half kick of every particle

    def dt_bins(self, factor=1.0):
        return [factor * self.dt_max / 2.0 ** b for b in range(self.max_bin + 1)]

    def _forces(self, act):
        ctx, g = self.ctx, self.grid
        if self.balsara or self.visc is not None:
            sph_density_divcurl(ctx, g, self.h, act, self.rho, self.omega, self.n_ngb, self.flags, None,
                                self.vel_pred, self.divv, self.curlv, self.params)
        else:
            sph_density(ctx, g, self.h, act, self.rho, self.omega, self.n_ngb, self.flags, None, self.params)
        if self.visc is not None:
            sw = (self.divv, self.curlv) if self.balsara else (None, None)
            sph_hydro_force_visc(ctx, g, self.vel_pred, self.u_pred, self.h, self.rho, self.omega, self.alpha_pred,
                                 *sw, act, self.acc, self.dudt, self.vsig, None, self.params)
            v = self.visc
            sph_visc_rate(ctx, act, self.h, self.u_pred, self.divv, self.alpha_pred, self.dalpha, self.params.gamma,
                          v["alpha_min"], v["alpha_max"], v["ell"])
        elif self.balsara:
            sph_hydro_force_balsara(ctx, g, self.vel_pred, self.u_pred, self.h, self.rho, self.omega, self.divv,
                                    self.curlv, act, self.acc, self.dudt, self.vsig, None, self.params)
        else:
            sph_hydro_force(ctx, g, self.vel_pred, self.u_pred, self.h, self.rho, self.omega, act, self.acc,
                            self.dudt, self.vsig, None, self.params)

    def collect(self):
        """Reads and clears the context's device counters (a host
        synchronisation); adds the pairs they counted to self.pairs."""
        _, st = sph_sync_status(self.ctx)
        self.pairs += st["density_pairs"] + st["force_pairs"]

    def _kick(self, act, factor, sync=False):
        sph_kick(self.ctx, act, act.numel(), self.bins, self.dt_bins(factor), self.acc, self.dudt, self.vel, self.u,
                 self.vel_pred if sync else None, self.u_pred if sync else None)
        if self.visc is not None:
            sph_kick_scalar(self.ctx, act, act.numel(), self.bins, self.dt_bins(factor), self.dalpha, self.alpha,
                            self.alpha_pred if sync else None)

    def step(self, sync=True):
        """Advance one tick (dt_max / 2^max_bin). With sync (a host round
        trip) the device counters are collected and the active count is
        returned; without, nothing is read back and the count stays in
        self.count and self.tick_counts."""
        ctx = self.ctx
        dt = self.dt_max / 2.0 ** self.max_bin
        sph_drift(ctx, self.pos, self.vel, dt, self.box, self.acc, self.dudt, self.vel_pred, self.u_pred)
        if self.visc is not None:
            sph_predict_scalar(ctx, dt, self.dalpha, self.alpha_pred)
        self.tick += 1
        sph_grid_update(ctx, self.grid, self.pos, self.mass)
        # the active particles, then -1 up to n: every call below takes the whole list
        sph_active_from_bins(ctx, self.grid, self.bins, self.tick, self.max_bin, self.active, self.count)
        act = self.active
        self._forces(act)
        self._kick(act, 0.5, sync=True)   # closing half kick: synchronized v, u become the predictions
        if self.rebin:
            sph_timebins(ctx, self.h, self.vsig, act, self.tick, self.courant, self.dt_max, self.max_bin, self.bins)
        self._kick(act, 0.5)           # opening half kick of the next step
        self.tick_counts[self.tick % (1 << self.max_bin)].copy_(self.count[0])
        if sync:
            self.collect()
            return int(self.count.item())
        return None

    def capture_cycle(self):
        """Captures the ticks of one dt_max cycle (2^max_bin of them) as a CUDA
        graph, at a cycle boundary. The decisions depend on the tick only
        modulo 2^max_bin, so run_cycle may replay it at every later boundary.
        Capturing runs nothing."""
        if self.tick % (1 << self.max_bin):
            raise RuntimeError("capture_cycle: not at a cycle boundary")
        t0 = self.tick
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.stream(side):
            with torch.cuda.graph(self.graph, stream=side):
                for _ in range(1 << self.max_bin):
                    self.step(sync=False)
        torch.cuda.current_stream().wait_stream(side)
        self.tick = t0

    def run_cycle(self):
        """Replays the captured cycle (no host round trip)."""
        if self.graph is None or self.tick % (1 << self.max_bin):
            raise RuntimeError("run_cycle: capture_cycle first, at a cycle boundary")
        self.graph.replay()
        self.tick += 1 << self.max_bin

    def synchronized_velocity(self):
        """Velocities at the current time: the half kick of every particle's
        running step taken back (exact at the end of a dt_max cycle)."""
        v = self.vel.clone()
        u = self.u.clone()
        everyone = torch.arange(self.n, dtype=torch.int32, device=self.vel.device)
        sph_kick(self.ctx, everyone, self.n, self.bins, self.dt_bins(-0.5), self.acc, self.dudt, v, u)
        return v, u

    def synchronized_alpha(self):
        """Viscosity parameters at the current time (as synchronized_velocity)."""
        a = self.alpha.clone()
        everyone = torch.arange(self.n, dtype=torch.int32, device=a.device)
        sph_kick_scalar(self.ctx, everyone, self.n, self.bins, self.dt_bins(-0.5), self.dalpha, a)
        return a
