"""FP64 kick-drift-kick integrator on power-of-two time bins (the paper's
adaptive time steps, Sec. 2.2), over the oracle's density and force passes.

TEST INFRASTRUCTURE ONLY (tests/ may import it). It shares no code with the
CUDA library.

The scheme, in the order the steps are taken:
  * time bins b in [0, max_bin], step dt_max / 2^b; the timeline counts
    ticks of dt_max / 2^max_bin; a particle in bin b ends a step at every
    tick that is a multiple of 2^(max_bin - b);
  * start: density and force for all, then the opening half kick
    v += a dt_b / 2, u += du/dt dt_b / 2;
  * each tick: drift every particle x += v dt_tick (periodic) and predict
    its velocity and energy to the new time, v_pred += a dt_tick,
    u_pred += du/dt dt_tick; then for the particles whose step ends: density
    (from their current h) and force at (x, v_pred, u_pred), the closing half
    kick (after which v, u are the synchronized values, which become v_pred,
    u_pred), and the opening half kick of the next step.
Inactive particles keep the h, rho, Omega, a, du/dt of their last step. The
prediction keeps the scheme second order although the force depends on v
(viscosity, du/dt) and u (pressure). Bins are given (the same bins for both
sides of a comparison).

Options: balsara=True limits the viscosity with Balsara's switch (div v and
curl v from the density pass's neighbours); visc=dict(alpha0, alpha_min,
alpha_max, ell) gives every particle its own viscosity parameter alpha, with
the rate of Morris & Monaghan (1997) (oracle.visc_rate) evaluated with the
force and integrated like u: kicked, predicted, reset at the closing kick.
"""
from __future__ import annotations

import numpy as np

from . import density, divcurl, force, quantize, visc_rate


def timebins(h, vsig, courant, dt_max, max_bin, tick=0):
    """The Courant bin rule in FP32 with correctly rounded operations: the
    smallest b with dt_max <= dt 2^b, dt = courant * h / vsig (max_bin if
    none, 0 if vsig <= 0), raised until the tick is on the bin's boundary."""
    h32 = np.asarray(h, np.float32)
    vs32 = np.asarray(vsig, np.float32)
    c32, dm32 = np.float32(courant), np.float32(dt_max)
    bins = np.zeros(h32.shape, np.uint8)
    for i in range(h32.size):
        b = 0
        if vs32[i] > 0:
            dt = np.float32(np.float32(c32 * h32[i]) / vs32[i])
            while b < max_bin and not (dm32 <= np.float32(np.ldexp(dt, b))):
                b += 1
        while b < max_bin and tick % (1 << (max_bin - b)) != 0:
            b += 1
        bins[i] = b
    return bins


class KDK:
    def __init__(self, pos, vel, mass, u, bins, dt_max, max_bin, box=1.0, n_target=64.0, alpha=1.0,
                 gamma=5.0 / 3.0, balsara=False, visc=None):
        self.pos = np.array(pos, np.float64)
        self.vel = np.array(vel, np.float64)
        self.mass = np.array(mass, np.float64)
        self.u = np.array(u, np.float64)
        self.bins = np.array(bins, np.int64)
        self.dt_max, self.max_bin, self.box = float(dt_max), int(max_bin), float(box)
        self.n_target, self.alpha, self.gamma = n_target, alpha, gamma
        self.balsara, self.visc = bool(balsara), visc
        n = self.pos.shape[0]
        self.h = np.zeros(n)
        self.rho = np.zeros(n)
        self.omega = np.zeros(n)
        self.acc = np.zeros((n, 3))
        self.dudt = np.zeros(n)
        self.vsig = np.zeros(n)
        self.scale_a = np.zeros(n)   # sum over force evaluations of scale_a * |dt kicked with it|
        self.scale_u = np.zeros(n)
        self.tick = 0
        self.vel_pred = self.vel.copy()
        self.u_pred = self.u.copy()
        self.divv = np.zeros(n)
        self.curlv = np.zeros(n)
        if visc is not None:
            self.av = np.full(n, float(visc["alpha0"]))   # the viscosity parameter, kicked like u
            self.av_pred = self.av.copy()
            self.dav = np.zeros(n)
        self._forces(np.arange(n))
        self._kick(np.arange(n), 0.5)

    def dt_bin(self, idx):
        return self.dt_max / 2.0 ** self.bins[idx]

    def _forces(self, act):
        X = quantize(self.pos, self.box)
        d = density(X, self.mass, self.h, box=self.box, n_target=self.n_target, tol=1e-10, active=act)
        for k in ("h", "rho", "omega"):
            getattr(self, k)[act] = d[k][act]
        sw = {}
        if self.balsara or self.visc is not None:
            dv, cv = divcurl(X, self.vel_pred, self.mass, self.h, self.rho, box=self.box, active=act)
            self.divv[act], self.curlv[act] = dv[act], cv[act]
            if self.balsara:
                sw = {"divv": self.divv, "curlv": self.curlv}
        alpha = self.alpha if self.visc is None else self.av_pred
        f = force(X, self.vel_pred, self.mass, self.u_pred, self.h, self.rho, self.omega, box=self.box,
                  alpha=alpha, gamma=self.gamma, active=act, **sw)
        if self.visc is not None:
            v = self.visc
            self.dav[act] = visc_rate(self.h[act], self.u_pred[act], self.divv[act], self.av_pred[act],
                                      v["alpha_min"], v["alpha_max"], v["ell"], self.gamma)
        self.acc[act] = f["acc"][act]
        self.dudt[act] = f["dudt"][act]
        self.vsig[act] = f["vsig"][act]
        self._sa, self._su = f["scale_a"], f["scale_u"]

    def _kick(self, act, factor, sync=False):
        dt = factor * self.dt_bin(act)
        self.vel[act] += self.acc[act] * dt[:, None]
        self.u[act] += self.dudt[act] * dt
        self.scale_a[act] += self._sa[act] * np.abs(dt)
        self.scale_u[act] += self._su[act] * np.abs(dt)
        if self.visc is not None:
            self.av[act] += self.dav[act] * dt
        if sync:   # the kicked values are the synchronized ones: the new predictions
            self.vel_pred[act] = self.vel[act]
            self.u_pred[act] = self.u[act]
            if self.visc is not None:
                self.av_pred[act] = self.av[act]

    def step(self):
        dt = self.dt_max / 2.0 ** self.max_bin
        self.pos = np.mod(self.pos + self.vel * dt, self.box)
        self.pos[self.pos >= self.box] -= self.box
        self.vel_pred += self.acc * dt
        self.u_pred += self.dudt * dt
        if self.visc is not None:
            self.av_pred += self.dav * dt
        self.tick += 1
        act = np.nonzero(self.tick % (1 << (self.max_bin - self.bins)) == 0)[0]
        if act.size:
            self._forces(act)
            self._kick(act, 0.5, sync=True)
            self._kick(act, 0.5)
        return act.size

    def synchronized_velocity(self):
        dt = -0.5 * self.dt_bin(np.arange(self.pos.shape[0]))
        return self.vel + self.acc * dt[:, None], self.u + self.dudt * dt

    def synchronized_alpha(self):
        return self.av - 0.5 * self.dav * self.dt_bin(np.arange(self.pos.shape[0]))
