"""Shared helpers for the GPU parity tests: run the CUDA path through the
C ABI and the FP64 oracle on the same seeded inputs.

Inputs are rounded to float32 once (positions, masses, velocities, u) and both
sides see exactly those values: the library gets the float32 arrays, the
oracle their exact float64 copies. Nothing the CUDA path computes is ever fed
to the oracle.
"""
from __future__ import annotations

import numpy as np
import torch

import oracle
import workloads as W

GAMMA = 5.0 / 3.0


def as_f32(p: W.Particles) -> W.Particles:
    f = lambda a: np.asarray(a, dtype=np.float32).astype(np.float64)
    pos = f(p.pos)
    pos[pos >= p.box] -= p.box  # float32 rounding can land exactly on L
    return W.Particles(pos, f(p.vel), f(p.mass), f(p.u), p.box)


def dev(a, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda").to(dtype)


def host(t):
    return t.detach().cpu().numpy()


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return np.abs(a - b) / np.maximum(np.abs(b), 1e-300)


def oracle_all(p: W.Particles, n_target=64.0, alpha=1.0, active=None, brute=False):
    X = oracle.quantize(p.pos, p.box)
    d = oracle.density(X, p.mass, None, box=p.box, n_target=n_target, tol=1e-10, brute=brute)
    f = oracle.force(X, p.vel, p.mass, p.u, d["h"], d["rho"], d["omega"], box=p.box, alpha=alpha,
                     active=active, brute=brute)
    return X, d, f


def gpu_grid(S, ctx, p: W.Particles, params, pos64=False):
    pos = dev(p.pos, torch.float64 if pos64 else torch.float32)
    return S.sph_build_grid(ctx, pos, dev(p.mass), params)


def gpu_density(S, ctx, grid, h0, params, active=None):
    h = dev(h0)
    act = None if active is None else dev(active, torch.int32)
    out = S.density(ctx, grid, h, act, params, want_hash=True)
    rc, stats = S.sph_sync_status(ctx, raise_on_error=False)
    res = {k: host(v) for k, v in out.items()}
    res["h"] = host(h)
    res["hash"] = res["hash"].view(np.uint64)
    res["rc"], res["stats"] = rc, stats
    return res


def gpu_force(S, ctx, grid, p: W.Particles, h, rho, omega, params, active=None):
    act = None if active is None else dev(active, torch.int32)
    out = S.hydro_force(ctx, grid, dev(p.vel), dev(p.u), dev(h), dev(rho), dev(omega), act, params,
                        want_hash=True)
    rc, stats = S.sph_sync_status(ctx, raise_on_error=False)
    res = {k: host(v) for k, v in out.items()}
    res["hash"] = res["hash"].view(np.uint64)
    res["rc"], res["stats"] = rc, stats
    return res


def check_force(g, f, idx, tol, check_hash=True):
    """|delta a| <= tol * S_a and |delta du| <= tol * S_u per particle (S = sum of
    the magnitudes of the pair terms), v_sig relative, pair sets exact."""
    da = np.linalg.norm(g["acc"][idx] - f["acc"][idx], axis=1)
    assert np.all(da <= tol * f["scale_a"][idx] + 1e-30), (da / f["scale_a"][idx]).max()
    ddu = np.abs(g["dudt"][idx] - f["dudt"][idx])
    assert np.all(ddu <= tol * f["scale_u"][idx] + 1e-30), (ddu / f["scale_u"][idx]).max()
    dv = np.abs(g["vsig"][idx] - f["vsig"][idx])
    assert np.all(dv <= max(tol / 10, 2e-6) * (np.abs(f["vsig"][idx]) + np.median(f["vsig"][idx])))
    if check_hash:
        assert np.array_equal(g["hash"][idx], f["hash"][idx])
