"""GB300-native SPH neighbour-interaction hot path (density + hydro force).

Python face of the C ABI in include/sph.h. The functions below carry the C
names and only marshal arguments: tensors must be contiguous CUDA tensors of
the stated dtype, and every computation runs in libsph_gb300.so on the
current CUDA stream.
"""
from __future__ import annotations

import ctypes

import torch

from . import abi
from .abi import (SPH_FIXED_H, SPH_FP64, SPH_H_GUESS, SPH_PLAIN_FP32, SPH_TIME_KERNELS, SPH_WARP_GROUP, SPH_DENSITY_BUFFERED, SPH_PER_THREAD_WALK, SPH_COOP_WALK, SPH_WARP_WALK, SPH_NO_LISTS, SPH_PARTIAL_LISTS, SPHError,
                  default_params, sph_gravity_params, sph_params, sph_stats)

__all__ = ["Context", "Grid", "sph_create", "sph_build_grid", "sph_build_grid_batched", "sph_grid_update",
           "sph_density", "sph_hydro_force", "sph_density_divcurl", "sph_hydro_force_balsara",
           "sph_hydro_force_conduction", "sph_hydro_force_visc", "sph_visc_rate", "sph_kick_scalar",
           "sph_predict_scalar", "sph_gravity", "gravity_params", "sph_gravity_params", "sph_timebins", "sph_active_from_bins", "sph_kick", "sph_drift",
           "sph_backward", "sph_sync_status", "sph_grid_export", "sph_sort_keys_static", "density",
           "hydro_force", "default_params", "sph_params", "sph_stats", "SPHError", "SPH_FP64",
           "SPH_PLAIN_FP32", "SPH_FIXED_H", "SPH_H_GUESS", "SPH_TIME_KERNELS", "SPH_WARP_GROUP", "SPH_DENSITY_BUFFERED", "SPH_PER_THREAD_WALK", "SPH_COOP_WALK", "SPH_WARP_WALK", "SPH_NO_LISTS", "SPH_PARTIAL_LISTS"]


def _ptr(t, dtype=None, name="tensor"):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise TypeError(f"{name} must be contiguous")
    if dtype is not None and t.dtype not in (dtype if isinstance(dtype, tuple) else (dtype,)):
        raise TypeError(f"{name} must have dtype {dtype}, got {t.dtype}")
    return ctypes.c_void_p(t.data_ptr())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


class Context:
    """An sph_ctx on one CUDA device."""

    def __init__(self, device: int = 0):
        self.lib = abi.load()
        self.device = device
        self.handle = ctypes.c_void_p()
        st = self.lib.sph_create(ctypes.byref(self.handle), int(device))
        if st != 0:
            raise SPHError(st, "sph_create failed")

    def check(self, st: int):
        if st != 0:
            raise SPHError(st, self.lib.sph_last_error(self.handle).decode())

    def close(self):
        if self.handle:
            self.lib.sph_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Grid:
    """An sph_grid built by sph_build_grid*."""

    def __init__(self, ctx: Context, handle: ctypes.c_void_p, n: int):
        self.ctx, self.handle, self.n = ctx, handle, n

    def free(self):
        if self.handle:
            self.ctx.lib.sph_grid_free(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def sph_create(device: int = 0) -> Context:
    return Context(device)


def sph_build_grid(ctx: Context, pos: torch.Tensor, mass: torch.Tensor, params: sph_params) -> Grid:
    n = pos.shape[0]
    f64 = pos.dtype == torch.float64
    out = ctypes.c_void_p()
    ctx.check(ctx.lib.sph_build_grid(ctx.handle, _ptr(pos, (torch.float32, torch.float64), "pos"), int(f64),
                                     _ptr(mass, torch.float32, "mass"), n, ctypes.byref(params), _stream(),
                                     ctypes.byref(out)))
    return Grid(ctx, out, n)


def sph_build_grid_batched(ctx: Context, pos: torch.Tensor, mass: torch.Tensor, box_offsets, box_sizes,
                           params: sph_params) -> Grid:
    nb = len(box_sizes)
    offs = (ctypes.c_int64 * (nb + 1))(*[int(v) for v in box_offsets])
    sizes = (ctypes.c_double * nb)(*[float(v) for v in box_sizes])
    f64 = pos.dtype == torch.float64
    out = ctypes.c_void_p()
    ctx.check(ctx.lib.sph_build_grid_batched(ctx.handle, _ptr(pos, (torch.float32, torch.float64), "pos"),
                                             int(f64), _ptr(mass, torch.float32, "mass"), offs, sizes, nb,
                                             ctypes.byref(params), _stream(), ctypes.byref(out)))
    return Grid(ctx, out, int(box_offsets[-1]))


def sph_grid_update(ctx: Context, grid: Grid, pos: torch.Tensor, mass: torch.Tensor):
    f64 = pos.dtype == torch.float64
    ctx.check(ctx.lib.sph_grid_update(ctx.handle, grid.handle, _ptr(pos, (torch.float32, torch.float64), "pos"),
                                      int(f64), _ptr(mass, torch.float32, "mass"), _stream()))


def sph_grid_export(grid: Grid, perm=None, keys=None, X=None):
    grid.ctx.check(grid.ctx.lib.sph_grid_export(grid.handle, _ptr(perm, torch.int32, "perm"),
                                                _ptr(keys, torch.int64, "keys"), _ptr(X, torch.int32, "X"),
                                                _stream()))


def sph_density(ctx: Context, grid: Grid, h, active, rho, omega, n_ngb, flags, hash=None,
                params: sph_params = None):
    na = 0 if active is None else active.numel()
    ctx.check(ctx.lib.sph_density(ctx.handle, grid.handle, _ptr(h, torch.float32, "h"),
                                  _ptr(active, torch.int32, "active"), na, _ptr(rho, torch.float32, "rho"),
                                  _ptr(omega, torch.float32, "omega"), _ptr(n_ngb, torch.int32, "n_ngb"),
                                  _ptr(flags, torch.uint8, "flags"), _ptr(hash, torch.int64, "hash"),
                                  ctypes.byref(params), _stream()))


def sph_hydro_force(ctx: Context, grid: Grid, vel, u, h, rho, omega, active, acc, dudt, vsig, hash=None,
                    params: sph_params = None):
    na = 0 if active is None else active.numel()
    f = torch.float32
    ctx.check(ctx.lib.sph_hydro_force(ctx.handle, grid.handle, _ptr(vel, f, "vel"), _ptr(u, f, "u"),
                                      _ptr(h, f, "h"), _ptr(rho, f, "rho"), _ptr(omega, f, "omega"),
                                      _ptr(active, torch.int32, "active"), na, _ptr(acc, f, "acc"),
                                      _ptr(dudt, f, "dudt"), _ptr(vsig, f, "vsig"),
                                      _ptr(hash, torch.int64, "hash"), ctypes.byref(params), _stream()))


def sph_density_divcurl(ctx: Context, grid: Grid, h, active, rho, omega, n_ngb, flags, hash, vel, divv, curlv,
                        params: sph_params = None):
    na = 0 if active is None else active.numel()
    f = torch.float32
    ctx.check(ctx.lib.sph_density_divcurl(ctx.handle, grid.handle, _ptr(h, f, "h"),
                                          _ptr(active, torch.int32, "active"), na, _ptr(rho, f, "rho"),
                                          _ptr(omega, f, "omega"), _ptr(n_ngb, torch.int32, "n_ngb"),
                                          _ptr(flags, torch.uint8, "flags"), _ptr(hash, torch.int64, "hash"),
                                          _ptr(vel, f, "vel"), _ptr(divv, f, "divv"), _ptr(curlv, f, "curlv"),
                                          ctypes.byref(params or default_params()), _stream()))


def sph_hydro_force_balsara(ctx: Context, grid: Grid, vel, u, h, rho, omega, divv, curlv, active, acc, dudt, vsig,
                            hash=None, params: sph_params = None):
    na = 0 if active is None else active.numel()
    f = torch.float32
    ctx.check(ctx.lib.sph_hydro_force_balsara(ctx.handle, grid.handle, _ptr(vel, f, "vel"), _ptr(u, f, "u"),
                                              _ptr(h, f, "h"), _ptr(rho, f, "rho"), _ptr(omega, f, "omega"),
                                              _ptr(divv, f, "divv"), _ptr(curlv, f, "curlv"),
                                              _ptr(active, torch.int32, "active"), na, _ptr(acc, f, "acc"),
                                              _ptr(dudt, f, "dudt"), _ptr(vsig, f, "vsig"),
                                              _ptr(hash, torch.int64, "hash"),
                                              ctypes.byref(params or default_params()), _stream()))


def sph_hydro_force_conduction(ctx: Context, grid: Grid, vel, u, h, rho, omega, divv, curlv, kappa, active, acc,
                               dudt, vsig, dudt_cond, hash=None, params: sph_params = None):
    na = 0 if active is None else active.numel()
    f = torch.float32
    ctx.check(ctx.lib.sph_hydro_force_conduction(ctx.handle, grid.handle, _ptr(vel, f, "vel"), _ptr(u, f, "u"),
                                                 _ptr(h, f, "h"), _ptr(rho, f, "rho"), _ptr(omega, f, "omega"),
                                                 _ptr(divv, f, "divv"), _ptr(curlv, f, "curlv"),
                                                 _ptr(kappa, f, "kappa"), _ptr(active, torch.int32, "active"), na,
                                                 _ptr(acc, f, "acc"), _ptr(dudt, f, "dudt"), _ptr(vsig, f, "vsig"),
                                                 _ptr(dudt_cond, f, "dudt_cond"), _ptr(hash, torch.int64, "hash"),
                                                 ctypes.byref(params or default_params()), _stream()))


def sph_hydro_force_visc(ctx: Context, grid: Grid, vel, u, h, rho, omega, alpha_v, divv, curlv, active, acc, dudt,
                         vsig, hash=None, params: sph_params = None):
    na = 0 if active is None else active.numel()
    f = torch.float32
    ctx.check(ctx.lib.sph_hydro_force_visc(ctx.handle, grid.handle, _ptr(vel, f, "vel"), _ptr(u, f, "u"),
                                           _ptr(h, f, "h"), _ptr(rho, f, "rho"), _ptr(omega, f, "omega"),
                                           _ptr(alpha_v, f, "alpha_v"), _ptr(divv, f, "divv"), _ptr(curlv, f, "curlv"),
                                           _ptr(active, torch.int32, "active"), na, _ptr(acc, f, "acc"),
                                           _ptr(dudt, f, "dudt"), _ptr(vsig, f, "vsig"),
                                           _ptr(hash, torch.int64, "hash"),
                                           ctypes.byref(params or default_params()), _stream()))


def sph_visc_rate(ctx: Context, active, h, u, divv, alpha_v, dalpha, gamma=5.0 / 3.0, alpha_min=0.1, alpha_max=1.0,
                  ell=0.2):
    na = h.numel() if active is None else active.numel()
    f = torch.float32
    ctx.check(ctx.lib.sph_visc_rate(ctx.handle, _ptr(active, torch.int32, "active"), na, _ptr(h, f, "h"),
                                    _ptr(u, f, "u"), _ptr(divv, f, "divv"), _ptr(alpha_v, f, "alpha_v"),
                                    float(gamma), float(alpha_min), float(alpha_max), float(ell),
                                    _ptr(dalpha, f, "dalpha"), _stream()))


def sph_kick_scalar(ctx: Context, active, n_active, bins, dt_bin, rate, value, value_pred=None):
    dts = (ctypes.c_double * len(dt_bin))(*[float(x) for x in dt_bin])
    f = torch.float32
    ctx.check(ctx.lib.sph_kick_scalar(ctx.handle, _ptr(active, torch.int32, "active"), int(n_active),
                                      _ptr(bins, torch.uint8, "bins"), dts, len(dt_bin), _ptr(rate, f, "rate"),
                                      _ptr(value, f, "value"), _ptr(value_pred, f, "value_pred"), _stream()))


def sph_predict_scalar(ctx: Context, dt, rate, value_pred):
    f = torch.float32
    ctx.check(ctx.lib.sph_predict_scalar(ctx.handle, value_pred.numel(), float(dt), _ptr(rate, f, "rate"),
                                         _ptr(value_pred, f, "value_pred"), _stream()))


def gravity_params(G=1.0, theta=0.5, r_split=0.0, r_cut=0.25, h_soft=0.0) -> sph_gravity_params:
    return sph_gravity_params(float(G), float(theta), float(r_split), float(r_cut), float(h_soft))


def sph_gravity(ctx: Context, grid: Grid, active, gp: sph_gravity_params, acc, n_nodes=None, n_pairs=None):
    na = 0 if active is None else active.numel()
    i32 = torch.int32
    ctx.check(ctx.lib.sph_gravity(ctx.handle, grid.handle, _ptr(active, i32, "active"), na, ctypes.byref(gp),
                                  _ptr(acc, torch.float32, "acc"), _ptr(n_nodes, i32, "n_nodes"),
                                  _ptr(n_pairs, i32, "n_pairs"), _stream()))


def sph_timebins(ctx: Context, h, vsig, active, tick, courant, dt_max, max_bin, bins):
    na = 0 if active is None else active.numel()
    f = torch.float32
    ctx.check(ctx.lib.sph_timebins(ctx.handle, _ptr(h, f, "h"), _ptr(vsig, f, "vsig"),
                                   _ptr(active, torch.int32, "active"), na, h.numel(), int(tick), float(courant),
                                   float(dt_max), int(max_bin), _ptr(bins, torch.uint8, "bins"), _stream()))


def sph_active_from_bins(ctx: Context, grid: Grid, bins, tick, max_bin, active, n_active):
    ctx.check(ctx.lib.sph_active_from_bins(ctx.handle, grid.handle, _ptr(bins, torch.uint8, "bins"), int(tick),
                                           int(max_bin), _ptr(active, torch.int32, "active"),
                                           _ptr(n_active, torch.int32, "n_active"), _stream()))


def sph_kick(ctx: Context, active, n_active, bins, dt_bin, acc, dudt, vel, u, vel_pred=None, u_pred=None):
    dts = (ctypes.c_double * len(dt_bin))(*[float(x) for x in dt_bin])
    f = torch.float32
    ctx.check(ctx.lib.sph_kick(ctx.handle, _ptr(active, torch.int32, "active"), int(n_active),
                               _ptr(bins, torch.uint8, "bins"), dts, len(dt_bin), _ptr(acc, f, "acc"),
                               _ptr(dudt, f, "dudt"), _ptr(vel, f, "vel"), _ptr(u, f, "u"),
                               _ptr(vel_pred, f, "vel_pred"), _ptr(u_pred, f, "u_pred"), _stream()))


def sph_drift(ctx: Context, pos, vel, dt, box=1.0, acc=None, dudt=None, vel_pred=None, u_pred=None):
    f = torch.float32
    ctx.check(ctx.lib.sph_drift(ctx.handle, _ptr(pos, torch.float64, "pos"), _ptr(vel, f, "vel"),
                                pos.shape[0], float(dt), float(box), _ptr(acc, f, "acc"), _ptr(dudt, f, "dudt"),
                                _ptr(vel_pred, f, "vel_pred"), _ptr(u_pred, f, "u_pred"), _stream()))


def sph_backward(ctx: Context, grid: Grid, vel, u, h, rho, omega, g_acc, g_rho, g_pos, g_u, g_mass,
                 params: sph_params = None):
    f = torch.float32
    ctx.check(ctx.lib.sph_backward(ctx.handle, grid.handle, _ptr(vel, f, "vel"), _ptr(u, f, "u"), _ptr(h, f, "h"),
                                   _ptr(rho, f, "rho"), _ptr(omega, f, "omega"), _ptr(g_acc, f, "g_acc"),
                                   _ptr(g_rho, f, "g_rho"), _ptr(g_pos, f, "g_pos"), _ptr(g_u, f, "g_u"),
                                   _ptr(g_mass, f, "g_mass"), ctypes.byref(params or default_params()), _stream()))


def sph_sync_status(ctx: Context, raise_on_error: bool = True):
    """Waits for the current stream; returns (status, stats dict) and clears the counters."""
    st = sph_stats()
    rc = ctx.lib.sph_sync_status(ctx.handle, _stream(), ctypes.byref(st))
    if rc != 0 and raise_on_error:
        raise SPHError(rc, ctx.lib.sph_last_error(ctx.handle).decode())
    return rc, st.as_dict()


def _check_sort_static(keys, sorted_keys, perm, device):
    """Host-side checks of sph_sort_keys_static's tensors, made before any
    launch: the outputs hold exactly as many elements as the keys (a shorter
    one would be written past its end), and all three live on `device`, the
    device whose scratch array the call uses."""
    for name, t in (("keys", keys), ("sorted_keys", sorted_keys), ("perm", perm)):
        if not isinstance(t, torch.Tensor):
            raise TypeError(f"{name} must be a tensor")
        if t.device != device:
            raise ValueError(f"{name} is on {t.device}, the call runs on {device}")
    if not (sorted_keys.numel() == perm.numel() == keys.numel()):
        raise ValueError(f"sorted_keys ({sorted_keys.numel()}) and perm ({perm.numel()}) must hold as many "
                         f"elements as keys ({keys.numel()})")


def sph_sort_keys_static(keys, sorted_keys, perm):
    """Stable sort of int64-viewed uint64 keys without any allocation (see
    include/sph.h): fills sorted_keys and perm. Needs no Context."""
    _check_sort_static(keys, sorted_keys, perm, torch.device("cuda", torch.cuda.current_device()))
    lib = abi.load()
    rc = lib.sph_sort_keys_static(_ptr(keys, torch.int64, "keys"), keys.numel(),
                                  _ptr(sorted_keys, torch.int64, "sorted_keys"), _ptr(perm, torch.int32, "perm"),
                                  _stream())
    if rc != 0:
        raise SPHError(rc, "sph_sort_keys_static: n must be in [1, SPH_SORT_STATIC_MAX_KEYS] "
                           "and pointers non-NULL" if rc == abi.SPH_ERR_INVALID else "CUDA call failed")


# ---- conveniences that allocate the outputs ----------------------------------

def density(ctx, grid, h, active=None, params=None, want_hash=False):
    """Runs sph_density in place on h; returns dict of rho, omega, n_ngb, flags (, hash)."""
    n = grid.n
    dev = h.device
    out = {"rho": torch.zeros(n, device=dev), "omega": torch.zeros(n, device=dev),
           "n_ngb": torch.full((n,), -1, dtype=torch.int32, device=dev),
           "flags": torch.zeros(n, dtype=torch.uint8, device=dev)}
    if want_hash:
        out["hash"] = torch.zeros(n, dtype=torch.int64, device=dev)
    sph_density(ctx, grid, h, active, out["rho"], out["omega"], out["n_ngb"], out["flags"],
                out.get("hash"), params or default_params())
    return out


def hydro_force(ctx, grid, vel, u, h, rho, omega, active=None, params=None, want_hash=False):
    n = grid.n
    dev = h.device
    out = {"acc": torch.zeros(n, 3, device=dev), "dudt": torch.zeros(n, device=dev),
           "vsig": torch.zeros(n, device=dev)}
    if want_hash:
        out["hash"] = torch.zeros(n, dtype=torch.int64, device=dev)
    sph_hydro_force(ctx, grid, vel, u, h, rho, omega, active, out["acc"], out["dudt"], out["vsig"],
                    out.get("hash"), params or default_params())
    return out
