"""FP64 CPU oracle for the SPH density and hydro-force passes and the
short-range gravity pass.

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package. It shares no code
with the CUDA library and never imports it; the library never imports this.

The arithmetic lives in ``sph_oracle.c`` (plain C, FP64, OpenMP over
particles); this module only builds it with gcc and marshals numpy arrays.
Function-level citations are in the C source.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sph_oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "libsph_oracle.so")
_lib = None

NOT_CONVERGED = 1
H_TOO_LARGE = 2


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2 -fopenmp, FP64, no fast-math)."""
    os.makedirs(_LIB_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               "-fno-fast-math", "-ffp-contract=off", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        i64, f64, i32 = ctypes.c_int64, ctypes.c_double, ctypes.c_int
        L.orc_quantize.argtypes = [P, i64, f64, P]
        L.orc_morton.argtypes = [ctypes.c_uint32] * 3
        L.orc_morton.restype = ctypes.c_uint64
        L.orc_keys.argtypes = [P, i64, i64, i32, P]
        L.orc_sort_keys.argtypes = [P, i64, P]
        L.orc_kernel_array.argtypes = [P, i64, P, P]
        L.orc_splitmix64.argtypes = [ctypes.c_uint64]
        L.orc_splitmix64.restype = ctypes.c_uint64
        L.orc_set_hash_offset.argtypes = [i64]
        L.orc_set_hash_offset.restype = None
        L.orc_density.argtypes = [i32, P, P, i64, f64, P, P, f64, f64, i32, P, i64, i32, i32,
                                  P, P, P, P, P, P, P, P]
        L.orc_density.restype = i32
        L.orc_force.argtypes = [i32, P, P, i64, f64, P, P, P, P, P, P, f64, P, f64, P, P, P, i64, i32,
                                P, P, P, P, P, P, P]
        L.orc_divcurl.argtypes = [i32, P, P, i64, f64, P, P, P, P, P, i64, i32, P, P, P, P]
        L.orc_conduction.argtypes = [i32, P, P, i64, f64, P, P, P, P, P, P, i64, i32, P, P]
        L.orc_neighbours.argtypes = [i32, P, P, i64, f64, i64, f64, i32, P, i64]
        L.orc_neighbours.restype = i64
        L.orc_num_threads.restype = i32
        L.orc_set_threads.argtypes = [i32]
        L.orc_set_threads.restype = i32
        L.orc_gravity.argtypes = [P, i64, f64, P, f64, f64, f64, f64, f64, P, i64, P, P, P, P]
        L.orc_soft_mass.argtypes = [f64]
        L.orc_soft_mass.restype = f64
        L.orc_pair_list.argtypes = [i32, P, P, i64, f64, P, i32, P, P, i64]
        L.orc_pair_list.restype = i64
        _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def num_threads() -> int:
    return int(lib().orc_num_threads())


def set_threads(t: int) -> int:
    """Threads of the oracle's later parallel regions; returns the previous count."""
    return int(lib().orc_set_threads(int(t)))


def quantize(pos, box: float = 1.0) -> np.ndarray:
    """Integer positions X (N, 3) uint32 of float positions in a periodic box."""
    p = _c(pos, np.float64)
    X = np.empty(p.shape, dtype=np.uint32)
    lib().orc_quantize(_p(p), p.size, float(box), _p(X))
    return X


def morton_keys(X, box_index: int = 0, box_bits: int = 0) -> np.ndarray:
    Xc = _c(X, np.uint32)
    k = np.empty(Xc.shape[0], dtype=np.uint64)
    lib().orc_keys(_p(Xc), Xc.shape[0], int(box_index), int(box_bits), _p(k))
    return k


def sort_perm(keys) -> np.ndarray:
    k = _c(keys, np.uint64)
    perm = np.empty(k.shape[0], dtype=np.int64)
    lib().orc_sort_keys(_p(k), k.shape[0], _p(perm))
    return perm


def kernel(q):
    """w(q) and dw/dq of the cubic spline (support 1)."""
    qq = _c(q, np.float64).ravel()
    w = np.empty_like(qq)
    dw = np.empty_like(qq)
    lib().orc_kernel_array(_p(qq), qq.size, _p(w), _p(dw))
    return w.reshape(np.shape(q)), dw.reshape(np.shape(q))


def splitmix64(x: int) -> int:
    return int(lib().orc_splitmix64(ctypes.c_uint64(x)))


def _geom(X, xc, box):
    if xc is not None:
        xc = _c(xc, np.float64)
        if X is None:
            X = quantize(xc, box)
        return 1, _c(X, np.uint32), xc
    return 0, _c(X, np.uint32), None


def density(X=None, mass=None, h_init=None, box=1.0, n_target=64.0, tol=1e-10, max_iter=200,
            active=None, brute=False, fixed_h=False, xc=None, hash_offset=0):
    """Density pass (and smoothing-length solve unless ``fixed_h``).

    Pass integer positions ``X`` (quantised geometry, exact predicate) or
    continuous FP64 positions ``xc``. Returns a dict of per-particle arrays
    (entries of inactive particles are NaN / -1). ``hash_offset`` is added to
    every index the neighbour-set checksums hash (a box that sits at an
    offset in a batch).
    """
    mode, Xc, xcc = _geom(X, xc, box)
    n = Xc.shape[0]
    m = _c(mass, np.float64)
    hi = None if h_init is None else _c(h_init, np.float64)
    act = None if active is None else _c(active, np.int64)
    out = {k: np.full(n, np.nan) for k in ("h", "rho", "drho_dh", "omega", "neff")}
    out["n_ngb"] = np.full(n, -1, dtype=np.int64)
    out["hash"] = np.zeros(n, dtype=np.uint64)
    out["status"] = np.zeros(n, dtype=np.int32)
    lib().orc_set_hash_offset(int(hash_offset))
    st = lib().orc_density(mode, _p(Xc), _p(xcc), n, float(box), _p(m), _p(hi), float(n_target),
                           float(tol), int(max_iter), _p(act), 0 if act is None else act.size,
                           int(bool(brute)), int(bool(fixed_h)), _p(out["h"]), _p(out["rho"]),
                           _p(out["drho_dh"]), _p(out["omega"]), _p(out["neff"]),
                           _p(out["n_ngb"]), _p(out["hash"]), _p(out["status"]))
    lib().orc_set_hash_offset(0)
    out["any_status"] = int(st)
    return out


def divcurl(X=None, vel=None, mass=None, h=None, rho=None, box=1.0, active=None, brute=False, xc=None,
            scales=False):
    """Velocity divergence and |curl| at the given h and rho (entries of
    inactive particles NaN); with scales=True also the per-particle sums of
    the pair terms' magnitudes (divergence, curl)."""
    mode, Xc, xcc = _geom(X, xc, box)
    n = Xc.shape[0]
    args = [_c(a, np.float64) for a in (vel, mass, h, rho)]
    act = None if active is None else _c(active, np.int64)
    divv = np.full(n, np.nan)
    curlv = np.full(n, np.nan)
    sd = np.full(n, np.nan)
    sc = np.full(n, np.nan)
    lib().orc_divcurl(mode, _p(Xc), _p(xcc), n, float(box), *[_p(a) for a in args], _p(act),
                      0 if act is None else act.size, int(bool(brute)), _p(divv), _p(curlv), _p(sd), _p(sc))
    return (divv, curlv, sd, sc) if scales else (divv, curlv)


def conduction(X=None, mass=None, u=None, h=None, rho=None, kappa=None, box=1.0, active=None, brute=False,
               xc=None):
    """Conduction heating rate over the force pair set and its per-particle
    scale (sum of the pair terms' magnitudes); inactive entries NaN."""
    mode, Xc, xcc = _geom(X, xc, box)
    n = Xc.shape[0]
    args = [_c(a, np.float64) for a in (mass, u, h, rho, kappa)]
    act = None if active is None else _c(active, np.int64)
    du = np.full(n, np.nan)
    sc = np.full(n, np.nan)
    lib().orc_conduction(mode, _p(Xc), _p(xcc), n, float(box), *[_p(a) for a in args], _p(act),
                         0 if act is None else act.size, int(bool(brute)), _p(du), _p(sc))
    return du, sc


def force(X=None, vel=None, mass=None, u=None, h=None, rho=None, omega=None, box=1.0,
          alpha=1.0, gamma=5.0 / 3.0, active=None, brute=False, xc=None, divv=None, curlv=None, hash_offset=0):
    """Hydro-force pass. Returns acc (N,3), dudt, vsig, scale_a, scale_u,
    n_pairs, hash (entries of inactive particles NaN / -1). With divv and
    curlv, Balsara's switch limits the viscosity. alpha: a number, or one
    value per particle (the pair taking the mean of its two)."""
    mode, Xc, xcc = _geom(X, xc, box)
    alpha_p = None
    if np.ndim(alpha) > 0:
        alpha_p, alpha = _c(alpha, np.float64), 0.0
    n = Xc.shape[0]
    args = [_c(a, np.float64) for a in (vel, mass, u, h, rho, omega)]
    sw = [None, None] if divv is None else [_c(divv, np.float64), _c(curlv, np.float64)]
    act = None if active is None else _c(active, np.int64)
    out = {"acc": np.full((n, 3), np.nan)}
    for k in ("dudt", "vsig", "scale_a", "scale_u"):
        out[k] = np.full(n, np.nan)
    out["n_pairs"] = np.full(n, -1, dtype=np.int64)
    out["hash"] = np.zeros(n, dtype=np.uint64)
    lib().orc_set_hash_offset(int(hash_offset))
    lib().orc_force(mode, _p(Xc), _p(xcc), n, float(box), *[_p(a) for a in args], float(alpha), _p(alpha_p),
                    float(gamma), _p(sw[0]), _p(sw[1]), _p(act), 0 if act is None else act.size, int(bool(brute)),
                    _p(out["acc"]), _p(out["dudt"]), _p(out["vsig"]), _p(out["scale_a"]),
                    _p(out["scale_u"]), _p(out["n_pairs"]), _p(out["hash"]))
    lib().orc_set_hash_offset(0)
    return out


def visc_rate(h, u, divv, alpha, alpha_min=0.1, alpha_max=1.0, ell=0.2, gamma=5.0 / 3.0):
    """Rate of change of the viscosity parameter (Morris & Monaghan 1997):
    d alpha/dt = -(alpha - alpha_min) / tau + S, with the decay time
    tau = h / (ell c) (h the kernel's support radius, c = sqrt(gamma (gamma - 1) u)
    the sound speed) and the source S = max(-div v, 0) (alpha_max - alpha),
    which raises alpha only where the flow converges."""
    h, u, divv, alpha = (np.asarray(a, np.float64) for a in (h, u, divv, alpha))
    c = np.sqrt(gamma * (gamma - 1.0) * u)
    tau = h / (ell * c)
    source = np.maximum(-divv, 0.0) * (alpha_max - alpha)
    return -(alpha - alpha_min) / tau + source


def gravity(X, mass, box=1.0, G=1.0, theta=0.5, r_split=0.0, r_cut=0.25, h_soft=0.0, active=None):
    """Short-range gravity (TreePM split) by the Barnes-Hut walk of
    orc_gravity. X: integer positions (N, 3). Returns acc (N, 3), scale (sum
    of |term|), n_nodes, n_pairs; inactive entries NaN / -1."""
    Xc = _c(X, np.uint32)
    n = Xc.shape[0]
    if not (0.0 < r_cut <= 0.25 * box) or not (0.0 <= theta <= 1.0):
        raise ValueError("need 0 < r_cut <= box/4 and 0 <= theta <= 1")
    act = None if active is None else _c(active, np.int64)
    out = {"acc": np.full((n, 3), np.nan), "scale": np.full(n, np.nan),
           "n_nodes": np.full(n, -1, np.int64), "n_pairs": np.full(n, -1, np.int64)}
    lib().orc_gravity(_p(Xc), n, float(box), _p(_c(mass, np.float64)), float(G), float(theta), float(r_split),
                      float(r_cut), float(h_soft), _p(act), 0 if act is None else act.size, _p(out["acc"]),
                      _p(out["scale"]), _p(out["n_nodes"]), _p(out["n_pairs"]))
    return out


def soft_mass(q) -> float:
    """Mass fraction of the cubic spline (support 1) inside radius q."""
    return lib().orc_soft_mass(float(q))


def neighbours(X=None, i=0, h=0.1, box=1.0, brute=True, xc=None) -> np.ndarray:
    """Sorted indices j != i with r_ij < h."""
    mode, Xc, xcc = _geom(X, xc, box)
    n = Xc.shape[0]
    cap = 1024
    while True:
        out = np.empty(cap, dtype=np.int64)
        k = lib().orc_neighbours(mode, _p(Xc), _p(xcc), n, float(box), int(i), float(h),
                                 int(bool(brute)), _p(out), cap)
        if k <= cap:
            return np.sort(out[:k])
        cap = int(k)


def pair_list(X=None, h=None, box=1.0, brute=False, xc=None):
    """Ordered pairs (i, j), i != j, with r_ij < max(h_i, h_j): int64 arrays."""
    mode, Xc, xcc = _geom(X, xc, box)
    n = Xc.shape[0]
    hh = _c(h, np.float64)
    cap = max(1024, 80 * n)
    while True:
        oi = np.empty(cap, dtype=np.int64)
        oj = np.empty(cap, dtype=np.int64)
        k = lib().orc_pair_list(mode, _p(Xc), _p(xcc), n, float(box), _p(hh), int(bool(brute)),
                                _p(oi), _p(oj), cap)
        if k <= cap:
            return oi[:k], oj[:k]
        cap = int(k)
