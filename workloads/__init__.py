"""Seeded synthetic particle sets shaped like the paper's SPH workloads.

This module is shared by the FP64 oracle tests and by the GPU path's tests and
benchmark. It holds no SPH arithmetic: it only draws positions, masses,
velocities and internal energies, and ranks a caller-supplied array into time
bins. Everything is float64 numpy; callers cast as they need.

The paper (Sec. 1 and Sec. 3) runs Magneticum cosmological boxes, which are not
available; these generators stand in for them:

* ``lattice``   -- jittered cubic lattice, equal masses (the uniform, plain case).
* ``clustered`` -- Gaussian blobs on a uniform background with log-normal
  masses: a density contrast of ~1e4, like halos forming in the paper's
  Fig. 1, so smoothing lengths span a ~70x range.
* ``batch``     -- many independent boxes of uneven size.
* ``timebins``  -- ranked adaptive time bins, so successive steps have exactly
  the requested fractions of active particles (Sec. 2.2, "Adaptive Timesteps").
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "Particles", "lattice", "clustered", "batch", "timebins",
    "active_sets", "perturb", "config1", "config2", "config3", "config4",
    "config5", "sample_indices",
]


@dataclasses.dataclass
class Particles:
    """One periodic box of gas particles (all arrays float64, caller order)."""
    pos: np.ndarray      # (N, 3) in [0, box)
    vel: np.ndarray      # (N, 3)
    mass: np.ndarray     # (N,)
    u: np.ndarray        # (N,) specific internal energy
    box: float = 1.0

    @property
    def n(self) -> int:
        return int(self.pos.shape[0])

    def take(self, idx: np.ndarray) -> "Particles":
        return Particles(self.pos[idx], self.vel[idx], self.mass[idx], self.u[idx], self.box)


def lattice(n_side: int, jitter: float = 0.3, seed: int = 1, box: float = 1.0,
            vel_sigma: float = 0.1, u_range=(0.9, 1.1)) -> Particles:
    """Cubic lattice at ((i+1/2)/n_side) with uniform jitter of +-jitter cells.

    Equal masses summing to 1. ``jitter=0`` and ``vel_sigma=0`` give the
    perfect lattice used by the symmetry pins.
    """
    rng = np.random.default_rng(seed)
    g = (np.arange(n_side, dtype=np.float64) + 0.5) / n_side
    gx, gy, gz = np.meshgrid(g, g, g, indexing="ij")
    pos = np.stack([gx.ravel(), gy.ravel(), gz.ravel()], axis=1)
    n = pos.shape[0]
    if jitter:
        pos = pos + rng.uniform(-jitter, jitter, size=(n, 3)) / n_side
    pos = np.mod(pos * box, box)
    vel = rng.normal(0.0, vel_sigma, size=(n, 3)) if vel_sigma else np.zeros((n, 3))
    u = rng.uniform(u_range[0], u_range[1], size=n) if u_range[1] > u_range[0] \
        else np.full(n, float(u_range[0]))
    mass = np.full(n, 1.0 / n)
    return Particles(pos, vel, mass, u, box)


def clustered(n: int, n_blobs: int, seed: int, box: float = 1.0, blob_frac: float = 0.7,
              radius_range=(0.002, 0.05), mass_sigma: float = 1.0,
              vel_sigma: float = 0.1, bulk_sigma: float = 0.1,
              log10_u_range=(-1.0, 1.0)) -> Particles:
    """Gaussian blobs on a uniform background.

    * ``blob_frac`` of the particles belong to blobs, membership uniform over
      blobs; the rest are uniform in the box.
    * Blob centres uniform; blob Gaussian sigma log-uniform in
      ``radius_range`` (box units).
    * Particle masses i.i.d. exp(mass_sigma * z), normalised to total mass 1.
    * Velocities N(0, vel_sigma^2) per component plus the blob's bulk velocity
      N(0, bulk_sigma^2) per component (background: no bulk flow).
    * u = 10**U(log10_u_range), i.e. log-uniform over two decades.
    """
    rng = np.random.default_rng(seed)
    n_blob = int(round(blob_frac * n))
    n_bg = n - n_blob
    centres = rng.uniform(0.0, 1.0, size=(n_blobs, 3))
    lo, hi = math.log(radius_range[0]), math.log(radius_range[1])
    sig = np.exp(rng.uniform(lo, hi, size=n_blobs))
    bulk = rng.normal(0.0, bulk_sigma, size=(n_blobs, 3))
    member = rng.integers(0, n_blobs, size=n_blob)
    pos_b = centres[member] + rng.normal(0.0, 1.0, size=(n_blob, 3)) * sig[member, None]
    pos_u = rng.uniform(0.0, 1.0, size=(n_bg, 3))
    pos = np.mod(np.concatenate([pos_b, pos_u]) * box, box)
    # np.mod can return exactly `box` for tiny negative inputs; fold it back.
    pos[pos >= box] = 0.0
    vel = rng.normal(0.0, vel_sigma, size=(n, 3))
    vel[:n_blob] += bulk[member]
    mass = np.exp(mass_sigma * rng.normal(0.0, 1.0, size=n))
    mass /= mass.sum()
    u = 10.0 ** rng.uniform(log10_u_range[0], log10_u_range[1], size=n)
    # Shuffle so that caller order carries no spatial or blob structure.
    perm = rng.permutation(n)
    return Particles(pos[perm], vel[perm], mass[perm], u[perm], box)


def blobs_for(n: int) -> int:
    """Blob count proportional to sqrt(N): 500 at 1e7, ~230 at 2M."""
    return max(1, int(round(0.158 * math.sqrt(n))))


def batch(n_boxes: int = 64, seed: int = 4, n_min: int = 4096, n_max: int = 524288,
          box_seed0: int = 100) -> list[Particles]:
    """Independent periodic unit boxes, N log-uniform in [n_min, n_max]."""
    rng = np.random.default_rng(seed)
    sizes = np.exp(rng.uniform(math.log(n_min), math.log(n_max), size=n_boxes))
    sizes = np.round(sizes).astype(np.int64)
    return [clustered(int(nb), blobs_for(int(nb)), box_seed0 + b) for b, nb in enumerate(sizes)]


def timebins(dt: np.ndarray, fractions=(0.001, 0.01, 0.1)) -> np.ndarray:
    """Rank particles by a time-step estimate into bins 0..len(fractions).

    The smallest ``fractions[0]`` of ``dt`` go to the highest bin, the next up
    to ``fractions[1]`` one bin lower, and so on; the rest get bin 0. Ties are
    broken by index, so the fractions are exact. Step k activates bins >= k.
    """
    n = dt.shape[0]
    order = np.lexsort((np.arange(n), dt))
    bins = np.zeros(n, dtype=np.int32)
    nb = len(fractions)
    prev = 0
    for k, f in enumerate(sorted(fractions)):
        cnt = int(round(f * n))
        bins[order[prev:cnt]] = nb - k
        prev = max(prev, cnt)
    return bins


def active_sets(bins: np.ndarray) -> list[np.ndarray]:
    """Active index lists (int32, ascending) for steps k = 0..max(bins)."""
    return [np.nonzero(bins >= k)[0].astype(np.int32) for k in range(int(bins.max()) + 1)]


def perturb(x: np.ndarray, sigma: float, seed: int) -> np.ndarray:
    """x * exp(sigma * z), z ~ N(0,1), seeded (used to unconverge h guesses)."""
    rng = np.random.default_rng(seed)
    return x * np.exp(sigma * rng.normal(0.0, 1.0, size=x.shape))


def sample_indices(n: int, k: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    k = min(k, n)
    return np.sort(rng.choice(n, size=k, replace=False)).astype(np.int64)


# ---- the five workloads ------------------------------------------------------

def config1(n_side: int = 32) -> Particles:
    """32^3 jittered lattice (+-0.3 cell), equal mass, u ~ U[0.9,1.1], seed 1."""
    return lattice(n_side, 0.3, seed=1)


def config2(n: int = 2_097_152) -> Particles:
    """2M clustered particles, 200 blobs, seed 2."""
    return clustered(n, 200, seed=2)


def config3(n: int = 10_000_000) -> Particles:
    """10M clustered particles, 500 blobs, seed 3."""
    return clustered(n, 500, seed=3)


def config4(n_boxes: int = 64, n_min: int = 4096, n_max: int = 524288) -> list[Particles]:
    """64 boxes, N log-uniform in [4096, 524288], box b from seed 100+b."""
    return batch(n_boxes, 4, n_min, n_max, 100)


def config5(n: int = 262_144) -> Particles:
    """262,144 clustered particles, seed 5, blob count ~ sqrt(N)."""
    return clustered(n, blobs_for(n), seed=5)
