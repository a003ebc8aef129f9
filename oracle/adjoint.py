"""Reference gradient of the SPH density + force passes (FP64, CPU).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py). Plain PyTorch CPU ops in
float64 over the oracle's explicit pair list: the forward formulas of
sph_oracle.c written once more as tensor expressions, and torch.autograd
for the reverse pass. The smoothing lengths enter through one Newton step
from the oracle's converged root h*:

    h = h* - (N_eff(h*, x) - N_t) / (dN_eff/dh)|_{h*, detached},

which equals h* in value and has the implicit-function derivative
dh/dx = -(dN/dx)/(dN/dh), so first derivatives are exact. The pair set is
held fixed (it only changes on a measure-zero set of positions).

Loss (the differentiation workload): L = sum_i |a_i - a*_i|^2 + sum_i (rho_i - rho*_i)^2.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import density as _density
from . import pair_list as _pair_list

TWO32 = 4294967296.0


def _w(q):
    return torch.where(q <= 0.5, 1 - 6 * q**2 + 6 * q**3,
                       torch.where(q < 1, 2 * (1 - q) ** 3, torch.zeros_like(q)))


def _dw(q):
    return torch.where(q <= 0.5, -12 * q + 18 * q**2,
                       torch.where(q < 1, -6 * (1 - q) ** 2, torch.zeros_like(q)))


def forward_torch(X, mass, u, vel, box, h_star, pairs, n_target=64.0, alpha=1.0, gamma=5.0 / 3.0,
                  requires_grad=True):
    """Returns (x, m, u_t, acc, rho) with x, m, u_t leaf tensors."""
    I = torch.as_tensor(pairs[0])
    J = torch.as_tensor(pairs[1])
    n = X.shape[0]
    x = torch.tensor(X.astype(np.float64) * (box / TWO32), dtype=torch.float64, requires_grad=requires_grad)
    m = torch.tensor(np.asarray(mass, np.float64), requires_grad=requires_grad)
    ut = torch.tensor(np.asarray(u, np.float64), requires_grad=requires_grad)
    v = torch.tensor(np.asarray(vel, np.float64))
    hs = torch.tensor(np.asarray(h_star, np.float64))
    d = x[J] - x[I]                       # x_j - x_i
    d = d - box * torch.round(d / box)    # minimum image (round has zero derivative)
    r = torch.sqrt((d * d).sum(1))
    zero = torch.zeros(n, dtype=torch.float64)
    # h through one Newton step from the root h*
    q0 = r / hs[I]
    N = 32.0 / 3.0 * (zero.index_add(0, I, _w(q0)) + 1.0)          # + w(0) of the particle itself
    dNdh = (-32.0 / 3.0 / hs * zero.index_add(0, I, q0 * _dw(q0))).detach()
    h = hs - (N - n_target) / dNdh
    # density, its h-derivative, the grad-h factor
    hi = h[I]
    q = r / hi
    wq, dwq = _w(q), _dw(q)
    Wp = 8.0 / (math.pi * hi**3) * wq
    rho = zero.index_add(0, I, m[J] * Wp) + m * 8.0 / (math.pi * h**3)
    Whp = -8.0 / (math.pi * hi**4) * (3 * wq + q * dwq)
    D = zero.index_add(0, I, m[J] * Whp) + m * (-24.0 / (math.pi * h**4))
    omega = 1.0 / (1.0 + h * D / (3.0 * rho))
    # hydro force
    P = (gamma - 1.0) * rho * ut
    c = torch.sqrt(gamma * P / rho)
    A = omega * P / rho**2
    Fi = 8.0 / (math.pi * hi**4) * _dw(r / hi) / r
    hj = h[J]
    Fj = 8.0 / (math.pi * hj**4) * _dw(r / hj) / r
    rij = -d
    vr = ((v[I] - v[J]) * rij).sum(1)
    wij = vr / r
    vsig = c[I] + c[J] - 3.0 * wij
    PI = torch.where(wij < 0, -0.5 * alpha * vsig * wij / (0.5 * (rho[I] + rho[J])), torch.zeros_like(wij))
    Fbar = 0.5 * (Fi + Fj)
    coef = m[J] * (A[I] * Fi + A[J] * Fj + PI * Fbar)
    acc = -torch.zeros(n, 3, dtype=torch.float64).index_add(0, I, coef[:, None] * rij)
    return x, m, ut, acc, rho


def reference_gradient(X, mass, u, vel, box, a_star, rho_star, n_target=64.0, alpha=1.0,
                       gamma=5.0 / 3.0, h_star=None):
    """FP64 gradient of L = sum |a - a*|^2 + sum (rho - rho*)^2 with respect to
    positions, u and masses. Returns dict(loss, g_pos, g_u, g_mass, acc, rho, h)."""
    if h_star is None:
        h_star = _density(X, np.asarray(mass, np.float64), None, box=box, n_target=n_target, tol=1e-12)["h"]
    pairs = _pair_list(X, h_star, box=box)
    x, m, ut, acc, rho = forward_torch(X, mass, u, vel, box, h_star, pairs, n_target, alpha, gamma)
    loss = ((acc - torch.as_tensor(a_star)) ** 2).sum() + ((rho - torch.as_tensor(rho_star)) ** 2).sum()
    loss.backward()
    return {"loss": float(loss.detach()), "g_pos": x.grad.numpy(), "g_u": ut.grad.numpy(), "g_mass": m.grad.numpy(),
            "acc": acc.detach().numpy(), "rho": rho.detach().numpy(), "h": np.asarray(h_star)}
