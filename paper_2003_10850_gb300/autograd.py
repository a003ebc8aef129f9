"""torch.autograd.Function over the C-ABI density, force and adjoint passes.

SPHDensityForce.apply(pos, vel, mass, u, h_init, ctx, params) -> (acc, rho)
runs sph_build_grid + sph_density + sph_hydro_force (all particles active)
and, in backward, sph_backward, which returns dL/dpos, dL/du and dL/dmass
through the implicit smoothing lengths. vel and h_init get no gradient.
Marshalling only: the arithmetic is in libsph_gb300.so.
"""
from __future__ import annotations

import torch

from . import (default_params, sph_backward, sph_build_grid, sph_density, sph_hydro_force,
               sph_sync_status)


class SPHDensityForce(torch.autograd.Function):
    @staticmethod
    def forward(fctx, pos, vel, mass, u, h_init, sctx, params=None):
        params = params or default_params()
        pos, vel, mass, u = (t.detach().contiguous() for t in (pos, vel, mass, u))
        n = pos.shape[0]
        grid = sph_build_grid(sctx, pos, mass, params)
        h = h_init.detach().clone().contiguous()
        dev = pos.device
        rho = torch.zeros(n, device=dev)
        omega = torch.zeros(n, device=dev)
        n_ngb = torch.zeros(n, dtype=torch.int32, device=dev)
        flags = torch.zeros(n, dtype=torch.uint8, device=dev)
        sph_density(sctx, grid, h, None, rho, omega, n_ngb, flags, None, params)
        acc = torch.zeros(n, 3, device=dev)
        dudt = torch.zeros(n, device=dev)
        vsig = torch.zeros(n, device=dev)
        sph_hydro_force(sctx, grid, vel, u, h, rho, omega, None, acc, dudt, vsig, None, params)
        sph_sync_status(sctx)
        fctx.save_for_backward(vel, u, h, rho, omega)
        fctx.grid, fctx.sctx, fctx.params = grid, sctx, params
        fctx.mark_non_differentiable(h)
        return acc, rho

    @staticmethod
    def backward(fctx, g_acc, g_rho):
        vel, u, h, rho, omega = fctx.saved_tensors
        n = h.shape[0]
        dev = h.device
        g_acc = torch.zeros(n, 3, device=dev) if g_acc is None else g_acc.contiguous().float()
        g_rho = None if g_rho is None else g_rho.contiguous().float()
        g_pos = torch.empty(n, 3, device=dev)
        g_u = torch.empty(n, device=dev)
        g_mass = torch.empty(n, device=dev)
        sph_backward(fctx.sctx, fctx.grid, vel, u, h, rho, omega, g_acc, g_rho, g_pos, g_u, g_mass, fctx.params)
        sph_sync_status(fctx.sctx)
        return g_pos, None, g_mass, g_u, None, None, None
