"""GPU parity of the velocity divergence / curl (sph_density_divcurl) and of
the force pass with Balsara's switch (sph_hydro_force_balsara) against the
FP64 oracle, through the C ABI.

Tolerances as for the force: div and |curl| within 1e-4 of the per-particle
scale (the sum of the magnitudes of their pair terms over rho); a and du/dt
within 1e-4 of the force's pair-term scale; pair sets exact.
"""
import numpy as np
import pytest
import torch

import oracle
import workloads as W
from sph_cases import as_f32, check_force, dev, gpu_grid, host, oracle_all, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    from paper_2003_10850_gb300 import build
    build.build()
    import paper_2003_10850_gb300 as S
    return S


@pytest.fixture(scope="module")
def ctx(S):
    return S.Context(0)


@pytest.fixture(scope="module")
def clustered():
    p = as_f32(W.clustered(50_000, 40, seed=202))
    return p, oracle_all(p)


@pytest.fixture(scope="module")
def shear_lattice():
    """Jittered 32^3 lattice in a shear flow plus noise: div and curl both matter."""
    q = W.config1(32)
    vel = q.vel.copy()
    vel[:, 0] += 0.5 * np.sin(2 * np.pi * q.pos[:, 1])
    vel[:, 1] += 0.3 * np.sin(2 * np.pi * q.pos[:, 0])
    p = as_f32(W.Particles(q.pos, vel, q.mass, q.u, q.box))
    return p, oracle_all(p)


def _divcurl_gpu(S, ctx, grid, p, h0, params):
    n = p.n
    h = dev(h0)
    rho, om = torch.zeros(n, device="cuda"), torch.zeros(n, device="cuda")
    nn = torch.zeros(n, dtype=torch.int32, device="cuda")
    fl = torch.zeros(n, dtype=torch.uint8, device="cuda")
    dv, cv = torch.zeros(n, device="cuda"), torch.zeros(n, device="cuda")
    S.sph_density_divcurl(ctx, grid, h, None, rho, om, nn, fl, None, dev(p.vel), dv, cv, params)
    rc, st = S.sph_sync_status(ctx, raise_on_error=False)
    return rc, host(h), host(rho), host(om), host(dv), host(cv)


@pytest.mark.parametrize("kind", ["shear_lattice", "clustered"])
def test_divcurl_fixed_h(S, ctx, kind, shear_lattice, clustered):
    p, (X, d, _) = shear_lattice if kind == "shear_lattice" else clustered
    h32 = d["h"].astype(np.float32)
    do = oracle.density(X, p.mass, h32.astype(np.float64), box=p.box, fixed_h=True)
    div_o, curl_o, sd, sc = oracle.divcurl(X, p.vel, p.mass, h32, do["rho"], box=p.box, scales=True)
    grid = gpu_grid(S, ctx, p, S.default_params(box=p.box))
    rc, h, rho, om, dv, cv = _divcurl_gpu(S, ctx, grid, p, h32, S.default_params(box=p.box, flags=S.SPH_FIXED_H))
    assert rc == 0
    assert rel(rho, do["rho"]).max() <= 1e-5
    assert np.all(np.abs(dv - div_o) <= 1e-4 * sd + 1e-30)
    assert np.all(np.abs(cv - curl_o) <= 1e-4 * sc + 1e-30)
    assert np.abs(div_o).max() > 0.01 * np.abs(sd).max()    # the field is not trivial


def test_divcurl_converged(S, ctx, clustered):
    """From no h guess: h, rho as sph_density; div and curl at that h."""
    p, (X, d, _) = clustered
    div_o, curl_o, sd, sc = oracle.divcurl(X, p.vel, p.mass, d["h"], d["rho"], box=p.box, scales=True)
    grid = gpu_grid(S, ctx, p, S.default_params(box=p.box))
    rc, h, rho, om, dv, cv = _divcurl_gpu(S, ctx, grid, p, np.zeros(p.n, np.float32), S.default_params(box=p.box))
    assert rc == 0
    assert rel(h, d["h"]).max() <= 1e-5 and rel(rho, d["rho"]).max() <= 1e-5
    assert np.all(np.abs(dv - div_o) <= 1e-4 * sd + 1e-30)
    assert np.all(np.abs(cv - curl_o) <= 1e-4 * sc + 1e-30)


@pytest.mark.parametrize("kind", ["shear_lattice", "clustered"])
def test_force_balsara(S, ctx, kind, shear_lattice, clustered):
    """The switched force from the recorded lists (after an all-active
    density pass at the same h) and from the walk (h changed), against the
    oracle's switched force on the same div and curl inputs."""
    p, (X, d, _) = shear_lattice if kind == "shear_lattice" else clustered
    h, rho, om = (d[k].astype(np.float32) for k in ("h", "rho", "omega"))
    div_o, curl_o = oracle.divcurl(X, p.vel, p.mass, h, rho, box=p.box)
    dv32, cv32 = div_o.astype(np.float32), curl_o.astype(np.float32)
    f = oracle.force(X, p.vel, p.mass, p.u, h, rho, om, box=p.box, divv=dv32, curlv=cv32)
    f_plain = oracle.force(X, p.vel, p.mass, p.u, h, rho, om, box=p.box)
    params = S.default_params(box=p.box)
    grid = gpu_grid(S, ctx, p, params)
    S.density(ctx, grid, dev(h), None, S.default_params(box=p.box, flags=S.SPH_FIXED_H))
    S.sph_sync_status(ctx)
    for hh, fo, lists in ((h, f, True), (None, None, False)):
        if hh is None:   # another h: the lists cannot serve the call, the walk does
            hh = (h * np.float32(1.001)).astype(np.float32)
            fo = oracle.force(X, p.vel, p.mass, p.u, hh, rho, om, box=p.box, divv=dv32, curlv=cv32)
        n = p.n
        acc, du, vs = torch.zeros(n, 3, device="cuda"), torch.zeros(n, device="cuda"), torch.zeros(n, device="cuda")
        hs = torch.zeros(n, dtype=torch.int64, device="cuda")
        S.sph_hydro_force_balsara(ctx, grid, dev(p.vel), dev(p.u), dev(hh), dev(rho), dev(om), dev(dv32), dev(cv32),
                                  None, acc, du, vs, hs, params)
        rc, st = S.sph_sync_status(ctx, raise_on_error=False)
        assert rc == 0 and (st["pair_tests"] == 0) == lists
        g = {"acc": host(acc), "dudt": host(du), "vsig": host(vs), "hash": host(hs).view(np.uint64)}
        check_force(g, fo, np.arange(n), 1e-4)
    # the switch acts: the switched and plain forces differ beyond the tolerance somewhere
    da = np.linalg.norm(f["acc"] - f_plain["acc"], axis=1) / f["scale_a"]
    assert da.max() > 1e-3


def test_switch_entry_points_reject_other_paths(S, ctx, clustered):
    p, _ = clustered
    grid = gpu_grid(S, ctx, p, S.default_params(box=p.box))
    n = p.n
    z = torch.zeros(n, device="cuda")
    with pytest.raises(S.SPHError):
        S.sph_density_divcurl(ctx, grid, z.clone(), None, z.clone(), z.clone(),
                              torch.zeros(n, dtype=torch.int32, device="cuda"),
                              torch.zeros(n, dtype=torch.uint8, device="cuda"), None, dev(p.vel), z.clone(), z.clone(),
                              S.default_params(box=p.box, flags=S.SPH_PER_THREAD_WALK))
