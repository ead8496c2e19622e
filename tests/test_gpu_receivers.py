"""GPU: receiver sampling (the recording of u_next at the receiver points after
each step, Sec. 2's update followed by the sampling step) through the table
that wave_propagate builds on the device, against the FP64 oracle.

The table groups the receivers by xy tile and sorts each tile's entries by
(z, receiver index); these cases reach every branch of that build: receivers
in random order with repeats, every point of a grid that fits in one tile
(a segment far larger than the shared-memory sort, sorted in global memory),
receivers on every plane, and device-resident receivers outside the interior
(left out of the table and reported by the next synchronizing call).
Tolerance: relative L2 <= 1e-5 against the oracle, as for the other FP32
parity tests.
"""
import numpy as np
import pytest

import workloads as wl

pytestmark = pytest.mark.gpu

TOL = 1e-5


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def _run(pkg, vel, sp, dt, nsteps, shot, rec, u0=None, up0=None, device_rec=True):
    import torch
    nz, ny, nx = vel.shape
    s = pkg.WaveSolver((nx, ny, nz), sp, dt, torch.from_numpy(vel).cuda())
    try:
        if u0 is not None:
            s.set_state(torch.from_numpy(u0).cuda(), torch.from_numpy(up0).cuda(), 0)
        r = torch.from_numpy(rec).cuda() if device_rec else rec
        tr = torch.zeros((nsteps, rec.shape[0]), dtype=torch.float32, device="cuda")
        s.propagate(shot, nsteps, r, tr)
        s.synchronize()
        return tr.cpu().numpy().astype(np.float64)
    finally:
        s.close()


def test_unordered_repeated_receivers(wave_lib, oracle_mod):
    nx, ny, nz = 101, 45, 30
    rng = np.random.default_rng(7)
    vel = rng.uniform(1500.0, 4500.0, size=(nz, ny, nx)).astype(np.float32)
    u0, up0 = wl.random_state((nz, ny, nx), seed=5)
    sp = (10.0, 11.0, 9.0)
    dt = 0.45 * wave_lib.wave_cfl_dt(sp, float(vel.max()))
    base = wl.random_receivers(nx, ny, nz, 300, seed=11)
    rec = np.ascontiguousarray(np.concatenate([base, base[::-1][:77], base[:5]]),
                               dtype=np.int32)
    shot = (50, 20, 15, 15.0, 0.01, 1e-3)
    g = _run(wave_lib, vel, sp, dt, 9, shot, rec, u0, up0)
    h = _run(wave_lib, vel, sp, dt, 9, shot, rec, u0, up0, device_rec=False)
    assert np.array_equal(g, h)  # device- and host-resident receivers: same table
    _, _, o = oracle_mod.propagate(vel, sp, dt, 9, u=u0, u_prev=up0, source=shot,
                                   receivers=rec)
    assert rel_l2(g, o) <= TOL
    # repeated points record identical traces
    assert np.array_equal(g[:, :5], g[:, 377:382])


def test_one_tile_holding_every_point(wave_lib, oracle_mod):
    # 16 x 16 x 40 fits in one 32 x 16 tile: all 10240 points are receivers,
    # a segment of 10240 entries (shuffled), sorted in global memory.
    nx, ny, nz = 16, 16, 40
    rng = np.random.default_rng(3)
    vel = rng.uniform(2000.0, 3000.0, size=(nz, ny, nx)).astype(np.float32)
    u0, up0 = wl.random_state((nz, ny, nx), seed=9)
    sp = (10.0, 10.0, 10.0)
    dt = 0.45 * wave_lib.wave_cfl_dt(sp, float(vel.max()))
    zz, yy, xx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    pts = np.stack([xx.ravel(), yy.ravel(), zz.ravel()], axis=1).astype(np.int32)
    rec = np.ascontiguousarray(pts[rng.permutation(len(pts))], dtype=np.int32)
    shot = (8, 8, 20, 15.0, 0.01, 1e-3)
    g = _run(wave_lib, vel, sp, dt, 5, shot, rec, u0, up0)
    ou, _, o = oracle_mod.propagate(vel, sp, dt, 5, u=u0, u_prev=up0, source=shot,
                                    receivers=rec)
    assert rel_l2(g, o) <= TOL
    # the last row is the whole final field, point by point
    field = np.zeros((nz, ny, nx))
    field[rec[:, 2], rec[:, 1], rec[:, 0]] = g[-1]
    assert rel_l2(field, ou) <= TOL


def test_receivers_on_every_plane_many_tiles(wave_lib, oracle_mod):
    nx, ny, nz = 130, 70, 24
    rng = np.random.default_rng(21)
    vel = rng.uniform(1500.0, 4500.0, size=(nz, ny, nx)).astype(np.float32)
    u0, up0 = wl.random_state((nz, ny, nx), seed=2)
    sp = (10.0, 10.0, 10.0)
    dt = 0.45 * wave_lib.wave_cfl_dt(sp, float(vel.max()))
    rec = np.ascontiguousarray(np.concatenate(
        [wl.receiver_plane(nx, ny, z, 7) for z in range(nz)])[::-1], dtype=np.int32)
    shot = (65, 35, 0, 15.0, 0.01, 1e-3)
    g = _run(wave_lib, vel, sp, dt, 6, shot, rec, u0, up0)
    _, _, o = oracle_mod.propagate(vel, sp, dt, 6, u=u0, u_prev=up0, source=shot,
                                   receivers=rec)
    assert rel_l2(g, o) <= TOL


def test_device_receiver_outside_is_reported(wave_lib, oracle_mod):
    import torch
    nx, ny, nz = 40, 24, 16
    vel = wl.layered3(nx, ny, nz)
    sp = (10.0, 10.0, 10.0)
    dt = 0.5 * wave_lib.wave_cfl_dt(sp, 3500.0)
    good = wl.receiver_plane(nx, ny, 5, 4)
    bad = np.array([[nx, 0, 0], [0, -1, 3], [0, 0, nz]], dtype=np.int32)
    rec = np.ascontiguousarray(np.concatenate([good, bad]), dtype=np.int32)
    shot = (20, 12, 8, 15.0, -1.0, 1.0)
    s = wave_lib.WaveSolver((nx, ny, nz), sp, dt, torch.from_numpy(vel).cuda())
    try:
        tr = torch.full((10, rec.shape[0]), 7.0, dtype=torch.float32, device="cuda")
        s.propagate(shot, 10, torch.from_numpy(rec).cuda(), tr)
        with pytest.raises(wave_lib.WaveError) as ei:
            s.synchronize()
        assert ei.value.code == -1
        trh = tr.cpu().numpy()
        # the points outside were never written; the valid ones were recorded
        assert np.all(trh[:, len(good):] == 7.0)
        _, _, o = oracle_mod.propagate(vel, sp, dt, 10, source=shot, receivers=good)
        assert rel_l2(trh[:, :len(good)], o) <= TOL
        # the error stays until the state is replaced, then the context works
        with pytest.raises(wave_lib.WaveError):
            s.synchronize()
        s.reset()
        tr2 = torch.zeros((10, len(good)), dtype=torch.float32, device="cuda")
        s.propagate(shot, 10, torch.from_numpy(good).cuda(), tr2)
        s.synchronize()
        assert rel_l2(tr2.cpu().numpy(), o) <= TOL
    finally:
        s.close()
