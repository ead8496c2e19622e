"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerance: relative L2 <= 1e-5 on fields and traces, the bar the FP32 path
is held to after 100 steps of the 64^3 layered workload. Per-step FP32
rounding of the 25-term sum is ~1e-7 relative; it accumulates roughly
linearly over steps, so 1e-5 leaves margin at 100 steps while still failing
on any wrong weight, index, sign or boundary (those give O(1e-2) or worse).
"""
import math

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


def _torch():
    import torch
    return torch


def gpu_run(pkg, vel, spacing, dt, nsteps, u0=None, up0=None, step0=0, shot=None,
            rec=None, device_io=True, chunks=None):
    """Run the CUDA path; returns (u, u_prev, traces) as float64 numpy arrays."""
    torch = _torch()
    nz, ny, nx = vel.shape
    v = torch.from_numpy(vel).cuda() if device_io else np.ascontiguousarray(vel)
    solver = pkg.WaveSolver((nx, ny, nz), spacing, dt, v)
    try:
        if u0 is not None:
            if device_io:
                solver.set_state(torch.from_numpy(u0).cuda(), torch.from_numpy(up0).cuda(), step0)
            else:
                solver.set_state(u0, up0, step0)
        nrec = 0 if rec is None else rec.shape[0]
        traces = np.zeros((nsteps, nrec), dtype=np.float32)
        steps = chunks or [nsteps]
        row = 0
        for k in steps:
            if device_io:
                r = torch.from_numpy(rec).cuda() if nrec else None
                t = torch.zeros((k, nrec), dtype=torch.float32, device="cuda") if nrec else None
                solver.propagate(shot, k, r, t)
                if nrec:
                    traces[row:row + k] = t.cpu().numpy()
            else:
                t = np.zeros((k, nrec), dtype=np.float32) if nrec else None
                solver.propagate(shot, k, rec if nrec else None, t)
                if nrec:
                    traces[row:row + k] = t
            row += k
        out_u = np.empty((nz, ny, nx), dtype=np.float32)
        out_up = np.empty((nz, ny, nx), dtype=np.float32)
        solver.get_field(0, out_u)
        solver.get_field(1, out_up)
        assert solver.step_count == step0 + nsteps
        solver.synchronize()
    finally:
        solver.close()
    return out_u.astype(np.float64), out_up.astype(np.float64), traces.astype(np.float64)


def test_cfl_matches_oracle(wave_lib, oracle_mod):
    for sp, v in (((10.0, 10.0, 10.0), 3500.0), ((7.0, 12.5, 9.0), 4321.0)):
        assert wave_lib.wave_cfl_dt(sp, v) == pytest.approx(oracle_mod.cfl_dt(sp, v), rel=1e-15)


def test_small_layered_workload_100_steps(wave_lib, oracle_mod):
    cfg = wl.CFG_SMALL
    nx, ny, nz = cfg["shape"]
    vel = wl.velocity_for(cfg)
    sp = cfg["spacing"]
    dt = cfg["cfl_fraction"] * wave_lib.wave_cfl_dt(sp, float(vel.max()))
    dt_o = cfg["cfl_fraction"] * oracle_mod.cfl_dt(sp, float(vel.max()))
    assert dt == pytest.approx(dt_o, rel=1e-15)
    plane = wl.receiver_plane(nx, ny, cfg["rec_z"], cfg["rec_stride"])
    line = np.array([[x, 32, 32] for x in range(nx)], dtype=np.int32)
    rec = np.ascontiguousarray(np.concatenate([line, plane]), dtype=np.int32)
    shot = (*cfg["source"], cfg["f_peak"], -1.0, 1.0)
    n = cfg["nsteps"]
    gu, gup, gtr = gpu_run(wave_lib, vel, sp, dt, n, shot=shot, rec=rec)
    ou, oup, otr = oracle_mod.propagate(vel, sp, dt_o, n, source=shot, receivers=rec)
    assert np.linalg.norm(ou) > 0
    assert rel_l2(gu, ou) <= TOL
    assert rel_l2(gup, oup) <= TOL
    assert rel_l2(gtr, otr) <= TOL
    # the z = 8 plane barely sees the wavelet yet: absolute check against the field scale
    scale = np.max(np.abs(ou))
    assert np.max(np.abs(gtr[:, nx:] - otr[:, nx:])) <= 1e-6 * scale


RAGGED = [
    # (nx, ny, nz), spacing, nsteps  -- tile edges, ragged tails, tiny grids
    ((70, 37, 23), (10.0, 12.0, 8.0), 7),
    ((64, 16, 9), (10.0, 10.0, 10.0), 6),
    ((5, 3, 2), (9.0, 10.0, 11.0), 5),
    ((1, 1, 1), (10.0, 10.0, 10.0), 3),
    ((131, 19, 40), (12.0, 9.0, 10.0), 34),   # > one graph chunk, even count
    ((33, 65, 17), (10.0, 10.0, 13.0), 33),   # graph chunk + odd remainder
    ((3, 100, 12), (10.0, 10.0, 10.0), 4),
]


@pytest.mark.parametrize("shape,spacing,nsteps", RAGGED)
def test_ragged_random_state(wave_lib, oracle_mod, shape, spacing, nsteps):
    nx, ny, nz = shape
    rng = np.random.default_rng(nx * 10007 + ny * 101 + nz)
    vel = rng.uniform(1500.0, 4500.0, size=(nz, ny, nx)).astype(np.float32)
    u0, up0 = wl.random_state((nz, ny, nx), seed=nx + ny + nz)
    dt = 0.45 * wave_lib.wave_cfl_dt(spacing, float(vel.max()))
    rec = wl.random_receivers(nx, ny, nz, 17, seed=3)
    shot = (nx // 2, ny // 3, nz - 1, 15.0, 0.01, 1e-3)
    gu, gup, gtr = gpu_run(wave_lib, vel, spacing, dt, nsteps, u0, up0, 11, shot, rec)
    ou, oup, otr = oracle_mod.propagate(vel, spacing, dt, nsteps, u=u0, u_prev=up0, step0=11,
                                        source=shot, receivers=rec)
    assert rel_l2(gu, ou) <= TOL
    assert rel_l2(gup, oup) <= TOL
    assert rel_l2(gtr, otr) <= TOL


def test_host_and_device_buffers_agree_bitwise(wave_lib):
    nx, ny, nz = 40, 30, 20
    vel = wl.layered3(nx, ny, nz)
    sp = (10.0, 10.0, 10.0)
    dt = 0.5 * wave_lib.wave_cfl_dt(sp, 3500.0)
    rec = wl.receiver_plane(nx, ny, 5, 3)
    shot = (20, 15, 10, 15.0, -1.0, 1.0)
    a = gpu_run(wave_lib, vel, sp, dt, 37, shot=shot, rec=rec, device_io=True)
    b = gpu_run(wave_lib, vel, sp, dt, 37, shot=shot, rec=rec, device_io=False)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_split_calls_equal_one_call(wave_lib):
    nx, ny, nz = 48, 40, 36
    vel = wl.layered3(nx, ny, nz)
    sp = (10.0, 10.0, 10.0)
    dt = 0.5 * wave_lib.wave_cfl_dt(sp, 3500.0)
    rec = wl.receiver_plane(nx, ny, 8, 4)
    shot = (24, 20, 18, 15.0, -1.0, 1.0)
    whole = gpu_run(wave_lib, vel, sp, dt, 75, shot=shot, rec=rec)
    split = gpu_run(wave_lib, vel, sp, dt, 75, shot=shot, rec=rec, chunks=[33, 1, 41])
    for x, y in zip(whole, split):
        assert np.array_equal(x, y)


def test_step_without_source_is_propagate_without_source(wave_lib):
    torch = _torch()
    nx, ny, nz = 36, 28, 20
    vel = wl.layered3(nx, ny, nz)
    u0, up0 = wl.random_state((nz, ny, nx), seed=9)
    sp = (10.0, 10.0, 10.0)
    dt = 0.5 * wave_lib.wave_cfl_dt(sp, 3500.0)
    outs = []
    for use_step in (True, False):
        s = wave_lib.WaveSolver((nx, ny, nz), sp, dt, torch.from_numpy(vel).cuda())
        s.set_state(u0, up0)
        if use_step:
            s.step(13)
        else:
            s.propagate(None, 13)
        o = np.empty((nz, ny, nx), dtype=np.float32)
        outs.append(s.get_field(0, o).copy())
        s.close()
    assert np.array_equal(outs[0], outs[1])


def test_reset_and_zero_steps(wave_lib):
    nx, ny, nz = 20, 20, 20
    vel = wl.layered3(nx, ny, nz)
    sp = (10.0, 10.0, 10.0)
    dt = 0.5 * wave_lib.wave_cfl_dt(sp, 3500.0)
    s = wave_lib.WaveSolver((nx, ny, nz), sp, dt, vel)
    s.propagate((10, 10, 10, 15.0, -1.0, 1.0), 0)
    assert s.step_count == 0
    s.propagate((10, 10, 10, 15.0, -1.0, 1.0), 40)
    o = np.empty((nz, ny, nx), dtype=np.float32)
    assert np.abs(s.get_field(0, o)).max() > 0
    s.reset()
    assert s.step_count == 0
    assert np.abs(s.get_field(0, o)).max() == 0
    assert np.abs(s.get_field(1, o)).max() == 0
    s.close()


def test_invalid_inputs_are_rejected(wave_lib):
    nx, ny, nz = 16, 16, 16
    vel = wl.layered3(nx, ny, nz)
    sp = (10.0, 10.0, 10.0)
    lim = wave_lib.wave_cfl_dt(sp, 3500.0)
    E = wave_lib.WaveError
    with pytest.raises(E) as ei:
        wave_lib.WaveSolver((nx, ny, nz), sp, lim * 1.01, vel)
    assert ei.value.code == -4
    bad = vel.copy()
    bad[3, 4, 5] = np.nan
    with pytest.raises(E) as ei:
        wave_lib.WaveSolver((nx, ny, nz), sp, 0.5 * lim, bad)
    assert ei.value.code == -1
    bad = vel.copy()
    bad[0, 0, 0] = 0.0
    with pytest.raises(E):
        wave_lib.WaveSolver((nx, ny, nz), sp, 0.5 * lim, bad)
    with pytest.raises(E) as ei:
        wave_lib.WaveSolver((nx, ny, nz), sp, 0.5 * lim, vel, storage=7)
    assert ei.value.code == -8
    with pytest.raises(E):
        wave_lib.WaveSolver((0, ny, nz), sp, 0.5 * lim, vel)
    s = wave_lib.WaveSolver((nx, ny, nz), sp, 0.5 * lim, vel)
    tr = np.zeros((4, 1), dtype=np.float32)
    for shot in ((16, 0, 0, 15.0, -1.0, 1.0), (0, -1, 0, 15.0, -1.0, 1.0),
                 (0, 0, 0, 0.0, -1.0, 1.0)):
        with pytest.raises(E):
            s.propagate(shot, 4)
    for r in ([[0, 0, 16]], [[-1, 0, 0]], [[0, 16, 0]]):
        with pytest.raises(E):
            s.propagate(None, 4, np.array(r, dtype=np.int32), tr)
    with pytest.raises(E):
        wave_lib.wave_step(s.ctx, -1)
    assert s.step_count == 0  # nothing was launched by the rejected calls
    s.close()


def test_bounded_wait_reports_timeout(wave_lib):
    # A barrier that nothing arrives on: the bounded wait must give up and the
    # library must return WAVE_ETIMEOUT with the context still usable.
    assert wave_lib.wave_selftest_wait(20_000_000) == -5
    nx = ny = nz = 8
    vel = wl.layered3(nx, ny, nz)
    s = wave_lib.WaveSolver((nx, ny, nz), (10.0,) * 3, 1e-4, vel)
    s.step(3)
    s.synchronize()
    s.close()


def _sub_box_oracle(oracle_mod, vel, u0, up0, sp, dt, n, p, shot, step0=0):
    """Exact oracle value at point p after n steps from a sub-box of radius 4n."""
    nz, ny, nx = vel.shape
    x, y, z = p
    r = 4 * n
    xl, xh = max(0, x - r), min(nx, x + r + 1)
    yl, yh = max(0, y - r), min(ny, y + r + 1)
    zl, zh = max(0, z - r), min(nz, z + r + 1)
    sl = (slice(zl, zh), slice(yl, yh), slice(xl, xh))
    src = None
    if shot is not None:
        sx, sy, sz = shot[:3]
        if xl <= sx < xh and yl <= sy < yh and zl <= sz < zh:
            src = (sx - xl, sy - yl, sz - zl, *shot[3:])
    rec = np.array([[x - xl, y - yl, z - zl]], dtype=np.int32)
    u, _, tr = oracle_mod.propagate(vel[sl], sp, dt, n, u=u0[sl], u_prev=up0[sl],
                                    step0=step0, source=src, receivers=rec)
    return u[z - zl, y - yl, x - xl], tr[:, 0]


@pytest.mark.parametrize("cfg", [wl.CFG_512, wl.CFG_1024], ids=lambda c: c["name"])
def test_full_size_sampled_points(wave_lib, oracle_mod, cfg):
    """Full-size grid in the benchmark's launch configuration, checked at sampled
    points (tile corners, domain edges, the source, receivers) against the
    oracle on the sub-box each point depends on."""
    torch = _torch()
    nx, ny, nz = cfg["shape"]
    vel = wl.velocity_for(cfg)
    sp = cfg["spacing"]
    dt = cfg["cfl_fraction"] * wave_lib.wave_cfl_dt(sp, float(vel.max()))
    g = torch.Generator(device="cuda")
    g.manual_seed(1234)
    u0 = torch.rand((nz, ny, nx), generator=g, device="cuda") * 2 - 1
    up0 = torch.rand((nz, ny, nx), generator=g, device="cuda") * 2 - 1
    n = 3
    shot = (*cfg["source"], cfg["f_peak"], -1.0, 1e4)
    rec_all = wl.receiver_plane(nx, ny, cfg["rec_z"], cfg["rec_stride"])
    s = wave_lib.WaveSolver((nx, ny, nz), sp, dt, torch.from_numpy(vel).cuda())
    s.set_state(u0, up0, 0)
    tr = torch.zeros((n, rec_all.shape[0]), dtype=torch.float32, device="cuda")
    s.propagate(shot, n, torch.from_numpy(rec_all).cuda(), tr)
    out = torch.empty((nz, ny, nx), dtype=torch.float32, device="cuda")
    s.get_field(0, out)
    s.synchronize()
    info = s.launch_info()
    s.close()
    u0h, up0h = u0.cpu().numpy(), up0.cpu().numpy()
    outh = out.cpu().numpy()
    trh = tr.cpu().numpy()
    rng = np.random.default_rng(0)
    tx, ty, zc = info["tile_x"], info["tile_y"], info["z_chunk"]
    pts = [(0, 0, 0), (nx - 1, ny - 1, nz - 1), (nx - 1, 0, nz // 2), cfg["source"],
           (cfg["source"][0] + 3, cfg["source"][1] - 2, cfg["source"][2] + 1),
           (tx - 1, ty, zc - 1), (tx, ty - 1, zc), (2 * tx - 1, 2 * ty - 1, min(nz - 1, 2 * zc))]
    pts += [tuple(int(v) for v in (rng.integers(nx), rng.integers(ny), rng.integers(nz)))
            for _ in range(12)]
    for p in pts:
        want, _ = _sub_box_oracle(oracle_mod, vel, u0h, up0h, sp, dt, n, p, shot)
        got = outh[p[2], p[1], p[0]]
        assert abs(got - want) <= 2e-5 * max(1.0, abs(want)), (p, got, want)
    near = np.argsort(np.abs(rec_all[:, 0] - cfg["source"][0])
                      + np.abs(rec_all[:, 1] - cfg["source"][1]))[:4]
    for r in list(near) + list(rng.integers(0, rec_all.shape[0], 4)):
        _, want_tr = _sub_box_oracle(oracle_mod, vel, u0h, up0h, sp, dt, n,
                                     tuple(int(v) for v in rec_all[r]), shot)
        np.testing.assert_allclose(trh[:, r], want_tr, rtol=2e-5, atol=2e-5)


def _hash_field(x, y, z, k):
    """Deterministic values in [-1, 1) from integer coordinates (numpy or
    torch int64 arrays): a multiplicative hash keeps 20 bits, so the float32
    value is exact and the same on the host and the device."""
    a, b, c = ((73856093, 19349663, 83492791), (50331653, 12582917, 25165843))[k]
    h = (x * a) ^ (y * b) ^ (z * c)
    return (h & 0xFFFFF).float() / 524288.0 - 1.0 if hasattr(h, "float") else \
        (h & 0xFFFFF).astype(np.float32) / np.float32(524288.0) - np.float32(1.0)


def test_grid_beyond_2_31_points(wave_lib, oracle_mod):
    """2048 x 1024 x 1040 = 2.18e9 points (more than 2^31; 26 GB of fields):
    3 steps from a hashed state with source and receivers, checked at points
    near the far end of the grid and at tile and layer edges against the
    oracle on sub-boxes (the state of a sub-box is recomputed on the host from
    the same hash)."""
    import torch
    nx, ny, nz = 2048, 1024, 1040
    assert nx * ny * nz > 2 ** 31
    sp = (10.0, 10.0, 10.0)
    vz = wl.layered_profile(nz, 5)
    dt = 0.5 * wave_lib.wave_cfl_dt(sp, float(vz.max()))
    vel = torch.from_numpy(vz).cuda()[:, None, None].expand(nz, ny, nx).contiguous()
    u0 = torch.empty((nz, ny, nx), device="cuda")
    up0 = torch.empty((nz, ny, nx), device="cuda")
    xs = torch.arange(nx, device="cuda", dtype=torch.int64)[None, None, :]
    ys = torch.arange(ny, device="cuda", dtype=torch.int64)[None, :, None]
    for z0 in range(0, nz, 64):
        zs = torch.arange(z0, min(nz, z0 + 64), device="cuda", dtype=torch.int64)[:, None, None]
        u0[z0:z0 + 64] = _hash_field(xs, ys, zs, 0)
        up0[z0:z0 + 64] = _hash_field(xs, ys, zs, 1)
    n = 3
    shot = (nx - 5, ny - 7, nz - 9, 15.0, -1.0, 1e3)
    rec = np.array([[nx - 1, ny - 1, nz - 1], [nx - 5, ny - 7, nz - 9], [17, 900, 1030],
                    [2000, 3, 600]], dtype=np.int32)
    s = wave_lib.WaveSolver((nx, ny, nz), sp, dt, vel)
    del vel
    s.set_state(u0, up0, 0)
    del u0, up0
    tr = torch.zeros((n, rec.shape[0]), device="cuda")
    s.propagate(shot, n, torch.from_numpy(rec).cuda(), tr)
    out = torch.empty((nz, ny, nx), device="cuda")
    s.get_field(0, out)
    s.synchronize()
    info = s.launch_info()
    s.close()
    trh = tr.cpu().numpy()
    tx, ty, zc = info["tile_x"], info["tile_y"], info["z_chunk"]
    pts = [(nx - 1, ny - 1, nz - 1), (nx - 5, ny - 7, nz - 9), (0, 0, nz - 1), (nx - 1, 0, 0),
           (tx, ty - 1, zc), (tx - 1, ty, zc - 1), (1234, 567, 890), (2047, 1023, 520)]

    def sub_box(p):
        x, y, z = p
        r = 4 * n
        lo = [max(0, c - r) for c in (x, y, z)]
        hi = [min(m, c + r + 1) for c, m in zip((x, y, z), (nx, ny, nz))]
        X = np.arange(lo[0], hi[0], dtype=np.int64)[None, None, :]
        Y = np.arange(lo[1], hi[1], dtype=np.int64)[None, :, None]
        Z = np.arange(lo[2], hi[2], dtype=np.int64)[:, None, None]
        vb = np.broadcast_to(vz[lo[2]:hi[2], None, None],
                             (hi[2] - lo[2], hi[1] - lo[1], hi[0] - lo[0])).copy()
        src = None
        if all(lo[i] <= shot[i] < hi[i] for i in range(3)):
            src = (shot[0] - lo[0], shot[1] - lo[1], shot[2] - lo[2], *shot[3:])
        r1 = np.array([[x - lo[0], y - lo[1], z - lo[2]]], dtype=np.int32)
        u, _, t = oracle_mod.propagate(vb, sp, dt, n, u=_hash_field(X, Y, Z, 0),
                                       u_prev=_hash_field(X, Y, Z, 1), source=src,
                                       receivers=r1)
        return u[z - lo[2], y - lo[1], x - lo[0]], t[:, 0]

    for p in pts:
        want, _ = sub_box(p)
        got = float(out[p[2], p[1], p[0]].item())
        assert abs(got - want) <= 2e-5 * max(1.0, abs(want)), (p, got, want)
    for r in range(rec.shape[0]):
        _, want_tr = sub_box(tuple(int(v) for v in rec[r]))
        np.testing.assert_allclose(trh[:, r], want_tr, rtol=2e-5, atol=2e-5)
