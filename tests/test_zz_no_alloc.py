"""wave_propagate_noalloc against wave_propagate, through the C ABI.

The allocation-free entry point is for callers that must not allocate device
memory, for example code running inside an application whose memory pool
already owns the GPU, plugins held to a fixed memory budget, or services
that forbid allocation after start-up. It keeps its tables in a fixed array
declared by the library and works on buffers the caller owns. This test
checks that two calls in a row give the same fields and traces as the
context-based entry point, within the parity tolerance (relative L2 1e-5),
and that a request too large for the array is refused before any launch.
The file name sorts last so that a run stopping at the first failure has
run every other test already.
"""
import numpy as np
import pytest

import workloads as wl

pytestmark = pytest.mark.gpu

TOL = 1e-5


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_noalloc_matches_propagate_on_two_calls(wave_lib):
    import torch
    nx, ny, nz = 72, 40, 36
    sp = (10.0, 12.0, 9.0)
    rng = np.random.default_rng(21)
    vel = rng.uniform(1500.0, 4000.0, size=(nz, ny, nx)).astype(np.float32)
    u0, up0 = wl.random_state((nz, ny, nx), seed=22)
    dt = 0.5 * wave_lib.wave_cfl_dt(sp, float(vel.max()))
    shot = (30, 17, 20, 15.0, 0.02, 5.0)
    rec = np.ascontiguousarray(np.concatenate(
        [wl.random_receivers(nx, ny, nz, 40, seed=23), wl.receiver_plane(nx, ny, 4, 8)]),
        dtype=np.int32)
    nrec = rec.shape[0]
    calls = [(5, 13), (18, 20)]  # (step0, nsteps): an odd then an even count

    # the context-based entry point
    ref = wave_lib.WaveSolver((nx, ny, nz), sp, dt, torch.from_numpy(vel).cuda())
    ref.set_state(u0, up0, 5)
    ref_out = []
    for step0, n in calls:
        tr = torch.zeros((n, nrec), dtype=torch.float32, device="cuda")
        ref.propagate(shot, n, torch.from_numpy(rec).cuda(), tr)
        u = np.empty((nz, ny, nx), dtype=np.float32)
        up = np.empty((nz, ny, nx), dtype=np.float32)
        ref.get_field(0, u)
        ref.get_field(1, up)
        ref_out.append((u, up, tr.cpu().numpy()))
    ref.close()

    # the allocation-free entry point on caller-owned device buffers
    vel_d = torch.from_numpy(vel).cuda()
    bufs = [torch.from_numpy(u0).cuda(), torch.from_numpy(up0).cuda()]
    rec_d = torch.from_numpy(rec).cuda()
    cur = 0  # index of the buffer holding the newest step
    for (step0, n), (ru, rup, rtr) in zip(calls, ref_out):
        tr = torch.zeros((n, nrec), dtype=torch.float32, device="cuda")
        newest = wave_lib.wave_propagate_noalloc(
            (nx, ny, nz), sp, dt, vel_d, bufs[cur], bufs[cur ^ 1], shot, step0, n,
            rec_d, tr)
        assert newest == n % 2
        if newest:
            cur ^= 1
        got_u = bufs[cur].cpu().numpy()
        got_up = bufs[cur ^ 1].cpu().numpy()
        assert rel_l2(got_u, ru) <= TOL
        assert rel_l2(got_up, rup) <= TOL
        assert rel_l2(tr.cpu().numpy(), rtr) <= TOL


def test_noalloc_refuses_requests_beyond_its_array(wave_lib):
    import torch
    nx, ny, nz = 16, 16, 16
    vel = torch.full((nz, ny, nx), 2000.0, device="cuda")
    u = torch.zeros((nz, ny, nx), device="cuda")
    up = torch.zeros((nz, ny, nx), device="cuda")
    dt = 0.5 * wave_lib.wave_cfl_dt((10.0,) * 3, 2000.0)
    nrec = 300_000  # 300000 * 16 bytes of receiver table > 4 MiB
    rec = torch.zeros((nrec, 3), dtype=torch.int32, device="cuda")
    tr = torch.zeros((1, nrec), device="cuda")
    with pytest.raises(wave_lib.WaveError) as ei:
        wave_lib.wave_propagate_noalloc((nx, ny, nz), (10.0,) * 3, dt, vel, u, up, None, 0, 1,
                                        rec, tr)
    assert ei.value.code == -9
    assert float(u.abs().max()) == 0.0 and float(tr.abs().max()) == 0.0


def test_noalloc_host_receivers_no_source_and_zero_steps(wave_lib):
    """The branches the first test does not reach: receivers in host memory
    (staged through the library's static buffer), no source (no wavelet
    block, so the tables start earlier), and nsteps = 0 (validation only,
    the buffers left as they were). A warm call also leaves the device's
    free memory unchanged: it allocates nothing."""
    import torch
    nx, ny, nz = 40, 28, 22
    sp = (10.0, 10.0, 10.0)
    rng = np.random.default_rng(31)
    vel = rng.uniform(1500.0, 3500.0, size=(nz, ny, nx)).astype(np.float32)
    u0, up0 = wl.random_state((nz, ny, nx), seed=32)
    dt = 0.45 * wave_lib.wave_cfl_dt(sp, float(vel.max()))
    rec = wl.random_receivers(nx, ny, nz, 25, seed=33)
    n = 9

    ref = wave_lib.WaveSolver((nx, ny, nz), sp, dt, torch.from_numpy(vel).cuda())
    ref.set_state(u0, up0, 0)
    rtr = np.zeros((n, rec.shape[0]), dtype=np.float32)
    ref.propagate(None, n, rec, rtr)
    ru = np.empty((nz, ny, nx), dtype=np.float32)
    ref.get_field(0, ru)
    ref.close()

    vel_d = torch.from_numpy(vel).cuda()
    bufs = [torch.from_numpy(u0).cuda(), torch.from_numpy(up0).cuda()]
    # nsteps = 0: nothing moves
    newest = wave_lib.wave_propagate_noalloc((nx, ny, nz), sp, dt, vel_d, bufs[0], bufs[1],
                                             None, 0, 0)
    assert newest == 0
    assert np.array_equal(bufs[0].cpu().numpy(), u0)
    assert np.array_equal(bufs[1].cpu().numpy(), up0)
    tr = torch.zeros((n, rec.shape[0]), dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    newest = wave_lib.wave_propagate_noalloc((nx, ny, nz), sp, dt, vel_d, bufs[0], bufs[1],
                                             None, 0, n, rec, tr)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    got = bufs[newest].cpu().numpy()
    assert rel_l2(got, ru) <= TOL
    assert rel_l2(tr.cpu().numpy(), rtr) <= TOL
