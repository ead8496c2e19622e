"""Shot server (include/wave_serve.h) on the GPU, through the C ABI.

The server advances every resident shot by one step per batched launch.
Each shot's arithmetic is that of the single-grid path, so its traces must
be bit-for-bit those of wave_propagate and of the same request served alone
(tolerance 0: the per-point operation order does not depend on the mix).
"""
import numpy as np
import pytest

import workloads as wl

pytestmark = pytest.mark.gpu

GB = 10 ** 9
SPEC = [  # (grid, storage, nsteps, seed)
    ((64, 48, 40), 0, 60, 1),
    ((96, 64, 72), 2, 45, 2),
    ((40, 40, 40), 0, 80, 3),
    ((72, 56, 48), 1, 50, 4),
    ((131, 37, 29), 0, 33, 5),
    ((80, 64, 96), 2, 40, 6),
]


def _inputs(grid, seed):
    import torch
    nx, ny, nz = grid
    vel = torch.from_numpy(wl.layered_volume(nx, ny, nz, seed)).cuda()
    rng = np.random.default_rng(seed)
    rec = np.concatenate([wl.receiver_plane(nx, ny, min(8, nz - 1), 5),
                          wl.random_receivers(nx, ny, nz, 11, seed)]).astype(np.int32)
    shot = (int(rng.integers(nx)), int(rng.integers(ny)), min(10, nz - 1), 15.0, -1.0, 1.0)
    return vel, torch.from_numpy(np.ascontiguousarray(rec)).cuda(), shot


def _serve(pkg, specs, budget=16 * GB, slots=16):
    import torch
    srv = pkg.ShotServer(budget, slots)
    tickets, outs = [], []
    for grid, storage, nsteps, seed in specs:
        vel, rec, shot = _inputs(grid, seed)
        tr = torch.zeros((nsteps, rec.shape[0]), device="cuda")
        tickets.append(srv.submit(grid, (10.0, 10.0, 10.0), vel, shot, nsteps, rec, tr,
                                  storage=storage))
        outs.append(tr)
    results = []
    for t in tickets:
        st, res = srv.wait(t, 120.0)
        assert st == 0, (st, res)
        results.append(res)
    stats = srv.stats()
    srv.close()
    return [o.cpu().numpy() for o in outs], results, stats


def test_alone_and_in_the_mix_are_identical(wave_lib):
    import torch
    mix, res, stats = _serve(wave_lib, SPEC)
    assert stats["resident_peak"] >= 2 and stats["completed"] == len(SPEC)
    # overlap: some shot started before another one finished
    assert min(r["done_s"] for r in res) > max(r["start_s"] for r in res[:2])
    for (grid, storage, nsteps, seed), tr_mix, r in zip(SPEC, mix, res):
        alone, res1, _ = _serve(wave_lib, [(grid, storage, nsteps, seed)])
        assert np.array_equal(alone[0], tr_mix)
        assert res1[0]["dt"] == r["dt"]
        # and the single-grid context path
        vel, rec, shot = _inputs(grid, seed)
        s = wave_lib.WaveSolver(grid, (10.0, 10.0, 10.0), r["dt"], vel, storage=storage)
        tr = torch.zeros((nsteps, rec.shape[0]), device="cuda")
        s.propagate(shot, nsteps, rec, tr)
        s.synchronize()
        s.close()
        assert np.array_equal(tr.cpu().numpy(), tr_mix)
        assert np.abs(tr_mix).max() > 0


def test_served_shots_match_the_oracle(wave_lib, oracle_mod):
    """Each shot of a served mix against the FP64 oracle on that shot's own
    model, source, receivers and time step: the batched launch (per-shot
    tensor maps, CTA-to-shot search, step offsets) computes the Eq. 1
    leapfrog update of every resident shot. Ragged sizes (nx not a multiple
    of 4, grids smaller than a tile in some axis), FP32 and FP16 in one mix.
    FP32: relative L2 <= 1e-5, the FP32 parity bar. FP16: every step rounds
    u_next to 11 significant bits (relative 2^-11) and the leapfrog carries
    the errors forward undamped, so the traces stay within 6 * 2^-11 *
    sqrt(steps), the bound of the 16-bit short-run parity tests."""
    specs = [((45, 37, 29), 0, 40, 51), ((70, 33, 41), 2, 35, 52),
             ((33, 50, 20), 0, 30, 53), ((61, 27, 35), 0, 37, 54),
             ((21, 9, 44), 2, 28, 55)]
    mix, res, stats = _serve(wave_lib, specs, slots=8)
    assert stats["completed"] == len(specs) and stats["resident_peak"] >= 3
    for (grid, storage, nsteps, seed), tr, r in zip(specs, mix, res):
        vel, rec, shot = _inputs(grid, seed)
        _, _, otr = oracle_mod.propagate(vel.cpu().numpy(), (10.0, 10.0, 10.0), r["dt"],
                                         nsteps, source=shot, receivers=rec.cpu().numpy())
        err = float(np.linalg.norm(tr.astype(np.float64) - otr) / np.linalg.norm(otr))
        tol = 1e-5 if storage == 0 else 6 * 2.0 ** -11 * np.sqrt(nsteps)
        assert err <= tol, (grid, storage, err, tol)


def test_stream_sized_shots_alone_and_in_the_mix(wave_lib):
    """Shots of the serving stream's sizes (up to 512 per axis; nz > 256 is
    split into two z layers per CTA column), FP32 and FP16 in one mix with a
    small shot: each mixed result is bit-identical to wave_propagate."""
    import torch
    specs = [((512, 384, 480), 0, 24, 31), ((448, 512, 320), 2, 20, 32),
             ((128, 160, 128), 0, 30, 33), ((256, 224, 512), 2, 18, 34)]
    mix, res, stats = _serve(wave_lib, specs, budget=40 * GB, slots=8)
    assert stats["completed"] == len(specs) and stats["resident_peak"] >= 2
    for (grid, storage, nsteps, seed), tr_mix, r in zip(specs, mix, res):
        vel, rec, shot = _inputs(grid, seed)
        s = wave_lib.WaveSolver(grid, (10.0, 10.0, 10.0), r["dt"], vel, storage=storage)
        tr = torch.zeros((nsteps, rec.shape[0]), device="cuda")
        s.propagate(shot, nsteps, rec, tr)
        s.synchronize()
        s.close()
        assert np.array_equal(tr.cpu().numpy(), tr_mix), grid
        assert np.abs(tr_mix).max() > 0


def test_budget_admission_queues_requests(wave_lib):
    # room for two of these shots at a time
    grid = (96, 96, 96)
    one = 3 * 96 * 96 * 96 * 4
    specs = [(grid, 0, 40, 10 + i) for i in range(6)]
    _, res, stats = _serve(wave_lib, specs, budget=int(2.2 * one + 4e6), slots=8)
    assert stats["bytes_peak"] <= int(2.2 * one + 4e6)
    assert stats["resident_peak"] == 2
    starts = sorted(r["start_s"] for r in res)
    dones = sorted(r["done_s"] for r in res)
    assert starts[2] >= dones[0]  # the third waited for the first to leave


def test_slot_limit(wave_lib):
    specs = [((48, 40, 36), 0, 30, 20 + i) for i in range(5)]
    _, res, stats = _serve(wave_lib, specs, slots=2)
    assert stats["resident_peak"] <= 2 and stats["completed"] == 5


def test_rejected_and_failed_requests(wave_lib):
    import torch
    srv = wave_lib.ShotServer(1 * GB, 4)
    vel, rec, shot = _inputs((32, 32, 32), 7)
    tr = torch.zeros((10, rec.shape[0]), device="cuda")
    E = wave_lib.WaveError
    with pytest.raises(E) as ei:  # source outside the grid
        srv.submit((32, 32, 32), (10.0,) * 3, vel, (40, 0, 0, 15.0, -1.0, 1.0), 10, rec, tr)
    assert ei.value.code == -1
    with pytest.raises(E) as ei:  # larger than the whole budget
        big = torch.ones((600, 600, 600), device="cuda")
        srv.submit((600, 600, 600), (10.0,) * 3, big, shot, 10)
    assert ei.value.code == -9
    bad = vel.clone()
    bad[3, 3, 3] = float("nan")
    t_bad = srv.submit((32, 32, 32), (10.0,) * 3, bad, shot, 10, rec, tr)
    t_fast = srv.submit((32, 32, 32), (10.0,) * 3, vel, shot, 10, rec, tr, dt=1.0)
    t_ok = srv.submit((32, 32, 32), (10.0,) * 3, vel, shot, 10, rec, tr)
    assert srv.wait(t_bad, 60)[0] == -1      # WAVE_EINVAL at admission
    assert srv.wait(t_fast, 60)[0] == -4     # WAVE_EUNSTABLE at admission
    assert srv.wait(t_ok, 60)[0] == 0
    st = srv.stats()
    assert st["failed"] == 2 and st["completed"] == 1
    srv.close()


def test_injected_allocation_failure(wave_lib, monkeypatch):
    # Host-side fault: the server's 3rd device allocation fails; that request
    # fails with WAVE_ENOMEM and the server keeps serving the others.
    monkeypatch.setenv("GBWAVE_SERVE_FAULT_ALLOC", "2")
    import torch
    srv = wave_lib.ShotServer(2 * GB, 4)
    monkeypatch.delenv("GBWAVE_SERVE_FAULT_ALLOC")
    tickets = []
    for i in range(3):
        vel, rec, shot = _inputs((40, 32, 24), 30 + i)
        tr = torch.zeros((12, rec.shape[0]), device="cuda")
        tickets.append(srv.submit((40, 32, 24), (10.0,) * 3, vel, shot, 12, rec, tr))
    codes = [srv.wait(t, 60)[0] for t in tickets]
    assert codes == [-2, 0, 0]
    srv.close()


def test_host_traces_match_device_traces(wave_lib):
    import torch
    grid, nsteps = (56, 40, 32), 25
    vel, rec, shot = _inputs(grid, 41)
    srv = wave_lib.ShotServer(2 * GB, 4)
    tr_d = torch.zeros((nsteps, rec.shape[0]), device="cuda")
    tr_h = np.zeros((nsteps, rec.shape[0]), dtype=np.float32)
    a = srv.submit(grid, (10.0,) * 3, vel, shot, nsteps, rec, tr_d)
    b = srv.submit(grid, (10.0,) * 3, vel, shot, nsteps, rec.cpu().numpy(), tr_h)
    assert srv.wait(a, 60)[0] == 0 and srv.wait(b, 60)[0] == 0
    srv.close()
    assert np.array_equal(tr_d.cpu().numpy(), tr_h)
