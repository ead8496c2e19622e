"""Shot server with the CPML layer (wave_request.npml > 0), through the C ABI.

A layered shot's batched step is the batched sweep followed by the layer's
three axis passes and the shell receivers, in launches shared by the layered
shots of a storage type; its profile comes from the shot's own largest
velocity and time step. Its arithmetic is that of wave_propagate on a
context with wave_set_cpml (the line walks there equal the unrolled segment
kernels bit for bit), so the traces must match it exactly, in any mix with
plain shots; against the FP64 oracle the bars of the single-grid CPML tests
hold (FP32: relative L2 <= 1e-5; FP16: 12 * 2^-11 * sqrt(steps), twice the
plain 16-bit bound for the shell points' extra roundings).
"""
import numpy as np
import pytest

import workloads as wl

pytestmark = pytest.mark.gpu

GB = 10 ** 9
SP = (10.0, 10.0, 10.0)
# (grid, storage, nsteps, seed, npml): layered and plain shots, FP32 and
# 16-bit, ragged sizes, layer widths on and off the unrolled forms
SPEC = [((64, 48, 40), 0, 45, 1, 8), ((70, 33, 41), 2, 35, 2, 6),
        ((45, 37, 29), 0, 40, 3, 0), ((80, 64, 44), 1, 30, 4, 16),
        ((61, 27, 35), 0, 37, 5, 5), ((48, 40, 36), 2, 33, 6, 0)]
R, FCPS = 1e-3, 15.0


def _inputs(grid, seed, npml):
    import torch
    nx, ny, nz = grid
    vel = torch.from_numpy(wl.layered_volume(nx, ny, nz, seed)).cuda()
    rng = np.random.default_rng(seed)
    # receivers on a plane inside the z layer, random ones, and a corner
    rec = np.concatenate([wl.receiver_plane(nx, ny, min(3, nz - 1), 5),
                          wl.random_receivers(nx, ny, nz, 11, seed),
                          np.array([[0, 0, 0], [nx - 1, ny - 1, nz - 1]])]).astype(np.int32)
    shot = (int(rng.integers(nx)), int(rng.integers(ny)), min(max(npml, 2), nz - 1), 15.0,
            -1.0, 1.0)
    return vel, torch.from_numpy(np.ascontiguousarray(rec)).cuda(), shot


def _serve(pkg, specs, budget=16 * GB, slots=16):
    import torch
    srv = pkg.ShotServer(budget, slots)
    tickets, outs = [], []
    for grid, storage, nsteps, seed, npml in specs:
        vel, rec, shot = _inputs(grid, seed, npml)
        tr = torch.zeros((nsteps, rec.shape[0]), device="cuda")
        tickets.append(srv.submit(grid, SP, vel, shot, nsteps, rec, tr, storage=storage,
                                  cpml=(npml, R, FCPS) if npml else None))
        outs.append(tr)
    results = []
    for t in tickets:
        st, res = srv.wait(t, 120.0)
        assert st == 0, (st, res)
        results.append(res)
    stats = srv.stats()
    srv.close()
    return [o.cpu().numpy() for o in outs], results, stats


def test_layered_shots_in_a_mix_equal_the_single_grid_path(wave_lib):
    import torch
    mix, res, stats = _serve(wave_lib, SPEC)
    assert stats["completed"] == len(SPEC) and stats["resident_peak"] >= 3
    for (grid, storage, nsteps, seed, npml), tr_mix, r in zip(SPEC, mix, res):
        vel, rec, shot = _inputs(grid, seed, npml)
        s = wave_lib.WaveSolver(grid, SP, r["dt"], vel, storage=storage)
        if npml:
            s.set_cpml(npml, R, FCPS)
        tr = torch.zeros((nsteps, rec.shape[0]), device="cuda")
        s.propagate(shot, nsteps, rec, tr)
        s.synchronize()
        s.close()
        assert np.array_equal(tr.cpu().numpy(), tr_mix), (grid, storage, npml)
        assert np.abs(tr_mix).max() > 0
    # a layered shot alone equals the same shot in the mix
    alone, _, _ = _serve(wave_lib, [SPEC[0]])
    assert np.array_equal(alone[0], mix[0])


def test_layered_served_shots_match_the_oracle(wave_lib, oracle_mod):
    specs = [s for s in SPEC if s[4] > 0 and s[1] in (0, 2)]
    mix, res, _ = _serve(wave_lib, specs)
    for (grid, storage, nsteps, seed, npml), tr, r in zip(specs, mix, res):
        vel, rec, shot = _inputs(grid, seed, npml)
        v = vel.cpu().numpy()
        _, _, _, _, otr = oracle_mod.propagate_cpml(v, SP, r["dt"], nsteps, npml, R=R, fcps=FCPS,
                                                    vmax=float(v.max()), source=shot,
                                                    receivers=rec.cpu().numpy())
        err = float(np.linalg.norm(tr.astype(np.float64) - otr) / np.linalg.norm(otr))
        tol = max(1e-5, 1e-7 * nsteps) if storage == 0 else 12 * 2.0 ** -11 * np.sqrt(nsteps)
        print("\nserved CPML %s storage %d npml %d: traces rel-L2 %.3e (bound %.3e)"
              % (grid, storage, npml, err, tol))
        assert err <= tol, (grid, storage, err, tol)


def test_layer_request_checks(wave_lib):
    import torch
    srv = wave_lib.ShotServer(GB, 4)
    try:
        vel = torch.full((20, 18, 16), 2000.0, device="cuda")
        shot = (5, 5, 5, 15.0, -1.0, 1.0)
        for cpml in ((9, R, FCPS), (4, 0.0, FCPS), (4, 1.0, FCPS), (4, R, -1.0),
                     (4, R, float("nan")), (-1, R, FCPS)):
            with pytest.raises(wave_lib.WaveError) as ei:
                srv.submit((16, 18, 20), SP, vel, shot, 5, cpml=cpml)
            assert ei.value.code == -1, cpml
        # 2 npml == the smallest axis: accepted and run
        t = srv.submit((16, 18, 20), SP, vel, shot, 5, cpml=(8, R, FCPS))
        st, _ = srv.wait(t, 60.0)
        assert st == 0
    finally:
        srv.close()


def test_layered_shot_with_host_buffers(wave_lib):
    """A layered shot whose receivers and traces are host arrays (the server
    stages the traces on the device and copies them back at completion),
    FP16 with npml 8: the same traces as the single-grid path."""
    import torch
    grid, storage, nsteps, seed, npml = (56, 44, 40), 2, 30, 9, 8
    vel, rec, shot = _inputs(grid, seed, npml)
    rec_h = rec.cpu().numpy()
    tr_h = np.zeros((nsteps, rec_h.shape[0]), dtype=np.float32)
    srv = wave_lib.ShotServer(GB, 4)
    try:
        t = srv.submit(grid, SP, vel, shot, nsteps, rec_h, tr_h, storage=storage,
                       cpml=(npml, R, FCPS))
        st, res = srv.wait(t, 60.0)
        assert st == 0, res
    finally:
        srv.close()
    s = wave_lib.WaveSolver(grid, SP, res["dt"], vel, storage=storage)
    s.set_cpml(npml, R, FCPS)
    tr = torch.zeros((nsteps, rec_h.shape[0]), device="cuda")
    s.propagate(shot, nsteps, rec, tr)
    s.synchronize()
    s.close()
    assert np.array_equal(tr.cpu().numpy(), tr_h)
    assert np.abs(tr_h).max() > 0


def test_layer_allocation_failure_fails_that_shot_alone(wave_lib, monkeypatch):
    """Host-side fault injection: the 11th device allocation of the server
    (one of the first shot's layer slabs, after its 7 field and table
    allocations) fails. That request ends with WAVE_ENOMEM, its memory is
    given back, and the other layered shots complete with the traces of the
    single-grid path."""
    import torch
    monkeypatch.setenv("GBWAVE_SERVE_FAULT_ALLOC", "10")
    srv = wave_lib.ShotServer(GB, 4)
    monkeypatch.delenv("GBWAVE_SERVE_FAULT_ALLOC")
    specs = [((40, 36, 32), 0, 12, 30 + i, 8) for i in range(3)]
    tickets, outs = [], []
    try:
        for grid, storage, nsteps, seed, npml in specs:
            vel, rec, shot = _inputs(grid, seed, npml)
            tr = torch.zeros((nsteps, rec.shape[0]), device="cuda")
            tickets.append(srv.submit(grid, SP, vel, shot, nsteps, rec, tr, storage=storage,
                                      cpml=(npml, R, FCPS)))
            outs.append(tr)
        results = [srv.wait(t, 60) for t in tickets]
        stats = srv.stats()
    finally:
        srv.close()
    assert [r[0] for r in results] == [-2, 0, 0]
    assert stats["bytes_resident"] == 0 and stats["failed"] == 1
    for (grid, storage, nsteps, seed, npml), tr, (st, res) in list(zip(specs, outs, results))[1:]:
        vel, rec, shot = _inputs(grid, seed, npml)
        s = wave_lib.WaveSolver(grid, SP, res["dt"], vel, storage=storage)
        s.set_cpml(npml, R, FCPS)
        want = torch.zeros((nsteps, rec.shape[0]), device="cuda")
        s.propagate(shot, nsteps, rec, want)
        s.synchronize()
        s.close()
        assert np.array_equal(tr.cpu().numpy(), want.cpu().numpy())
