"""GPU: wave_create_async, whose velocity pass (validation and the v^2 dt^2
conversion) runs in depth slabs beside the first steps of a propagation
from rest. A step k from rest only needs the model down to depth sz + 4k
(the star stencil of Eq. 1 reaches R = 4 planes per step, Sec. 4.1); these
tests show that the deferred context gives bit for bit the results of
wave_create for sources near the top and at depth, host (pinned and
pageable) and device models, calls split across the end of the upload,
states set by hand, 16-bit storage and the CPML layer, and that invalid
models are reported by the next synchronizing call.
"""
import numpy as np
import pytest

import workloads as wl

pytestmark = pytest.mark.gpu


def _run(pkg, vel, sp, dt, shot, calls, rec, defer, storage=0, state=None, cpml=None):
    """Propagate in `calls` (step counts); returns traces and both fields."""
    import torch
    nz, ny, nx = vel.shape
    s = pkg.WaveSolver((nx, ny, nz), sp, dt, vel, storage=storage, defer=defer)
    try:
        if cpml:
            s.set_cpml(*cpml)
        if state is not None:
            s.set_state(torch.from_numpy(state[0]).cuda(), torch.from_numpy(state[1]).cuda(), 0)
        rows = []
        rd = torch.from_numpy(rec).cuda()
        for k in calls:
            tr = torch.zeros((k, rec.shape[0]), dtype=torch.float32, device="cuda")
            s.propagate(shot, k, rd, tr)
            rows.append(tr)
        u = torch.empty((nz, ny, nx), device="cuda")
        up = torch.empty((nz, ny, nx), device="cuda")
        s.get_field(0, u)
        s.get_field(1, up)
        s.synchronize()
        return torch.cat(rows).cpu().numpy(), u.cpu().numpy(), up.cpu().numpy()
    finally:
        s.close()


def _case(nx=72, ny=40, nz=200, seed=0):
    vel = wl.random_layered(nx, ny, nz, seed=seed)
    sp = (10.0, 10.0, 10.0)
    return vel, sp, 0.5 * 0.4528 * 10.0 / float(vel.max())


def _same(a, b):
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("sz,calls", [(5, [70]), (5, [3, 50, 1]), (190, [40]),
                                      (100, [33, 33])])
def test_deferred_equals_synchronous(wave_lib, sz, calls):
    import torch
    vel, sp, dt = _case()
    nz, ny, nx = vel.shape
    rec = np.ascontiguousarray(np.concatenate(
        [wl.receiver_plane(nx, ny, 8, 4), wl.receiver_plane(nx, ny, nz - 1, 8),
         np.array([[nx // 2, ny // 2, z] for z in range(nz)], dtype=np.int32)]),
        dtype=np.int32)
    shot = (nx // 2, ny // 2, sz, 15.0, -1.0, 1.0)
    ref = _run(wave_lib, vel, sp, dt, shot, calls, rec, defer=False)
    assert np.abs(ref[0]).max() > 0
    for v in (vel, torch.from_numpy(vel).pin_memory(), torch.from_numpy(vel).cuda()):
        _same(_run(wave_lib, v, sp, dt, shot, calls, rec, defer=True), ref)


def test_deferred_with_state_storage_and_layer(wave_lib):
    vel, sp, dt = _case(48, 36, 64, seed=3)
    nz, ny, nx = vel.shape
    rec = wl.receiver_plane(nx, ny, 20, 3)
    shot = (20, 18, 30, 15.0, -1.0, 1.0)
    st = wl.random_state((nz, ny, nx), seed=4)
    _same(_run(wave_lib, vel, sp, dt, shot, [9], rec, True, state=st),
          _run(wave_lib, vel, sp, dt, shot, [9], rec, False, state=st))
    _same(_run(wave_lib, vel, sp, dt, shot, [12], rec, True, storage=2),
          _run(wave_lib, vel, sp, dt, shot, [12], rec, False, storage=2))
    _same(_run(wave_lib, vel, sp, dt, shot, [40], rec, True, cpml=(6, 1e-3, 15.0)),
          _run(wave_lib, vel, sp, dt, shot, [40], rec, False, cpml=(6, 1e-3, 15.0)))


def test_deferred_reports_bad_model(wave_lib):
    import torch
    vel, sp, dt = _case(32, 32, 48, seed=5)
    nz, ny, nx = vel.shape
    rec = wl.receiver_plane(nx, ny, 4, 4)
    shot = (16, 16, 4, 15.0, -1.0, 1.0)
    bad = vel.copy()
    bad[40, 3, 7] = np.nan
    for v, dtt, code in ((bad, dt, -1), (vel, 3.0 * dt, -4)):
        s = wave_lib.WaveSolver((nx, ny, nz), sp, dtt, torch.from_numpy(v).cuda(), defer=True)
        try:
            tr = torch.zeros((5, rec.shape[0]), device="cuda")
            s.propagate(shot, 5, torch.from_numpy(rec).cuda(), tr)
            for _ in range(2):  # reported by every synchronizing call, reset or not
                with pytest.raises(wave_lib.WaveError) as ei:
                    s.synchronize()
                assert ei.value.code == code
                s.reset()
        finally:
            s.close()
    # the synchronous form rejects the same models at creation
    with pytest.raises(wave_lib.WaveError):
        wave_lib.WaveSolver((nx, ny, nz), sp, dt, bad)
