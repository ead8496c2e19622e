"""Output-buffer guards and non-finite detection, through the C ABI.

compute-sanitizer is not available to these tests, so every output buffer
the library writes (traces of wave_propagate with and without the CPML layer,
wave_get_field, the gradient, served traces) is placed inside a larger
allocation filled with a canary value, and the canaries must be untouched
afterwards: a write past either end of a buffer shows up here. A source
large enough to overflow FP32 must come back as WAVE_ENAN (the traces are
checked after every call), and wave_reset clears it.
"""
import numpy as np
import pytest

import workloads as wl

pytestmark = pytest.mark.gpu

CANARY = 12345.678
PAD = 257  # guard elements on each side (odd: not aligned to anything)


def _guarded(torch, shape):
    """A tensor of `shape` inside a canary-filled flat buffer; returns both."""
    n = int(np.prod(shape))
    flat = torch.full((n + 2 * PAD,), CANARY, dtype=torch.float32, device="cuda")
    # the payload starts PAD floats in: these outputs take any float pointer
    return flat, flat[PAD:PAD + n].view(shape)


def _guards_intact(flat):
    f = flat.cpu().numpy()
    return bool(np.all(f[:PAD] == np.float32(CANARY)) and np.all(f[-PAD:] == np.float32(CANARY)))


def _case(torch, nx=45, ny=38, nz=29, amp=1.0, t0=-1.0):
    vel = torch.from_numpy(wl.layered3(nx, ny, nz)).cuda()
    sp = (10.0, 10.0, 10.0)
    rec = torch.from_numpy(np.ascontiguousarray(np.concatenate([
        wl.receiver_plane(nx, ny, 3, 4), wl.random_receivers(nx, ny, nz, 9, 2)]),
        dtype=np.int32)).cuda()
    shot = (nx // 2, ny // 2, nz // 2, 15.0, t0, amp)
    return vel, sp, rec, shot


@pytest.mark.parametrize("npml", [0, 5])
def test_traces_and_fields_stay_inside_their_buffers(wave_lib, npml):
    import torch
    vel, sp, rec, shot = _case(torch)
    nz, ny, nx = vel.shape
    dt = 0.5 * wave_lib.wave_cfl_dt(sp, 3500.0)
    s = wave_lib.WaveSolver((nx, ny, nz), sp, dt, vel)
    try:
        s.set_cpml(npml)
        for nsteps in (7, 40):  # direct launches, then graph chunks
            flat, tr = _guarded(torch, (nsteps, rec.shape[0]))
            s.propagate(shot, nsteps, rec, tr)
            s.synchronize()
            assert _guards_intact(flat)
            assert torch.isfinite(tr).all() and tr.abs().max() > 0
        for which in (0, 1):
            flat, out = _guarded(torch, (nz, ny, nx))
            s.get_field(which, out)
            s.synchronize()
            assert _guards_intact(flat)
    finally:
        s.close()


def test_gradient_output_stays_inside_its_buffer(wave_lib):
    import torch
    vel, sp, rec, shot = _case(torch, 32, 30, 28)
    nz, ny, nx = vel.shape
    dt = 0.5 * wave_lib.wave_cfl_dt(sp, 3500.0)
    obs = torch.zeros((30, rec.shape[0]), device="cuda")
    s = wave_lib.WaveSolver((nx, ny, nz), sp, dt, vel)
    try:
        flat, g = _guarded(torch, (nz, ny, nx))
        tflat, tr = _guarded(torch, (30, rec.shape[0]))
        s.gradient(shot, 30, rec, obs, g, ckpt_every=7, traces=tr)
        s.synchronize()
        assert _guards_intact(flat) and _guards_intact(tflat)
        assert torch.isfinite(g).all()
    finally:
        s.close()


def test_served_traces_stay_inside_their_buffers(wave_lib):
    import torch
    vel, sp, rec, shot = _case(torch)
    nz, ny, nx = vel.shape
    srv = wave_lib.ShotServer(4 * 10 ** 9, 4)
    try:
        bufs = []
        for storage in (0, 2):
            flat, tr = _guarded(torch, (25, rec.shape[0]))
            t = srv.submit((nx, ny, nz), sp, vel, shot, 25, rec, tr, storage=storage)
            bufs.append((t, flat))
        for t, flat in bufs:
            assert srv.wait(t)[0] == 0
            assert _guards_intact(flat)
    finally:
        srv.close()


def test_non_finite_traces_are_reported_and_reset_clears_them(wave_lib):
    import torch
    # the wavelet's peak at step 0: v^2 dt^2 * 3e38 overflows FP32
    vel, sp, rec, shot = _case(torch, amp=3e38, t0=0.0)
    nz, ny, nx = vel.shape
    dt = 0.5 * wave_lib.wave_cfl_dt(sp, 3500.0)
    s = wave_lib.WaveSolver((nx, ny, nz), sp, dt, vel)
    try:
        tr = torch.zeros((12, rec.shape[0]), device="cuda")
        s.propagate(shot, 12, rec, tr)  # device buffers: reported at the next sync
        with pytest.raises(wave_lib.WaveError) as ei:
            s.synchronize()
        assert ei.value.code == -7
        with pytest.raises(wave_lib.WaveError) as ei:  # still recorded
            s.synchronize()
        assert ei.value.code == -7
        s.reset()
        s.synchronize()  # cleared
        ok_shot = shot[:5] + (1.0,)
        s.propagate(ok_shot, 12, rec, tr)
        s.synchronize()
        assert torch.isfinite(tr).all()
        host_tr = np.zeros((12, rec.shape[0]), dtype=np.float32)
        with pytest.raises(wave_lib.WaveError) as ei:  # host traces: at once
            s.propagate(shot, 12, rec.cpu().numpy(), host_tr)
        assert ei.value.code == -7
    finally:
        s.close()


def test_served_shot_with_non_finite_traces_fails_alone(wave_lib):
    import torch
    vel, sp, rec, shot = _case(torch)
    nz, ny, nx = vel.shape
    srv = wave_lib.ShotServer(4 * 10 ** 9, 4)
    try:
        tr_bad = torch.zeros((20, rec.shape[0]), device="cuda")
        tr_ok = torch.zeros((20, rec.shape[0]), device="cuda")
        bad = srv.submit((nx, ny, nz), sp, vel, shot[:4] + (0.0, 3e38), 20, rec, tr_bad)
        good = srv.submit((nx, ny, nz), sp, vel, shot, 20, rec, tr_ok)
        assert srv.wait(bad)[0] == -7
        assert srv.wait(good)[0] == 0
        assert torch.isfinite(tr_ok).all()
    finally:
        srv.close()
