"""Adjoint gradient d(misfit)/d(v^2) on the GPU (wave_gradient / wave_adjoint,
through the C ABI) against the FP64 oracle's discrete adjoint, finite
differences of the GPU misfit, and autograd.

Tolerance against the oracle gradient: relative L2 <= 2e-4. The GPU carries
FP32 forward and adjoint fields (about 1e-6 relative per step, growing over
60 steps to ~1e-5) into a product summed over the steps in FP64; the oracle
is FP64 throughout. A sign, index, time-alignment or segment mistake gives
O(1) errors.
"""
import numpy as np
import pytest

import workloads as wl

pytestmark = pytest.mark.gpu


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _case(cfg=wl.CFG_GRAD_SMALL):
    nx, ny, nz = cfg["shape"]
    true = wl.anomaly_model(nx, ny, nz, seed=cfg["seed"], anomaly=cfg["anomaly_mps"])
    start = wl.smoothed_start(true)
    rec = wl.receiver_plane(nx, ny, cfg["rec_z"], cfg["rec_stride"])
    shot = (nx // 2, ny // 3, 3, 25.0, -1.0, 1e3)
    return true, start, rec, shot


def _dt(pkg, cfg, *models):
    return 0.5 * pkg.wave_cfl_dt(cfg["spacing"], max(float(m.max()) for m in models) * 1.02)


def _gpu_gradient(pkg, vel, cfg, dt, shot, rec, obs, ckpt, squared=False):
    import torch
    nx, ny, nz = cfg["shape"]
    s = pkg.WaveSolver((nx, ny, nz), cfg["spacing"], dt, torch.from_numpy(vel).cuda(),
                       squared=squared)
    g = torch.empty((nz, ny, nx), device="cuda")
    tr = torch.empty((cfg["nsteps"], rec.shape[0]), device="cuda")
    mis = s.gradient(shot, cfg["nsteps"], torch.from_numpy(rec).cuda(),
                     torch.from_numpy(obs).cuda(), g, ckpt_every=ckpt, traces=tr)
    assert s.step_count == 0
    s.close()
    return mis, g.cpu().numpy(), tr.cpu().numpy()


def test_gradient_matches_oracle_adjoint(wave_lib, oracle_mod):
    cfg = wl.CFG_GRAD_SMALL
    true, start, rec, shot = _case()
    dt = _dt(wave_lib, cfg, true, start)
    n = cfg["nsteps"]
    _, _, obs = oracle_mod.propagate(true, cfg["spacing"], dt, n, source=shot, receivers=rec)
    obs = obs.astype(np.float32)
    mis, g, tr = _gpu_gradient(wave_lib, start, cfg, dt, shot, rec, obs, cfg["ckpt_every"])
    _, _, otr = oracle_mod.propagate(start, cfg["spacing"], dt, n, source=shot, receivers=rec)
    omis = 0.5 * float(np.sum((otr - obs) ** 2))
    og = oracle_mod.gradient(start, cfg["spacing"], dt, n, shot, rec, otr - obs)
    assert rel_l2(tr, otr) <= 1e-5
    assert mis == pytest.approx(omis, rel=1e-4)
    assert np.abs(og).max() > 0
    err = rel_l2(g, og)
    print("\ngradient rel-L2 vs oracle adjoint: %.3e" % err)
    assert err <= 2e-4


def test_checkpoint_interval_does_not_change_the_gradient(wave_lib, oracle_mod):
    cfg = wl.CFG_GRAD_SMALL
    true, start, rec, shot = _case()
    dt = _dt(wave_lib, cfg, true, start)
    _, _, obs = oracle_mod.propagate(true, cfg["spacing"], dt, cfg["nsteps"], source=shot,
                                     receivers=rec)
    obs = obs.astype(np.float32)
    ref = _gpu_gradient(wave_lib, start, cfg, dt, shot, rec, obs, 60)
    for k in (1, 7, 13):
        got = _gpu_gradient(wave_lib, start, cfg, dt, shot, rec, obs, k)
        # the misfit sum is FP64 atomics (order varies); the gradient's
        # per-point time sums run in step order and must be bitwise equal
        assert got[0] == pytest.approx(ref[0], rel=1e-12)
        assert np.array_equal(got[1], ref[1])


def test_long_run_across_fold_boundaries(wave_lib, oracle_mod):
    """300 steps: the double-float partial of the time sum is folded into the
    FP64 sum at absolute step 256 and at the end. The gradient matches the
    oracle adjoint within the bar, and a checkpoint every 7 steps gives it
    bitwise equal to one segment (the fold points do not depend on the
    interval)."""
    cfg = dict(wl.CFG_GRAD_SMALL, shape=(24, 22, 20), nsteps=300)
    true, start, rec, shot = _case(cfg)
    dt = _dt(wave_lib, cfg, true, start)
    n = cfg["nsteps"]
    _, _, obs = oracle_mod.propagate(true, cfg["spacing"], dt, n, source=shot, receivers=rec)
    obs = obs.astype(np.float32)
    mis, g, tr = _gpu_gradient(wave_lib, start, cfg, dt, shot, rec, obs, 7)
    mis1, g1, _ = _gpu_gradient(wave_lib, start, cfg, dt, shot, rec, obs, n)
    assert np.array_equal(g, g1)
    assert mis == pytest.approx(mis1, rel=1e-12)
    _, _, otr = oracle_mod.propagate(start, cfg["spacing"], dt, n, source=shot, receivers=rec)
    og = oracle_mod.gradient(start, cfg["spacing"], dt, n, shot, rec, otr - obs)
    assert rel_l2(tr, otr) <= 1e-5 * n / 60
    err = rel_l2(g, og)
    print("\n300-step gradient rel-L2 vs oracle adjoint: %.3e" % err)
    assert err <= 2e-4


def test_directional_derivative_matches_finite_differences(wave_lib, oracle_mod):
    """<g, dm> against (J(m + e dm) - J(m - e dm)) / 2e with the GPU misfit
    (FP32 fields: step e = 1e-3 relative keeps rounding ~1e-4 and
    truncation ~1e-6)."""
    import torch
    cfg = wl.CFG_GRAD_SMALL
    true, start, rec, shot = _case()
    dt = _dt(wave_lib, cfg, true, start)
    n = cfg["nsteps"]
    _, _, obs = oracle_mod.propagate(true, cfg["spacing"], dt, n, source=shot, receivers=rec)
    obs = obs.astype(np.float32)
    mis, g, _ = _gpu_gradient(wave_lib, start, cfg, dt, shot, rec, obs, 7)
    m = start.astype(np.float64) ** 2
    nz, ny, nx = m.shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    dm = m * np.exp(-((x - 16.0) ** 2 + (y - 16.0) ** 2 + (z - 16.0) ** 2) / 40.0)
    eps = 1e-3

    def J(mm):
        v = np.sqrt(mm).astype(np.float32)
        return _gpu_gradient(wave_lib, v, cfg, dt, shot, rec, obs, 60)[0]

    fd = (J(m + eps * dm) - J(m - eps * dm)) / (2 * eps)
    assert fd == pytest.approx(float(np.sum(g.astype(np.float64) * dm)), rel=5e-3)


def test_autograd_matches_wave_gradient(wave_lib, oracle_mod):
    import torch
    cfg = wl.CFG_GRAD_SMALL
    true, start, rec, shot = _case()
    dt = _dt(wave_lib, cfg, true, start)
    n = cfg["nsteps"]
    _, _, obs = oracle_mod.propagate(true, cfg["spacing"], dt, n, source=shot, receivers=rec)
    obs32 = torch.from_numpy(obs.astype(np.float32)).cuda()
    m = torch.from_numpy(start.astype(np.float32)).cuda() ** 2
    m.requires_grad_(True)
    tr = wave_lib.wave_traces(m, cfg["spacing"], dt, shot, n, torch.from_numpy(rec).cuda(),
                              ckpt_every=7)
    loss = 0.5 * ((tr.double() - obs32.double()) ** 2).sum()
    (gm,) = torch.autograd.grad(loss, m)
    # the same model given as m = v^2 to wave_create_m: the same arithmetic
    mis, g, _ = _gpu_gradient(wave_lib, m.detach().cpu().numpy(), cfg, dt, shot, rec,
                              obs.astype(np.float32), 7, squared=True)
    assert float(loss.detach()) == pytest.approx(mis, rel=1e-6)
    assert rel_l2(gm.cpu().numpy(), g) <= 1e-5
    # and as velocities v = sqrt(m): v^2 dt^2 within an ulp or two of m dt^2
    v = torch.sqrt(m.detach()).float().cpu().numpy()
    mis_v, g_v, _ = _gpu_gradient(wave_lib, v, cfg, dt, shot, rec, obs.astype(np.float32), 7)
    assert mis_v == pytest.approx(mis, rel=1e-5)
    assert rel_l2(g_v, g) <= 1e-4


def test_host_buffers_and_unsupported_storage(wave_lib, oracle_mod):
    import torch
    cfg = dict(wl.CFG_GRAD_SMALL, shape=(20, 18, 16), nsteps=25)
    nx, ny, nz = cfg["shape"]
    true = wl.anomaly_model(nx, ny, nz)
    rec = wl.receiver_plane(nx, ny, 3, 3)
    shot = (10, 9, 2, 25.0, -1.0, 1e3)
    dt = _dt(wave_lib, cfg, true)
    obs = np.zeros((25, rec.shape[0]), dtype=np.float32)
    a = _gpu_gradient(wave_lib, true, cfg, dt, shot, rec, obs, 5)
    s = wave_lib.WaveSolver((nx, ny, nz), cfg["spacing"], dt, true)
    gh = np.empty((nz, ny, nx), dtype=np.float32)
    mis = s.gradient(shot, 25, rec, obs, gh, ckpt_every=5)
    s.close()
    assert mis == pytest.approx(a[0], rel=1e-12) and np.array_equal(gh, a[1])
    s16 = wave_lib.WaveSolver((nx, ny, nz), cfg["spacing"], dt, true, storage=2)
    with pytest.raises(wave_lib.WaveError) as ei:
        s16.gradient(shot, 25, rec, obs, gh, ckpt_every=5)
    assert ei.value.code == -8
    s16.close()


def test_full_size_directional_derivative(wave_lib):
    """The benchmark's gradient workload (256^3, 800 steps, checkpoint every
    40): <g, dm> against central differences of the GPU misfit along
    dm = m g / max|g| (a relative change of m of at most e, largest where the
    misfit is most sensitive, so the misfit change stands far above the FP32
    rounding noise of an 800-step run; a wrong sign, scale or pattern of g
    still shows, since the differences measure the true derivative along
    dm). Two step sizes must agree with each other and with <g, dm>."""
    import torch
    cfg = wl.CFG_GRAD
    nx, ny, nz = cfg["shape"]
    true = wl.anomaly_model(nx, ny, nz, seed=cfg["seed"], anomaly=cfg["anomaly_mps"])
    start = wl.smoothed_start(true)
    rec = torch.from_numpy(wl.receiver_plane(nx, ny, cfg["rec_z"], cfg["rec_stride"])).cuda()
    shot = (nx // 2, ny // 2, 10, cfg["f_peak"], -1.0, 1.0)
    n = cfg["nsteps"]
    dt = 0.5 * wave_lib.wave_cfl_dt(cfg["spacing"], max(float(true.max()), float(start.max())) * 1.05)
    obs = torch.zeros((n, rec.shape[0]), device="cuda")
    st = wave_lib.WaveSolver((nx, ny, nz), cfg["spacing"], dt, torch.from_numpy(true).cuda())
    st.propagate(shot, n, rec, obs)
    st.close()

    def misfit_and_grad(v, want_grad):
        s = wave_lib.WaveSolver((nx, ny, nz), cfg["spacing"], dt, torch.from_numpy(v).cuda())
        g = torch.empty((nz, ny, nx), device="cuda")
        mis = s.gradient(shot, n, rec, obs, g, ckpt_every=cfg["ckpt_every"])
        s.close()
        return mis, (g.cpu().numpy().astype(np.float64) if want_grad else None)

    j0, g = misfit_and_grad(start, True)
    assert np.all(np.isfinite(g)) and np.max(np.abs(g)) > 0
    m = start.astype(np.float64) ** 2
    dm = m * g / np.max(np.abs(g))
    dot = float(np.sum(g * dm))

    def fd(eps):
        jp, _ = misfit_and_grad(np.sqrt(m + eps * dm).astype(np.float32), False)
        jm, _ = misfit_and_grad(np.sqrt(m - eps * dm).astype(np.float32), False)
        return (jp - jm) / (2 * eps)

    f1, f2 = fd(2e-3), fd(1e-3)
    print("full-size gradient test: J %.6g, <g,dm> %.6g, FD(2e-3) %.6g, FD(1e-3) %.6g"
          % (j0, dot, f1, f2))
    assert f1 == pytest.approx(f2, rel=1e-3)
    assert dot == pytest.approx(f1, rel=1e-3)
