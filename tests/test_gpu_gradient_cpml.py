"""Adjoint gradient with the CPML absorbing layer on the GPU (wave_gradient on a
context with wave_set_cpml, through the C ABI) against the FP64 oracle's
discrete adjoint of the layered run, and central differences of the GPU
misfit at the benchmark's gradient size.

Tolerances: the plain gradient's bars (traces relative L2 <= 1e-5, misfit
1e-4, gradient relative L2 <= 2e-4); the layer adds a few FP32 operations per
shell point and step, far below them. A dropped memory-variable term, a wrong
sign of the first-derivative transpose, a missing layer term in the stored
forward increment or a checkpoint without the memory variables gives O(1e-2)
or larger errors in the shell, which holds much of the gradient's norm here
(the source and the receivers sit in the layer).
"""
import numpy as np
import pytest

import workloads as wl

pytestmark = pytest.mark.gpu

R, FCPS = 1e-3, 15.0


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _gpu(pkg, vel, sp, dt, npml, shot, n, rec, obs, ckpt):
    import torch
    nz, ny, nx = vel.shape
    s = pkg.WaveSolver((nx, ny, nz), sp, dt, torch.from_numpy(vel).cuda())
    s.set_cpml(npml, R, FCPS)
    g = torch.empty((nz, ny, nx), device="cuda")
    tr = torch.empty((n, rec.shape[0]), device="cuda")
    mis = s.gradient(shot, n, torch.from_numpy(rec).cuda(), torch.from_numpy(obs).cuda(), g,
                     ckpt_every=ckpt, traces=tr)
    assert s.step_count == 0
    s.close()
    return mis, g.cpu().numpy(), tr.cpu().numpy()


# (shape (nx, ny, nz), npml, checkpoint interval): the 32^3 x 60 case with
# ragged segments; a box whose y and z lines are one segment of the whole
# line (2 (npml + 4) > n) and whose x lines have two segments that read into
# each other's slab; a checkpoint every step (60 segments cycling the two D
# slots and the layer's checkpointed memory variables).
CASES = [((32, 32, 32), 6, 7), ((21, 18, 12), 6, 11), ((24, 22, 20), 4, 1)]


# npml 8 and 16 on axes of at least 2 (npml + 4) cells run the unrolled
# segment kernels (recompute and adjoint); x = 45 and 41 leave the high-face
# x rows unaligned.
SEG_CASES = [((45, 36, 30), 8, 9), ((41, 44, 40), 16, 13)]


@pytest.mark.parametrize("shape,npml,ckpt", SEG_CASES)
def test_unrolled_segments_in_the_gradient(wave_lib, oracle_mod, monkeypatch, shape, npml, ckpt):
    """The gradient with the unrolled segment kernels equals the one with the
    line walks (GBWAVE_CPML_GENERIC=1) bit for bit, and the oracle's layered
    adjoint within the gradient bar."""
    cfg = wl.CFG_GRAD_SMALL
    nx, ny, nz = shape
    sp = cfg["spacing"]
    n = cfg["nsteps"]
    true = wl.anomaly_model(nx, ny, nz, seed=cfg["seed"], anomaly=cfg["anomaly_mps"])
    start = wl.smoothed_start(true)
    rec = wl.receiver_plane(nx, ny, 4, 3)
    shot = (nx // 2, ny // 3, 3, 25.0, -1.0, 1e3)
    dt = 0.5 * wave_lib.wave_cfl_dt(sp, max(float(true.max()), float(start.max())) * 1.02)
    _, _, _, _, obs = oracle_mod.propagate_cpml(true, sp, dt, n, npml, R=R, fcps=FCPS,
                                                source=shot, receivers=rec)
    obs = obs.astype(np.float32)
    monkeypatch.setenv("GBWAVE_CPML_GENERIC", "1")
    mis_g, g_g, tr_g = _gpu(wave_lib, start, sp, dt, npml, shot, n, rec, obs, ckpt)
    monkeypatch.delenv("GBWAVE_CPML_GENERIC")
    mis, g, tr = _gpu(wave_lib, start, sp, dt, npml, shot, n, rec, obs, ckpt)
    assert np.array_equal(tr, tr_g) and np.array_equal(g, g_g)
    assert mis == pytest.approx(mis_g, rel=1e-12)
    vmax = float(start.max())
    _, _, _, _, otr = oracle_mod.propagate_cpml(start, sp, dt, n, npml, R=R, fcps=FCPS,
                                                vmax=vmax, source=shot, receivers=rec)
    og = oracle_mod.gradient_cpml(start, sp, dt, n, npml, shot, rec, otr - obs, R=R,
                                  fcps=FCPS, vmax=vmax)
    err = rel_l2(g, og)
    print("\nCPML gradient (unrolled segments) rel-L2 vs oracle adjoint %s: %.3e" % (shape, err))
    assert err <= 2e-4


@pytest.mark.parametrize("shape,npml,ckpt", CASES)
def test_cpml_gradient_matches_oracle_adjoint(wave_lib, oracle_mod, shape, npml, ckpt):
    cfg = wl.CFG_GRAD_SMALL
    nx, ny, nz = shape
    sp = cfg["spacing"]
    n = cfg["nsteps"]
    true = wl.anomaly_model(nx, ny, nz, seed=cfg["seed"], anomaly=cfg["anomaly_mps"])
    start = wl.smoothed_start(true)
    rec = wl.receiver_plane(nx, ny, min(4, nz - 1), 2)
    shot = (nx // 2, ny // 3, 3, 25.0, -1.0, 1e3)
    dt = 0.5 * wave_lib.wave_cfl_dt(sp, max(float(true.max()), float(start.max())) * 1.02)
    _, _, _, _, obs = oracle_mod.propagate_cpml(true, sp, dt, n, npml, R=R, fcps=FCPS,
                                                source=shot, receivers=rec)
    obs = obs.astype(np.float32)
    mis, g, tr = _gpu(wave_lib, start, sp, dt, npml, shot, n, rec, obs, ckpt)
    vmax = float(start.max())
    _, _, _, _, otr = oracle_mod.propagate_cpml(start, sp, dt, n, npml, R=R, fcps=FCPS,
                                                vmax=vmax, source=shot, receivers=rec)
    omis = 0.5 * float(np.sum((otr - obs) ** 2))
    og = oracle_mod.gradient_cpml(start, sp, dt, n, npml, shot, rec, otr - obs, R=R,
                                  fcps=FCPS, vmax=vmax)
    assert rel_l2(tr, otr) <= 1e-5
    assert mis == pytest.approx(omis, rel=1e-4)
    # the layer carries a real share of the gradient
    shell = np.ones(og.shape, dtype=bool)
    shell[npml:nz - npml, npml:ny - npml, npml:nx - npml] = False
    assert np.linalg.norm(og[shell]) > 0.1 * np.linalg.norm(og)
    err = rel_l2(g, og)
    print("\nCPML gradient rel-L2 vs oracle adjoint %s: %.3e" % (shape, err))
    assert err <= 2e-4
    # the same gradient from one segment (no recompute from a checkpoint):
    # the memory variables restored with each checkpoint reproduce the
    # forward run exactly (the misfit's FP64 atomics vary in order)
    mis1, g1, _ = _gpu(wave_lib, start, sp, dt, npml, shot, n, rec, obs, n)
    assert mis1 == pytest.approx(mis, rel=1e-12)
    assert np.array_equal(g1, g)


def test_cpml_full_size_directional_derivative(wave_lib):
    """The benchmark's gradient workload (256^3, 800 steps, checkpoint every
    40) with a 16-cell layer: <g, dm> against central differences of the GPU
    misfit along dm = m g / max|g|, set to zero where m is within 1% of its
    maximum so that the perturbed models keep the largest velocity, and with
    it the layer's profile, which the gradient holds fixed."""
    import torch
    cfg = wl.CFG_GRAD
    nx, ny, nz = cfg["shape"]
    npml = 16
    true = wl.anomaly_model(nx, ny, nz, seed=cfg["seed"], anomaly=cfg["anomaly_mps"])
    start = wl.smoothed_start(true)
    rec = torch.from_numpy(wl.receiver_plane(nx, ny, cfg["rec_z"], cfg["rec_stride"])).cuda()
    shot = (nx // 2, ny // 2, 10, cfg["f_peak"], -1.0, 1.0)
    n = cfg["nsteps"]
    dt = 0.5 * wave_lib.wave_cfl_dt(cfg["spacing"], max(float(true.max()), float(start.max())) * 1.05)
    obs = torch.zeros((n, rec.shape[0]), device="cuda")
    st = wave_lib.WaveSolver((nx, ny, nz), cfg["spacing"], dt, torch.from_numpy(true).cuda())
    st.set_cpml(npml, R, FCPS)
    st.propagate(shot, n, rec, obs)
    st.close()

    def misfit_and_grad(v, want_grad):
        s = wave_lib.WaveSolver((nx, ny, nz), cfg["spacing"], dt, torch.from_numpy(v).cuda())
        s.set_cpml(npml, R, FCPS)
        g = torch.empty((nz, ny, nx), device="cuda")
        mis = s.gradient(shot, n, rec, obs, g, ckpt_every=cfg["ckpt_every"])
        s.close()
        return mis, (g.cpu().numpy().astype(np.float64) if want_grad else None)

    j0, g = misfit_and_grad(start, True)
    assert np.all(np.isfinite(g)) and np.max(np.abs(g)) > 0
    m = start.astype(np.float64) ** 2
    dm = np.where(m < 0.99 * m.max(), m * g / np.max(np.abs(g)), 0.0)
    # the same direction restricted to the layer's cells
    shell = np.ones(m.shape, dtype=bool)
    shell[npml:nz - npml, npml:ny - npml, npml:nx - npml] = False
    dms = np.where(shell, dm, 0.0)

    def fd(eps, d):
        vp = np.sqrt(m + eps * d).astype(np.float32)
        vm = np.sqrt(m - eps * d).astype(np.float32)
        assert vp.max() == start.max() and vm.max() == start.max()
        jp, _ = misfit_and_grad(vp, False)
        jm, _ = misfit_and_grad(vm, False)
        return (jp - jm) / (2 * eps)

    # The misfit of one FP32 run carries rounding noise of about 1e-6 of J,
    # about 1e-3 of the difference quotient at e = 1e-3 and half that at
    # 2e-3: the two step sizes agree within 2e-3, and <g, dm> meets the
    # larger step within 1e-3.
    for name, d in (("m g / max|g|", dm), ("layer cells only", dms)):
        dot = float(np.sum(g * d))
        f1, f2 = fd(2e-3, d), fd(1e-3, d)
        print("full-size CPML gradient along %s: J %.6g, <g,dm> %.6g, FD(2e-3) %.6g, "
              "FD(1e-3) %.6g" % (name, j0, dot, f1, f2))
        assert f1 == pytest.approx(f2, rel=2e-3)
        assert dot == pytest.approx(f1, rel=1e-3)


def test_autograd_with_the_layer(wave_lib, oracle_mod):
    """wave_traces(m, ..., cpml=(npml, R, f_cps)) under torch.autograd: the
    misfit and dJ/dm equal the oracle's layered run and adjoint within the
    gradient bar, and wave_gradient on the same velocities within 1e-4 (the
    library squares v in FP32 there)."""
    import torch
    cfg = wl.CFG_GRAD_SMALL
    nx, ny, nz = 32, 32, 32
    npml = 6
    sp = cfg["spacing"]
    n = cfg["nsteps"]
    true = wl.anomaly_model(nx, ny, nz, seed=cfg["seed"], anomaly=cfg["anomaly_mps"])
    start = wl.smoothed_start(true)
    rec = wl.receiver_plane(nx, ny, 4, 2)
    shot = (nx // 2, ny // 3, 3, 25.0, -1.0, 1e3)
    dt = 0.5 * wave_lib.wave_cfl_dt(sp, max(float(true.max()), float(start.max())) * 1.02)
    _, _, _, _, obs = oracle_mod.propagate_cpml(true, sp, dt, n, npml, R=R, fcps=FCPS,
                                                source=shot, receivers=rec)
    obs32 = torch.from_numpy(obs.astype(np.float32)).cuda()
    m = torch.from_numpy(start.astype(np.float32)).cuda() ** 2
    m.requires_grad_(True)
    tr = wave_lib.wave_traces(m, sp, dt, shot, n, torch.from_numpy(rec).cuda(), ckpt_every=7,
                              cpml=(npml, R, FCPS))
    loss = 0.5 * ((tr.double() - obs32.double()) ** 2).sum()
    (gm,) = torch.autograd.grad(loss, m)
    vmax = float(start.max())
    _, _, _, _, otr = oracle_mod.propagate_cpml(start, sp, dt, n, npml, R=R, fcps=FCPS,
                                                vmax=vmax, source=shot, receivers=rec)
    og = oracle_mod.gradient_cpml(start, sp, dt, n, npml, shot, rec, otr - obs, R=R,
                                  fcps=FCPS, vmax=vmax)
    assert float(loss.detach()) == pytest.approx(0.5 * float(np.sum((otr - obs) ** 2)),
                                                 rel=1e-4)
    assert rel_l2(gm.cpu().numpy(), og) <= 2e-4
    _, g, _ = _gpu(wave_lib, start, sp, dt, npml, shot, n, rec, obs.astype(np.float32), 7)
    assert rel_l2(gm.cpu().numpy(), g) <= 1e-4
