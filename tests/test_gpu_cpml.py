"""GPU parity of the CPML absorbing layer against the FP64 oracle.

The layer (complex-frequency-shifted CPML for the second-order equation,
after Komatitsch and Martin 2007, which the paper's boundary follows, Sec. 2)
adds per-axis memory variables psi, zeta in slabs of npml cells at each
face. The CUDA path computes the points within npml + 4 cells of a face in
separate kernels and leaves the rest to the standard sweep; these tests check
the whole field, the traces (receivers inside and outside that shell) and
the continuation of the memory variables across calls and graph chunks.

Tolerance: the FP32 path's bar, relative L2 <= max(1e-5, 1e-7 per step):
one step rounds at ~1e-7 relative and the error grows about linearly with
the steps (the plain FP32 path measures 3.8e-5 after 500 steps); a wrong
profile, sign, index or slab offset gives errors of 1e-3 or more.
"""
import numpy as np
import pytest

import workloads as wl

pytestmark = pytest.mark.gpu



def tol(nsteps):
    return max(1e-5, 1e-7 * nsteps)


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def gpu_cpml(pkg, vel, spacing, dt, chunks, npml, R, fcps, shot, rec, u0=None, up0=None,
             step0=0):
    import torch
    nz, ny, nx = vel.shape
    solver = pkg.WaveSolver((nx, ny, nz), spacing, dt, torch.from_numpy(vel).cuda())
    try:
        solver.set_cpml(npml, R, fcps)
        if u0 is not None:
            solver.set_state(torch.from_numpy(u0).cuda(), torch.from_numpy(up0).cuda(), step0)
        nrec = rec.shape[0]
        r = torch.from_numpy(rec).cuda()
        rows = []
        for k in chunks:
            t = torch.zeros((k, nrec), dtype=torch.float32, device="cuda")
            solver.propagate(shot, k, r, t)
            rows.append(t.cpu().numpy())
        u = np.empty((nz, ny, nx), dtype=np.float32)
        up = np.empty((nz, ny, nx), dtype=np.float32)
        solver.get_field(0, u)
        solver.get_field(1, up)
        assert solver.step_count == step0 + sum(chunks)
        solver.synchronize()
    finally:
        solver.close()
    return u.astype(np.float64), up.astype(np.float64), np.concatenate(rows).astype(np.float64)


def shell_receivers(nx, ny, nz, w):
    """Receivers at corners, edges and faces of the layer shell, plus interior."""
    pts = {(0, 0, 0), (nx - 1, ny - 1, nz - 1), (nx // 2, ny // 2, 0),
           (nx // 2, 0, nz // 2), (0, ny // 2, nz // 2), (nx - 1, ny // 2, nz // 2),
           (min(w, nx - 1), ny // 2, nz // 2), (nx // 2, ny // 2, nz // 2),
           (max(nx - w - 1, 0), max(ny - w - 1, 0), max(nz - w - 1, 0))}
    return np.ascontiguousarray(sorted(pts), dtype=np.int32)


def test_layered_workload_reaches_the_layer(wave_lib, oracle_mod):
    """64^3 layered model, npml 10, 240 steps: the wave crosses the layer."""
    cfg = wl.CFG_SMALL
    nx, ny, nz = cfg["shape"]
    vel = wl.velocity_for(cfg)
    sp = cfg["spacing"]
    dt = cfg["cfl_fraction"] * wave_lib.wave_cfl_dt(sp, float(vel.max()))
    rec = np.concatenate([wl.receiver_plane(nx, ny, cfg["rec_z"], cfg["rec_stride"]),
                          shell_receivers(nx, ny, nz, 14)])
    rec = np.ascontiguousarray(rec, dtype=np.int32)
    shot = (*cfg["source"], cfg["f_peak"], -1.0, 1.0)
    n = 240
    gu, gup, gtr = gpu_cpml(wave_lib, vel, sp, dt, [n], 10, 1e-3, 15.0, shot, rec)
    ou, oup, _, _, otr = oracle_mod.propagate_cpml(vel, sp, dt, n, 10, R=1e-3, fcps=15.0,
                                                   source=shot, receivers=rec)
    assert np.linalg.norm(ou) > 0
    assert rel_l2(gu, ou) <= tol(n)
    assert rel_l2(gup, oup) <= tol(n)
    assert rel_l2(gtr, otr) <= tol(n)
    # the layer's own effect is resolved far below its size
    pu, _, ptr = oracle_mod.propagate(vel, sp, dt, n, source=shot, receivers=rec)
    assert rel_l2(gu, ou) <= 1e-3 * rel_l2(pu, ou)
    assert rel_l2(gtr, otr) <= 1e-3 * rel_l2(ptr, otr)


CASES = [
    # shape, spacing, npml, chunks, source (in the shell or not)
    ((70, 37, 23), (10.0, 12.0, 8.0), 5, [7, 40, 1], (2, 3, 20)),
    ((33, 65, 17), (10.0, 10.0, 13.0), 8, [33], (16, 30, 8)),     # shell is all of z
    ((9, 8, 2), (9.0, 10.0, 11.0), 1, [5, 3], (0, 7, 1)),          # tiny grid
    ((131, 19, 40), (12.0, 9.0, 10.0), 6, [34, 30], (130, 0, 39)),  # source at a corner
]


@pytest.mark.parametrize("shape,spacing,npml,chunks,src", CASES)
def test_ragged_random_state(wave_lib, oracle_mod, shape, spacing, npml, chunks, src):
    nx, ny, nz = shape
    rng = np.random.default_rng(nx * 7919 + ny * 31 + nz + npml)
    vel = rng.uniform(1500.0, 4500.0, size=(nz, ny, nx)).astype(np.float32)
    u0, up0 = wl.random_state((nz, ny, nx), seed=nx + 2 * ny + 3 * nz)
    dt = 0.45 * wave_lib.wave_cfl_dt(spacing, float(vel.max()))
    rec = np.concatenate([wl.random_receivers(nx, ny, nz, 23, seed=5),
                          shell_receivers(nx, ny, nz, npml + 4)])
    rec = np.ascontiguousarray(rec, dtype=np.int32)
    shot = (*src, 15.0, 0.01, 1e-3)
    fc = 20.0
    gu, gup, gtr = gpu_cpml(wave_lib, vel, spacing, dt, chunks, npml, 1e-4, fc, shot, rec,
                            u0, up0, step0=3)
    ou, oup, _, _, otr = oracle_mod.propagate_cpml(
        vel, spacing, dt, sum(chunks), npml, R=1e-4, fcps=fc, u=u0, u_prev=up0, step0=3,
        source=shot, receivers=rec)
    n = sum(chunks)
    assert rel_l2(gu, ou) <= tol(n)
    assert rel_l2(gup, oup) <= tol(n)
    assert rel_l2(gtr, otr) <= tol(n)


# npml 8 and 16 on axes of at least 2 (npml + 4) cells run the unrolled
# segment kernels (both faces of a line in parallel, x rows as float4 where
# the segment is aligned); the last case keeps the line walk on y (35 < 40).
SEG_CASES = [((75, 52, 44), 8), ((72, 41, 40), 16), ((88, 40, 57), 16), ((72, 35, 44), 16)]


@pytest.mark.parametrize("shape,npml", SEG_CASES)
def test_unrolled_segments_equal_the_line_walks(wave_lib, oracle_mod, monkeypatch, shape, npml):
    """The segment kernels round every operation as the line walks do, so the
    two give the same fields and traces bit for bit (GBWAVE_CPML_GENERIC=1
    keeps the line walks); both against the oracle at the FP32 bar. Random
    state, the source inside the low z layer, shell receivers, 37 steps in
    chunks across a graph's length."""
    nx, ny, nz = shape
    sp = (10.0, 12.0, 9.0)
    rng = np.random.default_rng(npml * 7 + nx)
    vel = rng.uniform(1500.0, 4000.0, size=(nz, ny, nx)).astype(np.float32)
    u0, up0 = wl.random_state((nz, ny, nx), seed=nx + ny)
    dt = 0.5 * wave_lib.wave_cfl_dt(sp, float(vel.max()))
    shot = (nx // 3, ny - 5, 3, 20.0, -1.0, 1e3)
    rec = shell_receivers(nx, ny, nz, npml + 4)
    chunks = [3, 34]
    R, fcps = 1e-3, 15.0
    monkeypatch.setenv("GBWAVE_CPML_GENERIC", "1")
    gu, gup, gtr = gpu_cpml(wave_lib, vel, sp, dt, chunks, npml, R, fcps, shot, rec, u0, up0, 2)
    monkeypatch.delenv("GBWAVE_CPML_GENERIC")
    su, sup, s_tr = gpu_cpml(wave_lib, vel, sp, dt, chunks, npml, R, fcps, shot, rec, u0, up0, 2)
    assert np.array_equal(su, gu) and np.array_equal(sup, gup) and np.array_equal(s_tr, gtr)
    ou, _, _, _, otr = oracle_mod.propagate_cpml(vel, sp, dt, sum(chunks), npml, R=R, fcps=fcps,
                                                 u=u0, u_prev=up0, step0=2, source=shot,
                                                 receivers=rec)
    assert rel_l2(su, ou) <= tol(sum(chunks))
    assert rel_l2(s_tr, otr) <= tol(sum(chunks))


def test_layer_absorbs_compared_with_the_zero_halo(wave_lib):
    """After the wavelet has crossed the grid, the field left with the layer is
    a small fraction of the field left with the bare zero (reflecting) halo."""
    import torch
    n = 48
    vel = np.full((n, n, n), 2000.0, dtype=np.float32)
    sp = (10.0, 10.0, 10.0)
    dt = 0.5 * wave_lib.wave_cfl_dt(sp, 2000.0)
    shot = (24, 24, 24, 20.0, -1.0, 1.0)
    out = []
    for npml in (0, 12):
        s = wave_lib.WaveSolver((n, n, n), sp, dt, torch.from_numpy(vel).cuda())
        try:
            s.set_cpml(npml, 1e-3, 20.0)
            s.propagate(shot, 500)
            u = np.empty((n, n, n), dtype=np.float32)
            s.get_field(0, u)
        finally:
            s.close()
        out.append(np.linalg.norm(u[12:-12, 12:-12, 12:-12]))
    assert out[1] < 1e-3 * out[0]


def test_switching_off_and_reset(wave_lib):
    """npml 0 gives the plain path bitwise; reset clears the memory variables."""
    import torch
    nx, ny, nz = 40, 30, 20
    vel = wl.layered3(nx, ny, nz)
    sp = (10.0, 10.0, 10.0)
    dt = 0.5 * wave_lib.wave_cfl_dt(sp, 3500.0)
    rec = torch.from_numpy(wl.receiver_plane(nx, ny, 2, 3)).cuda()
    shot = (20, 15, 3, 15.0, -1.0, 1.0)

    def run(s, k=70):
        t = torch.zeros((k, rec.shape[0]), device="cuda")
        s.propagate(shot, k, rec, t)
        return t.cpu().numpy()

    plain = wave_lib.WaveSolver((nx, ny, nz), sp, dt, torch.from_numpy(vel).cuda())
    s = wave_lib.WaveSolver((nx, ny, nz), sp, dt, torch.from_numpy(vel).cuda())
    try:
        ref = run(plain)
        s.set_cpml(6)
        a = run(s)
        s.reset()
        b = run(s)
        assert np.array_equal(a, b)
        assert not np.array_equal(a, ref)
        s.set_cpml(0)
        s.reset()
        assert np.array_equal(run(s), ref)
    finally:
        plain.close()
        s.close()


def test_invalid_arguments(wave_lib):
    import torch
    E = wave_lib.WaveError
    nx, ny, nz = 24, 20, 16
    vel = torch.from_numpy(wl.layered3(nx, ny, nz)).cuda()
    sp = (10.0, 10.0, 10.0)
    dt = 0.5 * wave_lib.wave_cfl_dt(sp, 3500.0)
    s = wave_lib.WaveSolver((nx, ny, nz), sp, dt, vel)
    try:
        for args in ((-1, 1e-3, 15.0), (9, 1e-3, 15.0), (4, 0.0, 15.0), (4, 1.0, 15.0),
                     (4, 1e-3, -1.0), (4, float("nan"), 15.0)):
            with pytest.raises(E) as ei:
                s.set_cpml(*args)
            assert ei.value.code == -1
        s.set_cpml(8, 1e-3, 15.0)  # 2 npml == nz: allowed
    finally:
        s.close()


# 16-bit storage with the layer: the axis passes read and write the stored
# fields through the step's power-of-two scales (one extra rounding per pass
# at the shell points, up to three at corners) and keep psi, zeta in FP32.
STORAGE16 = {"bf16": 1, "f16": 2}
EPS16 = {"bf16": 2.0 ** -8, "f16": 2.0 ** -11}


@pytest.mark.parametrize("mode", ["bf16", "f16"])
@pytest.mark.parametrize("shape,npml", [((75, 52, 44), 8), ((70, 37, 23), 5), ((72, 41, 40), 16),
                                        ((9, 8, 2), 1)])
def test_16bit_storage_with_the_layer(wave_lib, oracle_mod, monkeypatch, mode, shape, npml):
    """Against the oracle's layered run from the state as stored, within
    12 EPS sqrt(n): twice the plain 16-bit short-run bound, for the shell
    points' extra roundings; and the unrolled segment kernels (npml 8 and 16)
    equal the line walks bit for bit in 16-bit storage too. 3 + 34 steps in
    two calls (the second runs a captured 32-step graph)."""
    import torch
    nx, ny, nz = shape
    sp = (10.0, 12.0, 9.0)
    rng = np.random.default_rng(nx + npml)
    vel = rng.uniform(1500.0, 4000.0, size=(nz, ny, nx)).astype(np.float32)
    u0, up0 = wl.random_state((nz, ny, nx), seed=ny)
    dt = 0.45 * wave_lib.wave_cfl_dt(sp, float(vel.max()))
    shot = (nx // 3, ny - 4, min(3, nz - 1), 20.0, -1.0, 1e2)
    rec = shell_receivers(nx, ny, nz, npml + 4)
    chunks = (3, 34)  # split calls, the second through a 32-step graph
    n, R, fcps = sum(chunks), 1e-3, 15.0

    def run():
        s = wave_lib.WaveSolver((nx, ny, nz), sp, dt, torch.from_numpy(vel).cuda(),
                                storage=STORAGE16[mode])
        try:
            s.set_cpml(npml, R, fcps)
            s.set_state(u0, up0, 4)
            su = np.empty((nz, ny, nx), np.float32)
            sup = np.empty((nz, ny, nx), np.float32)
            s.get_field(0, su)
            s.get_field(1, sup)
            rows = []
            for k in chunks:
                tr = torch.zeros((k, rec.shape[0]), device="cuda")
                s.propagate(shot, k, torch.from_numpy(rec).cuda(), tr)
                rows.append(tr.cpu().numpy())
            u = np.empty((nz, ny, nx), np.float32)
            s.get_field(0, u)
            s.synchronize()
            return su, sup, u, np.concatenate(rows)
        finally:
            s.close()

    su, sup, u, tr = run()
    if npml in (8, 16):
        monkeypatch.setenv("GBWAVE_CPML_GENERIC", "1")
        _, _, gu, gtr = run()
        monkeypatch.delenv("GBWAVE_CPML_GENERIC")
        assert np.array_equal(u, gu) and np.array_equal(tr, gtr)
    ou, _, _, _, otr = oracle_mod.propagate_cpml(vel, sp, dt, n, npml, R=R, fcps=fcps,
                                                 u=su, u_prev=sup, step0=4, source=shot,
                                                 receivers=rec)
    tol = 12 * EPS16[mode] * np.sqrt(n)
    eu, et = rel_l2(u, ou), rel_l2(tr, otr)
    print("\n16-bit %s CPML %s npml %d: field %.3e traces %.3e (bound %.3e)"
          % (mode, shape, npml, eu, et, tol))
    assert eu <= tol and et <= tol


def _sub_box_cpml(oracle_mod, vel, u0, up0, sp, dt, n, p, shot, npml, R, fcps, vmax):
    """Oracle value (and trace) at p after n steps with the layer, from a sub-box.

    Along each axis the sub-box either contains the grid's face (so its layer
    is the real one) or is cut far enough from p that neither the zero halo
    nor the layer the oracle also puts at the cut can reach p in n steps: a
    difference spreads at most 8 cells per step (4 through Eq. 1, 4 more
    through psi), so the cut keeps npml + 8n + 1 cells of margin."""
    nz, ny, nx = vel.shape
    m = npml + 8 * n + 1
    sl, lo = [], []
    for c, size in zip(p[::-1], (nz, ny, nx)):
        a = 0 if c - m <= 0 else c - m
        b = size if c + m + 1 >= size else c + m + 1
        sl.append(slice(a, b))
        lo.append(a)
    zl, yl, xl = lo
    sl = tuple(sl)
    src = None
    if shot is not None:
        sx, sy, sz = shot[:3]
        if sl[2].start <= sx < sl[2].stop and sl[1].start <= sy < sl[1].stop \
                and sl[0].start <= sz < sl[0].stop:
            src = (sx - xl, sy - yl, sz - zl, *shot[3:])
    rec = np.array([[p[0] - xl, p[1] - yl, p[2] - zl]], dtype=np.int32)
    u, _, _, _, tr = oracle_mod.propagate_cpml(vel[sl], sp, dt, n, npml, R=R, fcps=fcps,
                                               vmax=vmax, u=u0[sl], u_prev=up0[sl],
                                               source=src, receivers=rec)
    return u[p[2] - zl, p[1] - yl, p[0] - xl], tr[:, 0]


def test_full_size_sampled_points(wave_lib, oracle_mod):
    """1024 x 1024 x 512 random 8-layer model with the layer the benchmark
    measures (npml 16), in its launch configuration: 3 steps from a random
    state, checked at points in the layers, at corners and edges, across the
    end of the correction segments, at the source (inside the z layer) and at
    receivers (all inside the layer's shell), against the oracle on sub-boxes."""
    import torch
    cfg = wl.CFG_1024
    nx, ny, nz = cfg["shape"]
    vel = wl.velocity_for(cfg)
    sp = cfg["spacing"]
    dt = cfg["cfl_fraction"] * wave_lib.wave_cfl_dt(sp, float(vel.max()))
    npml, R, fcps = 16, 1e-3, cfg["f_peak"]
    g = torch.Generator(device="cuda")
    g.manual_seed(4321)
    u0 = torch.rand((nz, ny, nx), generator=g, device="cuda") * 2 - 1
    up0 = torch.rand((nz, ny, nx), generator=g, device="cuda") * 2 - 1
    n = 3
    shot = (*cfg["source"], cfg["f_peak"], -1.0, 1e4)
    rec_all = wl.receiver_plane(nx, ny, cfg["rec_z"], cfg["rec_stride"])
    s = wave_lib.WaveSolver((nx, ny, nz), sp, dt, torch.from_numpy(vel).cuda())
    s.set_cpml(npml, R, fcps)
    s.set_state(u0, up0, 0)
    tr = torch.zeros((n, rec_all.shape[0]), dtype=torch.float32, device="cuda")
    s.propagate(shot, n, torch.from_numpy(rec_all).cuda(), tr)
    out = torch.empty((nz, ny, nx), dtype=torch.float32, device="cuda")
    s.get_field(0, out)
    s.synchronize()
    s.close()
    u0h, up0h = u0.cpu().numpy(), up0.cpu().numpy()
    outh = out.cpu().numpy()
    trh = tr.cpu().numpy()
    vmax = float(vel.max())
    w = npml + 4
    pts = [(0, 0, 0), (nx - 1, ny - 1, nz - 1), (nx - 1, 0, nz // 2), (0, ny // 2, nz - 1),
           (npml - 1, 300, 200), (npml, 301, 201), (w - 1, 302, 202), (w, 303, 203),
           (nx - w, 500, 100), (nx - w - 1, 501, 101), (700, npml - 1, 250), (701, ny - w, 251),
           (400, 402, nz - npml), (401, 403, w - 1), (5, 7, 9), (nx - 3, ny - 9, 2),
           cfg["source"], (cfg["source"][0] + 2, cfg["source"][1], cfg["source"][2] - 3),
           (512, 512, 256)]
    for p in pts:
        want, _ = _sub_box_cpml(oracle_mod, vel, u0h, up0h, sp, dt, n, p, shot, npml, R,
                                fcps, vmax)
        got = outh[p[2], p[1], p[0]]
        assert abs(got - want) <= 2e-5 * max(1.0, abs(want)), (p, got, want)
    rng = np.random.default_rng(1)
    near = np.argsort(np.abs(rec_all[:, 0] - cfg["source"][0])
                      + np.abs(rec_all[:, 1] - cfg["source"][1]))[:3]
    for r in list(near) + [0, rec_all.shape[0] - 1] + list(rng.integers(0, rec_all.shape[0], 3)):
        _, want_tr = _sub_box_cpml(oracle_mod, vel, u0h, up0h, sp, dt, n,
                                   tuple(int(v) for v in rec_all[r]), shot, npml, R, fcps, vmax)
        np.testing.assert_allclose(trh[:, r], want_tr, rtol=2e-5, atol=2e-5)


def test_full_size_fp16_with_the_layer(wave_lib, oracle_mod):
    """The benchmark's FP16 + CPML form (1024 x 1024 x 512, npml 16) in its
    launch configuration: 3 steps from a random state read back as stored,
    sampled points in the layer (faces, edges, corners, both ends of the
    correction segments) and receivers against the oracle's layered run on
    sub-boxes. Bound 88 EPS M: the plain 16-bit full-size bound (44 EPS M,
    each step's rounding carried at most 7-fold) doubled for the layer
    passes' extra roundings at shell points. That worst-case bound is of the
    order of the layer's own effect after 3 steps from rest memory variables,
    so the test also requires the layer's effect at the layer points (oracle
    with the layer against without) to exceed 20 times the largest measured
    error: a missing or misplaced layer term makes the error about as large
    as the effect."""
    import torch
    from test_gpu_parity import _sub_box_oracle
    cfg = wl.CFG_1024
    nx, ny, nz = cfg["shape"]
    vel = wl.velocity_for(cfg)
    sp = cfg["spacing"]
    dt = cfg["cfl_fraction"] * wave_lib.wave_cfl_dt(sp, float(vel.max()))
    npml, R, fcps = 16, 1e-3, cfg["f_peak"]
    g = torch.Generator(device="cuda")
    g.manual_seed(2468)
    u0 = torch.rand((nz, ny, nx), generator=g, device="cuda") * 2 - 1
    up0 = torch.rand((nz, ny, nx), generator=g, device="cuda") * 2 - 1
    n = 3
    shot = (*cfg["source"], cfg["f_peak"], -1.0, 1e2)
    rec_all = wl.receiver_plane(nx, ny, cfg["rec_z"], cfg["rec_stride"])
    s = wave_lib.WaveSolver((nx, ny, nz), sp, dt, torch.from_numpy(vel).cuda(), storage=2)
    s.set_cpml(npml, R, fcps)
    s.set_state(u0, up0, 0)
    su = torch.empty((nz, ny, nx), device="cuda")
    sup = torch.empty((nz, ny, nx), device="cuda")
    s.get_field(0, su)
    s.get_field(1, sup)
    tr = torch.zeros((n, rec_all.shape[0]), device="cuda")
    s.propagate(shot, n, torch.from_numpy(rec_all).cuda(), tr)
    out = torch.empty((nz, ny, nx), device="cuda")
    s.get_field(0, out)
    s.synchronize()
    s.close()
    u0h, up0h = su.cpu().numpy(), sup.cpu().numpy()
    outh, trh = out.cpu().numpy(), tr.cpu().numpy()
    M = max(float(np.abs(outh).max()), float(np.abs(u0h).max()))
    tol = 88 * EPS16["f16"] * M
    vmax = float(vel.max())
    w = npml + 4
    layer_pts = [(0, 0, 0), (nx - 1, ny - 1, nz - 1), (nx - 1, 0, nz // 2), (0, ny // 2, nz - 1),
                 (npml - 1, 300, 200), (npml, 301, 201), (w - 1, 302, 202), (nx - w, 500, 100),
                 (700, npml - 1, 250), (701, ny - w, 251), (400, 402, nz - npml),
                 (401, 403, w - 1), (5, 7, 9), (nx - 3, ny - 9, 2), cfg["source"]]
    worst, effect = 0.0, 0.0
    for p in layer_pts + [(512, 512, 256)]:
        want, _ = _sub_box_cpml(oracle_mod, vel, u0h, up0h, sp, dt, n, p, shot, npml, R, fcps,
                                vmax)
        got = outh[p[2], p[1], p[0]]
        worst = max(worst, abs(got - want))
        assert abs(got - want) <= tol, (p, got, want, tol)
        if p in layer_pts:
            plain, _ = _sub_box_oracle(oracle_mod, vel, u0h, up0h, sp, dt, n, p, shot)
            effect = max(effect, abs(want - plain))
    rng = np.random.default_rng(3)
    for r in [0, rec_all.shape[0] - 1] + list(rng.integers(0, rec_all.shape[0], 4)):
        _, want_tr = _sub_box_cpml(oracle_mod, vel, u0h, up0h, sp, dt, n,
                                   tuple(int(v) for v in rec_all[r]), shot, npml, R, fcps, vmax)
        assert np.max(np.abs(trh[:, r] - want_tr)) <= tol, r
    print("\nfull-size FP16 + CPML: worst |error| %.3e, bound %.3e, layer effect %.3e"
          % (worst, tol, effect))
    assert effect > 20 * worst
