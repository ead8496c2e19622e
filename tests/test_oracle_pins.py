"""Pins of the FP64 oracle against what the mathematics of Eq. 1 and the
leapfrog update fix, independently of the oracle's own code.

Each test is chosen so that a plausible slip in the oracle (a wrong weight, a
dropped or doubled centre term, a swapped axis spacing, a sign or index error
in the time update, the source injected at the wrong time, receivers sampled
before injection, a broken periodic wrap) fails at least one of them.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

R = 4


def _exact_second_derivative_weights(radius):
    """Solve the symmetric (2R+1)-point second-derivative conditions exactly.

    Unknowns a_0..a_R of  sum_{m=-R..R} a_|m| f(mh) ~ h^2 f''(0):  even
    moments sum_m a_|m| m^(2p) = 2 for p = 1 and 0 for p = 0, 2, .., R.
    """
    n = radius + 1
    rows, rhs = [], []
    for p in range(n):
        row = []
        for m in range(n):
            if m == 0:
                row.append(Fraction(1 if p == 0 else 0))
            else:
                row.append(Fraction(2 * m ** (2 * p)))
        rows.append(row)
        rhs.append(Fraction(2 if p == 1 else 0))
    # Gauss-Jordan in exact rationals
    a = [r[:] + [b] for r, b in zip(rows, rhs)]
    for col in range(n):
        piv = next(r for r in range(col, n) if a[r][col] != 0)
        a[col], a[piv] = a[piv], a[col]
        pv = a[col][col]
        a[col] = [x / pv for x in a[col]]
        for r in range(n):
            if r != col and a[r][col] != 0:
                f = a[r][col]
                a[r] = [x - f * y for x, y in zip(a[r], a[col])]
    return [a[i][n] for i in range(n)]


def test_weights_match_exact_solve(oracle_mod):
    exact = _exact_second_derivative_weights(R)
    assert exact == [Fraction(-205, 72), Fraction(8, 5), Fraction(-1, 5),
                     Fraction(8, 315), Fraction(-1, 560)]
    w = oracle_mod.weights()
    for wm, em in zip(w, exact):
        assert wm == float(em)


def test_weight_moments():
    w = _exact_second_derivative_weights(R)

    def moment(q):
        return (w[0] if q == 0 else 0) + sum(2 * w[m] * m ** q for m in range(1, R + 1))

    assert moment(0) == 0
    assert moment(2) == 2
    assert moment(4) == moment(6) == moment(8) == 0
    assert moment(10) == -1152


def _grid(n, h, c):
    return (np.arange(n, dtype=np.float64) - c) * h


def test_polynomial_exactness_up_to_degree_9(oracle_mod):
    nx, ny, nz = 21, 19, 17
    dx, dy, dz = 0.7, 1.3, 0.9
    x = _grid(nx, dx, 10.0)[None, None, :]
    y = _grid(ny, dy, 9.0)[None, :, None]
    z = _grid(nz, dz, 8.0)[:, None, None]
    u = x ** 9 + 2.0 * y ** 8 - z ** 7 + x ** 4 * y ** 5 * z ** 2 + 3.0 * x * y * z
    lap_exact = (72.0 * x ** 7 + 112.0 * y ** 6 - 42.0 * z ** 5
                 + 12.0 * x ** 2 * y ** 5 * z ** 2 + 20.0 * x ** 4 * y ** 3 * z ** 2
                 + 2.0 * x ** 4 * y ** 5)
    lap = oracle_mod.laplacian(u, (dx, dy, dz))
    inner = (slice(R, nz - R), slice(R, ny - R), slice(R, nx - R))
    err = np.abs(lap[inner] - lap_exact[inner])
    scale = np.max(np.abs(lap_exact[inner]))
    assert np.max(err) <= 1e-9 * scale


def test_degree_10_error_is_the_predicted_constant(oracle_mod):
    # The first non-vanishing moment gives, for f = x^10 exactly,
    # D_h f - f'' = (1/h^2) * (-1152) * h^10 * f^(10) / 10! = -1152 h^8.
    n, h = 25, 0.5
    for axis, shape in ((2, (9, 9, n)), (1, (9, n, 9)), (0, (n, 9, 9))):
        coord = _grid(n, h, 12.0)
        s = [1, 1, 1]
        s[axis] = n
        c = coord.reshape(s)
        u = np.broadcast_to(c ** 10, shape).copy()
        spacing = [1.0, 1.0, 1.0]
        spacing[2 - axis] = h
        lap = oracle_mod.laplacian(u, tuple(spacing))
        mid = [4, 4, 4]
        for i in range(R, n - R):
            mid[axis] = i
            got = lap[tuple(mid)] - 90.0 * coord[i] ** 8
            assert got == pytest.approx(-1152.0 * h ** 8, rel=1e-7, abs=1e-6)


def test_convergence_is_eighth_order(oracle_mod):
    # Periodic single Fourier mode u = sin(x) sin(2y) sin(z): error of L u
    # against -|k|^2 u. The leading error per axis is -h^8 u^(10) / 3150, i.e.
    # + h^8 k^10 u / 3150 for sin(k x), so the total is h^8 (1 + 2^10 + 1) u / 3150.
    errs = []
    for n in (32, 64):
        L = 2.0 * math.pi
        h = L / n
        xs = np.arange(n) * h
        z, y, x = np.meshgrid(xs, xs, xs, indexing="ij")
        u = np.sin(x) * np.sin(2.0 * y) * np.sin(z)
        lap = oracle_mod.laplacian(u, (h, h, h), periodic=True)
        err = lap + 6.0 * u
        errs.append(np.max(np.abs(err)))
        lead = h ** 8 * 1026.0 / 3150.0
        sel = np.abs(u) > 0.5
        np.testing.assert_allclose(err[sel] / u[sel], lead, rtol=0.08 if n == 32 else 0.02)
    ratio = errs[0] / errs[1]
    assert 240.0 < ratio < 262.0, ratio


def _symbol(kh, h):
    """Discrete Fourier symbol K of one axis from the exact weights."""
    w = [float(v) for v in _exact_second_derivative_weights(R)]
    return (-w[0] - 2.0 * sum(w[m] * math.cos(m * kh) for m in range(1, R + 1))) / h ** 2


def test_dispersion_relation_exact(oracle_mod):
    nx, ny, nz = 16, 12, 10
    dx, dy, dz = 10.0, 12.0, 8.0
    mx, my, mz = 3, 2, 1
    i = np.arange(nx)[None, None, :]
    j = np.arange(ny)[None, :, None]
    k = np.arange(nz)[:, None, None]
    ax, ay, az = 2 * math.pi * mx / nx, 2 * math.pi * my / ny, 2 * math.pi * mz / nz
    u0 = np.cos(ax * i) * np.cos(ay * j) * np.cos(az * k) * np.ones((nz, ny, nx))
    K = _symbol(ax, dx) + _symbol(ay, dy) + _symbol(az, dz)
    v = 2000.0
    # dt must respect the global limit, or round-off in other modes grows
    dt = 0.9 * oracle_mod.cfl_dt((dx, dy, dz), v)
    cos_t = 1.0 - 0.5 * v * v * dt * dt * K
    theta = math.acos(cos_t)
    vel = np.full((nz, ny, nx), v)
    nsteps = 37
    assert nsteps * theta > math.pi  # more than half a period: the phase is tested
    u, up, _ = oracle_mod.propagate(vel, (dx, dy, dz), dt, nsteps, u=u0,
                                    u_prev=cos_t * u0, periodic=True)
    np.testing.assert_allclose(u, math.cos(nsteps * theta) * u0, atol=1e-11)
    np.testing.assert_allclose(up, math.cos((nsteps - 1) * theta) * u0, atol=1e-11)


def test_scheme_is_second_order_in_time(oracle_mod):
    """Manufactured standing wave u = cos(k x) cos(omega t), omega = v k, on a
    periodic grid, started from the exact u(0) and u(-dt). At fixed T the
    error is the leapfrog phase error: theta - omega dt = (omega dt)^3 / 24 +
    O(dt^5) per step, so max |u^N - u(T)| = |sin(omega T)| omega T (omega dt)^2
    / 24 (1 + O(dt^2)); the spatial error ((k h)^8 / 3150 relative in the
    symbol, 7e-10 here) is far below. Halving dt divides it by 4."""
    nx, ny, nz, h, v = 32, 8, 8, 10.0, 2000.0
    k = 2 * math.pi / (nx * h)
    w = v * k
    T = 2.5 / w
    x = np.arange(nx) * h
    u0 = np.cos(k * x)[None, None, :] * np.ones((nz, ny, nx))
    vel = np.full((nz, ny, nx), v)
    err = {}
    for N in (80, 160, 320):
        dt = T / N
        assert dt < oracle_mod.cfl_dt((h, h, h), v)
        u, _, _ = oracle_mod.propagate(vel, (h, h, h), dt, N, u=u0,
                                       u_prev=math.cos(w * dt) * u0, periodic=True)
        err[N] = np.max(np.abs(u - math.cos(w * T) * u0))
        pred = abs(math.sin(w * T)) * w * T * (w * dt) ** 2 / 24
        assert err[N] == pytest.approx(pred, rel=0.02)
    assert 3.9 < err[80] / err[160] < 4.1
    assert 3.9 < err[160] / err[320] < 4.1


def test_stability_limit(oracle_mod):
    n, h, v = 8, 10.0, 3000.0
    i = np.arange(n)
    sign = ((-1.0) ** (i[:, None, None] + i[None, :, None] + i[None, None, :]))
    u0 = sign * np.ones((n, n, n))
    vel = np.full((n, n, n), v)
    dtc = oracle_mod.cfl_dt((h, h, h), v)
    # closed form: Courant number v dt / h = 2 / sqrt(3 S), S = |w0| + 2 sum |w_m|
    w = _exact_second_derivative_weights(R)
    S = abs(w[0]) + 2 * sum(abs(x) for x in w[1:])
    assert S == Fraction(205, 72) + Fraction(16, 5) + Fraction(2, 5) + Fraction(16, 315) + Fraction(1, 280)
    assert dtc * v / h == pytest.approx(2.0 / math.sqrt(3.0 * float(S)), rel=1e-14)
    below, _, _ = oracle_mod.propagate(vel, (h, h, h), 0.999 * dtc, 300, u=u0, u_prev=-u0,
                                       periodic=True)
    above, _, _ = oracle_mod.propagate(vel, (h, h, h), 1.001 * dtc, 300, u=u0, u_prev=-u0,
                                       periodic=True)
    assert np.max(np.abs(below)) < 2.0
    assert np.max(np.abs(above)) > 1e3


def test_discrete_energy_is_conserved(oracle_mod):
    n = 12
    dx, dy, dz = 10.0, 11.0, 9.0
    v = 2500.0
    rng = np.random.default_rng(3)
    u0 = rng.standard_normal((n, n, n))
    up0 = u0 + 0.01 * rng.standard_normal((n, n, n))
    vel = np.full((n, n, n), v)
    dt = 0.5 * oracle_mod.cfl_dt((dx, dy, dz), v)

    def energy(u_new, u_old):
        lu = oracle_mod.laplacian(u_old, (dx, dy, dz), periodic=True)
        return 0.5 * np.sum((u_new - u_old) ** 2) / dt ** 2 - 0.5 * v * v * np.sum(u_new * lu)

    e = []
    u, up = u0, up0
    for _ in range(6):
        u2, up2, _ = oracle_mod.propagate(vel, (dx, dy, dz), dt, 7, u=u, u_prev=up, periodic=True)
        e.append(energy(u2, up2))
        u, up = u2, up2
    e = np.array(e)
    assert np.max(np.abs(e - e[0])) <= 1e-11 * abs(e[0])


def test_mirror_and_axis_symmetry(oracle_mod):
    n = 17
    vel = np.full((n, n, n), 2000.0, dtype=np.float32)
    dt = 0.5 * oracle_mod.cfl_dt((10.0, 10.0, 10.0), 2000.0)
    u, up, _ = oracle_mod.propagate(vel, (10.0, 10.0, 10.0), dt, 40,
                                    source=(8, 8, 8, 15.0, -1.0, 1.0))
    scale = np.max(np.abs(u))
    assert scale > 0
    tol = 1e-13 * scale
    for axis in range(3):
        assert np.max(np.abs(u - np.flip(u, axis))) <= tol
    for perm in ((0, 2, 1), (1, 0, 2), (2, 1, 0), (1, 2, 0)):
        assert np.max(np.abs(u - np.transpose(u, perm))) <= tol


def test_ricker_closed_form(oracle_mod):
    f, amp = 15.0, 2.5
    t0 = 1.0 / f
    assert oracle_mod.ricker(t0, f, t0, amp) == pytest.approx(amp, rel=1e-15)
    tz = 1.0 / (math.sqrt(2.0) * math.pi * f)
    assert abs(oracle_mod.ricker(t0 + tz, f, t0, amp)) < 1e-14
    assert abs(oracle_mod.ricker(t0 - tz, f, t0, amp)) < 1e-14
    tm = math.sqrt(1.5) / (math.pi * f)
    assert oracle_mod.ricker(t0 + tm, f, t0, amp) == pytest.approx(-2.0 * amp * math.exp(-1.5), rel=1e-14)
    for dtt in (0.001, 0.013, 0.05):
        assert oracle_mod.ricker(t0 + dtt, f, t0, amp) == pytest.approx(
            oracle_mod.ricker(t0 - dtt, f, t0, amp), rel=1e-13)
    # default t0 is 1/f
    assert oracle_mod.ricker(t0, f) == pytest.approx(1.0, rel=1e-15)


def _dense_axis_operator(n, h, periodic):
    w = [float(v) for v in _exact_second_derivative_weights(R)]
    D = np.zeros((n, n))
    for i in range(n):
        D[i, i] += w[0] / h ** 2
        for m in range(1, R + 1):
            for j in (i + m, i - m):
                if periodic:
                    D[i, j % n] += w[m] / h ** 2
                elif 0 <= j < n:
                    D[i, j] += w[m] / h ** 2
    return D


def _dense_laplacian(nx, ny, nz, dx, dy, dz, periodic):
    Ix, Iy, Iz = np.eye(nx), np.eye(ny), np.eye(nz)
    Dx = _dense_axis_operator(nx, dx, periodic)
    Dy = _dense_axis_operator(ny, dy, periodic)
    Dz = _dense_axis_operator(nz, dz, periodic)
    # flat index (k*ny + j)*nx + i: z slowest, x fastest
    return (np.kron(Iz, np.kron(Iy, Dx)) + np.kron(Iz, np.kron(Dy, Ix))
            + np.kron(Dz, np.kron(Iy, Ix)))


@pytest.mark.parametrize("periodic", [False, True])
def test_brute_force_dense_matrix(oracle_mod, periodic):
    nx, ny, nz = 5, 6, 7
    dx, dy, dz = 9.0, 11.0, 10.0
    rng = np.random.default_rng(11)
    vel = rng.uniform(1500.0, 3000.0, size=(nz, ny, nx))
    dt = 0.45 * oracle_mod.cfl_dt((dx, dy, dz), vel.max())
    u0 = rng.standard_normal((nz, ny, nx))
    up0 = rng.standard_normal((nz, ny, nx))
    src = (2, 3, 4)
    f, t0, amp = 15.0, 0.02, 1.7
    rec = np.array([[0, 0, 0], [4, 5, 6], [2, 3, 4], [1, 2, 3]], dtype=np.int32)
    nsteps, step0 = 9, 5
    A = _dense_laplacian(nx, ny, nz, dx, dy, dz, periodic)
    c = (vel * vel * dt * dt).ravel()
    u, up = u0.ravel().copy(), up0.ravel().copy()
    ps = (src[2] * ny + src[1]) * nx + src[0]
    pr = (rec[:, 2] * ny + rec[:, 1]) * nx + rec[:, 0]
    tr = np.zeros((nsteps, len(rec)))
    for n in range(nsteps):
        un = 2.0 * u - up + c * (A @ u)
        t = (step0 + n) * dt
        a = (math.pi * f * (t - t0)) ** 2
        un[ps] += c[ps] * amp * (1.0 - 2.0 * a) * math.exp(-a)
        tr[n] = un[pr]
        up, u = u, un
    ou, oup, otr = oracle_mod.propagate(vel, (dx, dy, dz), dt, nsteps, u=u0, u_prev=up0,
                                        step0=step0, source=(*src, f, t0, amp),
                                        receivers=rec, periodic=periodic)
    scale = np.max(np.abs(u))
    np.testing.assert_allclose(ou.ravel(), u, rtol=0, atol=1e-12 * scale)
    np.testing.assert_allclose(oup.ravel(), up, rtol=0, atol=1e-12 * scale)
    np.testing.assert_allclose(otr, tr, rtol=0, atol=1e-12 * scale)


def test_source_first_two_steps_closed_form(oracle_mod):
    # From rest, step 0 leaves c_p s(0) at the source and nothing else; step 1
    # spreads it by one application of Eq. 1 and injects s(dt).
    nx, ny, nz = 11, 12, 13
    dx, dy, dz = 10.0, 8.0, 12.0
    rng = np.random.default_rng(5)
    vel = rng.uniform(1500.0, 3500.0, size=(nz, ny, nx))
    dt = 0.5 * oracle_mod.cfl_dt((dx, dy, dz), vel.max())
    p = (5, 6, 7)
    f, t0 = 15.0, 1.0 / 15.0
    c = vel * vel * dt * dt
    s0, s1 = oracle_mod.ricker(0.0, f, t0), oracle_mod.ricker(dt, f, t0)
    w = [float(v) for v in _exact_second_derivative_weights(R)]
    rec = np.array([[5, 6, 7], [7, 6, 7], [5, 6, 11], [6, 7, 7]], dtype=np.int32)
    u1, _, tr1 = oracle_mod.propagate(vel, (dx, dy, dz), dt, 1,
                                      source=(*p, f, t0, 1.0), receivers=rec)
    cp = c[p[2], p[1], p[0]]
    expect = np.zeros_like(u1)
    expect[p[2], p[1], p[0]] = cp * s0
    np.testing.assert_allclose(u1, expect, rtol=1e-15, atol=0)
    assert tr1[0, 0] == pytest.approx(cp * s0, rel=1e-15)
    u2, _, tr2 = oracle_mod.propagate(vel, (dx, dy, dz), dt, 2,
                                      source=(*p, f, t0, 1.0), receivers=rec)
    a1 = cp * s0
    centre = 2 * a1 + cp * (w[0] * (1 / dx ** 2 + 1 / dy ** 2 + 1 / dz ** 2)) * a1 + cp * s1
    assert u2[p[2], p[1], p[0]] == pytest.approx(centre, rel=1e-13)
    assert tr2[1, 0] == pytest.approx(centre, rel=1e-13)
    # x + 2 neighbour and z + 4 neighbour: one Eq. 1 term each
    assert tr2[1, 1] == pytest.approx(c[7, 6, 7] * w[2] / dx ** 2 * a1, rel=1e-13)
    assert tr2[1, 2] == pytest.approx(c[11, 6, 5] * w[4] / dz ** 2 * a1, rel=1e-13)
    assert tr2[1, 3] == 0.0  # a diagonal neighbour: outside the star of Eq. 1
    assert u2[7, 6, 9] == pytest.approx(c[7, 6, 9] * w[4] / dx ** 2 * a1, rel=1e-13)


def test_zero_halo_matches_embedding(oracle_mod):
    # The zero Dirichlet halo equals embedding the grid in a larger periodic one
    # whose extra cells are zero, for a single application of Eq. 1.
    rng = np.random.default_rng(7)
    nz, ny, nx = 6, 7, 9
    u = rng.standard_normal((nz, ny, nx))
    big = np.zeros((nz + 2 * R, ny + 2 * R, nx + 2 * R))
    big[R:-R, R:-R, R:-R] = u
    sp = (1.0, 2.0, 3.0)
    lap = oracle_mod.laplacian(u, sp)
    lap_big = oracle_mod.laplacian(big, sp, periodic=True)
    np.testing.assert_allclose(lap, lap_big[R:-R, R:-R, R:-R], rtol=1e-14, atol=1e-14)


def _misfit(oracle_mod, vel, sp, dt, nsteps, shot, rec, obs):
    _, _, tr = oracle_mod.propagate(vel, sp, dt, nsteps, source=shot, receivers=rec)
    return 0.5 * float(np.sum((tr - obs) ** 2)), tr


def _gradient_case(n=9, nsteps=30, seed=1):
    rng = np.random.default_rng(seed)
    sp = (10.0, 11.0, 9.0)
    vel = rng.uniform(1800.0, 3200.0, size=(n, n + 1, n + 2))
    true = vel * (1.0 + 0.05 * rng.standard_normal(vel.shape))
    shot = (3, 4, 2, 25.0, 0.03, 1e3)
    rec = np.array([[1, 1, 1], [n - 2, n - 3, n - 4], [5, n - 1, n - 3], [n + 1, 2, 3],
                    [n - 2, n - 3, n - 4]], dtype=np.int32)  # (x, y, z); one repeated
    return sp, vel, true, shot, rec


def test_adjoint_gradient_matches_finite_differences(oracle_mod):
    """The oracle gradient against central differences of the oracle misfit
    (FP64, step 1e-5 relative: truncation ~1e-10, rounding ~1e-9)."""
    sp, vel, true, shot, rec = _gradient_case()
    dt = 0.5 * oracle_mod.cfl_dt(sp, max(vel.max(), true.max()) * 1.01)
    nsteps = 30
    _, _, obs = oracle_mod.propagate(true, sp, dt, nsteps, source=shot, receivers=rec)
    _, tr = _misfit(oracle_mod, vel, sp, dt, nsteps, shot, rec, obs)
    g = oracle_mod.gradient(vel, sp, dt, nsteps, shot, rec, tr - obs)
    m = vel ** 2
    rng = np.random.default_rng(2)
    pts = [(2, 4, 3), (4, 6, 7), (0, 0, 0), (8, 9, 10)] + [
        tuple(int(rng.integers(s)) for s in m.shape) for _ in range(4)]
    for idx in pts:
        h = 1e-5 * m[idx]
        mp, mm = m.copy(), m.copy()
        mp[idx] += h
        mm[idx] -= h
        jp, _ = _misfit(oracle_mod, np.sqrt(mp), sp, dt, nsteps, shot, rec, obs)
        jm, _ = _misfit(oracle_mod, np.sqrt(mm), sp, dt, nsteps, shot, rec, obs)
        fd = (jp - jm) / (2 * h)
        assert fd == pytest.approx(g[idx], rel=2e-5, abs=1e-6 * np.max(np.abs(g))), idx
    # and along a smooth direction through the whole model
    z, y, x = np.meshgrid(*[np.arange(s) for s in m.shape], indexing="ij")
    dm = np.exp(-((x - 5.0) ** 2 + (y - 5.0) ** 2 + (z - 4.0) ** 2) / 8.0) * m
    eps = 1e-6
    jp, _ = _misfit(oracle_mod, np.sqrt(m + eps * dm), sp, dt, nsteps, shot, rec, obs)
    jm, _ = _misfit(oracle_mod, np.sqrt(m - eps * dm), sp, dt, nsteps, shot, rec, obs)
    assert (jp - jm) / (2 * eps) == pytest.approx(float(np.sum(g * dm)), rel=1e-6)


def test_oracle_rejects_points_outside_the_grid(oracle_mod):
    vel = np.full((5, 6, 7), 2000.0)
    dt = 0.5 * oracle_mod.cfl_dt((10.0,) * 3, 2000.0)
    with pytest.raises(ValueError):
        oracle_mod.propagate(vel, (10.0,) * 3, dt, 2, receivers=np.array([[7, 0, 0]]))
    with pytest.raises(ValueError):
        oracle_mod.propagate(vel, (10.0,) * 3, dt, 2, source=(0, 6, 0, 15.0, -1.0, 1.0))
    with pytest.raises(ValueError):
        oracle_mod.gradient(vel, (10.0,) * 3, dt, 2, (0, 0, 5, 15.0, -1.0, 1.0),
                            np.array([[0, 0, 0]]), np.zeros((2, 1)))


def test_adjoint_gradient_linear_in_residual_and_zero_without_it(oracle_mod):
    sp, vel, _, shot, rec = _gradient_case(n=7, nsteps=12)
    dt = 0.5 * oracle_mod.cfl_dt(sp, vel.max())
    rng = np.random.default_rng(9)
    r1 = rng.standard_normal((12, rec.shape[0]))
    r2 = rng.standard_normal((12, rec.shape[0]))
    g1 = oracle_mod.gradient(vel, sp, dt, 12, shot, rec, r1)
    g2 = oracle_mod.gradient(vel, sp, dt, 12, shot, rec, r2)
    g12 = oracle_mod.gradient(vel, sp, dt, 12, shot, rec, 2.0 * r1 - 3.0 * r2)
    np.testing.assert_allclose(g12, 2.0 * g1 - 3.0 * g2, rtol=1e-12, atol=1e-12 * np.abs(g1).max())
    g0 = oracle_mod.gradient(vel, sp, dt, 12, shot, rec, np.zeros_like(r1))
    assert np.all(g0 == 0.0)
