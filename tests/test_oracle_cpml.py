"""Pins of the oracle's CPML layer (FP64, CPU): the first-derivative weights
from an exact solve, reduction to the plain scheme when the layer does not
damp, a dense state-space brute force on a tiny grid, measured absorption
against the reflecting zero boundary, and mirror symmetry."""
import math
from fractions import Fraction

import numpy as np
import pytest

R4 = 4


def _exact_first_derivative_weights(radius):
    """Antisymmetric a_1..a_R with sum_m a_m (f(m) - f(-m)) ~ h f'(0):
    odd moments 2 sum_m a_m m^(2p+1) = 1 for p = 0, 0 for p = 1..R-1."""
    n = radius
    a = [[Fraction(2 * m ** (2 * p + 1)) for m in range(1, n + 1)] + [Fraction(1 if p == 0 else 0)]
         for p in range(n)]
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


def test_first_derivative_weights(oracle_mod):
    ex = _exact_first_derivative_weights(R4)
    assert ex == [Fraction(4, 5), Fraction(-1, 5), Fraction(4, 105), Fraction(-1, 280)]
    w = oracle_mod.first_weights()
    assert list(w[1:]) == [float(x) for x in ex]


def _layer_damping(oracle_mod, n, npml, h, dt, vmax, R):
    """Damping d of each cell, recovered from the oracle's b = exp(-d dt)
    (no frequency shift, so alpha = 0)."""
    b, a = oracle_mod.cpml_profile(n, npml, h, dt, vmax, R, 0.0)
    return -np.log(b) / dt, b, a


def test_profile_integral_meets_the_reflection_target(oracle_mod):
    """A PML of damping d(x) returns a wave that crossed it twice (in, off
    the wall behind it, and out) with amplitude exp(-2/v * integral of d),
    at every frequency when alpha = 0: that is the reflection coefficient
    the profile is designed for. The layer's summed damping, h * sum d over
    its cells, must therefore tend to (v / 2) ln(1/R) as the layer is
    resolved by more cells (the cell sum of a smooth profile exceeds its
    integral by O(1/npml)). A cell size left out of d0, a factor of the
    quadratic profile's integral (1/3) mistaken, or a linear profile give
    ratios of 10, 1.5 or 2/3 instead."""
    for h, v, R in ((10.0, 2000.0, 1e-3), (12.5, 4500.0, 0.1), (7.0, 1500.0, 1e-5)):
        ratios = []
        for npml in (10, 40, 400):
            n = 2 * npml + 8
            d, b, a = _layer_damping(oracle_mod, n, npml, h, 1e-4, v, R)
            left = h * np.sum(d[:npml])
            right = h * np.sum(d[n - npml:])
            assert left == pytest.approx(right, rel=1e-12)      # both faces alike
            assert np.all(b[npml:n - npml] == 1.0) and np.all(a[npml:n - npml] == 0.0)
            ratios.append(left / (0.5 * v * math.log(1.0 / R)))
        assert all(1.0 <= r <= 1.0 + 2.0 / npml for r, npml in zip(ratios, (10, 40, 400)))
        assert ratios[0] > ratios[1] > ratios[2]
    # damping grows toward the wall: zero inside, largest at the outer cell
    d, _, _ = _layer_damping(oracle_mod, 40, 12, 10.0, 1e-4, 3000.0, 1e-3)
    assert np.all(np.diff(d[:13]) < 0) and d[12] == 0.0


def test_frequency_shift_vanishes_at_the_wall(oracle_mod):
    """CFS shift alpha, recovered from b = exp(-(d + alpha) dt) and
    a = d / (d + alpha) (b - 1): zero at the outer cell (plain PML there),
    growing toward the interior edge of the layer, and bounded by pi f."""
    n, npml, h, dt, v, R, f = 60, 10, 10.0, 1e-4, 3000.0, 1e-3, 15.0
    b, a = oracle_mod.cpml_profile(n, npml, h, dt, v, R, f)
    tot = -np.log(b[:npml]) / dt          # d + alpha
    d = a[:npml] * tot / (b[:npml] - 1.0)
    alpha = tot - d
    assert abs(alpha[0]) <= 1e-9 * tot[0]
    assert np.all(np.diff(alpha) > 0) and alpha[-1] < math.pi * f


def _plane_pulse_reflection(b, a, n, h, v, dt, sigma, x0, rec, t_end):
    """1D experiment: the second-order CPML scheme (axis part of Eq. 1,
    8th-order first derivative, psi and zeta by the recursion with the
    given b and a) run on a right-moving Gaussian pulse; returns the peak
    of the pulse that comes back to the receiver over the peak that passed
    it."""
    w = [-205 / 72, 8 / 5, -1 / 5, 8 / 315, -1 / 560]
    w1 = [0.0, 4 / 5, -1 / 5, 4 / 105, -1 / 280]

    def d2(f):
        p = np.pad(f, 4)
        return (w[0] * f + sum(w[m] * (p[4 + m:4 + m + n] + p[4 - m:4 - m + n])
                               for m in range(1, 5))) / (h * h)

    def d1(f):
        p = np.pad(f, 4)
        return sum(w1[m] * (p[4 + m:4 + m + n] - p[4 - m:4 - m + n]) for m in range(1, 5)) / h

    x = np.arange(n) * h
    u = np.exp(-((x - x0) / sigma) ** 2)
    up = np.exp(-((x - x0 + v * dt) / sigma) ** 2)
    psi = np.zeros(n)
    zeta = np.zeros(n)
    c = (v * dt) ** 2
    tr = np.empty(int(t_end / dt))
    for k in range(tr.size):
        psi = b * psi + a * d1(u)
        lap = d2(u)
        dp = d1(psi)
        zeta = b * zeta + a * (lap + dp)
        u, up = 2 * u - up + c * (lap + dp + zeta), u
        tr[k] = u[rec]
    split = int(((rec * h - x0) / v + 5 * sigma / v) / dt)
    return np.max(np.abs(tr[split:])) / np.max(np.abs(tr[:split]))


@pytest.mark.parametrize("R,npml", [(0.3, 20), (0.1, 20), (0.1, 40)])
def test_normal_incidence_reflection(oracle_mod, R, npml):
    """A plane pulse sent into the layer (1D, normal incidence) comes back
    attenuated by the layer's round trip, exp(-2 h sum d / v) with the
    oracle's damping: within 3 % at this resolution (20 cells per pulse
    width, a quarter of the stability limit). That is R up to the O(1/npml)
    excess of the cell sum over the integral (8 % at npml 40)."""
    n, h, v = 1200, 10.0, 2000.0
    s_w = abs(-205 / 72) + 2 * (8 / 5 + 1 / 5 + 8 / 315 + 1 / 560)
    dt = 0.25 * 2.0 * h / (v * math.sqrt(s_w))
    b, a = oracle_mod.cpml_profile(n, npml, h, dt, v, R, 0.0)
    d = -np.log(b) / dt
    predicted = math.exp(-2.0 * h * np.sum(d[n - npml:]) / v)
    measured = _plane_pulse_reflection(b, a, n, h, v, dt, 120.0, 600 * h, 900, 5.0)
    assert measured == pytest.approx(predicted, rel=0.03)
    assert measured == pytest.approx(R, rel=0.25 if npml == 20 else 0.15)


def test_undamped_layer_is_the_plain_scheme(oracle_mod):
    rng = np.random.default_rng(4)
    nz, ny, nx = 11, 12, 13
    vel = rng.uniform(1500, 3000, size=(nz, ny, nx))
    sp = (10.0, 9.0, 11.0)
    dt = 0.5 * oracle_mod.cfl_dt(sp, vel.max())
    u0 = rng.standard_normal(vel.shape)
    up0 = rng.standard_normal(vel.shape)
    rec = np.array([[1, 2, 3], [12, 11, 10], [6, 6, 5]], dtype=np.int32)
    shot = (6, 5, 4, 20.0, -1.0, 1.0)
    u1, up1, ps, ze, tr1 = oracle_mod.propagate_cpml(vel, sp, dt, 17, npml=4, R=1.0, u=u0,
                                                     u_prev=up0, source=shot, receivers=rec)
    u2, up2, tr2 = oracle_mod.propagate(vel, sp, dt, 17, u=u0, u_prev=up0, source=shot,
                                        receivers=rec)
    assert np.all(ps == 0) and np.all(ze == 0)
    sc = np.abs(u2).max()
    np.testing.assert_allclose(u1, u2, rtol=0, atol=1e-12 * sc)
    np.testing.assert_allclose(tr1, tr2, rtol=0, atol=1e-12 * sc)


def _dense_axis(n, h, w, first):
    D = np.zeros((n, n))
    for i in range(n):
        if not first:
            D[i, i] += w[0] / h ** 2
        for m in range(1, R4 + 1):
            for j, sgn in ((i + m, 1.0), (i - m, -1.0 if first else 1.0)):
                if 0 <= j < n:
                    D[i, j] += (sgn * w[m] / h) if first else (w[m] / h ** 2)
    return D


def test_dense_state_space_brute_force(oracle_mod):
    nz, ny, nx = 7, 8, 9
    sp = (10.0, 12.0, 9.0)
    npml, R, fcps = 2, 1e-3, 20.0
    rng = np.random.default_rng(8)
    vel = rng.uniform(1500, 3000, size=(nz, ny, nx))
    dt = 0.45 * oracle_mod.cfl_dt(sp, vel.max())
    w2 = [-205 / 72, 8 / 5, -1 / 5, 8 / 315, -1 / 560]
    w1 = [0.0, 4 / 5, -1 / 5, 4 / 105, -1 / 280]
    dims = (nx, ny, nz)
    I = [np.eye(d) for d in dims]

    def lift(M, ax):  # 1D operator on axis ax -> full flat (z slowest, x fastest)
        mats = [I[2], I[1], I[0]]
        mats[2 - ax] = M
        return np.kron(mats[0], np.kron(mats[1], mats[2]))

    D1 = [lift(_dense_axis(dims[ax], sp[ax], w1, True), ax) for ax in range(3)]
    D2 = [lift(_dense_axis(dims[ax], sp[ax], w2, False), ax) for ax in range(3)]
    B, A = [], []
    for ax in range(3):
        # the layer's coefficients as the oracle forms them (pinned above by
        # the reflection target and the frequency shift); this test pins
        # the propagation that uses them
        b, a = oracle_mod.cpml_profile(dims[ax], npml, sp[ax], dt, vel.max(), R, fcps)
        B.append(np.diag(lift(np.diag(b), ax)))
        A.append(np.diag(lift(np.diag(a), ax)))
    c = (vel ** 2 * dt ** 2).ravel()
    N = c.size
    u = rng.standard_normal(N)
    up = rng.standard_normal(N)
    psi = [np.zeros(N) for _ in range(3)]
    zeta = [np.zeros(N) for _ in range(3)]
    src = (4, 3, 5)
    ps_i = (src[2] * ny + src[1]) * nx + src[0]
    rec = np.array([[0, 0, 0], [8, 7, 6], [4, 3, 5], [1, 6, 2]], dtype=np.int32)
    pr = (rec[:, 2] * ny + rec[:, 1]) * nx + rec[:, 0]
    f, t0 = 25.0, 0.04
    nsteps = 11
    tr = np.zeros((nsteps, len(rec)))
    u_init, up_init = u.copy(), up.copy()
    for n in range(nsteps):
        psi = [B[ax] * psi[ax] + A[ax] * (D1[ax] @ u) for ax in range(3)]
        zeta = [B[ax] * zeta[ax] + A[ax] * (D2[ax] @ u + D1[ax] @ psi[ax]) for ax in range(3)]
        s = sum(D2[ax] @ u + D1[ax] @ psi[ax] + zeta[ax] for ax in range(3))
        un = 2 * u - up + c * s
        t = n * dt
        aa = (math.pi * f * (t - t0)) ** 2
        un[ps_i] += c[ps_i] * (1 - 2 * aa) * math.exp(-aa)
        tr[n] = un[pr]
        up, u = u, un
    ou, oup, ops, oze, otr = oracle_mod.propagate_cpml(
        vel, sp, dt, nsteps, npml, R=R, fcps=fcps, u=u_init.reshape(vel.shape),
        u_prev=up_init.reshape(vel.shape), source=(*src, f, t0, 1.0), receivers=rec)
    sc = np.abs(u).max()
    np.testing.assert_allclose(ou.ravel(), u, rtol=0, atol=1e-12 * sc)
    np.testing.assert_allclose(otr, tr, rtol=0, atol=1e-12 * sc)
    for ax in range(3):
        np.testing.assert_allclose(ops[ax].ravel(), psi[ax], rtol=0,
                                   atol=1e-12 * max(1e-300, np.abs(psi[ax]).max()))
        np.testing.assert_allclose(oze[ax].ravel(), zeta[ax], rtol=0,
                                   atol=1e-12 * max(1e-300, np.abs(zeta[ax]).max()))


def test_layer_absorbs_what_the_zero_boundary_reflects(oracle_mod):
    n, npml = 40, 10
    vel = np.full((n, n, n), 2000.0)
    sp = (10.0, 10.0, 10.0)
    dt = 0.5 * oracle_mod.cfl_dt(sp, 2000.0)
    shot = (20, 20, 20, 25.0, 0.04, 1.0)
    steps = 360  # the pulse reaches the faces near step 90 and is back by 180
    u_d, _, _ = oracle_mod.propagate(vel, sp, dt, steps, source=shot)
    u_p, _, _, _, _ = oracle_mod.propagate_cpml(vel, sp, dt, steps, npml, R=1e-3, fcps=25.0,
                                                source=shot)
    inner = (slice(npml, n - npml),) * 3
    ratio = np.linalg.norm(u_p[inner]) / np.linalg.norm(u_d[inner])
    assert ratio < 0.03, ratio


def test_cpml_keeps_mirror_symmetry(oracle_mod):
    n = 21
    vel = np.full((n, n, n), 2500.0)
    dt = 0.5 * oracle_mod.cfl_dt((10.0,) * 3, 2500.0)
    u, _, _, _, _ = oracle_mod.propagate_cpml(vel, (10.0,) * 3, dt, 80, 5, source=(10, 10, 10, 25.0, -1.0, 1.0))
    sc = np.abs(u).max()
    for axis in range(3):
        assert np.max(np.abs(u - np.flip(u, axis))) <= 1e-12 * sc
    assert np.max(np.abs(u - np.transpose(u, (2, 1, 0)))) <= 1e-12 * sc


def test_sub_box_margin_reproduces_the_whole_grid(oracle_mod):
    """The sub-box reduction the full-size GPU test relies on: with a margin
    of npml + 8n + 1 cells at every cut, the oracle on the sub-box gives the
    whole-grid oracle's value at the point exactly (layers at true faces,
    source inside the layer, random state)."""
    from test_gpu_cpml import _sub_box_cpml
    nx, ny, nz = 120, 110, 100
    rng = np.random.default_rng(0)
    vel = rng.uniform(1500, 4500, size=(nz, ny, nx)).astype(np.float32)
    u0 = rng.uniform(-1, 1, size=vel.shape)
    up0 = rng.uniform(-1, 1, size=vel.shape)
    sp = (10.0, 10.0, 10.0)
    dt = 0.5 * oracle_mod.cfl_dt(sp, float(vel.max()))
    npml, n = 6, 3
    shot = (60, 55, 8, 15.0, -1.0, 1e4)
    vmax = float(vel.max())
    full, _, _, _, _ = oracle_mod.propagate_cpml(vel, sp, dt, n, npml, R=1e-3, fcps=15.0,
                                                 vmax=vmax, u=u0, u_prev=up0, source=shot)
    for p in [(0, 0, 0), (119, 109, 99), (5, 50, 50), (60, 55, 8), (40, 3, 97), (70, 70, 50)]:
        v, _ = _sub_box_cpml(oracle_mod, vel, u0, up0, sp, dt, n, p, shot, npml, 1e-3, 15.0,
                             vmax)
        assert v == full[p[2], p[1], p[0]]


def test_recursive_convolution_is_exact_for_a_step(oracle_mod):
    """psi^n = b psi^{n-1} + a g^n is the convolution psi = chi * g with the
    CFS kernel chi(t) = -d exp(-(d + alpha) t) (the inverse transform of
    1/s - 1, s = 1 + d / (alpha + i omega)), exact when g is constant over each
    step: for a unit step from t = 0 the continuous result at t = (n+1) dt is
    -d / (d + alpha) (1 - exp(-(d + alpha)(n + 1) dt)). A wrong sign or factor
    in a, or alpha missing from b, breaks the match."""
    n_cells, npml, h, dt, vmax, R, fc = 40, 10, 10.0, 1e-3, 3000.0, 1e-3, 15.0
    b, a = oracle_mod.cpml_profile(n_cells, npml, h, dt, vmax, R, fc)
    d0 = 3.0 * vmax * math.log(1.0 / R) / (2.0 * npml * h)
    for i in (0, 3, 7, 9, 33, 39):
        xi = (npml - i) / npml if i < npml else (i - (n_cells - npml - 1)) / npml
        d, al = d0 * xi * xi, math.pi * fc * (1.0 - xi)
        psi = 0.0
        for n in range(60):
            psi = b[i] * psi + a[i] * 1.0
            exact = -d / (d + al) * (1.0 - math.exp(-(d + al) * (n + 1) * dt))
            assert psi == pytest.approx(exact, rel=1e-12, abs=1e-15), (i, n)


def _cpml_gradient_case():
    rng = np.random.default_rng(17)
    nz, ny, nx = 13, 12, 14
    sp = (10.0, 11.0, 9.0)
    true = 2000.0 + 400.0 * rng.random((nz, ny, nx))
    vel = 2000.0 + 400.0 * rng.random((nz, ny, nx))
    shot = (7, 6, 6, 25.0, 0.02, 1e3)
    rec = np.array([[1, 1, 1], [4, 6, 2], [12, 3, 10], [7, 10, 12], [0, 11, 6]],
                   dtype=np.int32)
    return sp, vel, true, shot, rec


def _cpml_misfit(oracle_mod, vel, sp, dt, nsteps, npml, vmax, shot, rec, obs):
    tr = oracle_mod.propagate_cpml(vel, sp, dt, nsteps, npml, R=1e-2, fcps=20.0, vmax=vmax,
                                   source=shot, receivers=rec)[4]
    return 0.5 * float(np.sum((tr - obs) ** 2)), tr


def test_cpml_adjoint_gradient_matches_finite_differences(oracle_mod):
    """The CPML adjoint gradient against central differences of the oracle's
    CPML misfit, the layer's profile held at a fixed vmax (FP64, step 1e-5
    relative), at points inside and outside the layer and along a smooth
    direction through the whole model."""
    sp, vel, true, shot, rec = _cpml_gradient_case()
    vmax = 2500.0
    dt = 0.5 * oracle_mod.cfl_dt(sp, vmax)
    nsteps, npml = 28, 3
    obs = oracle_mod.propagate_cpml(true, sp, dt, nsteps, npml, R=1e-2, fcps=20.0, vmax=vmax,
                                    source=shot, receivers=rec)[4]
    _, tr = _cpml_misfit(oracle_mod, vel, sp, dt, nsteps, npml, vmax, shot, rec, obs)
    g = oracle_mod.gradient_cpml(vel, sp, dt, nsteps, npml, shot, rec, tr - obs, R=1e-2,
                                 fcps=20.0, vmax=vmax)
    m = vel ** 2
    # in the layer (corner, face, edge), at its inner edge, and inside
    for idx in [(0, 0, 0), (1, 6, 7), (6, 1, 12), (3, 3, 3), (6, 6, 7), (9, 8, 4), (12, 11, 13)]:
        h = 1e-5 * m[idx]
        mp, mm = m.copy(), m.copy()
        mp[idx] += h
        mm[idx] -= h
        jp, _ = _cpml_misfit(oracle_mod, np.sqrt(mp), sp, dt, nsteps, npml, vmax, shot, rec, obs)
        jm, _ = _cpml_misfit(oracle_mod, np.sqrt(mm), sp, dt, nsteps, npml, vmax, shot, rec, obs)
        fd = (jp - jm) / (2 * h)
        assert fd == pytest.approx(g[idx], rel=2e-5, abs=1e-6 * np.max(np.abs(g))), idx
    z, y, x = np.meshgrid(*[np.arange(s) for s in m.shape], indexing="ij")
    dm = np.exp(-((x - 3.0) ** 2 + (y - 6.0) ** 2 + (z - 5.0) ** 2) / 10.0) * m
    eps = 1e-6
    jp, _ = _cpml_misfit(oracle_mod, np.sqrt(m + eps * dm), sp, dt, nsteps, npml, vmax, shot,
                         rec, obs)
    jm, _ = _cpml_misfit(oracle_mod, np.sqrt(m - eps * dm), sp, dt, nsteps, npml, vmax, shot,
                         rec, obs)
    assert (jp - jm) / (2 * eps) == pytest.approx(float(np.sum(g * dm)), rel=1e-6)


def test_cpml_adjoint_without_damping_is_the_plain_adjoint(oracle_mod):
    """With R = 1 the layer does not damp (b = 1, a = 0): the CPML adjoint
    must equal the plain one (to FP64 rounding of a different order)."""
    sp, vel, _, shot, rec = _cpml_gradient_case()
    dt = 0.5 * oracle_mod.cfl_dt(sp, vel.max())
    rng = np.random.default_rng(3)
    res = rng.standard_normal((20, rec.shape[0]))
    g0 = oracle_mod.gradient(vel, sp, dt, 20, shot, rec, res)
    g1 = oracle_mod.gradient_cpml(vel, sp, dt, 20, 4, shot, rec, res, R=1.0, fcps=0.0)
    assert np.max(np.abs(g1 - g0)) <= 1e-12 * np.max(np.abs(g0))
