"""FP64 CPU oracle of the 3D acoustic wave update (Eq. 1 + leapfrog + source + receivers).

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package. The
product library (``paper_2404_04441_gb300``) never imports it and shares no
code with it.

The arithmetic lives in ``wave_oracle.c`` (plain C, FP64, OpenMP over z);
this module only marshals numpy arrays. See the header of ``wave_oracle.c``
for what each function computes and which passage it follows.
"""
import ctypes

import numpy as np

from . import build as _build

_lib = None
_lib_override = None


def _use_library(path):
    """Point the wrappers at another build of wave_oracle.c, or back at the
    normal build with None. Only the pin-strength tests use it: they load
    deliberately broken copies and check that the pins reject them."""
    global _lib, _lib_override
    _lib = None
    _lib_override = path


def _load():
    global _lib
    if _lib is None:
        path = _lib_override or _build.build()
        lib = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        lib.oracle_weights.argtypes = [dp]
        lib.oracle_weights.restype = None
        lib.oracle_laplacian.argtypes = [ctypes.c_int] * 3 + [ctypes.c_double] * 3 + [
            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]
        lib.oracle_laplacian.restype = None
        lib.oracle_ricker.argtypes = [ctypes.c_double] * 4
        lib.oracle_ricker.restype = ctypes.c_double
        lib.oracle_cfl_dt.argtypes = [ctypes.c_double] * 4
        lib.oracle_cfl_dt.restype = ctypes.c_double
        lib.oracle_propagate.argtypes = (
            [ctypes.c_int] * 3 + [ctypes.c_double] * 4
            + [ctypes.c_void_p] * 3 + [ctypes.c_int64, ctypes.c_int, ctypes.c_int]
            + [ctypes.c_int] * 3 + [ctypes.c_double] * 3
            + [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int])
        lib.oracle_propagate.restype = ctypes.c_int
        lib.oracle_threads.argtypes = []
        lib.oracle_threads.restype = ctypes.c_int
        lib.oracle_gradient.argtypes = (
            [ctypes.c_int] * 3 + [ctypes.c_double] * 4 + [ctypes.c_void_p, ctypes.c_int]
            + [ctypes.c_int] * 3 + [ctypes.c_double] * 3
            + [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p])
        lib.oracle_gradient.restype = ctypes.c_int
        lib.oracle_gradient_cpml.argtypes = (
            [ctypes.c_int] * 3 + [ctypes.c_double] * 4 + [ctypes.c_void_p, ctypes.c_int]
            + [ctypes.c_int] + [ctypes.c_double] * 3
            + [ctypes.c_int] * 3 + [ctypes.c_double] * 3
            + [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p])
        lib.oracle_gradient_cpml.restype = ctypes.c_int
        lib.oracle_first_weights.argtypes = [dp]
        lib.oracle_first_weights.restype = None
        lib.oracle_cpml_profile.argtypes = [ctypes.c_int, ctypes.c_int] + [ctypes.c_double] * 5 + [
            ctypes.c_void_p, ctypes.c_void_p]
        lib.oracle_cpml_profile.restype = None
        lib.oracle_propagate_cpml.argtypes = (
            [ctypes.c_int] * 3 + [ctypes.c_double] * 4 + [ctypes.c_void_p] * 5
            + [ctypes.c_int64, ctypes.c_int, ctypes.c_int] + [ctypes.c_double] * 3
            + [ctypes.c_int] * 4 + [ctypes.c_double] * 3
            + [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p])
        lib.oracle_propagate_cpml.restype = ctypes.c_int
        _lib = lib
    return _lib


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        assert a.shape == shape, (a.shape, shape)
    return a


def weights():
    """The five w_m of Eq. 1's axis operator (w_0 .. w_4), as used by the oracle."""
    w = np.zeros(5, dtype=np.float64)
    _load().oracle_weights(w.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return w


def laplacian(u, spacing, periodic=False):
    """Eq. 1 applied at every interior point of ``u`` (shape (nz, ny, nx))."""
    u = _f64(u)
    nz, ny, nx = u.shape
    out = np.empty_like(u)
    _load().oracle_laplacian(nx, ny, nz, *map(float, spacing), u.ctypes.data,
                             out.ctypes.data, int(bool(periodic)))
    return out


def ricker(t, f=15.0, t0=None, amp=1.0):
    """Ricker wavelet value at time t (seconds); t0 defaults to 1/f."""
    if t0 is None or t0 < 0:
        t0 = 1.0 / f
    return _load().oracle_ricker(float(t), float(f), float(t0), float(amp))


def cfl_dt(spacing, vmax):
    """Largest stable leapfrog dt for this stencil at velocity vmax."""
    return _load().oracle_cfl_dt(*map(float, spacing), float(vmax))


def propagate(vel, spacing, dt, nsteps, u=None, u_prev=None, step0=0,
              source=None, wavelet=None, receivers=None, periodic=False):
    """Advance the wave state by ``nsteps`` leapfrog steps in FP64.

    vel        (nz, ny, nx) velocities in m/s (any float dtype; read as FP64)
    u, u_prev  initial fields (default zero); not modified
    source     None or (sx, sy, sz, f, t0, amp) -- Ricker point source;
               t0 < 0 means 1/f
    wavelet    optional array of nsteps source values replacing the Ricker
    receivers  None or int array (nrec, 3) of (x, y, z)
    Returns (u, u_prev, traces) with traces of shape (nsteps, nrec).
    """
    vel = _f64(vel)
    nz, ny, nx = vel.shape
    u = np.zeros_like(vel) if u is None else _f64(u, vel.shape).copy()
    up = np.zeros_like(vel) if u_prev is None else _f64(u_prev, vel.shape).copy()
    if receivers is None:
        rec = np.zeros((0, 3), dtype=np.int32)
    else:
        rec = np.ascontiguousarray(receivers, dtype=np.int32).reshape(-1, 3)
    nrec = rec.shape[0]
    traces = np.zeros((nsteps, max(nrec, 0)), dtype=np.float64)
    if source is None:
        has_src, sx, sy, sz, f, t0, amp = 0, 0, 0, 0, 0.0, 0.0, 0.0
    else:
        sx, sy, sz, f, t0, amp = source
        has_src = 1
        if t0 is None or t0 < 0:
            t0 = 1.0 / f
    wl = None
    if wavelet is not None:
        wl = _f64(wavelet)
        assert wl.shape[0] >= nsteps
    rc = _load().oracle_propagate(
        nx, ny, nz, *map(float, spacing), float(dt), vel.ctypes.data, u.ctypes.data,
        up.ctypes.data, int(step0), int(nsteps), has_src, int(sx), int(sy), int(sz),
        float(f), float(t0), float(amp), None if wl is None else wl.ctypes.data,
        rec.ctypes.data if nrec else None, nrec, traces.ctypes.data if nrec else None,
        int(bool(periodic)))
    if rc != 0:
        raise ValueError("oracle_propagate rejected its input (rc=%d)" % rc)
    return u, up, traces


def gradient(vel, spacing, dt, nsteps, source, receivers, resid):
    """Discrete adjoint gradient dJ/d(v^2) of a run from rest, given
    resid[n, r] = dJ/d traces[n, r]. Returns (nz, ny, nx) FP64."""
    vel = _f64(vel)
    nz, ny, nx = vel.shape
    rec = np.ascontiguousarray(receivers, dtype=np.int32).reshape(-1, 3)
    res = _f64(resid).reshape(nsteps, rec.shape[0])
    sx, sy, sz, f, t0, amp = source
    if t0 is None or t0 < 0:
        t0 = 1.0 / f
    g = np.zeros_like(vel)
    rc = _load().oracle_gradient(nx, ny, nz, *map(float, spacing), float(dt), vel.ctypes.data,
                                 int(nsteps), int(sx), int(sy), int(sz), float(f), float(t0),
                                 float(amp), rec.ctypes.data, rec.shape[0], res.ctypes.data,
                                 g.ctypes.data)
    if rc != 0:
        raise ValueError("oracle_gradient rejected its input (rc=%d)" % rc)
    return g


def gradient_cpml(vel, spacing, dt, nsteps, npml, source, receivers, resid, R=1e-3,
                  fcps=15.0, vmax=None):
    """Discrete adjoint gradient dJ/d(v^2) of a CPML run from rest (the layer's
    profile held fixed at vmax, default the model's largest velocity), given
    resid[n, r] = dJ/d traces[n, r]. Returns (nz, ny, nx) FP64."""
    vel = _f64(vel)
    nz, ny, nx = vel.shape
    rec = np.ascontiguousarray(receivers, dtype=np.int32).reshape(-1, 3)
    res = _f64(resid).reshape(nsteps, rec.shape[0])
    sx, sy, sz, f, t0, amp = source
    if t0 is None or t0 < 0:
        t0 = 1.0 / f
    vm = float(vel.max()) if vmax is None else float(vmax)
    g = np.zeros_like(vel)
    rc = _load().oracle_gradient_cpml(
        nx, ny, nz, *map(float, spacing), float(dt), vel.ctypes.data, int(nsteps), int(npml),
        float(R), float(fcps), vm, int(sx), int(sy), int(sz), float(f), float(t0), float(amp),
        rec.ctypes.data, rec.shape[0], res.ctypes.data, g.ctypes.data)
    if rc != 0:
        raise ValueError("oracle_gradient_cpml rejected its input (rc=%d)" % rc)
    return g


def first_weights():
    """The 8th-order central first-derivative weights (index 1..4; index 0 unused)."""
    w = np.zeros(5, dtype=np.float64)
    _load().oracle_first_weights(w.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return w


def cpml_profile(n, npml, h, dt, vmax, R=1e-3, fcps=15.0):
    """(b, a) recursive-convolution coefficients of one axis of n cells."""
    b = np.zeros(n)
    a = np.zeros(n)
    _load().oracle_cpml_profile(int(n), int(npml), float(h), float(dt), float(vmax), float(R),
                                float(fcps), b.ctypes.data, a.ctypes.data)
    return b, a


def propagate_cpml(vel, spacing, dt, nsteps, npml, R=1e-3, fcps=15.0, vmax=None, u=None,
                   u_prev=None, psi=None, zeta=None, step0=0, source=None, receivers=None):
    """oracle propagate with the CPML layer; returns (u, u_prev, psi, zeta, traces)
    with psi and zeta of shape (3, nz, ny, nx) (axis x, y, z)."""
    vel = _f64(vel)
    nz, ny, nx = vel.shape
    u = np.zeros_like(vel) if u is None else _f64(u, vel.shape).copy()
    up = np.zeros_like(vel) if u_prev is None else _f64(u_prev, vel.shape).copy()
    ps = np.zeros((3,) + vel.shape) if psi is None else _f64(psi).copy()
    ze = np.zeros((3,) + vel.shape) if zeta is None else _f64(zeta).copy()
    rec = (np.zeros((0, 3), dtype=np.int32) if receivers is None
           else np.ascontiguousarray(receivers, dtype=np.int32).reshape(-1, 3))
    nrec = rec.shape[0]
    traces = np.zeros((nsteps, nrec))
    if source is None:
        has, sx, sy, sz, f, t0, amp = 0, 0, 0, 0, 0.0, 0.0, 0.0
    else:
        sx, sy, sz, f, t0, amp = source
        has = 1
        if t0 is None or t0 < 0:
            t0 = 1.0 / f
    vm = float(vel.max()) if vmax is None else float(vmax)
    rc = _load().oracle_propagate_cpml(
        nx, ny, nz, *map(float, spacing), float(dt), vel.ctypes.data, u.ctypes.data,
        up.ctypes.data, ps.ctypes.data, ze.ctypes.data, int(step0), int(nsteps), int(npml),
        float(R), float(fcps), vm, has, int(sx), int(sy), int(sz), float(f), float(t0),
        float(amp), rec.ctypes.data if nrec else None, nrec,
        traces.ctypes.data if nrec else None)
    if rc != 0:
        raise ValueError("oracle_propagate_cpml rejected its input (rc=%d)" % rc)
    return u, up, ps, ze, traces


def threads_used():
    """Number of OpenMP threads the oracle's parallel loops run with."""
    return int(_load().oracle_threads())
