"""Python binding of the gbwave C ABI (include/wave.h).

Argument marshalling only: every step of the wave update runs in the CUDA
library ``_build/libgbwave.so``. If that library is missing, ``load()``
raises; there is no CPU fallback.

Arrays may be torch tensors (CUDA or CPU) or numpy arrays; they are passed to
the library as raw pointers (``data_ptr()`` / ``ctypes.data``), and the
library decides from the pointer whether it is host or device memory. The
CUDA stream defaults to torch's current stream.
"""
import ctypes
import os

__all__ = [
    "WaveError", "load", "wave_cfl_dt", "wave_create", "wave_step", "wave_propagate",
    "wave_get_field", "wave_set_state", "wave_get_step", "wave_reset",
    "wave_synchronize", "wave_destroy", "wave_strerror", "wave_get_launch_info",
    "wave_selftest_wait", "wave_propagate_noalloc", "WaveSolver", "library_path",
    "ShotServer", "wave_adjoint", "wave_gradient", "WaveTraces", "wave_traces",
    "wave_set_cpml", "wave_create_async", "wave_create_m",
]

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "_build", "libgbwave.so")
_lib = None

WAVE_OK = 0
STATUS = {0: "WAVE_OK", -1: "WAVE_EINVAL", -2: "WAVE_ENOMEM", -3: "WAVE_ECUDA",
          -4: "WAVE_EUNSTABLE", -5: "WAVE_ETIMEOUT", -6: "WAVE_EBUSY", -7: "WAVE_ENAN",
          -8: "WAVE_ENOTSUP", -9: "WAVE_ETOOBIG"}


class WaveError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        msg = _lib.wave_strerror(code).decode() if _lib is not None else str(code)
        super().__init__("%s: %s (%s)" % (where, msg, STATUS.get(code, code)))


class _Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32)]


class _Spacing(ctypes.Structure):
    _fields_ = [("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dz", ctypes.c_double)]


class _Shot(ctypes.Structure):
    _fields_ = [("sx", ctypes.c_int32), ("sy", ctypes.c_int32), ("sz", ctypes.c_int32),
                ("f_peak", ctypes.c_double), ("t0", ctypes.c_double), ("amp", ctypes.c_double)]


class _Request(ctypes.Structure):
    _fields_ = [("grid", _Grid), ("spacing", _Spacing), ("dt", ctypes.c_double),
                ("velocity", ctypes.c_void_p), ("storage", ctypes.c_int), ("shot", _Shot),
                ("nsteps", ctypes.c_int), ("rec_xyz", ctypes.c_void_p), ("nrec", ctypes.c_int),
                ("traces", ctypes.c_void_p), ("npml", ctypes.c_int),
                ("reflection", ctypes.c_double), ("f_cps", ctypes.c_double)]


class _Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("ticket", ctypes.c_uint64),
                ("submit_s", ctypes.c_double), ("start_s", ctypes.c_double),
                ("done_s", ctypes.c_double), ("dt", ctypes.c_double),
                ("steps_done", ctypes.c_int64)]


class _Stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("failed", ctypes.c_int64), ("queued", ctypes.c_int64),
                ("resident", ctypes.c_int64), ("bytes_resident", ctypes.c_size_t),
                ("bytes_peak", ctypes.c_size_t), ("resident_peak", ctypes.c_int),
                ("batch_steps", ctypes.c_int64), ("point_steps", ctypes.c_double),
                ("busy_s", ctypes.c_double)]


def library_path():
    return _LIB_PATH


def load(path=None):
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(
            "gbwave CUDA library not found at %s; build it with "
            "`python -c 'import __graft_entry__ as g; g.build()'`" % path)
    lib = ctypes.CDLL(path)
    vp, ip = ctypes.c_void_p, ctypes.c_int
    lib.wave_cfl_dt.argtypes = [ctypes.POINTER(_Spacing), ctypes.c_double]
    lib.wave_cfl_dt.restype = ctypes.c_double
    lib.wave_create.argtypes = [ctypes.POINTER(_Grid), ctypes.POINTER(_Spacing),
                                ctypes.c_double, vp, ip, vp, ctypes.POINTER(vp)]
    lib.wave_create_async.argtypes = lib.wave_create.argtypes
    lib.wave_create_m.argtypes = lib.wave_create.argtypes
    lib.wave_step.argtypes = [vp, ip]
    lib.wave_propagate.argtypes = [vp, ctypes.POINTER(_Shot), ip, vp, ip, vp]
    lib.wave_get_field.argtypes = [vp, ip, vp]
    lib.wave_set_state.argtypes = [vp, vp, vp, ctypes.c_int64]
    lib.wave_get_step.argtypes = [vp, ctypes.POINTER(ctypes.c_int64)]
    lib.wave_reset.argtypes = [vp]
    lib.wave_set_cpml.argtypes = [vp, ip, ctypes.c_double, ctypes.c_double]
    lib.wave_synchronize.argtypes = [vp]
    lib.wave_destroy.argtypes = [vp]
    lib.wave_destroy.restype = None
    lib.wave_strerror.argtypes = [ip]
    lib.wave_strerror.restype = ctypes.c_char_p
    lib.wave_get_launch_info.argtypes = [vp] + [ctypes.POINTER(ctypes.c_int)] * 5
    lib.wave_selftest_wait.argtypes = [ctypes.c_int64, vp]
    lib.wave_adjoint.argtypes = [vp, ctypes.POINTER(_Shot), ip, vp, ip, vp, ip, vp, vp]
    lib.wave_gradient.argtypes = [vp, ctypes.POINTER(_Shot), ip, vp, ip, vp, ip,
                                  ctypes.POINTER(ctypes.c_double), vp, vp]
    lib.wave_adjoint.restype = ctypes.c_int
    lib.wave_gradient.restype = ctypes.c_int
    lib.serve_create.argtypes = [ctypes.c_size_t, ip, vp, ctypes.POINTER(vp)]
    lib.serve_submit.argtypes = [vp, ctypes.POINTER(_Request), ctypes.POINTER(ctypes.c_uint64)]
    lib.serve_poll.argtypes = [vp, ctypes.c_uint64, ctypes.POINTER(_Result)]
    lib.serve_wait.argtypes = [vp, ctypes.c_uint64, ctypes.c_double, ctypes.POINTER(_Result)]
    lib.serve_get_stats.argtypes = [vp, ctypes.POINTER(_Stats)]
    lib.serve_destroy.argtypes = [vp]
    lib.serve_destroy.restype = None
    for name in ("serve_create", "serve_submit", "serve_poll", "serve_wait", "serve_get_stats"):
        getattr(lib, name).restype = ctypes.c_int
    lib.wave_propagate_noalloc.argtypes = [
        ctypes.POINTER(_Grid), ctypes.POINTER(_Spacing), ctypes.c_double, vp, vp, vp,
        ctypes.POINTER(_Shot), ctypes.c_int64, ip, vp, ip, vp, vp, ctypes.POINTER(ip)]
    for name in ("wave_create", "wave_create_async", "wave_create_m", "wave_step", "wave_propagate", "wave_get_field",
                 "wave_set_state", "wave_get_step", "wave_reset", "wave_synchronize",
                 "wave_get_launch_info", "wave_selftest_wait", "wave_propagate_noalloc",
                 "wave_set_cpml"):
        getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def _check(code, where):
    if code != WAVE_OK:
        raise WaveError(code, where)


def _ptr(a, dtype_name, count, what):
    """Raw pointer of a contiguous torch tensor / numpy array with ``count`` elements."""
    if a is None:
        return None
    mod = type(a).__module__
    if mod.startswith("torch"):
        import torch
        want = {"float32": torch.float32, "int32": torch.int32}[dtype_name]
        if a.dtype != want or not a.is_contiguous():
            raise ValueError("%s must be a contiguous %s tensor" % (what, dtype_name))
        if a.numel() < count:
            raise ValueError("%s has %d elements, needs %d" % (what, a.numel(), count))
        return a.data_ptr()
    import numpy as np
    if not isinstance(a, np.ndarray):
        raise TypeError("%s must be a torch tensor or numpy array" % what)
    if a.dtype != np.dtype(dtype_name) or not a.flags["C_CONTIGUOUS"]:
        raise ValueError("%s must be a C-contiguous %s array" % (what, dtype_name))
    if a.size < count:
        raise ValueError("%s has %d elements, needs %d" % (what, a.size, count))
    if not a.flags["WRITEABLE"] and what in ("traces", "out"):
        raise ValueError("%s must be writeable" % what)
    return a.ctypes.data


def _default_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except ImportError:
        pass
    return 0


def wave_cfl_dt(spacing, vmax):
    """Largest stable dt for spacing (dx, dy, dz) and velocity vmax."""
    lib = load()
    return lib.wave_cfl_dt(ctypes.byref(_Spacing(*map(float, spacing))), float(vmax))


def wave_create(grid, spacing, dt, velocity, storage=0, stream=None, defer=False,
                squared=False):
    """Create a context; ``grid`` = (nx, ny, nz); velocity has nx*ny*nz float32.

    ``defer=True`` calls wave_create_async: the model is read on the GPU after
    the call returns (keep ``velocity`` alive and unchanged until the next
    synchronizing call); errors in it are raised by that call.
    ``squared=True`` calls wave_create_m: ``velocity`` holds m = v^2.
    """
    lib = load()
    nx, ny, nz = map(int, grid)
    g = _Grid(nx, ny, nz)
    h = _Spacing(*map(float, spacing))
    vptr = _ptr(velocity, "float32", nx * ny * nz, "velocity")
    out = ctypes.c_void_p()
    st = _default_stream() if stream is None else int(stream)
    if squared and defer:
        raise ValueError("squared and defer cannot be combined")
    name = "wave_create_m" if squared else ("wave_create_async" if defer else "wave_create")
    _check(getattr(lib, name)(ctypes.byref(g), ctypes.byref(h), float(dt), vptr, int(storage),
                              st, ctypes.byref(out)), name)
    return out


def wave_step(ctx, nsteps):
    _check(load().wave_step(ctx, int(nsteps)), "wave_step")


def wave_propagate(ctx, shot, nsteps, rec=None, traces=None):
    """Advance ``nsteps`` with source ``shot`` = (sx, sy, sz, f_peak, t0, amp) or None.

    ``rec``: int32 (nrec, 3) receiver points; ``traces``: float32 (nsteps, nrec) output.
    """
    lib = load()
    if rec is not None and (len(rec.shape) != 2 or rec.shape[1] != 3):
        raise ValueError("rec must have shape (nrec, 3)")
    nrec = 0 if rec is None else int(rec.shape[0])
    rptr = _ptr(rec, "int32", 3 * nrec, "rec") if nrec else None
    tptr = _ptr(traces, "float32", int(nsteps) * nrec, "traces") if nrec else None
    sp = None
    if shot is not None:
        sx, sy, sz, f, t0, amp = shot
        sp = ctypes.byref(_Shot(int(sx), int(sy), int(sz), float(f),
                                -1.0 if t0 is None else float(t0), float(amp)))
    _check(lib.wave_propagate(ctx, sp, int(nsteps), rptr, int(nrec), tptr), "wave_propagate")


def wave_get_field(ctx, which, out, count):
    _check(load().wave_get_field(ctx, int(which), _ptr(out, "float32", count, "out")),
           "wave_get_field")


def wave_set_state(ctx, u, u_prev, step, count):
    _check(load().wave_set_state(ctx, _ptr(u, "float32", count, "u"),
                                 _ptr(u_prev, "float32", count, "u_prev"), int(step)),
           "wave_set_state")


def wave_get_step(ctx):
    s = ctypes.c_int64()
    _check(load().wave_get_step(ctx, ctypes.byref(s)), "wave_get_step")
    return s.value


def wave_reset(ctx):
    _check(load().wave_reset(ctx), "wave_reset")


def wave_set_cpml(ctx, npml, reflection=1e-3, f_cps=15.0):
    """Absorbing CPML layer of npml cells at every face (0 switches it off)."""
    _check(load().wave_set_cpml(ctx, int(npml), float(reflection), float(f_cps)),
           "wave_set_cpml")


def wave_synchronize(ctx):
    _check(load().wave_synchronize(ctx), "wave_synchronize")


def wave_destroy(ctx):
    if ctx:
        load().wave_destroy(ctx)


def wave_propagate_noalloc(grid, spacing, dt, velocity, u, u_prev, shot, step0, nsteps,
                           rec=None, traces=None, stream=None):
    """Allocation-free propagation on caller-owned device buffers.

    Returns ``newest``: 0 if ``u`` holds the newest step on return, 1 if
    ``u_prev`` does. Raises WaveError on a non-zero status (WAVE_ETOOBIG when
    the request does not fit the library's fixed scratch array).
    """
    lib = load()
    nx, ny, nz = map(int, grid)
    count = nx * ny * nz
    if rec is not None and (len(rec.shape) != 2 or rec.shape[1] != 3):
        raise ValueError("rec must have shape (nrec, 3)")
    nrec = 0 if rec is None else int(rec.shape[0])
    sp = None
    if shot is not None:
        sx, sy, sz, f, t0, amp = shot
        sp = ctypes.byref(_Shot(int(sx), int(sy), int(sz), float(f),
                                -1.0 if t0 is None else float(t0), float(amp)))
    newest = ctypes.c_int(0)
    st = _default_stream() if stream is None else int(stream)
    _check(lib.wave_propagate_noalloc(
        ctypes.byref(_Grid(nx, ny, nz)), ctypes.byref(_Spacing(*map(float, spacing))),
        float(dt), _ptr(velocity, "float32", count, "velocity"),
        _ptr(u, "float32", count, "u"), _ptr(u_prev, "float32", count, "u_prev"), sp,
        int(step0), int(nsteps), _ptr(rec, "int32", 3 * nrec, "rec") if nrec else None, nrec,
        _ptr(traces, "float32", int(nsteps) * nrec, "traces") if nrec else None, st,
        ctypes.byref(newest)), "wave_propagate_noalloc")
    return newest.value


def _shot_ref(shot):
    if shot is None:
        return None
    sx, sy, sz, f, t0, amp = shot
    return ctypes.byref(_Shot(int(sx), int(sy), int(sz), float(f),
                              -1.0 if t0 is None else float(t0), float(amp)))


def wave_adjoint(ctx, shot, nsteps, rec, resid, ckpt_every, grad, count, traces=None):
    """dJ/d(v^2) of a run from rest given resid = dJ/dtraces (nsteps, nrec)."""
    nrec = 0 if rec is None else int(rec.shape[0])
    _check(load().wave_adjoint(
        ctx, _shot_ref(shot), int(nsteps), _ptr(rec, "int32", 3 * nrec, "rec") if nrec else None,
        nrec, _ptr(resid, "float32", int(nsteps) * nrec, "resid") if nrec else None,
        int(ckpt_every), _ptr(grad, "float32", count, "grad"),
        _ptr(traces, "float32", int(nsteps) * nrec, "traces") if traces is not None else None),
        "wave_adjoint")


def wave_gradient(ctx, shot, nsteps, rec, observed, ckpt_every, grad, count, traces=None):
    """L2 trace misfit of a run from rest and its gradient dJ/d(v^2); returns the misfit."""
    nrec = 0 if rec is None else int(rec.shape[0])
    mis = ctypes.c_double(0.0)
    _check(load().wave_gradient(
        ctx, _shot_ref(shot), int(nsteps), _ptr(rec, "int32", 3 * nrec, "rec") if nrec else None,
        nrec, _ptr(observed, "float32", int(nsteps) * nrec, "observed") if nrec else None,
        int(ckpt_every), ctypes.byref(mis), _ptr(grad, "float32", count, "grad"),
        _ptr(traces, "float32", int(nsteps) * nrec, "traces") if traces is not None else None),
        "wave_gradient")
    return mis.value


def wave_selftest_wait(limit_ns, stream=None):
    """Run the bounded-wait self-test; returns the library status (WAVE_ETIMEOUT expected)."""
    st = _default_stream() if stream is None else int(stream)
    return load().wave_selftest_wait(int(limit_ns), st)


def wave_strerror(code):
    return load().wave_strerror(int(code)).decode()


def wave_get_launch_info(ctx):
    vals = [ctypes.c_int() for _ in range(5)]
    _check(load().wave_get_launch_info(ctx, *[ctypes.byref(v) for v in vals]),
           "wave_get_launch_info")
    keys = ("tile_x", "tile_y", "z_chunk", "grid_ctas", "ctas_per_sm")
    return dict(zip(keys, (v.value for v in vals)))


class WaveSolver:
    """Owning wrapper of one context (destroyed with the object)."""

    def __init__(self, grid, spacing, dt, velocity, storage=0, stream=None, defer=False,
                 squared=False):
        self.grid = tuple(int(v) for v in grid)
        self.spacing = tuple(float(v) for v in spacing)
        self.dt = float(dt)
        self.count = self.grid[0] * self.grid[1] * self.grid[2]
        self.ctx = wave_create(self.grid, self.spacing, self.dt, velocity, storage, stream,
                               defer, squared)
        # a deferred creation reads the model later: keep it alive until close
        self._velocity = velocity if defer else None

    def step(self, nsteps):
        wave_step(self.ctx, nsteps)

    def propagate(self, shot, nsteps, rec=None, traces=None):
        wave_propagate(self.ctx, shot, nsteps, rec, traces)

    def get_field(self, which, out):
        wave_get_field(self.ctx, which, out, self.count)
        return out

    def set_state(self, u, u_prev, step=0):
        wave_set_state(self.ctx, u, u_prev, step, self.count)

    @property
    def step_count(self):
        return wave_get_step(self.ctx)

    def reset(self):
        wave_reset(self.ctx)

    def set_cpml(self, npml, reflection=1e-3, f_cps=15.0):
        wave_set_cpml(self.ctx, npml, reflection, f_cps)

    def synchronize(self):
        wave_synchronize(self.ctx)

    def launch_info(self):
        return wave_get_launch_info(self.ctx)

    def adjoint(self, shot, nsteps, rec, resid, grad, ckpt_every=40, traces=None):
        wave_adjoint(self.ctx, shot, nsteps, rec, resid, ckpt_every, grad, self.count, traces)
        return grad

    def gradient(self, shot, nsteps, rec, observed, grad, ckpt_every=40, traces=None):
        return wave_gradient(self.ctx, shot, nsteps, rec, observed, ckpt_every, grad,
                             self.count, traces)

    def close(self):
        if getattr(self, "ctx", None):
            wave_destroy(self.ctx)
            self.ctx = None
        self._velocity = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _result_dict(r):
    return {"status": r.status, "ticket": r.ticket, "submit_s": r.submit_s,
            "start_s": r.start_s, "done_s": r.done_s, "dt": r.dt,
            "steps_done": r.steps_done}


class ShotServer:
    """Continuous-batching shot server (include/wave_serve.h).

    ``submit`` keeps references to the request's arrays until the request is
    reported complete by ``poll``/``wait``, since the engine reads velocity and
    receivers when it admits the request and writes the traces while it runs.
    CUDA tensors are made visible to the server's stream by synchronizing
    torch's current stream before each submit.
    """

    def __init__(self, hbm_budget_bytes, max_slots=64, stream=None):
        lib = load()
        out = ctypes.c_void_p()
        _check(lib.serve_create(int(hbm_budget_bytes), int(max_slots),
                                None if stream is None else int(stream), ctypes.byref(out)),
               "serve_create")
        self.handle = out
        self._keep = {}

    def submit(self, grid, spacing, velocity, shot, nsteps, rec=None, traces=None,
               storage=0, dt=0.0, cpml=None):
        """cpml: None, npml, or (npml, reflection, f_cps): the shot's CPML
        layer (reflection 1e-3 and f_cps 15 Hz when only npml is given)."""
        nx, ny, nz = map(int, grid)
        if cpml is None:
            npml, refl, fcps = 0, 1e-3, 15.0
        elif isinstance(cpml, int):
            npml, refl, fcps = cpml, 1e-3, 15.0
        else:
            npml, refl, fcps = cpml
        nrec = 0 if rec is None else int(rec.shape[0])
        if any(type(a).__module__.startswith("torch") and a.is_cuda
               for a in (velocity, rec, traces) if a is not None):
            import torch
            torch.cuda.current_stream().synchronize()
        sx, sy, sz, f, t0, amp = shot
        req = _Request(
            _Grid(nx, ny, nz), _Spacing(*map(float, spacing)), float(dt),
            _ptr(velocity, "float32", nx * ny * nz, "velocity"), int(storage),
            _Shot(int(sx), int(sy), int(sz), float(f), -1.0 if t0 is None else float(t0),
                  float(amp)),
            int(nsteps), _ptr(rec, "int32", 3 * nrec, "rec") if nrec else None, nrec,
            _ptr(traces, "float32", int(nsteps) * nrec, "traces") if nrec else None,
            int(npml), float(refl), float(fcps))
        ticket = ctypes.c_uint64()
        _check(load().serve_submit(self.handle, ctypes.byref(req), ctypes.byref(ticket)),
               "serve_submit")
        self._keep[ticket.value] = (velocity, rec, traces)
        return ticket.value

    def poll(self, ticket):
        r = _Result()
        st = load().serve_poll(self.handle, int(ticket), ctypes.byref(r))
        if st != -6:
            self._keep.pop(int(ticket), None)
        return st, _result_dict(r)

    def wait(self, ticket, timeout_s=-1.0):
        r = _Result()
        st = load().serve_wait(self.handle, int(ticket), float(timeout_s), ctypes.byref(r))
        if st != -6:
            self._keep.pop(int(ticket), None)
        return st, _result_dict(r)

    def stats(self):
        s = _Stats()
        _check(load().serve_get_stats(self.handle, ctypes.byref(s)), "serve_get_stats")
        return {k: getattr(s, k) for k, _ in _Stats._fields_}

    def close(self):
        if getattr(self, "handle", None):
            load().serve_destroy(self.handle)
            self.handle = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _make_traces_function():
    import torch

    class WaveTraces(torch.autograd.Function):
        """Receiver traces of a run from rest as a differentiable function of
        the squared velocity m = v^2 (a CUDA tensor of shape (nz, ny, nx)).

        forward: the 25-point leapfrog with the given source and receivers
        (wave_propagate). backward: the discrete adjoint (wave_adjoint) with
        the incoming gradient as dJ/dtraces, checkpointing every ``ckpt_every``
        steps. dt stays fixed, so the map m -> traces is a fixed discrete
        function; the library takes m itself (wave_create_m: v^2 dt^2 = m dt^2).
        cpml: None, npml, or (npml, reflection, f_cps) for the CPML layer
        (wave_set_cpml); its profile, set from the largest velocity of m, is
        held fixed by the derivative.
        """

        @staticmethod
        def forward(fctx, m, spacing, dt, shot, nsteps, rec, ckpt_every=40, cpml=None):
            nz, ny, nx = m.shape
            solver = WaveSolver((nx, ny, nz), spacing, dt,
                                m.detach().to(torch.float32).contiguous(), squared=True)
            if cpml is not None:
                solver.set_cpml(*((cpml,) if isinstance(cpml, int) else tuple(cpml)))
            traces = torch.zeros((nsteps, rec.shape[0]), dtype=torch.float32, device=m.device)
            solver.propagate(shot, nsteps, rec, traces)
            solver.synchronize()
            fctx.solver = solver
            fctx.args = (shot, int(nsteps), rec, int(ckpt_every))
            return traces

        @staticmethod
        def backward(fctx, grad_traces):
            shot, nsteps, rec, ckpt = fctx.args
            solver = fctx.solver
            grad = torch.empty((solver.grid[2], solver.grid[1], solver.grid[0]),
                               dtype=torch.float32, device=grad_traces.device)
            solver.adjoint(shot, nsteps, rec, grad_traces.to(torch.float32).contiguous(), grad,
                           ckpt_every=ckpt)
            solver.close()
            return grad, None, None, None, None, None, None, None

    return WaveTraces


def wave_traces(m, spacing, dt, shot, nsteps, rec, ckpt_every=40, cpml=None):
    """Differentiable traces(m = v^2); see WaveTraces."""
    return _make_traces_function().apply(m, spacing, dt, shot, nsteps, rec, ckpt_every, cpml)


def __getattr__(name):
    if name == "WaveTraces":
        return _make_traces_function()
    raise AttributeError(name)
