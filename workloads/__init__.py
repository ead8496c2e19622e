"""Seeded synthetic inputs for the 3D acoustic wave path.

This module holds the input generators shared by the tests, the smoke check
and the benchmark. It contains none of the method's arithmetic (no stencil,
no time update, no source wavelet, no stability limit): only velocity
models, geometry (source and receiver positions) and random initial states.
Both the CUDA path and the oracle receive the same bytes from it.

The paper uses no dataset and prints no velocity model; its grids are cubes
of 100^3 .. 1024^3 points stepped 1000 times (Sec. 4.2, Sec. 5, Sec. 6.2).
The models below stand in for its unnamed workload:

* ``layered3``: three equal-thickness horizontal layers of 1500, 2500 and
  3500 m/s (z is depth), layer k < nz/3, k < 2nz/3, rest (integer division).
* ``random_layered``: 8 layers with 7 interfaces at sorted uniform-random
  depths and sorted uniform velocities in [1500, 4500] m/s, times (1 + eta)
  with eta an i.i.d. N(0,1) field smoothed by a Gaussian of sigma = 4 cells
  and scaled to max |eta| = 0.05.
* ``receiver_plane``: a plane of receivers at depth z, every 4th point in x
  and y starting at 0.
"""
import math

import numpy as np

# Workload descriptions: sizes are interior points (nx, ny, nz), x fastest.
CFG_SMALL = dict(name="layered3_64cube", shape=(64, 64, 64), spacing=(10.0, 10.0, 10.0),
                 cfl_fraction=0.5, f_peak=15.0, nsteps=100, seed=0,
                 source=(32, 32, 32), rec_z=8, rec_stride=4)
CFG_512 = dict(name="random8layer_512cube", shape=(512, 512, 512), spacing=(10.0, 10.0, 10.0),
               cfl_fraction=0.5, f_peak=15.0, nsteps=1000, seed=0,
               source=(256, 256, 10), rec_z=8, rec_stride=4)
CFG_1024 = dict(name="random8layer_1024x1024x512", shape=(1024, 1024, 512),
                spacing=(10.0, 10.0, 10.0), cfl_fraction=0.5, f_peak=15.0, nsteps=1000,
                seed=0, source=(512, 512, 10), rec_z=8, rec_stride=4)


def layered3(nx, ny, nz, v=(1500.0, 2500.0, 3500.0)):
    """Three horizontal layers in z; returns float32 (nz, ny, nx)."""
    out = np.empty((nz, ny, nx), dtype=np.float32)
    for k in range(nz):
        if k < nz // 3:
            out[k] = v[0]
        elif k < (2 * nz) // 3:
            out[k] = v[1]
        else:
            out[k] = v[2]
    return out


def _gauss_taps(sigma, truncate=4.0):
    r = int(math.ceil(truncate * sigma))
    x = np.arange(-r, r + 1, dtype=np.float64)
    g = np.exp(-0.5 * (x / sigma) ** 2)
    return g / g.sum()


def smooth_gaussian(a, sigma):
    """Separable Gaussian smoothing with zero padding, on CPU, float32.

    Uses torch's multithreaded CPU elementwise ops when torch is importable
    (plain shifted-slice sums: deterministic on one machine), else numpy.
    """
    taps = _gauss_taps(sigma)
    r = (len(taps) - 1) // 2
    try:
        import torch
        src = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32))
        for axis in range(3):
            out = torch.zeros_like(src)
            n = src.shape[axis]
            for t, g in zip(range(-r, r + 1), taps):
                lo, hi = max(0, -t), min(n, n - t)
                if hi <= lo:
                    continue
                dst = out.narrow(axis, lo, hi - lo)
                dst.add_(src.narrow(axis, lo + t, hi - lo), alpha=float(g))
            src = out
        return src.numpy()
    except ImportError:
        src = np.ascontiguousarray(a, dtype=np.float32)
        for axis in range(3):
            out = np.zeros_like(src)
            n = src.shape[axis]
            for t, g in zip(range(-r, r + 1), taps):
                lo, hi = max(0, -t), min(n, n - t)
                if hi <= lo:
                    continue
                d = [slice(None)] * 3
                s = [slice(None)] * 3
                d[axis] = slice(lo, hi)
                s[axis] = slice(lo + t, hi + t)
                out[tuple(d)] += np.float32(g) * src[tuple(s)]
            src = out
        return src


def random_layered(nx, ny, nz, seed=0, nlayers=8, vmin=1500.0, vmax=4500.0,
                   noise=0.05, sigma=4.0):
    """Random layered model with smoothed multiplicative noise; float32 (nz, ny, nx)."""
    rng = np.random.default_rng(seed)
    depths = np.sort(rng.integers(1, nz, size=nlayers - 1))
    vels = np.sort(rng.uniform(vmin, vmax, size=nlayers))
    layer = np.searchsorted(depths, np.arange(nz), side="right")
    vz = vels[layer].astype(np.float32)
    eta = rng.standard_normal((nz, ny, nx), dtype=np.float32)
    eta = smooth_gaussian(eta, sigma)
    m = float(np.max(np.abs(eta)))
    if m > 0:
        eta *= np.float32(noise / m)
    eta += np.float32(1.0)
    eta *= vz[:, None, None]
    return eta


def receiver_plane(nx, ny, z, stride=4):
    """int32 (nrec, 3) receivers (x, y, z) on plane z, every ``stride`` points."""
    xs = np.arange(0, nx, stride, dtype=np.int32)
    ys = np.arange(0, ny, stride, dtype=np.int32)
    yy, xx = np.meshgrid(ys, xs, indexing="ij")
    rec = np.stack([xx.ravel(), yy.ravel(), np.full(xx.size, z, dtype=np.int32)], axis=1)
    return np.ascontiguousarray(rec, dtype=np.int32)


def random_state(shape_zyx, seed, scale=1.0):
    """Two float32 random fields (u, u_prev), uniform in [-scale, scale]."""
    rng = np.random.default_rng(seed)
    u = rng.uniform(-scale, scale, size=shape_zyx).astype(np.float32)
    up = rng.uniform(-scale, scale, size=shape_zyx).astype(np.float32)
    return u, up


def random_receivers(nx, ny, nz, n, seed):
    """int32 (n, 3) receivers at uniform random interior points."""
    rng = np.random.default_rng(seed)
    rec = np.stack([rng.integers(0, nx, n), rng.integers(0, ny, n),
                    rng.integers(0, nz, n)], axis=1)
    return np.ascontiguousarray(rec, dtype=np.int32)


def layered_profile(nz, seed, nlayers=8, vmin=1500.0, vmax=4500.0):
    """float32 (nz,) velocities of a random horizontally layered model."""
    rng = np.random.default_rng(seed)
    depths = np.sort(rng.integers(1, max(2, nz), size=nlayers - 1))
    vels = np.sort(rng.uniform(vmin, vmax, size=nlayers))
    return vels[np.searchsorted(depths, np.arange(nz), side="right")].astype(np.float32)


def layered_volume(nx, ny, nz, seed):
    """float32 (nz, ny, nx) random layered model (no lateral variation)."""
    vz = layered_profile(nz, seed)
    return np.ascontiguousarray(np.broadcast_to(vz[:, None, None], (nz, ny, nx)))


# Shot-serving stream: Poisson arrivals of independent shots of uneven sizes.
SERVE_STREAM = dict(n=256, rate_per_s=20.0, seed=0, sizes=tuple(range(128, 513, 32)),
                    steps=(300, 800), src_z=10, rec_z=8, rec_stride=4,
                    budget_bytes=150 * 10 ** 9)


def serving_requests(n=256, rate_per_s=20.0, seed=0, sizes=tuple(range(128, 513, 32)),
                     steps=(300, 800), src_z=10, **_):
    """Seeded request list: arrival time (s), grid (nx, ny, nz), nsteps,
    source (x, y, z) and the seed of its layered velocity model."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(n):
        t += rng.exponential(1.0 / rate_per_s)
        nx, ny, nz = (int(rng.choice(sizes)) for _ in range(3))
        out.append(dict(arrival_s=t, grid=(nx, ny, nz),
                        nsteps=int(rng.integers(steps[0], steps[1] + 1)),
                        source=(int(rng.integers(0, nx)), int(rng.integers(0, ny)),
                                min(src_z, nz - 1)),
                        vel_seed=int(rng.integers(0, 2 ** 31))))
    return out


# Gradient workload: layered truth with a Gaussian anomaly, smoothed start.
CFG_GRAD = dict(name="anomaly_256cube", shape=(256, 256, 256), spacing=(10.0, 10.0, 10.0),
                nsteps=800, ckpt_every=40, f_peak=15.0, seed=0, anomaly_mps=300.0,
                rec_z=8, rec_stride=4)
CFG_GRAD_SMALL = dict(CFG_GRAD, name="anomaly_32cube", shape=(32, 32, 32), nsteps=60,
                      ckpt_every=7, rec_z=4, rec_stride=2)


def anomaly_model(nx, ny, nz, seed=0, anomaly=300.0):
    """Layered model (3 layers, seeded velocities) plus a Gaussian velocity
    anomaly of `anomaly` m/s at the grid centre (radius nz/6); float32."""
    rng = np.random.default_rng(seed)
    v = np.sort(rng.uniform(1800.0, 3200.0, size=3)).astype(np.float32)
    out = layered3(nx, ny, nz, v=tuple(float(x) for x in v))
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    r2 = ((x - nx / 2) ** 2 + (y - ny / 2) ** 2 + (z - nz / 2) ** 2) / (nz / 6.0) ** 2
    out += np.float32(anomaly) * np.exp(-r2).astype(np.float32)
    return out


def smoothed_start(model, sigma=3.0):
    """The starting model: the true model smoothed by a Gaussian (sigma cells)
    without the anomaly's sharp contrast; float32."""
    return smooth_gaussian(model, sigma)


def velocity_for(cfg):
    """The velocity model a workload description names."""
    nx, ny, nz = cfg["shape"]
    if cfg["name"].startswith("layered3"):
        return layered3(nx, ny, nz)
    return random_layered(nx, ny, nz, seed=cfg["seed"])
