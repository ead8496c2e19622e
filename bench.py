"""Benchmark of the FP32 wave stepper on one GB300 (or N independent replicas).

One bench step = one time step of the whole hot path (Eq. 1 Laplacian +
leapfrog update + Ricker source injection + receiver sampling) over the
1024 x 1024 x 512 random 8-layer workload; K steps are one call of
wave_propagate. The metric is Gpts/s = interior points x steps / time.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload 1024x1024x512|512cube|64cube]

Prints one JSON line (rank 0). See the printed keys: value (device-timed,
inputs resident in HBM), e2e (host buffers through the C ABI, copies inside
the timed region), roofline of the sweep kernel, cpu_baseline (the FP64
oracle on this machine's host cores over a bounded sample), clocks.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads as wl  # noqa: E402

METRIC = ("Gpts/s & % HBM roofline (r=4 3D wave, FP32 vs BF16 store); "
          "serve p50/p99 latency")
BYTES_PER_POINT = 16  # FP32: read u, u_prev, v^2dt^2, write u_next
BYTES_PER_POINT_16 = 10  # 16-bit u, u_prev, u_next; FP32 v^2dt^2
STORAGE = {"f32": 0, "bf16": 1, "f16": 2}
WORKLOADS = {"1024x1024x512": wl.CFG_1024, "512cube": wl.CFG_512, "64cube": wl.CFG_SMALL}
KERNEL_SOURCES = ["paper_2404_04441_gb300/csrc/sweep.cuh", "paper_2404_04441_gb300/csrc/ptx.cuh"]
TRAFFIC_FILE = "profiles/sweep_f32_traffic.txt"
TRAFFIC_FILE_16 = "profiles/sweep_16bit_traffic.txt"
GRAPH_STEPS = 32


def kernel_hash():
    h = hashlib.sha256()
    for p in KERNEL_SOURCES:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def read_traffic(workload_name, path=TRAFFIC_FILE, prefix=""):
    """Per-launch DRAM bytes of the sweep kernel from a committed ncu summary
    (prefix "bf16:" / "f16:" selects a storage form in the 16-bit file), or
    None if absent, unreadable or taken on different kernel sources."""
    path = os.path.join(ROOT, path)
    if not os.path.exists(path):
        return None
    vals = {}
    for line in open(path):
        if ":" in line and not line.startswith("#"):
            k, v = line.rsplit(":", 1)
            vals[k.strip()] = v.strip()
    if vals.get("kernel_source_sha256_16") != kernel_hash():
        return None
    key = "dram_bytes_per_launch[%s%s]" % (prefix, workload_name)
    try:
        return float(vals[key]) if key in vals else None
    except ValueError:
        return None


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0}, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        time.sleep(0.3)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def stop(self):
        if self.proc is None:
            return
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)

    def summary(self, t0, t1):
        sm, smax, power, reasons = [], [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ts, line in self.lines:
            if not (t0 <= ts <= t1):
                continue
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "power_w_max": max(power), "reasons": sorted(reasons), "samples": len(sm)}


def replica_max(value, device):
    """Largest `value` over the ranks of the default process group (the value
    itself when not distributed): each replica times its own work and the job
    takes the slowest, as the multi-GPU timing rule asks."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(points_per_replica, steps, seconds_max, world):
    """Whole-job throughput of `world` independent replicas (Gpts/s)."""
    return world * points_per_replica * steps / seconds_max / 1e9


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def oracle_sample(vel, cfg, dt, budget_s, nsteps_cap=None):
    """Time the FP64 oracle on z-slabs of the workload (full x-y extent), growing
    the slab until one call takes a meaningful share of budget_s. Returns
    (Gpts/s, cores, sample description, seconds)."""
    import oracle
    nx, ny, nz = cfg["shape"]
    sp = cfg["spacing"]
    shot = (*cfg["source"], cfg["f_peak"], -1.0, 1.0)
    planes = 4
    rng = np.random.default_rng(5)
    while True:
        sl = vel[:planes]
        u0 = rng.uniform(-1, 1, size=sl.shape)
        up0 = rng.uniform(-1, 1, size=sl.shape)
        src = shot if shot[2] < planes else None
        t = time.perf_counter()
        oracle.propagate(sl, sp, dt, 1, u=u0, u_prev=up0, source=src)
        el = time.perf_counter() - t
        if el * 4 >= budget_s or planes >= nz:
            break
        planes = min(nz, planes * 2)
    steps = max(1, int(budget_s / max(el, 1e-6)))
    if nsteps_cap:
        steps = min(steps, nsteps_cap)
    t = time.perf_counter()
    oracle.propagate(sl, sp, dt, steps, u=u0, u_prev=up0, source=src)
    el = time.perf_counter() - t
    pts = nx * ny * planes * steps
    sample = "%dx%dx%d slab (z = 0..%d) of the workload, %d oracle steps from a random state" % (
        nx, ny, planes, planes - 1, steps)
    return pts / el / 1e9, oracle.threads_used(), sample, el


def precision_errors(gw, torch):
    """Relative L2 of fields and traces against the FP64 oracle for each storage
    mode on the random 8-layer 128^3 model, Ricker at (64, 64, 10), receivers
    on z = 8 every 4th point, 500 steps."""
    import oracle
    n, nsteps = 128, 500
    vel = wl.random_layered(n, n, n, seed=0)
    sp = (10.0, 10.0, 10.0)
    dt = 0.5 * gw.wave_cfl_dt(sp, float(vel.max()))
    rec = wl.receiver_plane(n, n, 8, 4)
    shot = (64, 64, 10, 15.0, -1.0, 1.0)
    ou, _, otr = oracle.propagate(vel, sp, dt, nsteps, source=shot, receivers=rec)
    out = {}
    for name, st in STORAGE.items():
        s = gw.WaveSolver((n, n, n), sp, dt, torch.from_numpy(vel).cuda(), storage=st)
        tr = torch.zeros((nsteps, rec.shape[0]), device="cuda")
        s.propagate(shot, nsteps, torch.from_numpy(rec).cuda(), tr)
        u = np.empty((n, n, n), np.float32)
        s.get_field(0, u)
        s.close()
        trh = tr.cpu().numpy().astype(np.float64)
        out[name] = {
            "rel_l2_field": float(np.linalg.norm(u - ou) / np.linalg.norm(ou)),
            "rel_l2_traces": float(np.linalg.norm(trh - otr) / np.linalg.norm(otr)),
            "workload": "random8layer_128cube, 500 steps"}
    return out


def serve_stream(gw, torch, storage, n_requests, max_slots=32):
    """The shot-serving stream: Poisson arrivals (mean 20/s) of shots with
    grids drawn from {128..512 step 32}^3, 300-800 steps, a random layered
    model each, source at z = 10, receivers every 4th point on z = 8,
    150 GB admission budget. Returns latency percentiles and throughput."""
    spec = dict(wl.SERVE_STREAM, n=n_requests)
    reqs = wl.serving_requests(**spec)
    srv = gw.ShotServer(spec["budget_bytes"], max_slots)
    pending = []
    t0 = time.perf_counter()
    for r in reqs:
        delay = t0 + r["arrival_s"] - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        nx, ny, nz = r["grid"]
        vz = torch.from_numpy(wl.layered_profile(nz, r["vel_seed"])).cuda()
        vel = vz[:, None, None].expand(nz, ny, nx).contiguous()
        rec = torch.from_numpy(wl.receiver_plane(nx, ny, min(spec["rec_z"], nz - 1),
                                                 spec["rec_stride"])).cuda()
        tr = torch.empty((r["nsteps"], rec.shape[0]), device="cuda")
        t = srv.submit(r["grid"], (10.0, 10.0, 10.0), vel, (*r["source"], 15.0, -1.0, 1.0),
                       r["nsteps"], rec, tr, storage=storage)
        pending.append((t, nx * ny * nz * r["nsteps"]))
    lat, work, first, last, failed = [], 0.0, None, 0.0, 0
    for t, pts in pending:
        st, res = srv.wait(t)
        if st != 0:
            failed += 1
            continue
        lat.append(res["done_s"] - res["submit_s"])
        work += pts
        first = res["submit_s"] if first is None else min(first, res["submit_s"])
        last = max(last, res["done_s"])
    stats = srv.stats()
    srv.close()
    lat = np.array(lat)
    return {"requests": len(reqs), "failed": failed,
            "p50_latency_s": float(np.percentile(lat, 50)) if lat.size else None,
            "p99_latency_s": float(np.percentile(lat, 99)) if lat.size else None,
            "mean_latency_s": float(lat.mean()) if lat.size else None,
            "gpts": work / max(last - first, 1e-9) / 1e9 if lat.size else None,
            "gpts_busy": stats["point_steps"] / max(stats["busy_s"], 1e-9) / 1e9,
            "makespan_s": last - first if lat.size else None,
            "resident_peak": stats["resident_peak"], "max_slots": max_slots,
            "bytes_peak": stats["bytes_peak"], "budget_bytes": spec["budget_bytes"],
            "arrival_rate_per_s": spec["rate_per_s"]}


def serve_saturated(gw, torch, n_requests=48):
    """Capacity on the stream's shot mix: the first n requests submitted at
    once to the server (FP32 and FP16 storage, then the same with a 16-cell
    CPML layer on every shot) against the same shots run one after another
    through the plain FP32 single-grid path."""
    reqs = wl.serving_requests(**dict(wl.SERVE_STREAM, n=n_requests))
    made = []
    for r in reqs:
        nx, ny, nz = r["grid"]
        vz = torch.from_numpy(wl.layered_profile(nz, r["vel_seed"])).cuda()
        vel = vz[:, None, None].expand(nz, ny, nx).contiguous()
        rec = torch.from_numpy(wl.receiver_plane(nx, ny, min(8, nz - 1), 4)).cuda()
        made.append((r, vel, rec))
    work = sum(r["grid"][0] * r["grid"][1] * r["grid"][2] * r["nsteps"] for r in reqs)
    out = {"requests": n_requests, "point_steps": work}
    torch.cuda.synchronize()
    # plain FP32, one shot after another; timed on the second of two passes,
    # since the first allocation of device memory in a process is slow (the
    # server's stream-ordered pool is likewise warm when it is timed)
    for rep in range(2):
        t0 = time.perf_counter()
        for r, vel, rec in made:
            s = gw.WaveSolver(r["grid"], (10.0, 10.0, 10.0),
                              0.5 * gw.wave_cfl_dt((10.0, 10.0, 10.0), float(vel.max())), vel)
            tr = torch.empty((r["nsteps"], rec.shape[0]), device="cuda")
            s.propagate((*r["source"], 15.0, -1.0, 1.0), r["nsteps"], rec, tr)
            s.synchronize()
            s.close()
        out["plain_f32_sequential_gpts"] = work / (time.perf_counter() - t0) / 1e9
    # served, then the same shots each with a 16-cell CPML layer
    for name, npml in (("f32", 0), ("f16", 0), ("f32", 16), ("f16", 16)):
        srv = gw.ShotServer(wl.SERVE_STREAM["budget_bytes"], 64)
        trs = []
        t0 = time.perf_counter()
        for r, vel, rec in made:
            tr = torch.empty((r["nsteps"], rec.shape[0]), device="cuda")
            trs.append((srv.submit(r["grid"], (10.0, 10.0, 10.0), vel,
                                   (*r["source"], 15.0, -1.0, 1.0), r["nsteps"], rec, tr,
                                   storage=STORAGE[name],
                                   cpml=(npml, 1e-3, 15.0) if npml else None), tr))
        ok = all(srv.wait(t)[0] == 0 for t, _ in trs)
        el = time.perf_counter() - t0
        srv.close()
        key = "served_%s_gpts" % name if not npml else "served_%s_npml%d_gpts" % (name, npml)
        out[key] = work / el / 1e9 if ok else None
    for name in ("f32", "f16"):
        if out["served_%s_npml16_gpts" % name] and out["served_%s_gpts" % name]:
            out["served_%s_npml16_vs_served" % name] = (out["served_%s_npml16_gpts" % name]
                                                        / out["served_%s_gpts" % name])
    out["served_f32_vs_plain_f32"] = out["served_f32_gpts"] / out["plain_f32_sequential_gpts"]
    out["served_f16_vs_plain_f32"] = out["served_f16_gpts"] / out["plain_f32_sequential_gpts"]
    return out


def gradient_workload(gw, torch, cfg=wl.CFG_GRAD, npml=0):
    """L2 trace misfit gradient d/d(v^2): true model = layers + Gaussian
    300 m/s anomaly, start = smoothed truth, 256^3, 800 steps, checkpoint
    every 40 steps. Observed traces come from a forward run of the true model
    (not timed); the timed region is one wave_gradient call (forward with
    checkpoints, residual and FP64 misfit, segment recomputes, adjoint,
    FP64 time sums). npml > 0: the same with the CPML layer at all faces
    (R = 1e-3, f_cps = f_peak) in both runs."""
    nx, ny, nz = cfg["shape"]
    true = wl.anomaly_model(nx, ny, nz, seed=cfg["seed"], anomaly=cfg["anomaly_mps"])
    start = wl.smoothed_start(true)
    rec = torch.from_numpy(wl.receiver_plane(nx, ny, cfg["rec_z"], cfg["rec_stride"])).cuda()
    shot = (nx // 2, ny // 2, 10, cfg["f_peak"], -1.0, 1.0)
    n = cfg["nsteps"]
    dt = 0.5 * gw.wave_cfl_dt(cfg["spacing"], max(float(true.max()), float(start.max())))
    obs = torch.zeros((n, rec.shape[0]), device="cuda")
    st = gw.WaveSolver((nx, ny, nz), cfg["spacing"], dt, torch.from_numpy(true).cuda())
    if npml:
        st.set_cpml(npml, 1e-3, cfg["f_peak"])
    st.propagate(shot, n, rec, obs)
    st.close()
    s = gw.WaveSolver((nx, ny, nz), cfg["spacing"], dt, torch.from_numpy(start).cuda())
    if npml:
        s.set_cpml(npml, 1e-3, cfg["f_peak"])
    g = torch.empty((nz, ny, nx), device="cuda")
    # forward alone, for the cost ratio
    tr = torch.empty_like(obs)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s.propagate(shot, n, rec, tr)
    s.synchronize()
    t_fwd = time.perf_counter() - t0
    s.reset()
    t0 = time.perf_counter()
    misfit = s.gradient(shot, n, rec, obs, g, ckpt_every=cfg["ckpt_every"])
    t_grad = time.perf_counter() - t0
    s.close()
    pts = nx * ny * nz * n
    name = "%s, %d steps, checkpoint every %d" % (cfg["name"], n, cfg["ckpt_every"])
    if npml:
        name += ", CPML layer of %d cells" % npml
    return {"workload": name,
            "seconds": t_grad, "forward_seconds": t_fwd, "cost_vs_forward": t_grad / t_fwd,
            "gpts_model_steps": pts / t_grad / 1e9, "misfit": misfit,
            "grad_finite": bool(torch.isfinite(g).all().item()),
            "grad_max_abs": float(g.abs().max().item()),
            "device_memory_fields": 2 * ((n + cfg["ckpt_every"] - 1) // cfg["ckpt_every"])
            + 2 * cfg["ckpt_every"] + 6}


def cpml_gradient_bytes_per_step(shape, npml):
    """Algorithmic DRAM bytes per model step of the gradient with the CPML
    layer: the plain gradient's 72 B per point, plus per axis and per line
    along it: the forward's layer pass (cpml_bytes_per_step's line term), the
    recompute's, which also reads and writes D at the 2 w segment points
    (+8 B), and the adjoint's: p^{k+1} and C read and p^k read and written at
    the segment points (16 B), nu and mu read and written at the slab cells
    (16 B)."""
    nx, ny, nz = shape
    npts = nx * ny * nz
    w = npml + 4
    lines = npts / nx + npts / ny + npts / nz
    fwd = 16 * (2 * w + 2 * npml)
    return 72 * npts + (2 * fwd + 8 * 2 * w + 16 * (2 * w + 2 * npml)) * lines


def cpml_bytes_per_step(shape, npml, esize=4):
    """Algorithmic DRAM bytes of one step with the CPML layer: the sweep's
    16 B per point (10 with 16-bit fields, esize 2), plus per axis a and per
    line along a, at the 2 w = 2 (npml + 4) segment points u^n, C and
    u^{n+1} read and u^{n+1} written (16 B; 10 with 16-bit fields) and at the
    2 npml slab cells psi and zeta read and written (16 B, FP32)."""
    nx, ny, nz = shape
    npts = nx * ny * nz
    w = npml + 4
    lines = npts / nx + npts / ny + npts / nz
    per_pt = 3 * esize + 4
    return per_pt * npts + (per_pt * 2 * w + 16 * 2 * npml) * lines


def cpml_workload(gw, torch, cfg, vel_d, dt, steps, peak_gbs, plain_ms):
    """The same grid and model stepped with the CPML layer at all six faces
    (npml 8 and 16 with FP32 fields, npml 16 with FP16 fields; R = 1e-3,
    f_cps = f_peak); source and receiver plane moved below the top layer."""
    nx, ny, nz = cfg["shape"]
    npts = nx * ny * nz
    out = {}
    for npml, storage in ((8, 0), (16, 0), (16, 2)):
        rec = torch.from_numpy(wl.receiver_plane(nx, ny, npml + 8, cfg["rec_stride"])).cuda()
        shot = (cfg["source"][0], cfg["source"][1], npml + 10, cfg["f_peak"], -1.0, 1.0)
        s = gw.WaveSolver((nx, ny, nz), cfg["spacing"], dt, vel_d, storage=storage)
        s.set_cpml(npml, 1e-3, cfg["f_peak"])
        tr = torch.empty((steps, rec.shape[0]), device="cuda")
        s.propagate(shot, min(steps, 64), rec, tr)
        s.reset()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        s.propagate(shot, steps, rec, tr)
        e1.record()
        e1.synchronize()
        s.synchronize()
        ms = e0.elapsed_time(e1) / steps
        ok = bool(torch.isfinite(tr).all().item())
        s.close()
        b = cpml_bytes_per_step((nx, ny, nz), npml, 2 if storage else 4)
        ach = b / (ms * 1e-3) / 1e9
        out["npml%d%s" % (npml, "_f16" if storage else "")] = {
            "value": npts / (ms * 1e-3) / 1e9, "unit": "Gpts/s", "ms_per_step": ms,
            "steps": steps, ("vs_plain_f32_step" if storage else "vs_plain_step"): ms / plain_ms,
            "storage": "f16" if storage else "f32", "traces_finite": ok,
            "roofline": {"bound": "hbm", "achieved": ach, "peak": peak_gbs,
                         "unit": "GB/s", "frac": ach / peak_gbs,
                         "algorithmic_bytes_per_step": b,
                         "launches_per_step": "sweep + 3 axis kernels + shell receivers"}}
    return out


def run_reference(args, cfg):
    """The reference arm: the FP64 CPU oracle on this machine's host cores."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    nx, ny, nz = cfg["shape"]
    vel = wl.velocity_for(cfg)
    sp = cfg["spacing"]
    dt = cfg["cfl_fraction"] * oracle.cfl_dt(sp, float(vel.max()))
    total_budget = 150.0
    per_step = total_budget / max(1, args.steps + args.warmup)
    # size a slab so one oracle step takes about per_step seconds
    planes = 1
    rng = np.random.default_rng(5)
    u = rng.uniform(-1, 1, size=(planes, ny, nx))
    t = time.perf_counter()
    oracle.propagate(vel[:1], sp, dt, 1, u=u, u_prev=u)
    one = time.perf_counter() - t
    planes = int(max(1, min(nz, per_step / max(one, 1e-6))))
    sl = vel[:planes]
    u = rng.uniform(-1, 1, size=sl.shape)
    up = rng.uniform(-1, 1, size=sl.shape)
    src = (*cfg["source"], cfg["f_peak"], -1.0, 1.0) if cfg["source"][2] < planes else None
    for _ in range(args.warmup):
        u, up, _ = oracle.propagate(sl, sp, dt, 1, u=u, u_prev=up, source=src)
    t = time.perf_counter()
    for _ in range(args.steps):
        u, up, _ = oracle.propagate(sl, sp, dt, 1, u=u, u_prev=up, source=src)
    el = time.perf_counter() - t
    pts = nx * ny * planes
    value = pts * args.steps / el / 1e9
    sample = "%dx%dx%d slab of the workload per step" % (nx, ny, planes)
    cores = oracle.threads_used()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "Gpts/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": el / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": cfg["name"], "grid": list(cfg["shape"]),
                   "sample": sample},
        "cpu_baseline": {"value": value, "unit": "Gpts/s", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "Gpts/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_case(args):
    """Small fixed cases for profiler captures (no bench line): each runs one
    piece of the path on the bench's synthetic inputs and prints one line.
    sweep      --workload W --storage S --steps K [--variant V] [--npml P]: one
               context (with a CPML layer of P cells), K steps of
               wave_propagate (the captured launches are its sweeps)
    gradient   --steps K [--npml P]: the 256^3 gradient workload's start model
               with a layer of P cells, one wave_gradient call of K steps,
               checkpoint every 40 (observed traces zero)
    serve_cpml --serve-requests N: the first N requests of the serving stream
               at once, each with a 16-cell layer and at most 64 steps"""
    import torch
    import paper_2404_04441_gb300 as gw
    gw.load()
    if args.case == "sweep":
        cfg = WORKLOADS[args.workload]
        nx, ny, nz = cfg["shape"]
        vel = wl.velocity_for(cfg)
        dt = cfg["cfl_fraction"] * gw.wave_cfl_dt(cfg["spacing"], float(vel.max()))
        s = gw.WaveSolver((nx, ny, nz), cfg["spacing"], dt, torch.from_numpy(vel).cuda(),
                          storage=args.storage)
        if args.npml:
            s.set_cpml(args.npml, 1e-3, cfg["f_peak"])
        rec = torch.from_numpy(wl.receiver_plane(nx, ny, cfg["rec_z"], cfg["rec_stride"])).cuda()
        tr = torch.empty((args.steps, rec.shape[0]), device="cuda")
        s.propagate((*cfg["source"], cfg["f_peak"], -1.0, 1.0), args.steps, rec, tr)
        s.synchronize()
        out = {"case": "sweep", "workload": cfg["name"], "storage": args.storage,
               "npml": args.npml, "steps": args.steps, "launch": s.launch_info(),
               "finite": bool(torch.isfinite(tr).all().item())}
        s.close()
    elif args.case == "gradient":
        cfg = wl.CFG_GRAD
        nx, ny, nz = cfg["shape"]
        true = wl.anomaly_model(nx, ny, nz, seed=cfg["seed"], anomaly=cfg["anomaly_mps"])
        start = wl.smoothed_start(true)
        rec = torch.from_numpy(wl.receiver_plane(nx, ny, cfg["rec_z"], cfg["rec_stride"])).cuda()
        shot = (nx // 2, ny // 2, 10, cfg["f_peak"], -1.0, 1.0)
        dt = 0.5 * gw.wave_cfl_dt(cfg["spacing"], max(float(true.max()), float(start.max())))
        obs = torch.zeros((args.steps, rec.shape[0]), device="cuda")
        s = gw.WaveSolver((nx, ny, nz), cfg["spacing"], dt, torch.from_numpy(start).cuda())
        if args.npml:
            s.set_cpml(args.npml, 1e-3, cfg["f_peak"])
        g = torch.empty((nz, ny, nx), device="cuda")
        mis = s.gradient(shot, args.steps, rec, obs, g, ckpt_every=cfg["ckpt_every"])
        s.close()
        out = {"case": "gradient", "steps": args.steps, "npml": args.npml, "misfit": mis,
               "finite": bool(torch.isfinite(g).all().item())}
    else:
        reqs = wl.serving_requests(**dict(wl.SERVE_STREAM, n=args.serve_requests))
        srv = gw.ShotServer(wl.SERVE_STREAM["budget_bytes"], 64)
        tickets = []
        for r in reqs:
            nx, ny, nz = r["grid"]
            vz = torch.from_numpy(wl.layered_profile(nz, r["vel_seed"])).cuda()
            vel = vz[:, None, None].expand(nz, ny, nx).contiguous()
            rec = torch.from_numpy(wl.receiver_plane(
                nx, ny, min(wl.SERVE_STREAM["rec_z"], nz - 1),
                wl.SERVE_STREAM["rec_stride"])).cuda()
            n = min(r["nsteps"], 64)
            tr = torch.empty((n, rec.shape[0]), device="cuda")
            tickets.append((srv.submit(r["grid"], (10.0, 10.0, 10.0), vel,
                                       (*r["source"], 15.0, -1.0, 1.0), n, rec, tr,
                                       cpml=16), vel, rec, tr))
        status = [srv.wait(t)[0] for t, *_ in tickets]
        srv.close()
        out = {"case": "serve_cpml", "requests": len(reqs), "failed": sum(x != 0 for x in status)}
    print(json.dumps(out), flush=True)
    return 0 if out.get("finite", True) and not out.get("failed") else 1


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="1024x1024x512", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--variant", type=int, default=None, help="sweep kernel variant (tuning)")
    ap.add_argument("--no-precision", action="store_true",
                    help="skip the BF16/FP16 storage measurements")
    ap.add_argument("--no-serve", action="store_true",
                    help="skip the shot-serving stream")
    ap.add_argument("--serve-requests", type=int, default=wl.SERVE_STREAM["n"])
    ap.add_argument("--no-gradient", action="store_true",
                    help="skip the adjoint-gradient workload")
    ap.add_argument("--no-cpml", action="store_true",
                    help="skip the CPML absorbing-layer measurement")
    ap.add_argument("--case", default=None, choices=["sweep", "gradient", "serve_cpml"],
                    help="run one small case for a profiler capture instead of the bench")
    ap.add_argument("--storage", type=int, default=0, help="--case sweep: 0 FP32, 1 BF16, 2 FP16")
    ap.add_argument("--npml", type=int, default=0, help="--case sweep, gradient: layer width")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.case is not None:
        if args.variant is not None:
            os.environ["GBWAVE_VARIANT"] = str(args.variant)
        return run_case(args)
    cfg = WORKLOADS[args.workload]
    if args.impl == "reference":
        return run_reference(args, cfg)
    if args.variant is not None:
        os.environ["GBWAVE_VARIANT"] = str(args.variant)

    import torch
    import paper_2404_04441_gb300 as gw

    rank, world, local = dist_env()
    if not torch.cuda.is_available():
        raise RuntimeError("bench.py needs a CUDA device")
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    gw.load()

    nx, ny, nz = cfg["shape"]
    npts = nx * ny * nz
    sp = cfg["spacing"]
    vel = wl.velocity_for(cfg)
    dt = cfg["cfl_fraction"] * gw.wave_cfl_dt(sp, float(vel.max()))
    rec = wl.receiver_plane(nx, ny, cfg["rec_z"], cfg["rec_stride"])
    nrec = rec.shape[0]
    shot = (*cfg["source"], cfg["f_peak"], -1.0, 1.0)
    K, W = args.steps, args.warmup

    stream = torch.cuda.current_stream()
    vel_d = torch.from_numpy(vel).cuda()
    rec_d = torch.from_numpy(rec).cuda()
    traces_d = torch.empty((max(K, W), nrec), dtype=torch.float32, device="cuda")
    solver = gw.WaveSolver((nx, ny, nz), sp, dt, vel_d, stream=stream.cuda_stream)
    info = solver.launch_info()

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    # ---- device-resident timing -------------------------------------------------
    solver.propagate(shot, W, rec_d, traces_d)
    solver.synchronize()
    solver.reset()
    sampler = ClockSampler(local)
    sampler.start()
    barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    tw0 = time.time()
    ev0.record(stream)
    solver.propagate(shot, K, rec_d, traces_d)
    ev1.record(stream)
    ev1.synchronize()
    tw1 = time.time()
    barrier()
    torch.cuda.synchronize()
    sampler.stop()
    solver.synchronize()
    ms = replica_max(ev0.elapsed_time(ev1), "cuda")
    clocks = sampler.summary(tw0, tw1)
    value = replica_value(npts, K, ms * 1e-3, world)
    # graph chunks of GRAPH_STEPS sweeps + a step-counter node, the remainder
    # as direct sweeps + one counter kernel, the receiver table's four build
    # kernels and the final check of the traces
    launches = (K // GRAPH_STEPS) * (GRAPH_STEPS + 1) + \
        ((K % GRAPH_STEPS) + 1 if K % GRAPH_STEPS else 0) + (5 if nrec else 0)
    tr_ok = bool(torch.isfinite(traces_d[:K]).all().item())
    solver.close()
    del traces_d

    # ---- end to end through the C ABI with host buffers -------------------------
    e2e = None
    if not args.no_e2e:
        vel_h = torch.from_numpy(vel).pin_memory()
        rec_h = torch.from_numpy(rec).pin_memory()
        tr_h = torch.empty((K, nrec), dtype=torch.float32).pin_memory()
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s2 = gw.WaveSolver((nx, ny, nz), sp, dt, vel_h, stream=stream.cuda_stream,
                           defer=True)
        t1 = time.perf_counter()
        s2.propagate(shot, K, rec_h, tr_h)  # host traces: returns after the D2H copy
        t2 = time.perf_counter()
        s2.close()
        torch.cuda.synchronize()
        t3 = time.perf_counter()
        el = replica_max(t3 - t0, "cuda")
        e2e = {"value": replica_value(npts, K, el, world), "unit": "Gpts/s",
               "h2d_bytes_per_step": (vel.nbytes + rec.nbytes) / K,
               "d2h_bytes_per_step": nrec * 4,
               "split_ms": {"create": (t1 - t0) * 1e3, "propagate": (t2 - t1) * 1e3,
                            "destroy": (t3 - t2) * 1e3},
               "note": "wave_create_async(pinned host velocity: its upload overlaps the "
                       "first steps) + wave_propagate(host receivers, host traces) + "
                       "wave_destroy, all K steps"}

    # ---- roofline of the sweep kernel -------------------------------------------
    peaks, peak_kind = measured_peaks()
    per_launch_s = ms * 1e-3 / K
    achieved = BYTES_PER_POINT * npts / per_launch_s / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"], "traffic": read_traffic(cfg["name"]),
                "peak_kind": peak_kind + " (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured"
                else "fallback",
                "algorithmic_bytes_per_launch": BYTES_PER_POINT * npts,
                "kernel": "wave_sweep_kernel"}

    # ---- 16-bit storage forms: same workload and K; error on 128^3 x 500 ---
    precision = None
    # The storage forms, serving, gradient and CPML lines are single-GPU
    # measurements beside the headline; with N replicas only the headline
    # (and its e2e) is run, so the GPUs are held for the scaling line alone.
    side = world == 1
    if side and not args.no_precision:
        precision = {}
        for name in ("bf16", "f16"):
            s16 = gw.WaveSolver((nx, ny, nz), sp, dt, vel_d, storage=STORAGE[name],
                                stream=stream.cuda_stream)
            tr16 = torch.empty((max(K, W), nrec), dtype=torch.float32, device="cuda")
            s16.propagate(shot, W, rec_d, tr16)
            s16.reset()
            barrier()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            s16.propagate(shot, K, rec_d, tr16)
            e1.record(stream)
            e1.synchronize()
            s16.synchronize()
            ms16 = replica_max(e0.elapsed_time(e1), "cuda")
            s16.close()
            del tr16
            v16 = replica_value(npts, K, ms16 * 1e-3, world)
            ach = BYTES_PER_POINT_16 * npts / (ms16 * 1e-3 / K) / 1e9
            precision[name] = {"value": v16, "unit": "Gpts/s", "ms_per_step": ms16 / K,
                               "vs_f32": v16 / value,
                               "roofline": {"bound": "hbm", "achieved": ach,
                                            "peak": peaks["hbm_gbs"], "unit": "GB/s",
                                            "frac": ach / peaks["hbm_gbs"],
                                            "traffic": read_traffic(cfg["name"], TRAFFIC_FILE_16,
                                                                    name + ":"),
                                            "algorithmic_bytes_per_point": BYTES_PER_POINT_16}}
        if rank == 0:
            err = precision_errors(gw, torch)
            for name in ("bf16", "f16"):
                precision[name]["error_vs_fp64_oracle"] = err[name]
            precision["f32_error_vs_fp64_oracle"] = err["f32"]

    # ---- shot serving: continuous batching of a Poisson request stream -------
    serving = None
    if side and not args.no_serve:
        serving = {name: serve_stream(gw, torch, STORAGE[name], args.serve_requests)
                   for name in ("f32", "f16")}
        # HBM roofline of the engine's busy time: the batched step moves the
        # single-grid kernel's algorithmic bytes per point-step.
        for name, bpp in (("f32", BYTES_PER_POINT), ("f16", BYTES_PER_POINT_16)):
            ach = serving[name]["gpts_busy"] * bpp
            serving[name]["roofline_busy"] = {
                "bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": ach / peaks["hbm_gbs"], "algorithmic_bytes_per_point": bpp}
        serving["saturated_mix"] = serve_saturated(gw, torch)

    gradient = None
    if side and not args.no_gradient:
        gradient = gradient_workload(gw, torch)
        # 72 B per model-point-step: forward 16, recompute storing D 20, adjoint
        # with injection, D read and the FP64 time sum 36.
        ach = 72.0 * gradient["gpts_model_steps"]
        gradient["roofline"] = {"bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"],
                                "unit": "GB/s", "frac": ach / peaks["hbm_gbs"],
                                "algorithmic_bytes_per_model_point_step": 72}
        if not args.no_cpml:
            npml = 16
            gl = gradient_workload(gw, torch, npml=npml)
            b = cpml_gradient_bytes_per_step(wl.CFG_GRAD["shape"], npml)
            gsteps = wl.CFG_GRAD["nsteps"] / gl["seconds"]
            ach = b * gsteps / 1e9
            gradient["cpml_npml%d" % npml] = {
                "workload": gl["workload"], "seconds": gl["seconds"],
                "vs_plain_gradient": gl["seconds"] / gradient["seconds"],
                "cost_vs_forward": gl["cost_vs_forward"], "misfit": gl["misfit"],
                "grad_finite": gl["grad_finite"],
                "roofline": {"bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"],
                             "unit": "GB/s", "frac": ach / peaks["hbm_gbs"],
                             "algorithmic_bytes_per_model_step": b}}

    cpml = None
    if side and not args.no_cpml:
        cpml = cpml_workload(gw, torch, cfg, vel_d, dt, min(K, 200), peaks["hbm_gbs"], ms / K)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        g, cores, sample, el = oracle_sample(vel, cfg, dt, budget_s=15.0)
        cpu = {"value": g, "unit": "Gpts/s", "cores": cores, "kind": "oracle",
               "sample": sample, "seconds": round(el, 2)}

    if world > 1:
        torch.distributed.barrier()
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "Gpts/s", "n_gpus": world,
            "steps": K, "warmup": W, "ms_per_step": ms / K, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": cfg["name"], "grid": [nx, ny, nz], "spacing_m": list(sp),
                       "dt_s": dt, "nsteps_timed": K, "receivers": nrec,
                       "source": list(cfg["source"]), "f_peak_hz": cfg["f_peak"],
                       "parallelism": "replicas" if world > 1 else "single",
                       "l2": "inputs larger than L2 (16 B/pt x %d pts = %.2f GB per step)"
                             % (npts, BYTES_PER_POINT * npts / 1e9),
                       "launch": info},
            "e2e": e2e, "gpu_launches": launches, "roofline": roofline,
            "cpu_baseline": cpu, "clocks": clocks, "traces_finite": tr_ok,
            "precision_forms": precision, "serving": serving, "gradient": gradient,
            "cpml": cpml,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
