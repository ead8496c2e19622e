// Shot server (declared in include/wave_serve.h): requests queue on the
// host, an engine thread admits them by device-memory budget and free slots,
// advances every resident shot by one step per batched launch, and completes
// shots as they reach their step counts.
#include <chrono>
#include <condition_variable>
#include <cstdlib>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>

#include "../../include/wave_serve.h"
#include "common.cuh"
#include "cpml.cuh"
#include "sweep.cuh"

using namespace gbw;

namespace {

// One kernel configuration per storage type (index = WAVE_STORAGE_*), the
// single-grid defaults: FP32 32 x 16 tiles of 4 warps, 16-bit on the tensor
// cores with 64 x 16 tiles of 8 warps.
using ServeF32 = SweepCfg<32, 16, 1, 4, 4>;
using ServeB16 = TcCfg<64, 4, 2, __nv_bfloat16, 9>;
using ServeH16 = TcCfg<64, 4, 2, __half, 9>;
constexpr int kKinds = 3;
constexpr int kMaxGroup = 16;     // batch steps between two engine checks
constexpr int kLayerPlanes = 256; // target z planes per CTA for batched shots
// Admission stops adding shots once one batched step would launch more than
// this many waves of CTAs (4 per SM): enough to keep the GPU full with small
// shots, few enough that each resident shot gets a large share of it. On the
// Poisson stream of shots it lowers p99 latency from 1.48 s to 1.22 s
// (FP32) and 1.38 s to 1.11 s (FP16) against admitting up to the slot
// limit, for about 5 % less throughput when many shots wait at once.
constexpr int kTargetWaves = 6;

struct Kind {
  int tx, ty, hx, esize, threads;
  int box_u, box_p;  // TMA box widths: u plane with halo, u_prev / c tiles
  size_t smem;
  const void *func;
  void (*launch)(int, cudaStream_t, const BatchShot *, int, long long,
                 const StencilCoefs &);
};

template <class C>
void launch_batch(int ctas, cudaStream_t st, const BatchShot *table, int n,
                  long long k, const StencilCoefs &co) {
  wave_sweep_batched_kernel<C><<<ctas, C::THREADS, C::SMEM_BYTES, st>>>(
      table, n, k, co);
}

// Resident shots of one storage type and one grid spacing: one launch.
struct Group {
  int kind, first, count, ctas;
  StencilCoefs co;
};

template <class C>
Kind make_kind() {
  return Kind{C::TX,
              C::TY,
              C::HX,
              (int)sizeof(typename C::T),
              C::THREADS,
              C::BOX_U,
              C::BOX_P,
              C::SMEM_BYTES,
              reinterpret_cast<const void *>(&wave_sweep_batched_kernel<C>),
              &launch_batch<C>};
}

const Kind &kind_of(int storage) {
  static const Kind kinds[kKinds] = {make_kind<ServeF32>(), make_kind<ServeB16>(),
                                     make_kind<ServeH16>()};
  return kinds[storage];
}

size_t round_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

struct Request {
  uint64_t ticket = 0;
  wave_request r{};
  int status = WAVE_EBUSY;
  double t_submit = 0, t_start = -1, t_done = -1, dt = 0;
  int64_t steps_done = 0;
  size_t bytes = 0;
  // Resident state (engine thread only).
  void *buf[2] = {nullptr, nullptr};
  float *c = nullptr;
  StepDesc *desc = nullptr;
  float *wavelet = nullptr;
  int4 *rec = nullptr;
  int *rec_start = nullptr;
  float *stage = nullptr;  // device trace staging when traces are host memory
  bool host_traces = false;
  BatchShot shot{};
  int ctas = 0;
  double points = 0;
  // CPML layer (npml > 0): slabs, profiles, shell receivers, batch entry.
  void *layer_mem[13] = {};
  CpmlBatchShot layer{};
};

// Device bytes of a request's CPML layer: psi and zeta slabs of 2 npml cells
// per axis, the per-axis profiles b and a, and the shell receiver list.
size_t layer_bytes(const wave_request &r) {
  if (r.npml <= 0) return 0;
  const size_t nx = r.grid.nx, ny = r.grid.ny, nz = r.grid.nz, p = (size_t)r.npml;
  return 2 * 2 * p * (ny * nz + nz * nx + ny * nx) * 4 + 2 * (nx + ny + nz) * 4 +
         (size_t)r.nrec * sizeof(int4);
}

// Device bytes of a request once resident (the budget unit).
// z layers of a batched shot: at most kLayerPlanes planes each, equal sizes.
int request_layers(int nz) {
  return std::min(kMaxLayers, std::max(1, (nz + kLayerPlanes - 1) / kLayerPlanes));
}

// CTAs one batched step launches for the request.
int request_ctas(const wave_request &r) {
  const Kind &k = kind_of(r.storage);
  const int ntiles = ((r.grid.nx + k.tx - 1) / k.tx) * ((r.grid.ny + k.ty - 1) / k.ty);
  return ntiles * request_layers(r.grid.nz);
}

// The same in CTA places of 128 threads (an FP32 CTA; a 16-bit CTA of 8
// warps takes two), the unit of the admission's CTA target.
int request_places(const wave_request &r) {
  return request_ctas(r) * (kind_of(r.storage).threads / 128);
}

size_t request_bytes(const wave_request &r) {
  const Kind &k = kind_of(r.storage);
  const size_t nx = r.grid.nx, ny = r.grid.ny, nz = r.grid.nz;
  const size_t pxu = r.storage == WAVE_STORAGE_F32 ? round_up(nx, 4)
                                                   : round_up(nx, 8);
  const size_t ntiles = ((nx + k.tx - 1) / k.tx) * ((ny + k.ty - 1) / k.ty);
  size_t b = 2 * pxu * ny * nz * k.esize;          // wavefields
  b += round_up(nx, 4) * ny * nz * 4;               // v^2 dt^2
  b += sizeof(StepDesc) + (size_t)r.nsteps * 4;     // descriptor, wavelet
  b += (size_t)r.nrec * sizeof(int4) + (ntiles + 1) * 4;
  b += layer_bytes(r);
  return b;  // plus a staging buffer for host traces (added at submit)
}

}  // namespace

struct serve_ctx {
  size_t budget = 0;
  int max_slots = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  // Shots' device memory comes from a pool of the server's own that keeps
  // up to the budget mapped between shots: memory freed by a finished shot
  // serves the next admission without being returned to the driver and
  // mapped again (which cost ~18 ms per shot of the stream).
  cudaMemPool_t pool = nullptr;
  int sms = 1;
  int device = 0;
  std::chrono::steady_clock::time_point t0;
  std::mutex mu;
  std::condition_variable cv_engine, cv_done;
  std::deque<Request *> queue;
  std::unordered_map<uint64_t, std::unique_ptr<Request>> all;
  uint64_t next_ticket = 1;
  bool stopping = false;
  serve_stats_t st{};
  std::thread engine;
  // Engine thread only.
  std::vector<Request *> resident;
  size_t bytes = 0;
  long long ctas = 0;         // CTA places (128 threads) of one batched step
                              // over the resident shots
  long long target_ctas = 0;  // admission adds no shot beyond this (kTargetWaves)
  long long k = 0;  // batch steps taken
  BatchShot *d_table[kKinds] = {nullptr, nullptr, nullptr};
  std::vector<BatchShot> h_table[kKinds];
  // layered shots per storage type: batch table and blocks per axis launch
  CpmlBatchShot *d_layer[kKinds] = {nullptr, nullptr, nullptr};
  std::vector<CpmlBatchShot> h_layer[kKinds];
  int layer_blocks[kKinds][3] = {};
  int layer_rec_blocks[kKinds] = {1, 1, 1};  // record blocks per layered shot
  std::vector<Group> groups;
  bool dirty = true;
  void *d_scan = nullptr;     // 16 bytes: velocity max, invalid count
  long long fault_alloc = -1; // host fault injection: fail this allocation
  long long allocs = 0;

  double now() const {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0)
        .count();
  }
};

namespace {

int serve_alloc(serve_ctx *s, void **p, size_t bytes) {
  *p = nullptr;
  if (s->fault_alloc >= 0 && s->allocs++ == s->fault_alloc) return WAVE_ENOMEM;
  WAVE_TRY_CUDA(cudaMallocFromPoolAsync(p, std::max<size_t>(bytes, 256), s->pool, s->stream));
  return WAVE_OK;
}

void release(serve_ctx *s, Request *q) {
  void *ps[] = {q->buf[0], q->buf[1], q->c,        q->desc,
                q->wavelet, q->rec,   q->rec_start, q->stage};
  for (void *p : ps)
    if (p) cudaFreeAsync(p, s->stream);
  for (void *&p : q->layer_mem) {
    if (p) cudaFreeAsync(p, s->stream);
    p = nullptr;
  }
  q->buf[0] = q->buf[1] = nullptr;
  q->c = nullptr;
  q->desc = nullptr;
  q->wavelet = nullptr;
  q->rec = nullptr;
  q->rec_start = nullptr;
  q->stage = nullptr;
}

void finish(serve_ctx *s, Request *q, int status) {
  std::lock_guard<std::mutex> lk(s->mu);
  q->status = status;
  q->t_done = s->now();
  if (status == WAVE_OK)
    s->st.completed++;
  else
    s->st.failed++;
  s->cv_done.notify_all();
}

// The CPML layer of an admitted request: zeroed memory-variable slabs,
// profiles from the shot's largest velocity and time step (as
// wave_set_cpml), derivative weights, and the receivers within w of a face.
int admit_layer(serve_ctx *s, Request *q, float vmax, double dt,
                const std::vector<int32_t> &xyz) {
  const wave_request &r = q->r;
  cudaStream_t st = s->stream;
  const int nx = r.grid.nx, ny = r.grid.ny, nz = r.grid.nz, npml = r.npml;
  CpmlBatchShot &L = q->layer;
  L = CpmlBatchShot{};
  CpmlGeom &g = L.g;
  g.nx = nx;
  g.ny = ny;
  g.nz = nz;
  g.px = (int)round_up(nx, 4);
  g.pxu = r.storage == WAVE_STORAGE_F32 ? g.px : (int)round_up(nx, 8);
  g.npml = npml;
  g.w = npml + 4;
  const size_t sl[3] = {2ull * npml * ny * nz, 2ull * npml * nz * nx, 2ull * npml * ny * nx};
  const int dims[3] = {nx, ny, nz};
  const double hs[3] = {r.spacing.dx, r.spacing.dy, r.spacing.dz};
  int e, m = 0;
  for (int ax = 0; ax < 3; ++ax) {
    if ((e = serve_alloc(s, &q->layer_mem[m++], sl[ax] * 4)) ||
        (e = serve_alloc(s, &q->layer_mem[m++], sl[ax] * 4)) ||
        (e = serve_alloc(s, &q->layer_mem[m++], (size_t)dims[ax] * 4)) ||
        (e = serve_alloc(s, &q->layer_mem[m++], (size_t)dims[ax] * 4)))
      return e;
    g.psi[ax] = static_cast<float *>(q->layer_mem[m - 4]);
    g.zeta[ax] = static_cast<float *>(q->layer_mem[m - 3]);
    g.bprof[ax] = static_cast<float *>(q->layer_mem[m - 2]);
    g.aprof[ax] = static_cast<float *>(q->layer_mem[m - 1]);
    WAVE_TRY_CUDA(cudaMemsetAsync(g.psi[ax], 0, sl[ax] * 4, st));
    WAVE_TRY_CUDA(cudaMemsetAsync(g.zeta[ax], 0, sl[ax] * 4, st));
    std::vector<float> hb(dims[ax]), ha(dims[ax]);
    cpml_profile(dims[ax], npml, r.reflection, r.f_cps, (double)vmax, hs[ax], dt, hb.data(),
                 ha.data());
    const long long fstep[3] = {1, g.pxu, (long long)ny * g.pxu};
    const long long sstep[3] = {(long long)nz * ny, (long long)nz * nx, (long long)ny * nx};
    L.seg[ax] = cpml_seg_fits(npml, dims[ax], fstep[ax], sstep[ax]) ? npml : 0;
    if (L.seg[ax] == 16) cpml_side_prof(hb.data(), ha.data(), dims[ax], L.p16[ax]);
    if (L.seg[ax] == 8) cpml_side_prof(hb.data(), ha.data(), dims[ax], L.p8[ax]);
    WAVE_TRY_CUDA(cudaMemcpyAsync((void *)g.bprof[ax], hb.data(), dims[ax] * 4,
                                  cudaMemcpyHostToDevice, st));
    WAVE_TRY_CUDA(cudaMemcpyAsync((void *)g.aprof[ax], ha.data(), dims[ax] * 4,
                                  cudaMemcpyHostToDevice, st));
    cpml_axis_coefs(g, ax, hs[ax]);
  }
  // receivers within w of a face are re-recorded after the layer passes
  std::vector<int4> shell;
  for (int i = 0; i < r.nrec; ++i) {
    const int x = xyz[3 * i], y = xyz[3 * i + 1], z = xyz[3 * i + 2];
    if (x < g.w || x >= nx - g.w || y < g.w || y >= ny - g.w || z < g.w || z >= nz - g.w)
      shell.push_back(make_int4(x, y, z, i));
  }
  if ((e = serve_alloc(s, &q->layer_mem[m++], shell.size() * sizeof(int4)))) return e;
  if (!shell.empty())
    WAVE_TRY_CUDA(cudaMemcpyAsync(q->layer_mem[m - 1], shell.data(),
                                  shell.size() * sizeof(int4), cudaMemcpyHostToDevice, st));
  L.buf[0] = q->buf[0];
  L.buf[1] = q->buf[1];
  L.c = q->c;
  L.desc = q->desc;
  L.srec = static_cast<const int4 *>(q->layer_mem[m - 1]);
  L.nsrec = (int)shell.size();
  L.b0 = q->shot.b0;
  L.nsteps = r.nsteps;
  return WAVE_OK;
}

// Make a queued request resident: buffers, v^2 dt^2, tables, tensor maps.
int admit(serve_ctx *s, Request *q) {
  const wave_request &r = q->r;
  const Kind &kd = kind_of(r.storage);
  cudaStream_t st = s->stream;
  const int nx = r.grid.nx, ny = r.grid.ny, nz = r.grid.nz;
  const int px = (int)round_up(nx, 4);
  const int pxu = r.storage == WAVE_STORAGE_F32 ? px : (int)round_up(nx, 8);
  const int ntx = (nx + kd.tx - 1) / kd.tx, nty = (ny + kd.ty - 1) / kd.ty;
  const int ntiles = ntx * nty;
  const size_t fbytes = (size_t)pxu * ny * nz * kd.esize;
  const size_t cbytes = (size_t)px * ny * nz * 4;
  int e;
  if ((e = serve_alloc(s, &q->buf[0], fbytes)) ||
      (e = serve_alloc(s, &q->buf[1], fbytes)) ||
      (e = serve_alloc(s, (void **)&q->c, cbytes)) ||
      (e = serve_alloc(s, (void **)&q->desc, sizeof(StepDesc))) ||
      (e = serve_alloc(s, (void **)&q->wavelet, (size_t)r.nsteps * 4)) ||
      (e = serve_alloc(s, (void **)&q->rec, (size_t)r.nrec * sizeof(int4))) ||
      (e = serve_alloc(s, (void **)&q->rec_start, (size_t)(ntiles + 1) * 4)))
    return e;
  q->host_traces = r.nrec > 0 && !is_device_ptr(r.traces);
  if (q->host_traces &&
      (e = serve_alloc(s, (void **)&q->stage, (size_t)r.nsteps * r.nrec * 4)))
    return e;
  WAVE_TRY_CUDA(cudaMemsetAsync(q->buf[0], 0, fbytes, st));
  WAVE_TRY_CUDA(cudaMemsetAsync(q->buf[1], 0, fbytes, st));
  WAVE_TRY_CUDA(cudaMemsetAsync(q->c, 0, cbytes, st));

  // Velocity: validate, then v^2 dt^2.
  WAVE_TRY_CUDA(cudaMemcpy2DAsync(q->c, (size_t)px * 4, r.velocity,
                                  (size_t)nx * 4, (size_t)nx * 4,
                                  (size_t)ny * nz, cudaMemcpyDefault, st));
  WAVE_TRY_CUDA(cudaMemsetAsync(s->d_scan, 0, 16, st));
  int sms = 0;
  WAVE_TRY_CUDA(
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->device));
  scan_velocity_kernel<<<sms * 4, 256, 0, st>>>(
      q->c, nx, px, (long long)ny * nz, reinterpret_cast<unsigned *>(s->d_scan),
      reinterpret_cast<unsigned long long *>((char *)s->d_scan + 8));
  WAVE_TRY_CUDA(cudaGetLastError());
  unsigned char res[16];
  WAVE_TRY_CUDA(cudaMemcpyAsync(res, s->d_scan, 16, cudaMemcpyDeviceToHost, st));
  WAVE_TRY_CUDA(cudaStreamSynchronize(st));
  unsigned vb;
  unsigned long long bad;
  std::memcpy(&vb, res, 4);
  std::memcpy(&bad, res + 8, 8);
  if (bad) return WAVE_EINVAL;
  float vmax;
  std::memcpy(&vmax, &vb, 4);
  const double lim = wave_cfl_dt(&r.spacing, (double)vmax);
  const double dt = r.dt > 0 ? r.dt : 0.5 * lim;
  if (!(dt <= lim * (1.0 + 1e-12))) return WAVE_EUNSTABLE;
  q->dt = dt;
  launch_velocity_to_c(q->c, (long long)px * ny * nz, dt * dt, sms, st);
  WAVE_TRY_CUDA(cudaGetLastError());

  // Receivers and source wavelet.
  std::vector<int32_t> xyz((size_t)r.nrec * 3);
  if (r.nrec > 0) {
    WAVE_TRY_CUDA(cudaMemcpy(xyz.data(), r.rec_xyz, xyz.size() * 4,
                             cudaMemcpyDefault));
  }
  std::vector<int4> entries;
  std::vector<int> starts;
  if ((e = build_receiver_table(xyz.data(), r.nrec, nx, ny, nz, kd.tx, kd.ty,
                                ntx, ntiles, entries, starts)))
    return e;
  std::vector<float> wl(r.nsteps);
  const double t0 = r.shot.t0 < 0 ? 1.0 / r.shot.f_peak : r.shot.t0;
  for (int n = 0; n < r.nsteps; ++n)
    wl[n] = (float)ricker(n * dt, r.shot.f_peak, t0, r.shot.amp);
  if (r.nrec > 0)
    WAVE_TRY_CUDA(cudaMemcpyAsync(q->rec, entries.data(),
                                  entries.size() * sizeof(int4),
                                  cudaMemcpyHostToDevice, st));
  WAVE_TRY_CUDA(cudaMemcpyAsync(q->rec_start, starts.data(), starts.size() * 4,
                                cudaMemcpyHostToDevice, st));
  WAVE_TRY_CUDA(cudaMemcpyAsync(q->wavelet, wl.data(), wl.size() * 4,
                                cudaMemcpyHostToDevice, st));
  StepDesc d{};
  d.wavelet = q->wavelet;
  d.traces = q->host_traces ? q->stage : r.traces;
  d.rec = q->rec;
  d.rec_start = q->rec_start;
  d.nrec = r.nrec;
  d.src_active = 1;
  d.sx = r.shot.sx;
  d.sy = r.shot.sy;
  d.sz = r.shot.sz;
  WAVE_TRY_CUDA(
      cudaMemcpyAsync(q->desc, &d, sizeof(d), cudaMemcpyHostToDevice, st));

  // Batch entry: tensor maps for both buffer parities, arguments.
  BatchShot &b = q->shot;
  std::memset(&b, 0, sizeof(b));
  const CUtensorMapDataType dtf = field_dtype(r.storage);
  for (int i = 0; i < 2; ++i) {
    if ((e = encode_map(&b.halo[i], q->buf[i], nx, ny, nz, pxu, kd.esize, dtf,
                        kd.box_u, kd.ty + 2 * kR)))
      return e;
    if ((e = encode_map(&b.tile[i], q->buf[i], nx, ny, nz, pxu, kd.esize, dtf,
                        kd.box_p, kd.ty)))
      return e;
  }
  if ((e = encode_map(&b.cmap, q->c, nx, ny, nz, px, 4,
                      CU_TENSOR_MAP_DATA_TYPE_FLOAT32, kd.box_p, kd.ty)))
    return e;
  SweepArgs &a = b.args;
  a.nx = nx;
  a.ny = ny;
  a.nz = nz;
  a.px = pxu;
  const int nl = request_layers(nz);
  const int zc = (nz + nl - 1) / nl;
  std::vector<int> layers;
  for (int z = 0; z < nz; z += zc) layers.push_back(std::min(zc, nz - z));
  set_layers(a, layers);
  a.ntx = ntx;
  a.k = make_coefs(r.spacing.dx, r.spacing.dy, r.spacing.dz);
  a.desc = q->desc;
  a.cmax = (float)((double)vmax * vmax * dt * dt);
  b.buf[0] = q->buf[0];
  b.buf[1] = q->buf[1];
  b.b0 = s->k;
  b.nsteps = r.nsteps;
  b.ntx = ntx;
  b.nty = nty;
  q->ctas = ntiles * (int)layers.size();
  q->points = (double)nx * ny * nz;
  if (r.npml > 0 && (e = admit_layer(s, q, vmax, dt, xyz))) return e;
  return WAVE_OK;
}

// Order the resident shots by (storage, spacing), cut them into launch
// groups and upload the batch tables.
int upload_tables(serve_ctx *s) {
  s->groups.clear();
  for (int kd = 0; kd < kKinds; ++kd) {
    std::vector<Request *> shots;
    for (Request *q : s->resident)
      if (q->r.storage == kd) shots.push_back(q);
    // Group by coefficients; within a group, shots with longer z layers
    // first. A shot's CTAs all stream one layer length, so this hands the
    // block scheduler the longest CTAs first and shortens the partial last
    // wave of each batched step.
    std::stable_sort(shots.begin(), shots.end(), [](Request *x, Request *y) {
      const int c = std::memcmp(&x->shot.args.k, &y->shot.args.k, sizeof(StencilCoefs));
      if (c != 0) return c < 0;
      return x->shot.args.zl[1] - x->shot.args.zl[0] > y->shot.args.zl[1] - y->shot.args.zl[0];
    });
    auto &t = s->h_table[kd];
    t.clear();
    for (Request *q : shots) {
      const bool same = !s->groups.empty() && s->groups.back().kind == kd &&
                        std::memcmp(&s->groups.back().co, &q->shot.args.k,
                                    sizeof(StencilCoefs)) == 0;
      if (!same) s->groups.push_back(Group{kd, (int)t.size(), 0, 0, q->shot.args.k});
      Group &g = s->groups.back();
      q->shot.cta_begin = g.ctas;
      g.ctas += q->ctas;
      g.count++;
      t.push_back(q->shot);
    }
    if (!t.empty())
      WAVE_TRY_CUDA(cudaMemcpyAsync(s->d_table[kd], t.data(),
                                    t.size() * sizeof(BatchShot),
                                    cudaMemcpyHostToDevice, s->stream));
    // the layered shots of this storage type: blocks of each axis launch
    auto &lt = s->h_layer[kd];
    lt.clear();
    int *nb = s->layer_blocks[kd];
    nb[0] = nb[1] = nb[2] = 0;
    int max_srec = 0;
    for (Request *q : shots) {
      if (q->r.npml <= 0) continue;
      CpmlBatchShot L = q->layer;
      max_srec = std::max(max_srec, L.nsrec);
      const int nx = q->r.grid.nx, ny = q->r.grid.ny, nz = q->r.grid.nz;
      const int rows[3] = {nz, nz, ny}, across[3] = {ny, nx, nx};
      for (int ax = 0; ax < 3; ++ax) {  // the segment form: a block set per face
        L.blk_begin[ax] = nb[ax];
        nb[ax] += rows[ax] * ((across[ax] + 127) / 128) * (L.seg[ax] ? 2 : 1);
      }
      lt.push_back(L);
    }
    // about 256 shell receivers per record block, at most 64 blocks a shot
    s->layer_rec_blocks[kd] = std::min(64, std::max(1, (max_srec + 255) / 256));
    if (!lt.empty())
      WAVE_TRY_CUDA(cudaMemcpyAsync(s->d_layer[kd], lt.data(), lt.size() * sizeof(CpmlBatchShot),
                                    cudaMemcpyHostToDevice, s->stream));
  }
  s->dirty = false;
  return WAVE_OK;
}

// The layer passes and shell receivers of batch step k over the layered
// shots of storage type kd.
template <class T>
void launch_layers(serve_ctx *s, int kd, long long k) {
  const CpmlBatchShot *t = s->d_layer[kd];
  const int n = (int)s->h_layer[kd].size();
  const int *nb = s->layer_blocks[kd];
  cpml_line_batched_kernel<0, T><<<nb[0], 128, 0, s->stream>>>(t, n, k);
  cpml_line_batched_kernel<1, T><<<nb[1], 128, 0, s->stream>>>(t, n, k);
  cpml_line_batched_kernel<2, T><<<nb[2], 128, 0, s->stream>>>(t, n, k);
  const int rb = s->layer_rec_blocks[kd];
  cpml_record_batched_kernel<T><<<n * rb, 128, 0, s->stream>>>(t, k, rb);
}

// Complete a resident shot whose steps are all done (stream synchronized).
void complete(serve_ctx *s, Request *q) {
  int status = WAVE_OK;
  int err = 0;
  if (q->r.nrec > 0) {  // NaN / infinity in the traces: WAVE_ENAN
    finite_check_kernel<<<s->sms * 4, 256, 0, s->stream>>>(
        q->host_traces ? q->stage : q->r.traces, (long long)q->r.nsteps * q->r.nrec,
        &q->desc->error);
  }
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&err, &q->desc->error, sizeof(int), cudaMemcpyDeviceToHost,
                        s->stream);
  if (e == cudaSuccess && q->host_traces)
    e = cudaMemcpyAsync(q->r.traces, q->stage,
                        (size_t)q->r.nsteps * q->r.nrec * 4,
                        cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess)
    status = cuda_status(e);
  else if (err)
    status = device_error_status(err);
  release(s, q);
  finish(s, q, status);
}

void engine_main(serve_ctx *s) {
  cudaSetDevice(s->device);
  for (;;) {
    // Admission: first in, first out, while budget, slots and the CTA
    // target allow (a request that fits nothing else runs alone).
    for (;;) {
      Request *q = nullptr;
      {
        std::lock_guard<std::mutex> lk(s->mu);
        if (!s->queue.empty() && (int)s->resident.size() < s->max_slots &&
            s->bytes + s->queue.front()->bytes <= s->budget &&
            (s->resident.empty() ||
             s->ctas + request_places(s->queue.front()->r) <= s->target_ctas)) {
          q = s->queue.front();
          s->queue.pop_front();
          s->st.queued--;
        }
      }
      if (!q) break;
      const int e = admit(s, q);
      if (e != WAVE_OK) {
        cudaGetLastError();
        release(s, q);
        cudaStreamSynchronize(s->stream);
        finish(s, q, e);
        continue;
      }
      {
        std::lock_guard<std::mutex> lk(s->mu);
        q->t_start = s->now();
        s->resident.push_back(q);
        s->bytes += q->bytes;
        s->ctas += request_places(q->r);
        s->st.resident = (int64_t)s->resident.size();
        s->st.bytes_resident = s->bytes;
        s->st.bytes_peak = std::max(s->st.bytes_peak, s->bytes);
        s->st.resident_peak =
            std::max(s->st.resident_peak, (int)s->resident.size());
      }
      s->dirty = true;
    }
    if (s->resident.empty()) {
      std::unique_lock<std::mutex> lk(s->mu);
      if (s->stopping && s->queue.empty()) break;
      s->cv_engine.wait(lk, [&] { return s->stopping || !s->queue.empty(); });
      continue;
    }

    const double tb = s->now();
    int status = WAVE_OK;
    if (s->dirty) status = upload_tables(s);
    // A fixed group of steps: a shot that finishes inside it is skipped by
    // the remaining launches (its CTAs return at once) and completes at the
    // group's end, so the engine synchronizes once per group.
    int K = 1;
    for (Request *q : s->resident)
      K = (int)std::max<int64_t>(K, std::min<int64_t>(kMaxGroup,
                                                      q->r.nsteps - q->steps_done));
    for (int kk = 0; kk < K && status == WAVE_OK; ++kk) {
      for (const Group &g : s->groups)
        kind_of(g.kind).launch(g.ctas, s->stream, s->d_table[g.kind] + g.first,
                               g.count, s->k + kk, g.co);
      if (!s->h_layer[WAVE_STORAGE_F32].empty())
        launch_layers<float>(s, WAVE_STORAGE_F32, s->k + kk);
      if (!s->h_layer[WAVE_STORAGE_BF16].empty())
        launch_layers<__nv_bfloat16>(s, WAVE_STORAGE_BF16, s->k + kk);
      if (!s->h_layer[WAVE_STORAGE_F16].empty())
        launch_layers<__half>(s, WAVE_STORAGE_F16, s->k + kk);
    }
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (status == WAVE_OK && e != cudaSuccess) status = cuda_status(e);
    s->k += K;
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->st.batch_steps += K;
      s->st.busy_s += s->now() - tb;
      for (Request *q : s->resident) {
        const int64_t did = std::min<int64_t>(K, q->r.nsteps - q->steps_done);
        q->steps_done += did;
        s->st.point_steps += q->points * did;
      }
    }
    // Completion (or failure of everything resident if the launch failed).
    std::vector<Request *> keep;
    for (Request *q : s->resident) {
      if (status != WAVE_OK) {
        release(s, q);
        finish(s, q, status);
      } else if (q->steps_done >= q->r.nsteps) {
        complete(s, q);
      } else {
        keep.push_back(q);
        continue;
      }
      s->bytes -= q->bytes;
      s->ctas -= request_places(q->r);
      s->dirty = true;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    s->resident.swap(keep);
    s->st.resident = (int64_t)s->resident.size();
    s->st.bytes_resident = s->bytes;
  }
}

int validate_request(const wave_request *r) {
  if (!r || !r->velocity) return WAVE_EINVAL;
  if (r->grid.nx < 1 || r->grid.ny < 1 || r->grid.nz < 1) return WAVE_EINVAL;
  if ((long long)r->grid.nx * r->grid.ny * r->grid.nz > (1ll << 36))
    return WAVE_EINVAL;
  if (!finite_pos(r->spacing.dx) || !finite_pos(r->spacing.dy) ||
      !finite_pos(r->spacing.dz) || !std::isfinite(r->dt))
    return WAVE_EINVAL;
  if (r->storage < 0 || r->storage >= kKinds) return WAVE_ENOTSUP;
  if (r->nsteps < 1 || r->nrec < 0) return WAVE_EINVAL;
  if (r->nrec > 0 && (!r->rec_xyz || !r->traces)) return WAVE_EINVAL;
  const wave_shot &sh = r->shot;
  if (sh.sx < 0 || sh.sx >= r->grid.nx || sh.sy < 0 || sh.sy >= r->grid.ny ||
      sh.sz < 0 || sh.sz >= r->grid.nz || !finite_pos(sh.f_peak) ||
      !std::isfinite(sh.t0) || !std::isfinite(sh.amp))
    return WAVE_EINVAL;
  if (r->npml < 0) return WAVE_EINVAL;
  if (r->npml > 0) {  // the layer: as wave_set_cpml
    if (2 * r->npml > std::min(r->grid.nx, std::min(r->grid.ny, r->grid.nz)) ||
        !(r->reflection > 0.0 && r->reflection < 1.0) || !(r->f_cps >= 0.0) ||
        !std::isfinite(r->f_cps))
      return WAVE_EINVAL;
    if (r->grid.ny > 65535 || r->grid.nz > 65535) return WAVE_ENOTSUP;
  }
  return WAVE_OK;
}

void fill_result(const Request *q, wave_result *out) {
  if (!out) return;
  out->status = q->status;
  out->ticket = q->ticket;
  out->submit_s = q->t_submit;
  out->start_s = q->t_start;
  out->done_s = q->t_done;
  out->dt = q->dt;
  out->steps_done = std::min<int64_t>(q->steps_done, q->r.nsteps);
}

}  // namespace

extern "C" {

int serve_create(size_t hbm_budget_bytes, int max_slots, void *stream,
                 serve_ctx **out) {
  if (!out) return WAVE_EINVAL;
  *out = nullptr;
  if (hbm_budget_bytes == 0 || max_slots < 1 || max_slots > 4096)
    return WAVE_EINVAL;
  std::unique_ptr<serve_ctx> s(new (std::nothrow) serve_ctx());
  if (!s) return WAVE_ENOMEM;
  s->budget = hbm_budget_bytes;
  s->max_slots = max_slots;
  s->t0 = std::chrono::steady_clock::now();
  WAVE_TRY_CUDA(cudaGetDevice(&s->device));
  {
    int sms = 0;
    WAVE_TRY_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->device));
    s->sms = std::max(sms, 1);
    s->target_ctas = (long long)kTargetWaves * 4 * s->sms;
  }
  if (stream) {
    s->stream = reinterpret_cast<cudaStream_t>(stream);
  } else {
    WAVE_TRY_CUDA(cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking));
    s->own_stream = true;
  }
  int e = WAVE_OK;
  for (int kd = 0; kd < kKinds && e == WAVE_OK; ++kd) {
    const Kind &k = kind_of(kd);
    e = cuda_status(cudaFuncSetAttribute(
        k.func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)k.smem));
    if (e == WAVE_OK)
      e = cuda_status(cudaMalloc((void **)&s->d_table[kd],
                                 sizeof(BatchShot) * (size_t)max_slots));
    if (e == WAVE_OK)
      e = cuda_status(cudaMalloc((void **)&s->d_layer[kd],
                                 sizeof(CpmlBatchShot) * (size_t)max_slots));
  }
  if (e == WAVE_OK) e = cuda_status(cudaMalloc(&s->d_scan, 16));
  if (e == WAVE_OK) {
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = s->device;
    e = cuda_status(cudaMemPoolCreate(&s->pool, &props));
    if (e == WAVE_OK) {
      cuuint64_t keep = (cuuint64_t)hbm_budget_bytes;
      e = cuda_status(cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &keep));
    }
  }
  if (const char *f = std::getenv("GBWAVE_SERVE_FAULT_ALLOC"))
    s->fault_alloc = std::atoll(f);
  if (e != WAVE_OK) {
    for (int kd = 0; kd < kKinds; ++kd) {
      cudaFree(s->d_table[kd]);
      cudaFree(s->d_layer[kd]);
    }
    cudaFree(s->d_scan);
    if (s->pool) cudaMemPoolDestroy(s->pool);
    if (s->own_stream) cudaStreamDestroy(s->stream);
    return e;
  }
  serve_ctx *raw = s.release();
  raw->engine = std::thread(engine_main, raw);
  *out = raw;
  return WAVE_OK;
}

int serve_submit(serve_ctx *s, const wave_request *req, uint64_t *ticket) {
  if (!s || !ticket) return WAVE_EINVAL;
  *ticket = 0;
  const int v = validate_request(req);
  if (v != WAVE_OK) return v;
  std::unique_ptr<Request> q(new (std::nothrow) Request());
  if (!q) return WAVE_ENOMEM;
  q->r = *req;
  q->bytes = request_bytes(*req);
  if (req->nrec > 0 && !is_device_ptr(req->traces))
    q->bytes += (size_t)req->nsteps * req->nrec * 4;
  if (q->bytes > s->budget) return WAVE_ETOOBIG;
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->stopping) return WAVE_EBUSY;
  q->ticket = s->next_ticket++;
  q->t_submit = s->now();
  *ticket = q->ticket;
  s->queue.push_back(q.get());
  s->all.emplace(q->ticket, std::move(q));
  s->st.submitted++;
  s->st.queued++;
  s->cv_engine.notify_one();
  return WAVE_OK;
}

int serve_poll(serve_ctx *s, uint64_t ticket, wave_result *out) {
  if (!s) return WAVE_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return WAVE_EINVAL;
  fill_result(it->second.get(), out);
  return it->second->status;
}

int serve_wait(serve_ctx *s, uint64_t ticket, double timeout_s,
               wave_result *out) {
  if (!s) return WAVE_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return WAVE_EINVAL;
  Request *q = it->second.get();
  auto done = [&] { return q->status != WAVE_EBUSY; };
  if (timeout_s < 0)
    s->cv_done.wait(lk, done);
  else
    s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), done);
  fill_result(q, out);
  return q->status;
}

int serve_get_stats(serve_ctx *s, serve_stats_t *out) {
  if (!s || !out) return WAVE_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  *out = s->st;
  return WAVE_OK;
}

void serve_destroy(serve_ctx *s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stopping = true;
    s->cv_engine.notify_all();
  }
  if (s->engine.joinable()) s->engine.join();
  cudaStreamSynchronize(s->stream);
  for (int kd = 0; kd < kKinds; ++kd) {
    cudaFree(s->d_table[kd]);
    cudaFree(s->d_layer[kd]);
  }
  cudaFree(s->d_scan);
  if (s->pool) cudaMemPoolDestroy(s->pool);
  if (s->own_stream) cudaStreamDestroy(s->stream);
  delete s;
}

}  // extern "C"
