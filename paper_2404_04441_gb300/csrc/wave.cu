// C-ABI implementation of gbwave (declared in include/wave.h): context and
// buffer management, validation, TMA descriptors, launch geometry, CUDA
// graphs of the step loop, and the setup kernels.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <mutex>
#include <new>
#include <vector>

#include "../../include/wave.h"
#include "common.cuh"
#include "cpml.cuh"
#include "sweep.cuh"

using namespace gbw;

namespace {

// Kernel variants. Variant 0 of each storage is the default, measured
// fastest on GB300 at 1024 x 1024 x 512 and 512^3; the others stay
// selectable (GBWAVE_VARIANT) for tuning runs.
//  FP32 (tile x, tile y, rows per thread, prefetch depth, CTAs/SM): 32 x 16
//  tiles, 4 CTAs of 4 warps per SM.
using Cfg0 = SweepCfg<32, 16, 1, 4, 4>;
using CfgA = SweepCfg<64, 16, 1, 4, 2>;
using Cfg2 = SweepCfg<64, 8, 1, 4, 4>;
using Cfg3 = SweepCfg<32, 16, 1, 3, 4>;
//  16-bit, x and y parts of Eq. 1 on the tensor cores (tile x, prefetch
//  depth, CTAs/SM): 64 x 16 tiles of 8 warps, 2 per SM. FP16 / BF16 at
//  1024 x 1024 x 512 (Gpts/s): 64 x 16 529 / 523, 32 x 16 with 4 CTAs/SM
//  496 / 495, 128 x 16 with 1 CTA/SM 462 / 454. Forcing more CTAs per SM
//  spilled registers and was slower (32 x 16 with 5: 439 / 401; 64 x 16
//  with 3: 453 / 374), so those forms are not built.
using CfgBT64 = TcCfg<64, 4, 2, __nv_bfloat16, 9>;
using CfgHT64 = TcCfg<64, 4, 2, __half, 9>;
using CfgBT = TcCfg<32, 4, 4, __nv_bfloat16>;
using CfgHT = TcCfg<32, 4, 4, __half>;
using CfgBT128 = TcCfg<128, 4, 1, __nv_bfloat16, 9>;
using CfgHT128 = TcCfg<128, 4, 1, __half, 9>;
//  16-bit on the CUDA cores (the stencil's pair sums as mixed-precision
//  adds): 64-wide tiles, so a half-warp reads one contiguous 128-byte row of
//  16-bit elements (no shared-memory bank conflicts). 478 / 487 Gpts/s.
using CfgB0 = SweepCfg<64, 8, 1, 4, 4, __nv_bfloat16>;
using CfgB1 = SweepCfg<32, 16, 1, 4, 4, __nv_bfloat16>;
using CfgB2 = SweepCfg<64, 16, 2, 4, 3, __nv_bfloat16>;
using CfgH0 = SweepCfg<64, 8, 1, 4, 4, __half>;
using CfgH1 = SweepCfg<32, 16, 1, 4, 4, __half>;
using CfgH2 = SweepCfg<64, 16, 2, 4, 3, __half>;

struct Variant {
  const void *func;
  int tx, ty, threads;
  size_t smem;
  int esize, halo_x;  // bytes per wavefield element; box columns left of a tile
  int box_u, box_p;   // TMA box widths: u plane with halo, u_prev / c tiles
  void (*launch)(dim3, cudaStream_t, const CUtensorMap &, const CUtensorMap &,
                 const CUtensorMap &, const SweepArgs &);
};

// Launch with programmatic dependent launch allowed: the grid's CTAs may
// become resident while the previous kernel in the stream finishes, and wait
// in the kernel (griddepcontrol.wait) for its completion before reading
// anything. Used for the adjoint-gradient sweeps, issued back to back
// without graphs (wave_gradient at 256^3: 0.186 against 0.189 s). Kernels of
// other kinds in the stream (folds, copies) keep full stream ordering.
template <class K, class... Args>
void launch_pdl(K kernel, dim3 grid, int threads, size_t smem, cudaStream_t st,
                const Args &...args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kernel, args...);
}

template <class C>
void launch_sweep(dim3 grid, cudaStream_t st, const CUtensorMap &tu,
                  const CUtensorMap &tup, const CUtensorMap &tc,
                  const SweepArgs &a) {
  wave_sweep_kernel<C><<<grid, C::THREADS, C::SMEM_BYTES, st>>>(tu, tup, tc, a);
}

template <class C>
Variant make_variant() {
  return Variant{reinterpret_cast<const void *>(&wave_sweep_kernel<C>),
                 C::TX,
                 C::TY,
                 C::THREADS,
                 C::SMEM_BYTES,
                 (int)sizeof(typename C::T),
                 C::HX,
                 C::BOX_U,
                 C::BOX_P,
                 &launch_sweep<C>};
}

Variant pick_variant(int storage, int which) {
  if (storage == WAVE_STORAGE_BF16) {
    switch (which) {
      case 1: return make_variant<CfgB1>();
      case 2: return make_variant<CfgB2>();
      case 3: return make_variant<CfgBT>();
      case 5: return make_variant<CfgB0>();
      case 6: return make_variant<CfgBT128>();
      default: return make_variant<CfgBT64>();
    }
  }
  if (storage == WAVE_STORAGE_F16) {
    switch (which) {
      case 1: return make_variant<CfgH1>();
      case 2: return make_variant<CfgH2>();
      case 3: return make_variant<CfgHT>();
      case 5: return make_variant<CfgH0>();
      case 6: return make_variant<CfgHT128>();
      default: return make_variant<CfgHT64>();
    }
  }
  switch (which) {
    case 1: return make_variant<CfgA>();
    case 2: return make_variant<Cfg2>();
    case 3: return make_variant<Cfg3>();
    default: return make_variant<Cfg0>();
  }
}

__global__ void advance_kernel(StepDesc *d, int k) { d->n += k; }

// Waits on a barrier no one arrives on; records 2 if the wait gave up.
__global__ void selftest_wait_kernel(uint64_t limit_ns, int *out) {
  __shared__ uint64_t bar;
  mbar_init(&bar, 1);
  fence_barrier_init();
  const bool done = mbar_wait_bounded(&bar, 0, limit_ns);
  *out = done ? 1 : 2;
}

}  // namespace

constexpr int kUploadChunks = 32;  // z slabs of the deferred velocity pass

struct wave_ctx {
  int nx = 0, ny = 0, nz = 0;
  int px = 0;       // row pitch of the v^2 dt^2 field (floats, multiple of 4)
  int pxu = 0;      // row pitch of the wavefields (elements, 16-byte rows)
  int storage = WAVE_STORAGE_F32;
  int sms = 0;
  double vmax = 0;
  double dx = 0, dy = 0, dz = 0, dt = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t capture_stream = nullptr;
  int device = 0;
  void *base = nullptr;  // one allocation: both wavefields, c, desc, scratch
  void *buf[2] = {nullptr, nullptr};  // buf[cur] = u, buf[cur ^ 1] = u_prev
  float *c = nullptr;
  cudaEvent_t ev_aux = nullptr;  // joins work of capture_stream into stream
  // Deferred velocity pass (wave_create_async).
  cudaStream_t upload_stream = nullptr;
  cudaEvent_t ev_upload_start = nullptr;
  cudaEvent_t chunk_ev[kUploadChunks] = {};
  int chunk_z0[kUploadChunks] = {};
  int nchunks = 0;
  int chunk_next = 0;           // first slab the main stream has not waited for
  bool upload_pending = false;  // the main stream has not waited for every slab
  bool model_checked = true;    // the host holds the velocity pass's verdict
  int model_status = WAVE_OK;   // that verdict (WAVE_EINVAL, WAVE_EUNSTABLE)
  bool at_rest = true;          // zero fields since creation or reset
  int model_m = 0;              // the model was given as m = v^2 (wave_create_m)
  int cur = 0;
  int64_t step = 0;
  StepDesc *d_desc = nullptr;
  void *d_scratch = nullptr;  // 16 bytes for the velocity scan
  CUtensorMap tm_halo[2], tm_tile[2], tm_c;
  Variant var{};
  dim3 grid;
  int zchunk = 0, ctas_per_sm = 0, ntiles = 0;
  SweepArgs args{};
  // Per-call tables in one device buffer (one cudaFree at destroy): the
  // source wavelet, the receiver table and its build arrays, staged host
  // receivers, and staged traces for a host destination.
  DeviceBuf tables;
  float *d_wavelet = nullptr;
  int4 *d_rec = nullptr;            // receiver table, sorted by (tile, z)
  int *d_rec_start = nullptr;       // per-tile starts (ntiles + 1)
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  int graph_steps = 32;
  StepDesc host_desc{};
  std::vector<int32_t> h_rec_raw;  // host receivers, staged for upload
  std::vector<float> h_wavelet;
  unsigned char scale_image[32];  // host staging of the 16-bit scale state
  // CPML layer (wave_set_cpml).
  bool cpml = false;
  CpmlGeom cg{};
  std::vector<void *> cpml_mem;
  DeviceBuf srec;            // receivers within w of a face: {x, y, z, id}
  int *d_nsrec = nullptr;    // their count (device: graphs stay valid)
  int cpml_seg_axes = 0;     // bit a: axis a runs the unrolled segment kernels
  CpmlSideProf<8> prof8[3];  // their profile values (npml 8 or 16)
  CpmlSideProf<16> prof16[3];
};

namespace {

size_t round_up256(size_t x) { return (x + 255) & ~size_t(255); }

int make_map(CUtensorMap *m, const void *base, const wave_ctx *c, int box_x,
             int box_y, CUtensorMapDataType dtype, int pitch, int esize) {
  return encode_map(m, base, c->nx, c->ny, c->nz, pitch, esize, dtype, box_x,
                    box_y);
}

int build_maps(wave_ctx *c) {
  const int ty = c->var.ty;
  const CUtensorMapDataType dt = field_dtype(c->storage);
  for (int b = 0; b < 2; ++b) {
    int st = make_map(&c->tm_halo[b], c->buf[b], c, c->var.box_u, ty + 2 * kR,
                      dt, c->pxu, c->var.esize);
    if (st) return st;
    st = make_map(&c->tm_tile[b], c->buf[b], c, c->var.box_p, ty, dt, c->pxu,
                  c->var.esize);
    if (st) return st;
  }
  return make_map(&c->tm_c, c->c, c, c->var.box_p, ty,
                  CU_TENSOR_MAP_DATA_TYPE_FLOAT32, c->px, 4);
}

void set_coeffs(wave_ctx *c) {
  SweepArgs &a = c->args;
  a.nx = c->nx;
  a.ny = c->ny;
  a.nz = c->nz;
  a.px = c->pxu;
  a.ntx = (int)c->grid.x;
  a.cmax = (float)(c->vmax * c->vmax * c->dt * c->dt);
  a.k = make_coefs(c->dx, c->dy, c->dz);
  a.desc = c->d_desc;
}

// The layer's pass along axis AX of one forward step (dout: the layer's
// term also into the stored increment D), and of one adjoint step.
// T: the wavefields' storage; d, koff: the step's descriptor and offset
// (the 16-bit fields' scales).
template <int AX, class T, bool kD>
void launch_cpml_axis(const wave_ctx *c, const CpmlGeom &g, cudaStream_t st, const T *u,
                      T *un, float *dout, const StepDesc *d, int koff) {
  const int inner = AX == 0 ? c->ny : c->nx, outer = AX == 2 ? c->ny : c->nz;
  const bool seg = (c->cpml_seg_axes >> AX) & 1;
  const dim3 grid((inner + 127) / 128, outer, seg ? 2 : 1);
  if (!seg)
    cpml_line_kernel<AX, T, kD><<<grid, 128, 0, st>>>(g, u, un, c->c, dout, d, koff);
  else if (g.npml == 8)
    cpml_seg_kernel<AX, 8, T, kD><<<grid, 128, 0, st>>>(g, c->prof8[AX], u, un, c->c, dout, d,
                                                        koff);
  else
    cpml_seg_kernel<AX, 16, T, kD><<<grid, 128, 0, st>>>(g, c->prof16[AX], u, un, c->c, dout,
                                                         d, koff);
}

// g: the context's layer, or the same layer on other memory-variable slabs
template <class T, bool kD>
void launch_cpml_forward(const wave_ctx *c, const CpmlGeom &g, cudaStream_t st, const T *u,
                         T *un, float *dout, const StepDesc *d, int koff) {
  launch_cpml_axis<0, T, kD>(c, g, st, u, un, dout, d, koff);
  launch_cpml_axis<1, T, kD>(c, g, st, u, un, dout, d, koff);
  launch_cpml_axis<2, T, kD>(c, g, st, u, un, dout, d, koff);
}

// One step's layer passes and shell receivers on the context's fields, in
// their storage type.
template <class T>
void launch_cpml_step(const wave_ctx *c, cudaStream_t st, int cur, int koff) {
  const T *u = static_cast<const T *>(c->buf[cur]);
  T *un = static_cast<T *>(c->buf[cur ^ 1]);
  launch_cpml_forward<T, false>(c, c->cg, st, u, un, nullptr, c->d_desc, koff);
  cpml_record_kernel<T><<<c->sms, 256, 0, st>>>(c->cg, un, c->d_desc, (const int4 *)c->srec.p,
                                               c->d_nsrec, koff);
}

template <int AX>
void launch_cpml_adjoint_axis(const wave_ctx *c, cudaStream_t st, const float *p1, float *p0,
                              float *nus, float *mus) {
  const CpmlGeom &g = c->cg;
  const int inner = AX == 0 ? c->ny : c->nx, outer = AX == 2 ? c->ny : c->nz;
  const bool seg = (c->cpml_seg_axes >> AX) & 1;
  const dim3 grid((inner + 127) / 128, outer, seg ? 2 : 1);
  if (!seg)
    cpml_adjoint_line_kernel<AX><<<grid, 128, 0, st>>>(g, p1, p0, c->c, nus, mus);
  else if (g.npml == 8)
    cpml_seg_adjoint_kernel<AX, 8><<<grid, 128, 0, st>>>(g, c->prof8[AX], p1, p0, c->c, nus, mus);
  else
    cpml_seg_adjoint_kernel<AX, 16><<<grid, 128, 0, st>>>(g, c->prof16[AX], p1, p0, c->c, nus,
                                                          mus);
}

// Enqueue one step on stream st: u = buf[cur], u_prev = buf[cur ^ 1]. With
// the CPML layer: memory variables and shell points before the sweep, the
// shell values committed after it.
void enqueue_step(wave_ctx *c, cudaStream_t st, int cur, int koff) {
  SweepArgs a = c->args;
  a.unext = c->buf[cur ^ 1];
  a.koff = koff;
  c->var.launch(c->grid, st, c->tm_halo[cur], c->tm_tile[cur ^ 1], c->tm_c, a);
  if (c->cpml) {
    if (c->storage == WAVE_STORAGE_BF16)
      launch_cpml_step<__nv_bfloat16>(c, st, cur, koff);
    else if (c->storage == WAVE_STORAGE_F16)
      launch_cpml_step<__half>(c, st, cur, koff);
    else
      launch_cpml_step<float>(c, st, cur, koff);
  }
}

void drop_graphs(wave_ctx *c) {
  for (int p = 0; p < 2; ++p)
    if (c->graph[p]) {
      cudaGraphExecDestroy(c->graph[p]);
      c->graph[p] = nullptr;
    }
}

void free_cpml(wave_ctx *c) {
  for (void *p : c->cpml_mem) cudaFree(p);
  c->cpml_mem.clear();
  c->cpml = false;
  c->cg = CpmlGeom{};
  c->cpml_seg_axes = 0;
}

int zero_cpml(wave_ctx *c) {
  if (!c->cpml) return WAVE_OK;
  const size_t sl[3] = {2ull * c->cg.npml * c->ny * c->nz,
                        2ull * c->cg.npml * c->nz * c->nx,
                        2ull * c->cg.npml * c->ny * c->nx};
  for (int ax = 0; ax < 3; ++ax) {
    WAVE_TRY_CUDA(cudaMemsetAsync(c->cg.psi[ax], 0, sl[ax] * 4, c->stream));
    WAVE_TRY_CUDA(cudaMemsetAsync(c->cg.zeta[ax], 0, sl[ax] * 4, c->stream));
  }
  return WAVE_OK;
}

int build_graph(wave_ctx *c, int parity) {
  cudaGraph_t g = nullptr;
  WAVE_TRY_CUDA(cudaStreamBeginCapture(c->capture_stream,
                                       cudaStreamCaptureModeThreadLocal));
  for (int k = 0; k < c->graph_steps; ++k)
    enqueue_step(c, c->capture_stream, parity ^ (k & 1), k);
  advance_kernel<<<1, 1, 0, c->capture_stream>>>(c->d_desc, c->graph_steps);
  cudaError_t e = cudaStreamEndCapture(c->capture_stream, &g);
  if (e != cudaSuccess) return cuda_status(e);
  e = cudaGraphInstantiate(&c->graph[parity], g, 0);
  cudaGraphDestroy(g);
  return cuda_status(e);
}

// Run nsteps steps whose per-call state (StepDesc) is already uploaded.
int run_steps(wave_ctx *c, int nsteps) {
  int done = 0;
  while (nsteps - done >= c->graph_steps) {
    if (!c->graph[c->cur]) {
      int st = build_graph(c, c->cur);
      if (st) return st;
    }
    WAVE_TRY_CUDA(cudaGraphLaunch(c->graph[c->cur], c->stream));
    done += c->graph_steps;  // even count: parity unchanged
  }
  const int rem = nsteps - done;
  if (rem > 0) {
    int cur = c->cur;
    for (int k = 0; k < rem; ++k, cur ^= 1) enqueue_step(c, c->stream, cur, k);
    advance_kernel<<<1, 1, 0, c->stream>>>(c->d_desc, rem);
    c->cur = cur;
  }
  WAVE_TRY_CUDA(cudaGetLastError());
  c->step += nsteps;
  if (nsteps > 0) c->at_rest = false;
  return WAVE_OK;
}

// Deferred velocity pass, field at rest, source at depth sz: enqueue steps
// one by one, each after the slabs it can reach (planes up to sz + 4k for
// the call's step k), until every slab has been waited for or the call's
// steps run out. Returns the number of steps enqueued (the caller runs the
// rest as usual).
int steps_while_loading(wave_ctx *c, int sz, int nsteps) {
  int k = 0, cur = c->cur;
  for (; k < nsteps && c->chunk_next < c->nchunks; ++k, cur ^= 1) {
    const long long reach = (long long)sz + 4ll * k;
    while (c->chunk_next < c->nchunks && c->chunk_z0[c->chunk_next] <= reach) {
      WAVE_TRY_CUDA(cudaStreamWaitEvent(c->stream, c->chunk_ev[c->chunk_next], 0));
      ++c->chunk_next;
    }
    enqueue_step(c, c->stream, cur, k);
  }
  if (k > 0) {
    advance_kernel<<<1, 1, 0, c->stream>>>(c->d_desc, k);
    WAVE_TRY_CUDA(cudaGetLastError());
    c->cur = cur;
    c->step += k;
    c->at_rest = false;
  }
  if (c->chunk_next == c->nchunks) c->upload_pending = false;
  return k;
}

// Result of the velocity pass (16 bytes: max bits, bad count) to a status;
// sets vmax.
int check_model(wave_ctx *c, const unsigned char *res) {
  unsigned vb;
  unsigned long long bad;
  std::memcpy(&vb, res, 4);
  std::memcpy(&bad, res + 8, 8);
  if (bad) return WAVE_EINVAL;
  float top;
  std::memcpy(&top, &vb, 4);
  const double vmax = c->model_m ? std::sqrt((double)top) : (double)top;
  wave_spacing h{c->dx, c->dy, c->dz};
  const double lim = wave_cfl_dt(&h, vmax);
  if (!(c->dt <= lim * (1.0 + 1e-12))) return WAVE_EUNSTABLE;
  c->vmax = vmax;
  return WAVE_OK;
}

// Deferred velocity pass (wave_create_async): make the main stream wait for
// every slab.
int wait_model(wave_ctx *c) {
  if (!c->upload_pending) return WAVE_OK;
  WAVE_TRY_CUDA(cudaStreamWaitEvent(c->stream, c->chunk_ev[c->nchunks - 1], 0));
  c->chunk_next = c->nchunks;
  c->upload_pending = false;
  return WAVE_OK;
}

// Deferred velocity pass: wait for it on the host and take its verdict (and
// vmax); the verdict of a synchronous creation is already known.
int finish_model(wave_ctx *c) {
  if (c->model_checked) return c->model_status;
  unsigned char res[16];
  WAVE_TRY_CUDA(cudaMemcpyAsync(res, c->d_scratch, 16, cudaMemcpyDeviceToHost,
                                c->upload_stream));
  WAVE_TRY_CUDA(cudaStreamSynchronize(c->upload_stream));
  c->model_status = check_model(c, res);
  c->model_checked = true;
  return c->model_status;
}

int read_device_error(wave_ctx *c) {
  const int ms = finish_model(c);
  if (ms) return ms;
  int err = 0;
  WAVE_TRY_CUDA(cudaMemcpyAsync(&err, &c->d_desc->error, sizeof(int),
                                cudaMemcpyDeviceToHost, c->stream));
  WAVE_TRY_CUDA(cudaStreamSynchronize(c->stream));
  return device_error_status(err);
}

int upload_desc(wave_ctx *c) {
  c->host_desc.step0 = c->step;
  // Everything before the error word (which persists until read, followed
  // by the scale state of 16-bit storage).
  WAVE_TRY_CUDA(cudaMemcpyAsync(c->d_desc, &c->host_desc,
                                offsetof(StepDesc, error),
                                cudaMemcpyHostToDevice, c->stream));
  return WAVE_OK;
}

}  // namespace

extern "C" {

double wave_cfl_dt(const wave_spacing *h, double vmax) {
  if (!h || !finite_pos(h->dx) || !finite_pos(h->dy) || !finite_pos(h->dz) ||
      !finite_pos(vmax))
    return -1.0;
  double s = std::fabs(kW[0]);
  for (int m = 1; m <= 4; ++m) s += 2.0 * std::fabs(kW[m]);
  const double inv =
      1.0 / (h->dx * h->dx) + 1.0 / (h->dy * h->dy) + 1.0 / (h->dz * h->dz);
  return 2.0 / (vmax * std::sqrt(s * inv));
}

const char *wave_strerror(int st) {
  switch (st) {
    case WAVE_OK: return "ok";
    case WAVE_EINVAL: return "invalid argument";
    case WAVE_ENOMEM: return "out of device memory";
    case WAVE_ECUDA: return "CUDA error";
    case WAVE_EUNSTABLE: return "dt above the leapfrog stability limit";
    case WAVE_ETIMEOUT: return "device wait timed out";
    case WAVE_EBUSY: return "not ready";
    case WAVE_ENAN: return "non-finite values";
    case WAVE_ENOTSUP: return "not supported";
    case WAVE_ETOOBIG: return "request exceeds the fixed scratch array";
    default: return "unknown status";
  }
}

void wave_destroy(wave_ctx *c) {
  if (!c) return;
  if (c->upload_stream) cudaStreamSynchronize(c->upload_stream);
  if (c->stream || c->buf[0]) cudaStreamSynchronize(c->stream);
  for (int p = 0; p < 2; ++p)
    if (c->graph[p]) cudaGraphExecDestroy(c->graph[p]);
  cudaFree(c->base);
  cudaFree(c->tables.p);
  if (c->ev_aux) cudaEventDestroy(c->ev_aux);
  if (c->ev_upload_start) cudaEventDestroy(c->ev_upload_start);
  for (cudaEvent_t e : c->chunk_ev)
    if (e) cudaEventDestroy(e);
  if (c->upload_stream) cudaStreamDestroy(c->upload_stream);
  if (c->capture_stream) cudaStreamDestroy(c->capture_stream);
  free_cpml(c);
  cudaFree(c->srec.p);
  cudaFree(c->d_nsrec);
  delete c;
}

size_t field_bytes(const wave_ctx *c) {
  return (size_t)c->pxu * c->ny * c->nz * (size_t)c->var.esize;
}

// Where the velocity pass reads the caller's model: device memory, pinned
// host memory through its device mapping, or pageable host memory when the
// GPU reads the host's page tables (address translation services); nullptr
// when the model has to be staged by a copy first.
static const float *velocity_source(const float *velocity, int device) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, velocity) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged)
    return velocity;
  if (at.type == cudaMemoryTypeHost) {
    void *dp = nullptr;
    if (cudaHostGetDevicePointer(&dp, const_cast<float *>(velocity), 0) == cudaSuccess)
      return static_cast<const float *>(dp);
    cudaGetLastError();
    return nullptr;
  }
  int pageable = 0, host_tables = 0;
  cudaDeviceGetAttribute(&pageable, cudaDevAttrPageableMemoryAccess, device);
  cudaDeviceGetAttribute(&host_tables,
                         cudaDevAttrPageableMemoryAccessUsesHostPageTables, device);
  return pageable && host_tables ? velocity : nullptr;
}

// Streams, events and the one allocation that holds both wavefields,
// v^2 dt^2, the step descriptor and the scan result (one cudaMalloc /
// cudaFree instead of five). The zero initial state is written on the side
// stream (joined through ev_aux) while the velocity pass runs on the main one.
static int alloc_context(wave_ctx *c) {
  const size_t bytes = (size_t)c->px * c->ny * c->nz * sizeof(float);
  cudaStream_t st = c->stream;
  const char *ev = std::getenv("GBWAVE_VARIANT");
  c->var = pick_variant(c->storage, ev ? std::atoi(ev) : 0);
  WAVE_TRY_CUDA(cudaGetDevice(&c->device));
  WAVE_TRY_CUDA(cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount,
                                       c->device));
  WAVE_TRY_CUDA(cudaStreamCreateWithFlags(&c->capture_stream,
                                          cudaStreamNonBlocking));
  WAVE_TRY_CUDA(cudaEventCreateWithFlags(&c->ev_aux, cudaEventDisableTiming));
  const size_t fbytes = field_bytes(c);
  const size_t off1 = round_up256(fbytes), offc = off1 + round_up256(fbytes);
  const size_t offd = offc + round_up256(bytes);
  const size_t offs = offd + round_up256(sizeof(StepDesc));
  WAVE_TRY_CUDA(cudaMalloc(&c->base, offs + 256));
  char *base = static_cast<char *>(c->base);
  c->buf[0] = base;
  c->buf[1] = base + off1;
  c->c = reinterpret_cast<float *>(base + offc);
  c->d_desc = reinterpret_cast<StepDesc *>(base + offd);
  c->d_scratch = base + offs;
  WAVE_TRY_CUDA(cudaMemsetAsync(c->buf[0], 0, fbytes, c->capture_stream));
  WAVE_TRY_CUDA(cudaMemsetAsync(c->buf[1], 0, fbytes, c->capture_stream));
  WAVE_TRY_CUDA(cudaEventRecord(c->ev_aux, c->capture_stream));
  WAVE_TRY_CUDA(cudaMemsetAsync(c->d_desc, 0, offs + 256 - offd, st));
  return WAVE_OK;
}

// Launch geometry, z-layer plan, coefficients and tensor maps.
static int setup_launch(wave_ctx *c) {
  WAVE_TRY_CUDA(cudaFuncSetAttribute(c->var.func,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)c->var.smem));
  WAVE_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
      &c->ctas_per_sm, c->var.func, c->var.threads, c->var.smem));
  if (c->ctas_per_sm < 1) return WAVE_ECUDA;
  const int ntx = (c->nx + c->var.tx - 1) / c->var.tx;
  const int nty = (c->ny + c->var.ty - 1) / c->var.ty;
  c->ntiles = ntx * nty;
  int layers[kMaxLayers];
  double preroll = c->storage == WAVE_STORAGE_F32 ? 4.0 : 8.0;
  if (const char *pr = std::getenv("GBWAVE_PREROLL")) preroll = std::atof(pr);
  const int nl = plan_layers(c->nz, (long long)c->ntiles,
                             (long long)c->sms * c->ctas_per_sm, preroll, layers);
  c->zchunk = *std::max_element(layers, layers + nl);
  c->grid = dim3(ntx, nty, (unsigned)nl);
  if (c->grid.y > 65535) return WAVE_EINVAL;
  set_coeffs(c);
  set_layers(c->args, layers, nl);
  int stt = build_maps(c);
  if (stt) return stt;
  const char *gs = std::getenv("GBWAVE_GRAPH_STEPS");
  if (gs) c->graph_steps = std::max(2, (std::atoi(gs) / 2) * 2);
  return WAVE_OK;
}

static void launch_velocity_pass(wave_ctx *c, const float *src, long long sx,
                                 int z0, int z1, cudaStream_t st, int blocks) {
  const double dt2 = c->dt * c->dt;
  const float dh = (float)dt2, dl = (float)(dt2 - (double)dh);
  unsigned *vmax = reinterpret_cast<unsigned *>(c->d_scratch);
  unsigned long long *nbad =
      reinterpret_cast<unsigned long long *>((char *)c->d_scratch + 8);
  const float *s0 = src + (long long)z0 * c->ny * sx;
  float *c0 = c->c + (size_t)z0 * c->ny * c->px;
  if (sx == c->px && c->px == c->nx && reinterpret_cast<uintptr_t>(s0) % 16 == 0) {
    velocity_to_c_dense_kernel<<<blocks, 256, 0, st>>>(
        reinterpret_cast<const float4 *>(s0), reinterpret_cast<float4 *>(c0),
        (long long)(z1 - z0) * c->ny * c->px / 4, dh, dl, c->model_m, vmax, nbad);
  } else {
    velocity_to_c_checked_kernel<<<blocks, 256, 0, st>>>(
        s0, sx, c0, c->nx, c->px, (long long)(z1 - z0) * c->ny, dh, dl, c->model_m,
        vmax, nbad);
  }
}

static int create_impl(wave_ctx *c, const float *velocity) {
  int s;
  if ((s = alloc_context(c))) return s;
  cudaStream_t st = c->stream;
  // One pass validates the velocities, finds their maximum and writes
  // v^2 dt^2, reading the caller's model where it lies when the GPU can
  // reach it, else from a staged copy in the c buffer.
  const float *src = velocity_source(velocity, c->device);
  long long sx = c->nx;
  if (!src) {
    WAVE_TRY_CUDA(cudaMemcpy2DAsync(c->c, (size_t)c->px * 4, velocity,
                                    (size_t)c->nx * 4, (size_t)c->nx * 4,
                                    (size_t)c->ny * c->nz, cudaMemcpyDefault, st));
    src = c->c;
    sx = c->px;
  }
  launch_velocity_pass(c, src, sx, 0, c->nz, st, c->sms * 4);
  WAVE_TRY_CUDA(cudaGetLastError());
  WAVE_TRY_CUDA(cudaStreamWaitEvent(st, c->ev_aux, 0));
  unsigned char res[16];
  WAVE_TRY_CUDA(cudaMemcpyAsync(res, c->d_scratch, 16, cudaMemcpyDeviceToHost, st));
  WAVE_TRY_CUDA(cudaStreamSynchronize(st));
  if ((s = check_model(c, res))) return s;
  c->model_checked = true;
  return setup_launch(c);
}

// Deferred form (wave_create_async): v^2 dt^2 starts at zero everywhere (so
// every value the sweep can read is finite) and the velocity pass runs on
// its own stream in kUploadChunks z slabs, each followed by an event. While
// the field is still at rest, a propagation waits before step k only for
// the slabs that reach depth sz + 4k: the star stencil spreads the field by
// at most 4 planes per step, so every plane below that bound still holds
// u = u_prev = L u = 0 and computes u_next = 0 whatever its v^2 dt^2.
// A host model crosses the link by copy engine into the c buffer, slab by
// slab, and is converted there in place by a short kernel: the SMs stay
// with the sweep while the (link-bound) transfer runs. A device model is
// converted directly. The pass kernels take one block per SM.
static int create_async_impl(wave_ctx *c, const float *velocity) {
  int s;
  if ((s = alloc_context(c))) return s;
  cudaStream_t st = c->stream;
  // Pinned host models cross the link by copy engine and are converted in
  // place by one-block-per-SM kernels; pageable host models (read by the
  // GPU through the host's page tables) are read by the pass kernel itself
  // with a quarter of the SMs, enough blocks to fill the link while taking
  // few CTA places from the sweep; device models are converted directly.
  // Measured at 1024 x 1024 x 512, 20 steps from rest, create + propagate +
  // destroy: pinned 35.7 ms (copy engine) against 36.6 (kernel reads, 38
  // blocks); pageable 37.2 ms (kernel reads, 38 blocks) against 39.4 (76),
  // 40.4 (152) and 56.5 (copy engine: the pageable copy blocks the host).
  // GBWAVE_UPLOAD=sm|ce and GBWAVE_UPLOAD_BLOCKS override both (tuning).
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, velocity) != cudaSuccess) cudaGetLastError();
  const bool on_device =
      at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
  const float *direct = velocity_source(velocity, c->device);
  bool copy_engine = at.type == cudaMemoryTypeHost;
  int pass_blocks = copy_engine || on_device ? c->sms : std::max(1, c->sms / 4);
  if (const char *um = std::getenv("GBWAVE_UPLOAD"))
    copy_engine = !on_device && std::strcmp(um, "ce") == 0;
  if (const char *ub = std::getenv("GBWAVE_UPLOAD_BLOCKS"))
    pass_blocks = std::max(1, std::atoi(ub));
  WAVE_TRY_CUDA(cudaStreamCreateWithFlags(&c->upload_stream, cudaStreamNonBlocking));
  WAVE_TRY_CUDA(cudaEventCreateWithFlags(&c->ev_upload_start, cudaEventDisableTiming));
  for (int j = 0; j < kUploadChunks; ++j)
    WAVE_TRY_CUDA(cudaEventCreateWithFlags(&c->chunk_ev[j], cudaEventDisableTiming));
  WAVE_TRY_CUDA(cudaMemsetAsync(c->c, 0, (size_t)c->px * c->ny * c->nz * 4, st));
  WAVE_TRY_CUDA(cudaEventRecord(c->ev_upload_start, st));
  WAVE_TRY_CUDA(cudaStreamWaitEvent(c->upload_stream, c->ev_upload_start, 0));
  const int nch = std::min(c->nz, kUploadChunks);
  for (int j = 0; j < nch; ++j) {
    const int z0 = (int)((long long)c->nz * j / nch);
    const int z1 = (int)((long long)c->nz * (j + 1) / nch);
    c->chunk_z0[j] = z0;
    if (on_device || !copy_engine) {
      launch_velocity_pass(c, direct, c->nx, z0, z1, c->upload_stream, pass_blocks);
    } else {
      const size_t rows = (size_t)(z1 - z0) * c->ny;
      WAVE_TRY_CUDA(cudaMemcpy2DAsync(
          c->c + (size_t)z0 * c->ny * c->px, (size_t)c->px * 4,
          velocity + (size_t)z0 * c->ny * c->nx, (size_t)c->nx * 4, (size_t)c->nx * 4,
          rows, cudaMemcpyHostToDevice, c->upload_stream));
      launch_velocity_pass(c, c->c, c->px, z0, z1, c->upload_stream, pass_blocks);
    }
    WAVE_TRY_CUDA(cudaGetLastError());
    WAVE_TRY_CUDA(cudaEventRecord(c->chunk_ev[j], c->upload_stream));
  }
  c->nchunks = nch;
  c->chunk_next = 0;
  c->upload_pending = true;
  c->model_checked = false;
  c->at_rest = true;
  WAVE_TRY_CUDA(cudaStreamWaitEvent(st, c->ev_aux, 0));
  return setup_launch(c);
}

// Arguments shared by wave_create and wave_create_async; a new context with
// its sizes filled in, or a status.
static int new_context(const wave_grid *g, const wave_spacing *h, double dt,
                       const float *velocity, int storage, void *stream,
                       wave_ctx **out) {
  if (!out) return WAVE_EINVAL;
  *out = nullptr;
  if (!g || !h || !velocity) return WAVE_EINVAL;
  if (g->nx < 1 || g->ny < 1 || g->nz < 1) return WAVE_EINVAL;
  if (!finite_pos(h->dx) || !finite_pos(h->dy) || !finite_pos(h->dz) ||
      !finite_pos(dt))
    return WAVE_EINVAL;
  if (storage != WAVE_STORAGE_F32 && storage != WAVE_STORAGE_BF16 &&
      storage != WAVE_STORAGE_F16)
    return WAVE_ENOTSUP;
  // Row pitches: 16-byte rows (TMA): 4 floats, or 8 16-bit elements.
  const long long px = ((long long)g->nx + 3) / 4 * 4;
  const long long pxu =
      storage == WAVE_STORAGE_F32 ? px : ((long long)g->nx + 7) / 8 * 8;
  if (px * (long long)g->ny * (long long)g->nz > (1ll << 36)) return WAVE_EINVAL;
  wave_ctx *c = new (std::nothrow) wave_ctx();
  if (!c) return WAVE_ENOMEM;
  c->nx = g->nx;
  c->ny = g->ny;
  c->nz = g->nz;
  c->px = (int)px;
  c->pxu = (int)pxu;
  c->storage = storage;
  c->dx = h->dx;
  c->dy = h->dy;
  c->dz = h->dz;
  c->dt = dt;
  c->stream = reinterpret_cast<cudaStream_t>(stream);
  *out = c;
  return WAVE_OK;
}

int wave_create(const wave_grid *g, const wave_spacing *h, double dt,
                const float *velocity, int storage, void *stream,
                wave_ctx **out) {
  wave_ctx *c = nullptr;
  int st = new_context(g, h, dt, velocity, storage, stream, &c);
  if (st != WAVE_OK) return st;
  st = create_impl(c, velocity);
  if (st != WAVE_OK) {
    cudaGetLastError();
    wave_destroy(c);
    return st;
  }
  *out = c;
  return WAVE_OK;
}

int wave_create_m(const wave_grid *g, const wave_spacing *h, double dt,
                  const float *m, int storage, void *stream, wave_ctx **out) {
  wave_ctx *c = nullptr;
  int st = new_context(g, h, dt, m, storage, stream, &c);
  if (st != WAVE_OK) return st;
  c->model_m = 1;
  st = create_impl(c, m);
  if (st != WAVE_OK) {
    cudaGetLastError();
    wave_destroy(c);
    return st;
  }
  *out = c;
  return WAVE_OK;
}

int wave_create_async(const wave_grid *g, const wave_spacing *h, double dt,
                      const float *velocity, int storage, void *stream,
                      wave_ctx **out) {
  wave_ctx *c = nullptr;
  int st = new_context(g, h, dt, velocity, storage, stream, &c);
  if (st != WAVE_OK) return st;
  int dev = 0;
  const bool defer = storage == WAVE_STORAGE_F32 && cudaGetDevice(&dev) == cudaSuccess &&
                     velocity_source(velocity, dev) != nullptr;
  st = defer ? create_async_impl(c, velocity) : create_impl(c, velocity);
  if (st != WAVE_OK) {
    cudaGetLastError();
    wave_destroy(c);
    return st;
  }
  *out = c;
  return WAVE_OK;
}

int wave_step(wave_ctx *c, int nsteps) {
  if (!c || nsteps < 0) return WAVE_EINVAL;
  if (nsteps == 0) return WAVE_OK;
  StepDesc &d = c->host_desc;
  std::memset(&d, 0, sizeof(d));
  if (c->cpml)
    WAVE_TRY_CUDA(cudaMemsetAsync(c->d_nsrec, 0, sizeof(int), c->stream));
  int st = wait_model(c);
  if (st) return st;
  st = upload_desc(c);
  if (st) return st;
  return run_steps(c, nsteps);
}

}  // extern "C"

namespace {

// The part of a propagation call before its steps: validation, receiver
// table, wavelet and descriptor for nsteps steps from the context's step.
// host_traces / stage: traces staged on the device for a host buffer.
int propagate_begin(wave_ctx *c, const wave_shot *shot, int nsteps,
                    const int32_t *rec_xyz, int nrec, float *traces, bool &host_traces,
                    float *&stage) {
  if (!c || nsteps < 0 || nrec < 0) return WAVE_EINVAL;
  if (nrec > 0 && (!rec_xyz || !traces)) return WAVE_EINVAL;
  if (shot) {
    if (shot->sx < 0 || shot->sx >= c->nx || shot->sy < 0 ||
        shot->sy >= c->ny || shot->sz < 0 || shot->sz >= c->nz)
      return WAVE_EINVAL;
    if (!finite_pos(shot->f_peak) || !std::isfinite(shot->t0) ||
        !std::isfinite(shot->amp))
      return WAVE_EINVAL;
  }
  host_traces = false;
  stage = nullptr;
  if (nsteps == 0) return WAVE_OK;
  cudaStream_t st = c->stream;
  int s;

  // Receivers: host-resident ones are validated here (WAVE_EINVAL before
  // anything is launched) and staged through a copy the call owns, so the
  // caller's buffer is read completely before the call returns. The table
  // sorted by (tile, z) is then built on the device, with no round trip to
  // the host and no wait for the stream; device-resident receivers outside
  // the interior are left out and reported as WAVE_EINVAL by the next
  // synchronizing call.
  const bool host_rec = nrec > 0 && !is_device_ptr(rec_xyz);
  host_traces = nrec > 0 && !is_device_ptr(traces);
  if (host_rec) {
    c->h_rec_raw.resize((size_t)nrec * 3);
    for (int r = 0; r < nrec; ++r) {
      const int32_t x = rec_xyz[3 * r], y = rec_xyz[3 * r + 1], z = rec_xyz[3 * r + 2];
      if (x < 0 || x >= c->nx || y < 0 || y >= c->ny || z < 0 || z >= c->nz)
        return WAVE_EINVAL;
      c->h_rec_raw[3 * r] = x;
      c->h_rec_raw[3 * r + 1] = y;
      c->h_rec_raw[3 * r + 2] = z;
    }
  }
  // Layout of the tables buffer for this call (256-byte aligned blocks).
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off += round_up256(bytes);
    return o;
  };
  const size_t o_w = take(shot ? (size_t)nsteps * 4 : 0);
  const size_t o_raw = take(host_rec ? (size_t)nrec * 12 : 0);
  const size_t o_rec = take((size_t)nrec * sizeof(int4));
  const size_t o_keys = take((size_t)nrec * 8);
  const size_t o_start = take(nrec > 0 ? (size_t)(c->ntiles + 1) * 4 : 0);
  const size_t o_cnt = take(nrec > 0 ? (size_t)(c->ntiles + 1) * 4 : 0);
  const size_t o_tr = take(host_traces ? (size_t)nsteps * nrec * 4 : 0);
  if ((s = ensure(c->tables, off, st))) return s;
  char *tb = static_cast<char *>(c->tables.p);
  c->d_wavelet = reinterpret_cast<float *>(tb + o_w);
  c->d_rec = reinterpret_cast<int4 *>(tb + o_rec);
  c->d_rec_start = reinterpret_cast<int *>(tb + o_start);
  float *d_traces_stage = reinterpret_cast<float *>(tb + o_tr);
  stage = d_traces_stage;
  const int32_t *drec = rec_xyz;
  if (host_rec) {
    drec = reinterpret_cast<const int32_t *>(tb + o_raw);
    WAVE_TRY_CUDA(cudaMemcpyAsync(tb + o_raw, c->h_rec_raw.data(), (size_t)nrec * 12,
                                  cudaMemcpyHostToDevice, st));
  }

  // Source wavelet for this call's steps, FP64 on the host, stored FP32.
  StepDesc &d = c->host_desc;
  std::memset(&d, 0, sizeof(d));
  if (shot) {
    c->h_wavelet.resize(nsteps);
    const double t0 = shot->t0 < 0 ? 1.0 / shot->f_peak : shot->t0;
    for (int k = 0; k < nsteps; ++k)
      c->h_wavelet[k] = (float)ricker((double)(c->step + k) * c->dt,
                                      shot->f_peak, t0, shot->amp);
    WAVE_TRY_CUDA(cudaMemcpyAsync(c->d_wavelet, c->h_wavelet.data(),
                                  (size_t)nsteps * 4, cudaMemcpyHostToDevice, st));
    d.wavelet = c->d_wavelet;
    d.src_active = 1;
    d.sx = shot->sx;
    d.sy = shot->sy;
    d.sz = shot->sz;
  }
  const RecGeom geom{c->nx, c->ny, c->nz, c->var.tx, c->var.ty, (int)c->grid.x,
                     c->ntiles};
  if (nrec > 0) {
    if ((s = build_receiver_table_device(
             drec, nrec, geom, reinterpret_cast<int *>(tb + o_cnt), c->d_rec_start,
             reinterpret_cast<unsigned long long *>(tb + o_keys), c->d_rec,
             &c->d_desc->error, c->sms, st)))
      return s;
    d.traces = host_traces ? d_traces_stage : traces;
    d.rec = c->d_rec;
    d.rec_start = c->d_rec_start;
    d.nrec = nrec;
  }
  if (c->cpml) {
    // receivers inside the CPML shell are recorded from the shell values
    if (nrec > 0) {
      void *old = c->srec.p;
      if ((s = ensure(c->srec, (size_t)nrec * sizeof(int4), st))) return s;
      if (c->srec.p != old) drop_graphs(c);  // graphs hold the list's address
    }
    WAVE_TRY_CUDA(cudaMemsetAsync(c->d_nsrec, 0, sizeof(int), st));
    if (nrec > 0) {
      rec_shell_kernel<<<std::min(c->sms * 4, (nrec + 255) / 256), 256, 0, st>>>(
          drec, nrec, geom, c->cg.w, (int4 *)c->srec.p, c->d_nsrec);
      WAVE_TRY_CUDA(cudaGetLastError());
    }
  }
  return upload_desc(c);
}

// The part after the steps: the traces' finite check and, for a host
// buffer, their copy (which synchronizes and reports errors).
int propagate_end(wave_ctx *c, int nsteps, int nrec, float *traces, bool host_traces,
                  const float *stage) {
  cudaStream_t st = c->stream;
  if (nrec > 0) {  // NaN / infinity in the traces: WAVE_ENAN at the next sync
    finite_check_kernel<<<c->sms * 4, 256, 0, st>>>(
        c->host_desc.traces, (long long)nsteps * nrec, &c->d_desc->error);
    WAVE_TRY_CUDA(cudaGetLastError());
  }
  if (host_traces) {
    WAVE_TRY_CUDA(cudaMemcpyAsync(traces, stage, (size_t)nsteps * nrec * 4,
                                  cudaMemcpyDeviceToHost, st));
    return read_device_error(c);
  }
  return WAVE_OK;
}

}  // namespace

extern "C" {

int wave_propagate(wave_ctx *c, const wave_shot *shot, int nsteps,
                   const int32_t *rec_xyz, int nrec, float *traces) {
  bool host_traces;
  float *stage;
  int s = propagate_begin(c, shot, nsteps, rec_xyz, nrec, traces, host_traces, stage);
  if (s || nsteps == 0) return s;
  int early = 0;
  if (c->upload_pending) {
    if (c->at_rest && shot)
      early = steps_while_loading(c, shot->sz, nsteps);
    else if ((s = wait_model(c)))
      return s;
    if (early < 0) return early;
  }
  if ((s = run_steps(c, nsteps - early))) return s;
  return propagate_end(c, nsteps, nrec, traces, host_traces, stage);
}

}  // extern "C"

// Index of the scale slot of the field holding u (which = 0) or u_prev (1).
static int field_slot(const wave_ctx *c, int which) {
  return (int)((c->step + (which ? 3 : 0)) & 3);
}

template <class T>
static void launch_from_stored(const wave_ctx *c, float *dst, const void *src,
                               int slot) {
  from_stored_kernel<T><<<c->sms * 4, 256, 0, c->stream>>>(
      dst, reinterpret_cast<const T *>(src), c->pxu, c->nx,
      (long long)c->ny * c->nz, c->d_desc, slot);
}

template <class T>
static void launch_to_stored(const wave_ctx *c, void *dst, const float *src,
                             int slot) {
  to_stored_kernel<T><<<c->sms * 4, 256, 0, c->stream>>>(
      reinterpret_cast<T *>(dst), c->pxu, src, c->nx,
      (long long)c->ny * c->nz, c->d_desc, slot);
}

extern "C" {

int wave_get_field(const wave_ctx *c, int which, float *out) {
  if (!c || !out || (which != 0 && which != 1)) return WAVE_EINVAL;
  const void *src = c->buf[which == 0 ? c->cur : (c->cur ^ 1)];
  const bool host_out = !is_device_ptr(out);
  if (c->storage == WAVE_STORAGE_F32) {
    WAVE_TRY_CUDA(cudaMemcpy2DAsync(out, (size_t)c->nx * 4, src,
                                    (size_t)c->px * 4, (size_t)c->nx * 4,
                                    (size_t)c->ny * c->nz, cudaMemcpyDefault,
                                    c->stream));
    if (host_out) return read_device_error(const_cast<wave_ctx *>(c));
    return WAVE_OK;
  }
  // 16-bit storage: expand to FP32 with the field's scale.
  const size_t n = (size_t)c->nx * c->ny * c->nz;
  float *dst = out;
  if (host_out) WAVE_TRY_CUDA(cudaMalloc((void **)&dst, n * 4));
  if (c->storage == WAVE_STORAGE_BF16)
    launch_from_stored<__nv_bfloat16>(c, dst, src, field_slot(c, which));
  else
    launch_from_stored<__half>(c, dst, src, field_slot(c, which));
  cudaError_t e = cudaGetLastError();
  if (host_out) {
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(out, dst, n * 4, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(dst);
  }
  if (e != cudaSuccess) return cuda_status(e);
  return host_out ? read_device_error(const_cast<wave_ctx *>(c)) : WAVE_OK;
}

}  // extern "C"

// Scale exponent for a field whose largest magnitude is m: stored values
// are at most 2^14 in magnitude.
static int scale_exponent(float m) {
  if (!(m > 0.f) || !std::isfinite(m)) return 0;
  int e;
  std::frexp(m, &e);
  return e - 14;
}

static int set_state_16(wave_ctx *c, const float *u, const float *u_prev,
                        int64_t step) {
  const size_t n = (size_t)c->nx * c->ny * c->nz;
  cudaStream_t st = c->stream;
  const float *src[2] = {u, u_prev};
  float *tmp[2] = {nullptr, nullptr};
  int status = WAVE_OK;
  for (int b = 0; b < 2 && status == WAVE_OK; ++b) {
    if (!is_device_ptr(src[b])) {
      cudaError_t e = cudaMalloc((void **)&tmp[b], n * 4);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(tmp[b], src[b], n * 4, cudaMemcpyHostToDevice, st);
      if (e != cudaSuccess) status = cuda_status(e);
      src[b] = tmp[b];
    }
  }
  unsigned mb[2] = {0, 0};
  if (status == WAVE_OK) {
    unsigned *dm = reinterpret_cast<unsigned *>(c->d_scratch);
    cudaError_t e = cudaMemsetAsync(dm, 0, 8, st);
    for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
      absmax_kernel<<<c->sms * 4, 256, 0, st>>>(src[b], (long long)n, dm + b);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(mb, dm, 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) status = cuda_status(e);
  }
  if (status == WAVE_OK) {
    float m[2];
    std::memcpy(m, mb, 8);
    if (!std::isfinite(m[0]) || !std::isfinite(m[1])) status = WAVE_EINVAL;
    // Scale state: u at absolute step `step`, u_prev at step - 1.
    int exps[4] = {0, 0, 0, 0};
    unsigned maxb[4] = {0, 0, 0, 0};
    exps[step & 3] = scale_exponent(m[0]);
    exps[(step + 3) & 3] = scale_exponent(m[1]);
    maxb[step & 3] = mb[0];
    maxb[(step + 3) & 3] = mb[1];
    std::memcpy(c->scale_image, exps, 16);
    std::memcpy(c->scale_image + 16, maxb, 16);
    cudaError_t e = cudaSuccess;
    if (status == WAVE_OK)
      e = cudaMemcpyAsync(reinterpret_cast<char *>(c->d_desc) +
                              offsetof(StepDesc, exps),
                          c->scale_image, 32, cudaMemcpyHostToDevice, st);
    c->cur = 0;
    c->step = step;
    for (int b = 0; b < 2 && e == cudaSuccess && status == WAVE_OK; ++b) {
      const int slot = b == 0 ? (int)(step & 3) : (int)((step + 3) & 3);
      if (c->storage == WAVE_STORAGE_BF16)
        launch_to_stored<__nv_bfloat16>(c, c->buf[b], src[b], slot);
      else
        launch_to_stored<__half>(c, c->buf[b], src[b], slot);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess && status == WAVE_OK) status = cuda_status(e);
  }
  cudaFree(tmp[0]);
  cudaFree(tmp[1]);
  return status;
}

extern "C" {

int wave_set_state(wave_ctx *c, const float *u, const float *u_prev,
                   int64_t step) {
  if (!c || !u || !u_prev || step < 0) return WAVE_EINVAL;
  int ws = wait_model(c);  // the state is no longer at rest
  if (ws) return ws;
  c->at_rest = false;
  WAVE_TRY_CUDA(cudaMemsetAsync(&c->d_desc->error, 0, sizeof(int), c->stream));
  if (c->storage != WAVE_STORAGE_F32) return set_state_16(c, u, u_prev, step);
  c->cur = 0;
  const float *src[2] = {u, u_prev};
  for (int b = 0; b < 2; ++b)
    WAVE_TRY_CUDA(cudaMemcpy2DAsync(c->buf[b], (size_t)c->px * 4, src[b],
                                    (size_t)c->nx * 4, (size_t)c->nx * 4,
                                    (size_t)c->ny * c->nz, cudaMemcpyDefault,
                                    c->stream));
  c->step = step;
  int zs = zero_cpml(c);
  if (zs) return zs;
  if (!is_device_ptr(u) || !is_device_ptr(u_prev))
    WAVE_TRY_CUDA(cudaStreamSynchronize(c->stream));
  return WAVE_OK;
}

int wave_get_step(const wave_ctx *c, int64_t *step) {
  if (!c || !step) return WAVE_EINVAL;
  *step = c->step;
  return WAVE_OK;
}

int wave_reset(wave_ctx *c) {
  if (!c) return WAVE_EINVAL;
  const size_t bytes = field_bytes(c);
  // the state is replaced: an error recorded for the old one no longer holds
  WAVE_TRY_CUDA(cudaMemsetAsync(&c->d_desc->error, 0, sizeof(int), c->stream));
  WAVE_TRY_CUDA(cudaMemsetAsync(c->buf[0], 0, bytes, c->stream));
  WAVE_TRY_CUDA(cudaMemsetAsync(c->buf[1], 0, bytes, c->stream));
  WAVE_TRY_CUDA(cudaMemsetAsync(
      reinterpret_cast<char *>(c->d_desc) + offsetof(StepDesc, exps), 0,
      sizeof(int) * 4 + sizeof(unsigned) * 4, c->stream));
  c->cur = 0;
  c->step = 0;
  c->at_rest = true;
  return zero_cpml(c);
}

int wave_set_cpml(wave_ctx *c, int npml, double R, double f_cps) {
  if (!c || npml < 0) return WAVE_EINVAL;
  // the layer's profile needs the model's largest velocity
  int ms = finish_model(c);
  if (ms || (ms = wait_model(c))) return ms;
  if (npml == 0) {
    WAVE_TRY_CUDA(cudaStreamSynchronize(c->stream));
    free_cpml(c);
  } else {
    if (2 * npml > std::min(c->nx, std::min(c->ny, c->nz)) || !(R > 0.0 && R < 1.0) ||
        !(f_cps >= 0.0) || !std::isfinite(f_cps))
      return WAVE_EINVAL;
    // the axis kernels index one grid row of blocks per y or z
    if (c->ny > 65535 || c->nz > 65535) return WAVE_ENOTSUP;
    WAVE_TRY_CUDA(cudaStreamSynchronize(c->stream));
    free_cpml(c);
    CpmlGeom &g = c->cg;
    g.nx = c->nx;
    g.ny = c->ny;
    g.nz = c->nz;
    g.px = c->px;
    g.pxu = c->pxu;
    g.npml = npml;
    g.w = npml + 4;
    const size_t sl[3] = {2ull * npml * c->ny * c->nz, 2ull * npml * c->nz * c->nx,
                          2ull * npml * c->ny * c->nx};
    auto dalloc = [&](void **p, size_t bytes) -> int {
      cudaError_t e = cudaMalloc(p, std::max<size_t>(bytes, 256));
      if (e != cudaSuccess) return cuda_status(e);
      c->cpml_mem.push_back(*p);
      return WAVE_OK;
    };
    int e;
    const int dims[3] = {c->nx, c->ny, c->nz};
    const double hs[3] = {c->dx, c->dy, c->dz};
    for (int ax = 0; ax < 3; ++ax) {
      if ((e = dalloc((void **)&g.psi[ax], sl[ax] * 4)) ||
          (e = dalloc((void **)&g.zeta[ax], sl[ax] * 4)) ||
          (e = dalloc((void **)&g.bprof[ax], dims[ax] * 4)) ||
          (e = dalloc((void **)&g.aprof[ax], dims[ax] * 4))) {
        free_cpml(c);
        return e;
      }
      // Profiles (FP64, stored FP32) and derivative coefficients.
      std::vector<float> hb(dims[ax]), ha(dims[ax]);
      cpml_profile(dims[ax], npml, R, f_cps, c->vmax, hs[ax], c->dt, hb.data(), ha.data());
      // the unrolled segment kernels where they apply (cpml_seg_fits), with
      // the field and slab steps along the axis (the wavefields' pitch is at
      // least that of v^2 dt^2)
      const long long fstep[3] = {1, c->pxu, (long long)c->ny * c->pxu};
      const long long sstep[3] = {(long long)c->nz * c->ny, (long long)c->nz * c->nx,
                                  (long long)c->ny * c->nx};
      if (cpml_seg_fits(npml, dims[ax], fstep[ax], sstep[ax])) {
        c->cpml_seg_axes |= 1 << ax;
        if (npml == 8)
          cpml_side_prof(hb.data(), ha.data(), dims[ax], c->prof8[ax]);
        else
          cpml_side_prof(hb.data(), ha.data(), dims[ax], c->prof16[ax]);
      }
      WAVE_TRY_CUDA(cudaMemcpy((void *)g.bprof[ax], hb.data(), dims[ax] * 4,
                               cudaMemcpyHostToDevice));
      WAVE_TRY_CUDA(cudaMemcpy((void *)g.aprof[ax], ha.data(), dims[ax] * 4,
                               cudaMemcpyHostToDevice));
      cpml_axis_coefs(g, ax, hs[ax]);
    }
    if (!c->d_nsrec) WAVE_TRY_CUDA(cudaMalloc((void **)&c->d_nsrec, sizeof(int)));
    WAVE_TRY_CUDA(cudaMemset(c->d_nsrec, 0, sizeof(int)));
    c->cpml = true;
    if ((e = zero_cpml(c))) return e;
  }
  drop_graphs(c);  // captured graphs hold the previous step sequence
  return WAVE_OK;
}

int wave_synchronize(wave_ctx *c) {
  if (!c) return WAVE_EINVAL;
  return read_device_error(c);
}

int wave_get_launch_info(const wave_ctx *c, int *tile_x, int *tile_y,
                         int *z_chunk, int *grid_ctas, int *ctas_per_sm) {
  if (!c) return WAVE_EINVAL;
  if (tile_x) *tile_x = c->var.tx;
  if (tile_y) *tile_y = c->var.ty;
  if (z_chunk) *z_chunk = c->zchunk;
  if (grid_ctas) *grid_ctas = (int)(c->grid.x * c->grid.y * c->grid.z);
  if (ctas_per_sm) *ctas_per_sm = c->ctas_per_sm;
  return WAVE_OK;
}

int wave_selftest_wait(int64_t limit_ns, void *stream) {
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  limit_ns = std::min<int64_t>(std::max<int64_t>(limit_ns, 1000000), 10000000000ll);
  int *d = nullptr;
  WAVE_TRY_CUDA(cudaMalloc(&d, sizeof(int)));
  int h = 0;
  cudaError_t e = cudaMemsetAsync(d, 0, sizeof(int), st);
  if (e == cudaSuccess) {
    selftest_wait_kernel<<<1, 1, 0, st>>>((uint64_t)limit_ns, d);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&h, d, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(d);
  if (e != cudaSuccess) return cuda_status(e);
  return h == 2 ? WAVE_ETIMEOUT : WAVE_ECUDA;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Adjoint gradient (wave_adjoint, wave_gradient).
namespace {

template <int kMode>
void launch_mode(const wave_ctx *c, cudaStream_t st, dim3 grid, const CUtensorMap &tu,
                 const CUtensorMap &tup, const SweepArgs &a) {
  launch_pdl(wave_sweep_kernel<Cfg0, false, kMode>, grid, Cfg0::THREADS,
             Cfg0::SMEM_BYTES, st, tu, tup, c->tm_c, a);
}

// The backward pass's second stream and its events, released on scope exit.
struct GradStreams {
  cudaStream_t rs = nullptr;      // segment recomputes
  cudaEvent_t start = nullptr;    // the backward's inputs are ready
  cudaEvent_t rec_done[2] = {};   // recompute into D buffer slot s finished
  cudaEvent_t adj_done[2] = {};   // adjoint steps reading slot s finished
  ~GradStreams() {
    if (rs) cudaStreamDestroy(rs);
    for (cudaEvent_t e : {start, rec_done[0], rec_done[1], adj_done[0], adj_done[1]})
      if (e) cudaEventDestroy(e);
  }
  int init() {
    WAVE_TRY_CUDA(cudaStreamCreateWithFlags(&rs, cudaStreamNonBlocking));
    for (cudaEvent_t *e : {&start, &rec_done[0], &rec_done[1], &adj_done[0], &adj_done[1]})
      WAVE_TRY_CUDA(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
    return WAVE_OK;
  }
};

// z-layer plan of a gradient sweep mode: the u-only stages that refill the
// register queue weigh less against a stage that also moves D and the
// gradient partial, so those sweeps plan with a smaller preroll (more,
// shorter layers fill the CTA places better).
dim3 plan_mode(const wave_ctx *c, double preroll, SweepArgs &a) {
  int layers[kMaxLayers];
  const int nl = plan_layers(c->nz, (long long)c->ntiles,
                             (long long)c->sms * c->ctas_per_sm, preroll, layers);
  set_layers(a, layers, nl);
  return dim3(c->grid.x, c->grid.y, (unsigned)nl);
}

// r = traces - observed; misfit += 1/2 sum r^2 in FP64.
__global__ void residual_kernel(const float *tr, const float *obs, float *r,
                                long long n, double *misfit) {
  double local = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const float d = tr[i] - obs[i];
    r[i] = d;
    local += (double)d * (double)d;
  }
  for (int o = 16; o > 0; o >>= 1)
    local += __shfl_xor_sync(0xffffffffu, local, o);
  if ((threadIdx.x & 31) == 0 && local != 0.0) atomicAdd(misfit, 0.5 * local);
}

// Injection rows in adjoint launch order: row a = resid row N-1-a, row N = 0.
__global__ void reverse_rows_kernel(const float *res, float *inj, int N,
                                    int nrec) {
  const long long total = (long long)(N + 1) * nrec;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
       i < total; i += (long long)gridDim.x * blockDim.x) {
    const int a = (int)(i / nrec), r = (int)(i - (long long)a * nrec);
    inj[i] = a < N ? res[(long long)(N - 1 - a) * nrec + r] : 0.f;
  }
}

// FP64 time sum += the double-float partial hi + lo (exact in FP64), and the
// partial restarts from zero; 4 points per thread and iteration (n4 groups:
// the fields' rows are multiples of 4 elements).
__global__ void grad_fold_kernel(double *gacc, float *ghi, float *glo, long long n4) {
  float4 *h4 = reinterpret_cast<float4 *>(ghi), *l4 = reinterpret_cast<float4 *>(glo);
  double2 *a2 = reinterpret_cast<double2 *>(gacc);
  const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n4;
       i += (long long)gridDim.x * blockDim.x) {
    const float4 h = h4[i], l = l4[i];
    double2 a0 = a2[2 * i], a1 = a2[2 * i + 1];
    a0.x += (double)h.x + (double)l.x;
    a0.y += (double)h.y + (double)l.y;
    a1.x += (double)h.z + (double)l.z;
    a1.y += (double)h.w + (double)l.w;
    a2[2 * i] = a0;
    a2[2 * i + 1] = a1;
    h4[i] = zero;
    l4[i] = zero;
  }
}

// Steps per FP64 fold of the gradient's time sum, counted in absolute steps
// so the sum's rounding does not depend on the checkpoint interval. The
// double-float partial carries the rounding errors of its hi word in its lo
// word, which after k steps is at most about k 2^-24 of the sum and rounds at
// 2^-24 of itself: over a block of B steps at most about B^2 2^-49 of the
// sum, 2^-33 for B = 256, far below the FP32 rounding of the gradient (2^-24)
// and usually much less; each fold reads and writes 32 bytes per point, so
// fewer folds save bandwidth (25 folds of 132 us at 256^3 for 800 steps with
// blocks of 32, 3 with blocks of 256).
constexpr int kGradFold = 256;

// dJ/dm = sum / (m^2 dt^2) = sum * dt^2 / c^2 with c = m dt^2; dense output,
// one row (y, z) per block iteration. The FP64 time sum is rounded to FP32
// once and scaled in FP32 by dt^2 / c^2 (a few FP32 roundings, within 2 ulp
// of the FP32 output): this GPU's FP64 rate is a small fraction of its FP32
// rate, and with FP64 products, an FP64 division and a 64-bit integer
// division (of the flat index by nx) per point this kernel took 738 us at
// 256^3. c^2 outside the FP32 normal range (not reached by a model that
// passes wave_create) is scaled in FP64.
__global__ void grad_assemble_kernel(const double *gacc, const float *c,
                                     float *grad, int nx, int px,
                                     long long rows, double dt2) {
  const float dt2f = (float)dt2;
  for (long long r = blockIdx.x; r < rows; r += gridDim.x) {
    const double *ga = gacc + r * px;
    const float *cr = c + r * px;
    float *gr = grad + r * nx;
    for (int x = threadIdx.x; x < nx; x += blockDim.x) {
      const float cv = cr[x];
      const float q = cv * cv;
      if (q > 1e-30f && q < 1e30f)
        gr[x] = (float)ga[x] * (dt2f * __frcp_rn(q));
      else
        gr[x] = (float)(ga[x] * dt2 / ((double)cv * (double)cv));
    }
  }
}

struct DevFree {  // frees the registered device buffers on scope exit
  std::vector<void *> ptrs;
  ~DevFree() {
    for (void *p : ptrs) cudaFree(p);
  }
  template <class T>
  int alloc(T **p, size_t bytes) {
    *p = nullptr;
    cudaError_t e = cudaMalloc((void **)p, std::max<size_t>(bytes, 256));
    if (e != cudaSuccess) return cuda_status(e);
    ptrs.push_back(*p);
    return WAVE_OK;
  }
};

int gradient_impl(wave_ctx *c, const wave_shot *shot, int N,
                  const int32_t *rec_xyz, int nrec, const float *data,
                  bool data_is_resid, int K, double *misfit, float *grad,
                  float *traces_out) {
  if (!c || N < 1 || nrec < 0 || K < 1 || !grad) return WAVE_EINVAL;
  if (nrec > 0 && (!rec_xyz || !data)) return WAVE_EINVAL;
  if (c->storage != WAVE_STORAGE_F32 ||
      c->var.func != reinterpret_cast<const void *>(&wave_sweep_kernel<Cfg0>))
    return WAVE_ENOTSUP;
  int ms = finish_model(c);
  if (ms || (ms = wait_model(c))) return ms;
  cudaStream_t st = c->stream;
  const size_t fe = (size_t)c->px * c->ny * c->nz;  // field elements
  const size_t fb = fe * 4;
  const int ncp = (N + K - 1) / K;
  const size_t tn = (size_t)N * nrec;
  DevFree mem;
  float *ckpt, *dbuf, *padj[2], *trd, *res, *inj, *wl, *ghi, *glo;
  double *gacc, *dmis;
  StepDesc *dadj, *dfwd;
  int e;
  // two D buffers (slots) when there are several segments: the recompute of
  // one segment runs beside the adjoint steps of the next. A segment's
  // recompute steps its checkpoint's two fields (and layer slabs) in place:
  // each checkpoint is read by that recompute alone, and the forward keeps
  // its own fields, so the last segment's recompute can also run beside the
  // forward's last segment.
  const int nslot = ncp > 1 ? 2 : 1;
  if ((e = mem.alloc(&ckpt, fb * 2 * ncp)) || (e = mem.alloc(&dbuf, fb * K * nslot)) ||
      (e = mem.alloc(&padj[0], fb)) || (e = mem.alloc(&padj[1], fb)) ||
      (e = mem.alloc(&trd, tn * 4)) || (e = mem.alloc(&res, tn * 4)) ||
      (e = mem.alloc(&inj, (tn + nrec) * 4)) || (e = mem.alloc(&wl, (size_t)N * 4)) ||
      (e = mem.alloc(&gacc, fe * 8)) || (e = mem.alloc(&dmis, 8)) ||
      (e = mem.alloc(&ghi, fb)) || (e = mem.alloc(&glo, fb)) ||
      (e = mem.alloc(&dadj, sizeof(StepDesc))) ||
      (e = mem.alloc(&dfwd, sizeof(StepDesc))))
    return e;
  // With the CPML layer: the memory variables psi, zeta (per axis) are saved
  // with each checkpoint, the recompute steps the saved copies in place, and
  // the adjoint carries its nu, mu slabs.
  const CpmlGeom &cg = c->cg;
  size_t sl[3] = {0, 0, 0};
  float *ckpt_l = nullptr, *nus[3] = {}, *mus[3] = {};
  if (c->cpml) {
    sl[0] = 2ull * cg.npml * c->ny * c->nz;
    sl[1] = 2ull * cg.npml * c->nz * c->nx;
    sl[2] = 2ull * cg.npml * c->ny * c->nx;
    if ((e = mem.alloc(&ckpt_l, (sl[0] + sl[1] + sl[2]) * 2 * 4 * ncp))) return e;
    for (int ax = 0; ax < 3; ++ax)
      if ((e = mem.alloc(&nus[ax], sl[ax] * 4)) || (e = mem.alloc(&mus[ax], sl[ax] * 4)))
        return e;
  }
  // the layer slabs held by a segment's checkpoint (per axis psi, then zeta)
  auto layer_of = [&](int sgm) {
    CpmlGeom gg = cg;
    float *q = ckpt_l + (sl[0] + sl[1] + sl[2]) * 2 * sgm;
    for (int ax = 0; ax < 3; ++ax) {
      gg.psi[ax] = q;
      gg.zeta[ax] = q + sl[ax];
      q += 2 * sl[ax];
    }
    return gg;
  };
  // copies the context's memory variables into a segment's checkpoint
  auto layer_ckpt = [&](int sgm, cudaStream_t cs) -> int {
    const CpmlGeom gg = layer_of(sgm);
    for (int ax = 0; ax < 3; ++ax) {
      WAVE_TRY_CUDA(cudaMemcpyAsync(gg.psi[ax], cg.psi[ax], sl[ax] * 4,
                                    cudaMemcpyDeviceToDevice, cs));
      WAVE_TRY_CUDA(cudaMemcpyAsync(gg.zeta[ax], cg.zeta[ax], sl[ax] * 4,
                                    cudaMemcpyDeviceToDevice, cs));
    }
    return WAVE_OK;
  };
  GradStreams gs;
  if ((e = gs.init())) return e;
  const void *fns[3] = {
      reinterpret_cast<const void *>(&wave_sweep_kernel<Cfg0, false, kModeStoreD>),
      reinterpret_cast<const void *>(&wave_sweep_kernel<Cfg0, false, kModeInject>),
      reinterpret_cast<const void *>(
          &wave_sweep_kernel<Cfg0, false, kModeInject | kModeGradAcc>)};
  for (const void *f : fns)
    WAVE_TRY_CUDA(cudaFuncSetAttribute(
        f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg0::SMEM_BYTES));
  // tensor maps (halo and tile boxes) of a field
  auto field_maps = [&](const void *f, CUtensorMap *halo, CUtensorMap *tile) -> int {
    int me = make_map(halo, f, c, c->var.tx + 2 * c->var.halo_x, c->var.ty + 2 * kR,
                      CU_TENSOR_MAP_DATA_TYPE_FLOAT32, c->pxu, 4);
    if (!me)
      me = make_map(tile, f, c, c->var.tx, c->var.ty, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, c->pxu,
                    4);
    return me;
  };
  CUtensorMap ahalo[2], atile[2];
  for (int b = 0; b < 2; ++b)
    if ((e = field_maps(padj[b], &ahalo[b], &atile[b]))) return e;

  // Layer plans of the recompute (D stored) and adjoint sweeps. Preroll
  // weights timed on 256^3 x 800 steps, checkpoint every 40 (wave_gradient,
  // best of 4): 4/4 (the forward plan) 0.1864 s, 2/2 0.1827 s, 3.2/1.8
  // 0.1866, 2/1 0.1909, 1/1 0.1907, 4/1 0.1949 (bitwise equal gradients:
  // the plan only regroups the planes). GBWAVE_GRAD_PREROLL=d,a overrides.
  double pre_d = 2.0, pre_a = 2.0;
  if (const char *gp = std::getenv("GBWAVE_GRAD_PREROLL"))
    std::sscanf(gp, "%lf,%lf", &pre_d, &pre_a);
  SweepArgs args_d = c->args, args_a = c->args;
  const dim3 grid_d = plan_mode(c, pre_d, args_d);
  const dim3 grid_a = plan_mode(c, pre_a, args_a);

  // Descriptor of the recompute (source, no receivers).
  std::vector<float> hw(N, 0.f);
  StepDesc hf{}, ha{};
  if (shot) {
    const double t0 = shot->t0 < 0 ? 1.0 / shot->f_peak : shot->t0;
    for (int n = 0; n < N; ++n)
      hw[n] = (float)ricker(n * c->dt, shot->f_peak, t0, shot->amp);
    hf.wavelet = wl;
    hf.src_active = 1;
    hf.sx = shot->sx;
    hf.sy = shot->sy;
    hf.sz = shot->sz;
  }
  WAVE_TRY_CUDA(cudaMemcpyAsync(wl, hw.data(), (size_t)N * 4,
                                cudaMemcpyHostToDevice, st));
  WAVE_TRY_CUDA(cudaMemcpyAsync(dfwd, &hf, sizeof(hf), cudaMemcpyHostToDevice, st));

  // Recompute of a segment's forward steps from its checkpoint on stream
  // rs, keeping D^n = C L u^n + source (+ the layer's term) for n in
  // [s0, s1) in the segment's D slot.
  auto dslot_of = [&](int sgm) {
    return dbuf + (size_t)(nslot == 2 ? (sgm & 1) : 0) * K * fe;
  };
  auto recompute = [&](int sgm, cudaStream_t rs) -> int {
    const int s0 = sgm * K, s1 = std::min(N, s0 + K);
    float *dslot = dslot_of(sgm);
    // the checkpoint's fields: rbuf[0] = u^{s0}, rbuf[1] = u^{s0-1}
    float *rbuf[2] = {ckpt + (size_t)2 * sgm * fe, ckpt + (size_t)(2 * sgm + 1) * fe};
    CUtensorMap rhalo[2], rtile[2];
    for (int b = 0; b < 2; ++b) {
      const int me = field_maps(rbuf[b], &rhalo[b], &rtile[b]);
      if (me) return me;
    }
    const CpmlGeom rg = c->cpml ? layer_of(sgm) : cg;
    int cur = 0;
    for (int n = s0; n < s1; ++n) {
      SweepArgs a = args_d;
      a.desc = dfwd;
      a.koff = n;
      a.unext = rbuf[cur ^ 1];
      a.dout = dslot + (size_t)(n - s0) * fe;
      launch_mode<kModeStoreD>(c, rs, grid_d, rhalo[cur], rtile[cur ^ 1], a);
      if (c->cpml)  // the layer's terms, into u^{n+1} and D^n
        launch_cpml_forward<float, true>(c, rg, rs, rbuf[cur], rbuf[cur ^ 1], a.dout, nullptr,
                                         0);
      cur ^= 1;
    }
    if (nslot == 2) WAVE_TRY_CUDA(cudaEventRecord(gs.rec_done[sgm & 1], rs));
    return WAVE_OK;
  };

  // Forward run from rest, prepared once for all N steps (receiver table,
  // wavelet, descriptor), with a checkpoint (u^{sK}, u^{sK-1}) and the
  // layer's memory variables before each segment. The last segment's
  // recompute starts beside the forward's last segment.
  if ((e = wave_reset(c))) return e;
  bool host_tr;
  float *stage;
  if ((e = propagate_begin(c, shot, N, rec_xyz, nrec, nrec ? trd : nullptr, host_tr, stage)))
    return e;
  for (int sgm = 0; sgm < ncp; ++sgm) {
    WAVE_TRY_CUDA(cudaMemcpyAsync(ckpt + (size_t)2 * sgm * fe, c->buf[c->cur],
                                  fb, cudaMemcpyDeviceToDevice, st));
    WAVE_TRY_CUDA(cudaMemcpyAsync(ckpt + (size_t)(2 * sgm + 1) * fe,
                                  c->buf[c->cur ^ 1], fb,
                                  cudaMemcpyDeviceToDevice, st));
    if (c->cpml && (e = layer_ckpt(sgm, st))) return e;
    if (sgm == ncp - 1 && nslot == 2) {
      WAVE_TRY_CUDA(cudaEventRecord(gs.start, st));
      WAVE_TRY_CUDA(cudaStreamWaitEvent(gs.rs, gs.start, 0));
      if ((e = recompute(sgm, gs.rs))) return e;
    }
    if ((e = run_steps(c, std::min(K, N - sgm * K)))) return e;
  }
  if ((e = propagate_end(c, N, nrec, nrec ? trd : nullptr, false, nullptr))) return e;

  // Residual (dJ/dtraces) and, for the L2 misfit, its FP64 sum.
  if (nrec > 0) {
    WAVE_TRY_CUDA(cudaMemcpyAsync(res, data, tn * 4, cudaMemcpyDefault, st));
    if (!data_is_resid) {
      WAVE_TRY_CUDA(cudaMemsetAsync(dmis, 0, 8, st));
      residual_kernel<<<c->sms * 4, 256, 0, st>>>(trd, res, res, (long long)tn,
                                                  dmis);
      WAVE_TRY_CUDA(cudaGetLastError());
    }
    reverse_rows_kernel<<<c->sms * 4, 256, 0, st>>>(res, inj, N, nrec);
    WAVE_TRY_CUDA(cudaGetLastError());
  } else if (!data_is_resid) {
    WAVE_TRY_CUDA(cudaMemsetAsync(dmis, 0, 8, st));
  }

  // Descriptor of the adjoint (receiver injections, no source).
  if (nrec > 0) {
    ha.inj_val = inj;
    ha.inj = c->d_rec;  // receiver table of the forward run
    ha.inj_start = c->d_rec_start;
    ha.ninj = nrec;
  }
  WAVE_TRY_CUDA(cudaMemcpyAsync(dadj, &ha, sizeof(ha), cudaMemcpyHostToDevice, st));
  WAVE_TRY_CUDA(cudaMemsetAsync(padj[0], 0, fb, st));
  WAVE_TRY_CUDA(cudaMemsetAsync(padj[1], 0, fb, st));
  WAVE_TRY_CUDA(cudaMemsetAsync(gacc, 0, fe * 8, st));
  WAVE_TRY_CUDA(cudaMemsetAsync(ghi, 0, fb, st));
  WAVE_TRY_CUDA(cudaMemsetAsync(glo, 0, fb, st));
  for (int ax = 0; ax < 3 && c->cpml; ++ax) {
    WAVE_TRY_CUDA(cudaMemsetAsync(nus[ax], 0, sl[ax] * 4, st));
    WAVE_TRY_CUDA(cudaMemsetAsync(mus[ax], 0, sl[ax] * 4, st));
  }

  // Adjoint launch a = N - k computes p^k from p^{k+1} (padj[ca]) and
  // p^{k+2}; with kModeGradAcc it adds p^{k+1} D^k to the double-float
  // partial, which is folded into the FP64 sum after every step k that is
  // a multiple of kGradFold (the last fold is after k = 0).
  int ca = 0;
  auto adjoint_step = [&](int k, const float *dsrc) {
    SweepArgs a = args_a;
    a.desc = dadj;
    a.koff = N - k;
    a.unext = padj[ca ^ 1];
    a.dsrc = dsrc;
    a.ghi = ghi;
    a.glo = glo;
    if (dsrc)
      launch_mode<kModeInject | kModeGradAcc>(c, st, grid_a, ahalo[ca], atile[ca ^ 1], a);
    else
      launch_mode<kModeInject>(c, st, grid_a, ahalo[ca], atile[ca ^ 1], a);
    if (c->cpml) {  // the layer's adjoint terms, from p^{k+1} into p^k
      const float *p1 = padj[ca];
      float *p0 = padj[ca ^ 1];
      launch_cpml_adjoint_axis<0>(c, st, p1, p0, nus[0], mus[0]);
      launch_cpml_adjoint_axis<1>(c, st, p1, p0, nus[1], mus[1]);
      launch_cpml_adjoint_axis<2>(c, st, p1, p0, nus[2], mus[2]);
    }
    if (dsrc && k % kGradFold == 0)
      grad_fold_kernel<<<c->sms * 4, 256, 0, st>>>(gacc, ghi, glo, (long long)(fe / 4));
    ca ^= 1;
  };
  adjoint_step(N, nullptr);  // p^N (no D^N term)
  // Segments from the last: the recompute of a segment (stream gs.rs, D into
  // slot sgm & 1) runs beside the adjoint steps of the segment after it
  // (stream st), which read the other slot. A recompute waits for the
  // adjoint steps that last read its slot; the adjoint steps wait for their
  // recompute. The sweeps of one 256^3 step fill the GPU's CTA places less
  // than once, so two chains of launches keep it busier. With one segment
  // everything runs on st.
  for (int sgm = ncp - 1; sgm >= 0; --sgm) {
    const int s0 = sgm * K, s1 = std::min(N, s0 + K), slot = sgm & 1;
    if (nslot == 1) {
      if ((e = recompute(sgm, st))) return e;
    } else {
      if (sgm < ncp - 1) {  // the last segment's recompute is under way
        if (sgm + 2 < ncp) WAVE_TRY_CUDA(cudaStreamWaitEvent(gs.rs, gs.adj_done[slot], 0));
        if ((e = recompute(sgm, gs.rs))) return e;
      }
      WAVE_TRY_CUDA(cudaStreamWaitEvent(st, gs.rec_done[slot], 0));
    }
    float *dslot = dslot_of(sgm);
    for (int k = s1 - 1; k >= s0; --k)
      adjoint_step(k, dslot + (size_t)(k - s0) * fe);
    if (nslot == 2) WAVE_TRY_CUDA(cudaEventRecord(gs.adj_done[slot], st));
  }
  WAVE_TRY_CUDA(cudaGetLastError());

  // Gradient, traces, misfit.
  const size_t ne = (size_t)c->nx * c->ny * c->nz;
  float *gout = grad;
  const bool host_grad = !is_device_ptr(grad);
  if (host_grad && (e = mem.alloc(&gout, ne * 4))) return e;
  grad_assemble_kernel<<<c->sms * 4, 256, 0, st>>>(
      gacc, c->c, gout, c->nx, c->px, (long long)c->ny * c->nz, c->dt * c->dt);
  WAVE_TRY_CUDA(cudaGetLastError());
  if (host_grad)
    WAVE_TRY_CUDA(cudaMemcpyAsync(grad, gout, ne * 4, cudaMemcpyDeviceToHost, st));
  if (traces_out && nrec > 0)
    WAVE_TRY_CUDA(cudaMemcpyAsync(traces_out, trd, tn * 4, cudaMemcpyDefault, st));
  double hm = 0.0;
  if (!data_is_resid)
    WAVE_TRY_CUDA(cudaMemcpyAsync(&hm, dmis, 8, cudaMemcpyDeviceToHost, st));
  int errs[2] = {0, 0};
  WAVE_TRY_CUDA(cudaMemcpyAsync(&errs[0], &dfwd->error, 4, cudaMemcpyDeviceToHost, st));
  WAVE_TRY_CUDA(cudaMemcpyAsync(&errs[1], &dadj->error, 4, cudaMemcpyDeviceToHost, st));
  WAVE_TRY_CUDA(cudaStreamSynchronize(st));
  if (misfit && !data_is_resid) *misfit = hm;
  // errors of the forward run (a timeout, or NaN in its traces), read before
  // the reset clears them
  const int ferr = read_device_error(c);
  if ((e = wave_reset(c))) return e;
  if (ferr) return ferr;
  if (errs[0] || errs[1]) return device_error_status(errs[0] ? errs[0] : errs[1]);
  return WAVE_OK;
}

}  // namespace

extern "C" int wave_adjoint(wave_ctx *ctx, const wave_shot *shot, int nsteps,
                            const int32_t *rec_xyz, int nrec,
                            const float *resid, int ckpt_every, float *grad_v2,
                            float *traces) {
  return gradient_impl(ctx, shot, nsteps, rec_xyz, nrec, resid, true,
                       ckpt_every, nullptr, grad_v2, traces);
}

extern "C" int wave_gradient(wave_ctx *ctx, const wave_shot *shot, int nsteps,
                             const int32_t *rec_xyz, int nrec,
                             const float *observed, int ckpt_every,
                             double *misfit, float *grad_v2, float *traces) {
  if (!misfit) return WAVE_EINVAL;
  return gradient_impl(ctx, shot, nsteps, rec_xyz, nrec, observed, false,
                       ckpt_every, misfit, grad_v2, traces);
}

// ---------------------------------------------------------------------------
// Allocation-free entry point (wave_propagate_noalloc).
//
// Its tables live in g_noalloc_scratch, a fixed device array declared here;
// the host builds their image in g_noalloc_image (also static) and copies it
// over in one transfer per call. Layout (byte offsets):
//   [0, 256)      StepDesc
//   [256, 272)    velocity scan result: max bits (u32), bad count (u64 at 264)
//   [512, ...)    wavelet (nsteps floats), rec_start (tiles + 1 ints),
//                 receivers (nrec int4), each block starting on 256 bytes
namespace {

using NoallocCfg = CfgA;
constexpr size_t kNoallocBytes = WAVE_NOALLOC_SCRATCH_BYTES;
constexpr int kNoallocMaxDevices = 64;
constexpr size_t kNoallocScanOff = 256;
constexpr size_t kNoallocTablesOff = 512;
constexpr size_t kNoallocMaxRec = kNoallocBytes / sizeof(int4);

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];
alignas(256) unsigned char g_noalloc_image[kNoallocBytes];
int32_t g_noalloc_rec_raw[kNoallocMaxRec * 3];
unsigned char g_noalloc_scan[16];

struct NoallocDevice {
  unsigned char *scratch;  // device address of g_noalloc_scratch
  int sms, ctas_per_sm;
};
NoallocDevice g_noalloc_dev[kNoallocMaxDevices];

size_t round256(size_t x) { return (x + 255) & ~size_t(255); }

// Once per device, with that device current. A mutex (static storage, no
// allocation) serialises first calls from several host threads; the cached
// address stays valid for the life of the process's context on the device.
std::mutex g_noalloc_setup_mutex;

int noalloc_setup(int dev, NoallocDevice **out) {
  if (dev < 0 || dev >= kNoallocMaxDevices) return WAVE_ECUDA;
  NoallocDevice &d = g_noalloc_dev[dev];
  std::lock_guard<std::mutex> lock(g_noalloc_setup_mutex);
  if (!d.scratch) {
    void *p = nullptr;
    WAVE_TRY_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    const void *fn =
        reinterpret_cast<const void *>(&wave_sweep_kernel<NoallocCfg, true>);
    WAVE_TRY_CUDA(cudaFuncSetAttribute(
        fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
        (int)NoallocCfg::SMEM_BYTES));
    int sms = 0, per = 0;
    WAVE_TRY_CUDA(
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    WAVE_TRY_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &per, fn, NoallocCfg::THREADS, NoallocCfg::SMEM_BYTES));
    if (per < 1) return WAVE_ECUDA;
    d.sms = sms;
    d.ctas_per_sm = per;
    d.scratch = static_cast<unsigned char *>(p);
  }
  *out = &d;
  return WAVE_OK;
}

// Tensor map over a caller-owned dense field (row pitch nx floats).
int noalloc_map(CUtensorMap *m, const float *base, int nx, int ny, int nz,
                int box_x, int box_y) {
  auto enc = get_encode();
  if (!enc) return WAVE_ECUDA;
  cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz};
  cuuint64_t strides[2] = {(cuuint64_t)nx * 4, (cuuint64_t)nx * 4 * ny};
  cuuint32_t box[3] = {(cuuint32_t)box_x, (cuuint32_t)box_y, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
                   const_cast<float *>(base), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? WAVE_OK : WAVE_ECUDA;
}

}  // namespace

extern "C" int wave_propagate_noalloc(const wave_grid *g, const wave_spacing *h,
                                      double dt, const float *velocity,
                                      float *u, float *u_prev,
                                      const wave_shot *shot, int64_t step0,
                                      int nsteps, const int32_t *rec_xyz,
                                      int nrec, float *traces, void *stream,
                                      int *newest) {
  using C = NoallocCfg;
  if (!newest) return WAVE_EINVAL;
  *newest = 0;
  if (!g || !h || !velocity || !u || !u_prev) return WAVE_EINVAL;
  const int nx = g->nx, ny = g->ny, nz = g->nz;
  if (nx < 1 || ny < 1 || nz < 1 || nx % 4 != 0) return WAVE_EINVAL;
  if ((long long)nx * ny * nz > (1ll << 36)) return WAVE_EINVAL;
  if (!finite_pos(h->dx) || !finite_pos(h->dy) || !finite_pos(h->dz) ||
      !finite_pos(dt) || nsteps < 0 || nrec < 0 || step0 < 0)
    return WAVE_EINVAL;
  if (nrec > 0 && (!rec_xyz || !traces)) return WAVE_EINVAL;
  if (shot && (shot->sx < 0 || shot->sx >= nx || shot->sy < 0 ||
               shot->sy >= ny || shot->sz < 0 || shot->sz >= nz ||
               !finite_pos(shot->f_peak) || !std::isfinite(shot->t0) ||
               !std::isfinite(shot->amp)))
    return WAVE_EINVAL;
  for (const void *p : {(const void *)velocity, (const void *)u,
                        (const void *)u_prev})
    if (reinterpret_cast<uintptr_t>(p) % 16 != 0) return WAVE_EINVAL;
  const int ntx = (nx + C::TX - 1) / C::TX, nty = (ny + C::TY - 1) / C::TY;
  const size_t ntiles = (size_t)ntx * nty;
  const size_t off_w = kNoallocTablesOff;
  const size_t off_rs = off_w + (shot ? round256((size_t)nsteps * 4) : 0);
  const size_t off_r = off_rs + (nrec > 0 ? round256((ntiles + 1) * 4) : 0);
  const size_t end = off_r + (size_t)nrec * sizeof(int4);
  if (end > kNoallocBytes) return WAVE_ETOOBIG;
  if (!is_device_ptr(velocity) || !is_device_ptr(u) || !is_device_ptr(u_prev) ||
      (nrec > 0 && !is_device_ptr(traces)))
    return WAVE_EINVAL;

  int dev = 0;
  WAVE_TRY_CUDA(cudaGetDevice(&dev));
  NoallocDevice *nd = nullptr;
  int st = noalloc_setup(dev, &nd);
  if (st) return st;
  cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
  unsigned char *scr = nd->scratch;

  // Receivers to the host (static buffer), then bounds.
  if (nrec > 0) {
    if (is_device_ptr(rec_xyz)) {
      WAVE_TRY_CUDA(cudaMemcpyAsync(g_noalloc_rec_raw, rec_xyz,
                                    (size_t)nrec * 12, cudaMemcpyDeviceToHost,
                                    cs));
      WAVE_TRY_CUDA(cudaStreamSynchronize(cs));
    } else {
      std::memcpy(g_noalloc_rec_raw, rec_xyz, (size_t)nrec * 12);
    }
    for (int r = 0; r < nrec; ++r) {
      const int x = g_noalloc_rec_raw[3 * r], y = g_noalloc_rec_raw[3 * r + 1],
                z = g_noalloc_rec_raw[3 * r + 2];
      if (x < 0 || x >= nx || y < 0 || y >= ny || z < 0 || z >= nz)
        return WAVE_EINVAL;
    }
  }

  // Velocity scan (max, invalid count) into the scratch's scan block.
  WAVE_TRY_CUDA(cudaMemsetAsync(scr + kNoallocScanOff, 0, 16, cs));
  scan_velocity_kernel<<<nd->sms * 4, 256, 0, cs>>>(
      velocity, nx, nx, (long long)ny * nz,
      reinterpret_cast<unsigned *>(scr + kNoallocScanOff),
      reinterpret_cast<unsigned long long *>(scr + kNoallocScanOff + 8));
  WAVE_TRY_CUDA(cudaGetLastError());
  WAVE_TRY_CUDA(cudaMemcpyAsync(g_noalloc_scan, scr + kNoallocScanOff, 16,
                                cudaMemcpyDeviceToHost, cs));
  WAVE_TRY_CUDA(cudaStreamSynchronize(cs));
  unsigned vb;
  unsigned long long bad;
  std::memcpy(&vb, g_noalloc_scan, 4);
  std::memcpy(&bad, g_noalloc_scan + 8, 8);
  if (bad) return WAVE_EINVAL;
  float vmax;
  std::memcpy(&vmax, &vb, 4);
  if (!(dt <= wave_cfl_dt(h, (double)vmax) * (1.0 + 1e-12)))
    return WAVE_EUNSTABLE;
  if (nsteps == 0) return WAVE_OK;

  // Host image of the tables; every field the kernels read is written here,
  // so nothing depends on what an earlier call left in the array.
  std::memset(g_noalloc_image, 0, kNoallocTablesOff);
  StepDesc d{};
  if (shot) {
    float *w = reinterpret_cast<float *>(g_noalloc_image + off_w);
    const double t0 = shot->t0 < 0 ? 1.0 / shot->f_peak : shot->t0;
    for (int k = 0; k < nsteps; ++k)
      w[k] = (float)ricker((double)(step0 + k) * dt, shot->f_peak, t0,
                           shot->amp);
    d.wavelet = reinterpret_cast<const float *>(scr + off_w);
    d.src_active = 1;
    d.sx = shot->sx;
    d.sy = shot->sy;
    d.sz = shot->sz;
  }
  if (nrec > 0) {
    int *rs = reinterpret_cast<int *>(g_noalloc_image + off_rs);
    int4 *re = reinterpret_cast<int4 *>(g_noalloc_image + off_r);
    if (fill_receiver_table(g_noalloc_rec_raw, nrec, nx, ny, nz, C::TX, C::TY,
                            (int)ntx, (int)ntiles, re, rs))
      return WAVE_EINVAL;
    d.traces = traces;
    d.rec = reinterpret_cast<const int4 *>(scr + off_r);
    d.rec_start = reinterpret_cast<const int *>(scr + off_rs);
    d.nrec = nrec;
  }
  std::memcpy(g_noalloc_image, &d, sizeof(d));
  WAVE_TRY_CUDA(cudaMemcpyAsync(scr, g_noalloc_image, end,
                                cudaMemcpyHostToDevice, cs));

  // Launch geometry and tensor maps over the caller's buffers.
  float *buf[2] = {u, u_prev};
  CUtensorMap halo[2], tile[2], vmap;
  for (int b = 0; b < 2; ++b) {
    if ((st = noalloc_map(&halo[b], buf[b], nx, ny, nz, C::TX + 2 * kR,
                          C::TY + 2 * kR)))
      return st;
    if ((st = noalloc_map(&tile[b], buf[b], nx, ny, nz, C::TX, C::TY)))
      return st;
  }
  if ((st = noalloc_map(&vmap, velocity, nx, ny, nz, C::TX, C::TY))) return st;
  int layers[kMaxLayers];
  const int nl = plan_layers(nz, (long long)ntiles,
                             (long long)nd->sms * nd->ctas_per_sm, 4.0, layers);
  const dim3 grid(ntx, nty, (unsigned)nl);
  if (grid.y > 65535) return WAVE_EINVAL;
  SweepArgs a{};
  set_layers(a, layers, nl);
  a.nx = nx;
  a.ny = ny;
  a.nz = nz;
  a.px = nx;
  a.ntx = ntx;
  a.k = make_coefs(h->dx, h->dy, h->dz);
  a.desc = reinterpret_cast<StepDesc *>(scr);
  a.dt2 = (float)(dt * dt);
  for (int k = 0; k < nsteps; ++k) {
    const int cur = k & 1;
    a.unext = buf[cur ^ 1];
    a.koff = k;
    wave_sweep_kernel<C, true><<<grid, C::THREADS, C::SMEM_BYTES, cs>>>(
        halo[cur], tile[cur ^ 1], vmap, a);
  }
  WAVE_TRY_CUDA(cudaGetLastError());
  if (nrec > 0) {  // NaN / infinity in the traces: WAVE_ENAN
    finite_check_kernel<<<nd->sms * 4, 256, 0, cs>>>(traces, (long long)nsteps * nrec,
                                                     &a.desc->error);
    WAVE_TRY_CUDA(cudaGetLastError());
  }
  int err = 0;
  WAVE_TRY_CUDA(cudaMemcpyAsync(&err, &a.desc->error, sizeof(int),
                                cudaMemcpyDeviceToHost, cs));
  WAVE_TRY_CUDA(cudaStreamSynchronize(cs));
  *newest = nsteps & 1;
  return device_error_status(err);
}
