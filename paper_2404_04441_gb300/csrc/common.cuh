// Host and setup-kernel helpers shared by the translation units of the
// library (context API, allocation-free entry point, shot server). Internal:
// every definition has internal linkage, so each .cu file gets its own copy.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <functional>
#include <vector>

#include "../../include/wave.h"
#include "sweep.cuh"

namespace {
using namespace gbw;

// 8th-order central second-derivative weights w_0..w_4 (Eq. 1's
// discretization parameters, c_am = w_m / h_a^2).
constexpr double kW[5] = {-205.0 / 72.0, 8.0 / 5.0, -1.0 / 5.0, 8.0 / 315.0,
                          -1.0 / 560.0};
// 8th-order central first-derivative weights (index 1..4), for the CPML.
constexpr double kW1[5] = {0.0, 4.0 / 5.0, -1.0 / 5.0, 4.0 / 105.0, -1.0 / 280.0};

// Device error word values: a receiver trace holds a NaN or an infinity; a
// device-resident receiver point lies outside the interior.
constexpr int kErrNonFinite = 2;
constexpr int kErrBadReceiver = 3;

// Records kErrNonFinite in *err (if no error is recorded yet) when any of the
// n values is not finite.
__global__ void finite_check_kernel(const float *v, long long n, int *err) {
  bool bad = false;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    bad |= !isfinite(v[i]);
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicCAS(err, 0, kErrNonFinite);
}

// Device error word (kErr* values) to a status.
inline int device_error_status(int err) {
  if (err == 0) return WAVE_OK;
  if (err == kErrTimeout) return WAVE_ETIMEOUT;
  if (err == kErrNonFinite) return WAVE_ENAN;
  if (err == kErrBadReceiver) return WAVE_EINVAL;
  return WAVE_ECUDA;
}

// Velocity scan over the dense-in-x pitched buffer: max, and count of values
// that are not finite and positive. Blocks take whole rows, threads adjacent
// x (no per-element index division).
__global__ void scan_velocity_kernel(const float *v, int nx, int px,
                                     long long rows, unsigned *vmax_bits,
                                     unsigned long long *nbad) {
  unsigned local_max = 0;
  unsigned long long local_bad = 0;
  for (long long r = blockIdx.x; r < rows; r += gridDim.x) {
    const float *row = v + r * px;
    for (int x = threadIdx.x; x < nx; x += blockDim.x) {
      const float val = row[x];
      if (!(val > 0.f) || !isfinite(val)) {
        ++local_bad;
      } else {
        local_max = max(local_max, __float_as_uint(val));
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    local_max = max(local_max, __shfl_xor_sync(0xffffffffu, local_max, o));
    local_bad += __shfl_xor_sync(0xffffffffu, local_bad, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(vmax_bits, local_max);
    if (local_bad) atomicAdd(nbad, local_bad);
  }
}

// c = v^2 dt^2 in FP32 arithmetic (FP64 runs at a small fraction of the
// FP32 rate on this part): v^2 = p + e exactly (TwoProduct with an FMA,
// Ogita, Rump and Oishi 2005), dt^2 = dh + dl (the FP64 value split into two
// floats), c = p dh + (p dl + e dh), small terms first: within about one unit
// in the last place of the exact product, and the same on every path.
__device__ __forceinline__ float v2dt2(float v, float dh, float dl) {
  const float p = v * v;
  const float e = fmaf(v, v, -p);
  return fmaf(p, dh, fmaf(p, dl, e * dh));
}

// The model value to v^2 dt^2: a velocity v (sq = 0) through v2dt2, or a
// squared velocity m = v^2 (sq = 1) as m dh + m dl, again within about one
// unit in the last place of the exact m dt^2.
__device__ __forceinline__ float model_to_c(float x, int sq, float dh, float dl) {
  return sq ? fmaf(x, dh, x * dl) : v2dt2(x, dh, dl);
}

// v2dt2 in place over a field; n is a multiple of 4 and c is 16-byte aligned
// (pitched field).
__global__ void velocity_to_c_kernel(float *c, long long n, float dh, float dl) {
  float4 *c4 = reinterpret_cast<float4 *>(c);
  const long long n4 = n / 4;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n4;
       i += (long long)gridDim.x * blockDim.x) {
    float4 t = c4[i];
    t.x = v2dt2(t.x, dh, dl);
    t.y = v2dt2(t.y, dh, dl);
    t.z = v2dt2(t.z, dh, dl);
    t.w = v2dt2(t.w, dh, dl);
    c4[i] = t;
  }
}

// One pass over a velocity model: c = v2dt2(v) into the pitched field (its
// pitch columns [nx, px) written as zero), the largest velocity (float bits)
// and the count of values that are not finite and positive. With sq = 1 the
// model holds m = v^2 instead (c = m dt^2, largest m). Rows of src are
// sx floats apart: nx for a caller's dense array (device memory, or host
// memory the GPU can read), px when converting a staged copy in place.
// Blocks take whole rows; each thread loads four columns a block-width apart
// before it stores any (more loads in flight on the host link).
__global__ void __launch_bounds__(256, 4)
    velocity_to_c_checked_kernel(const float *src, long long sx, float *c,
                                 int nx, int px, long long rows, float dh,
                                 float dl, int sq, unsigned *vmax_bits,
                                 unsigned long long *nbad) {
  unsigned local_max = 0;
  unsigned long long local_bad = 0;
  const int bw = blockDim.x;
  for (long long r = blockIdx.x; r < rows; r += gridDim.x) {
    const float *row = src + r * sx;
    float *out = c + r * px;
    for (int x0 = threadIdx.x; x0 < px; x0 += 4 * bw) {
      float v[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int x = x0 + j * bw;
        v[j] = x < nx ? row[x] : 0.f;
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int x = x0 + j * bw;
        if (x < nx) {
          if (!(v[j] > 0.f) || !isfinite(v[j]))
            ++local_bad;
          else
            local_max = max(local_max, __float_as_uint(v[j]));
        }
        if (x < px) out[x] = x < nx ? model_to_c(v[j], sq, dh, dl) : 0.f;
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    local_max = max(local_max, __shfl_xor_sync(0xffffffffu, local_max, o));
    local_bad += __shfl_xor_sync(0xffffffffu, local_bad, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(vmax_bits, local_max);
    if (local_bad) atomicAdd(nbad, local_bad);
  }
}

// The velocity pass over a slab stored without row padding (px == nx): one
// contiguous run of n4 float4 in src and in c (both 16-byte aligned). Each
// thread keeps four 16-byte loads in flight, so a few blocks saturate the
// host link when src is host memory the GPU reads directly.
__global__ void __launch_bounds__(256, 4)
    velocity_to_c_dense_kernel(const float4 *src, float4 *c, long long n4,
                               float dh, float dl, int sq, unsigned *vmax_bits,
                               unsigned long long *nbad) {
  unsigned local_max = 0;
  unsigned long long local_bad = 0;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i0 = blockIdx.x * (long long)blockDim.x + threadIdx.x; i0 < n4;
       i0 += 4 * stride) {
    float4 v[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const long long i = i0 + j * stride;
      v[j] = i < n4 ? src[i] : make_float4(1.f, 1.f, 1.f, 1.f);
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const long long i = i0 + j * stride;
      if (i >= n4) continue;
      const float e[4] = {v[j].x, v[j].y, v[j].z, v[j].w};
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if (!(e[k] > 0.f) || !isfinite(e[k]))
          ++local_bad;
        else
          local_max = max(local_max, __float_as_uint(e[k]));
      }
      c[i] = make_float4(model_to_c(e[0], sq, dh, dl), model_to_c(e[1], sq, dh, dl),
                         model_to_c(e[2], sq, dh, dl), model_to_c(e[3], sq, dh, dl));
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    local_max = max(local_max, __shfl_xor_sync(0xffffffffu, local_max, o));
    local_bad += __shfl_xor_sync(0xffffffffu, local_bad, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(vmax_bits, local_max);
    if (local_bad) atomicAdd(nbad, local_bad);
  }
}

// Launch velocity_to_c_kernel for dt^2 given in FP64.
inline void launch_velocity_to_c(float *c, long long n, double dt2, int sms,
                                 cudaStream_t st) {
  const float dh = (float)dt2;
  const float dl = (float)(dt2 - (double)dh);
  velocity_to_c_kernel<<<sms * 4, 256, 0, st>>>(c, n, dh, dl);
}

template <class T>
__device__ __forceinline__ T from_f32(float v);
template <>
__device__ __forceinline__ __nv_bfloat16 from_f32(float v) {
  return __float2bfloat16_rn(v);
}
template <>
__device__ __forceinline__ __half from_f32(float v) {
  return __float2half_rn(v);
}

// Dense FP32 (x fastest) -> pitched 16-bit field with scale 2^exps[slot].
template <class T>
__global__ void to_stored_kernel(T *dst, int pxu, const float *src, int nx,
                                 long long rows, const StepDesc *d, int slot) {
  const float inv = ldexpf(1.0f, -d->exps[slot]);
  const long long total = rows * (long long)nx;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
       i < total; i += (long long)gridDim.x * blockDim.x) {
    const long long r = i / nx;
    const int x = (int)(i - r * nx);
    dst[r * pxu + x] = from_f32<T>(src[i] * inv);
  }
}

// Pitched 16-bit field with scale 2^exps[slot] -> dense FP32.
template <class T>
__global__ void from_stored_kernel(float *dst, const T *src, int pxu, int nx,
                                   long long rows, const StepDesc *d,
                                   int slot) {
  const float sc = ldexpf(1.0f, d->exps[slot]);
  const long long total = rows * (long long)nx;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
       i < total; i += (long long)gridDim.x * blockDim.x) {
    const long long r = i / nx;
    const int x = (int)(i - r * nx);
    dst[i] = to_f32(src[r * pxu + x]) * sc;
  }
}

// Largest |v| (as float bits) of a dense FP32 array.
__global__ void absmax_kernel(const float *v, long long n, unsigned *out) {
  unsigned m = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    m = max(m, __float_as_uint(fabsf(v[i])));
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

struct DeviceBuf {
  void *p = nullptr;
  size_t cap = 0;
};

int cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return WAVE_OK;
  if (e == cudaErrorMemoryAllocation) return WAVE_ENOMEM;
  return WAVE_ECUDA;
}

#define WAVE_TRY_CUDA(expr)                         \
  do {                                              \
    cudaError_t e_ = (expr);                        \
    if (e_ != cudaSuccess) return cuda_status(e_);  \
  } while (0)

bool is_device_ptr(const void *p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

int ensure(DeviceBuf &b, size_t bytes, cudaStream_t st) {
  if (b.cap >= bytes) return WAVE_OK;
  if (b.p) {
    // Work queued earlier may still read the old buffer.
    WAVE_TRY_CUDA(cudaStreamSynchronize(st));
    cudaFree(b.p);
    b.p = nullptr;
    b.cap = 0;
  }
  size_t cap = std::max<size_t>(bytes, 256);
  WAVE_TRY_CUDA(cudaMalloc(&b.p, cap));
  b.cap = cap;
  return WAVE_OK;
}

PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                         cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

CUtensorMapDataType field_dtype(int storage) {
  if (storage == WAVE_STORAGE_BF16) return CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  if (storage == WAVE_STORAGE_F16) return CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
  return CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
}

// Makespan of one launch, in units of one CTA stage (one plane) run alone.
// CTAs start in launch order (layer by layer, tiles within a layer) as soon
// as one of the `slots` resident places is free, and each takes planes +
// preroll stages. All resident CTAs advance together, one stage per
// 1 + C / slots units while C are resident: a CTA alone is bound by load
// latency, and CTAs that share the GPU share its HBM bandwidth. On GB300 a
// stage takes 0.37 us with few CTAs resident and 0.72 us with all 608
// places busy.
//
// preroll: for the FP32 sweep the 8 u-only stages that refill the register
// queue move about 40 % of the bytes of a full stage and count as 4. The
// 16-bit sweeps, bound by instruction issue and with a longer CTA prologue
// (the scale state), run fastest with fewer, longer CTAs; a preroll of 8
// picks those plans (1024 x 1024 x 512: 448/64 against 272/216/24, FP16 477
// against 470 Gpts/s, BF16 487 against 481).
//
// Measured on 128^3 .. 448^3 and 1024 x 1024 x 512, this model picks the
// fastest plan tried on all but 384^3 (2.6 % slower than its best).
// Counting each CTA's time as fixed left small grids with a third of the
// places idle (128^3: 106 against 174 Gpts/s, 192^3: 203 against 316).
//
// The simulation keeps the resident CTAs as groups that finish at the same
// time (CTAs started together with the same layer length), so its cost
// grows with the number of distinct finish times, not with the number of
// CTAs; it uses fixed storage only. Returns a huge value if the groups
// outgrow that storage (the plan is then never chosen).
constexpr int kPlanGroups = 1024;

double layer_makespan(const int *chunks, int nchunks, long long ntiles,
                      long long slots, double preroll = 4.0) {
  double fin[kPlanGroups];
  long long cnt[kPlanGroups];
  int ng = 0;
  int layer = 0;
  long long tile = 0;  // next tile of `layer` to start
  long long live = 0;  // resident CTAs
  bool overflow = false;
  // start k CTAs at progress point p, in launch order
  auto start = [&](long long k, double p) {
    while (k > 0 && layer < nchunks) {
      const long long m = std::min(k, ntiles - tile);
      const double f = p + (chunks[layer] + preroll);
      int g = 0;
      while (g < ng && fin[g] != f) ++g;
      if (g == ng) {
        if (ng == kPlanGroups) {
          overflow = true;
          return;
        }
        fin[ng] = f;
        cnt[ng++] = 0;
      }
      cnt[g] += m;
      live += m;
      k -= m;
      tile += m;
      if (tile == ntiles) {
        tile = 0;
        ++layer;
      }
    }
  };
  double t = 0.0, prog = 0.0;
  start(slots, 0.0);
  while (ng > 0 && !overflow) {
    double nxt = fin[0];
    for (int g = 1; g < ng; ++g) nxt = std::min(nxt, fin[g]);
    t += (nxt - prog) * (1.0 + (double)live / (double)slots);
    prog = nxt;
    long long freed = 0;
    for (int g = 0; g < ng;) {
      if (fin[g] <= prog) {
        freed += cnt[g];
        fin[g] = fin[ng - 1];
        cnt[g] = cnt[ng - 1];
        --ng;
      } else {
        ++g;
      }
    }
    live -= freed;
    start(freed, prog);
  }
  return overflow ? 1e300 : t;
}

double layer_makespan(const std::vector<int> &chunks, long long ntiles,
                      long long slots, double preroll = 4.0) {
  return layer_makespan(chunks.data(), (int)chunks.size(), ntiles, slots,
                        preroll);
}

// Candidate plans for plan_layers, numbered in a fixed order: first the
// uniform splits into k = 1..min(nz, 16) layers, then "layers of a planes,
// the rest, then `tail` layers of b planes" for a = 16, 24, .. < nz, b in
// {8, 16, 24, 32, 48, 64} below a, tail = 1..4, keeping those of at most 16
// layers. Writes candidate `idx` to out and returns its layer count (0 when
// idx is past the last candidate).
struct PlanCandidate {
  int a, b, tail;  // a = 0: uniform split into b layers
};

int plan_candidate_chunks(int nz, const PlanCandidate &pc, int *out) {
  int n = 0;
  if (pc.a == 0) {
    const int zc = (nz + pc.b - 1) / pc.b;
    for (int z = 0; z < nz; z += zc) out[n++] = std::min(zc, nz - z);
    return n;
  }
  int rest = nz - pc.tail * pc.b;
  const int full = rest / pc.a;
  if (full + (rest % pc.a > 0) + pc.tail > kMaxLayers) return 0;
  while (rest >= pc.a) {
    out[n++] = pc.a;
    rest -= pc.a;
  }
  if (rest > 0) out[n++] = rest;
  for (int t = 0; t < pc.tail; ++t) out[n++] = pc.b;
  return n;
}

// Split nz into at most kMaxLayers z layers, chosen by layer_makespan: a
// cheap score (work plus waves) ranks all candidates; every uniform split
// and the best-ranked others (among the 48 best scores) are simulated, and
// the first plan with the smallest makespan wins. Writes the plan to out and
// returns its layer count. Fixed storage only (no allocation).
int plan_layers(int nz, long long ntiles, long long slots, double preroll,
                int out[kMaxLayers]) {
  constexpr int kTop = 48;
  static const int kTail[6] = {8, 16, 24, 32, 48, 64};
  const int nuni = std::min(nz, kMaxLayers);
  // the kTop best (score, index) pairs, ascending
  double tscore[kTop] = {};
  int tidx[kTop] = {};
  PlanCandidate tcand[kTop] = {};
  int ntop = 0;
  int idx = 0;
  int ch[kMaxLayers];
  auto consider = [&](const PlanCandidate &pc) {
    const int n = plan_candidate_chunks(nz, pc, ch);
    if (n == 0) return;
    double w = 0;
    for (int i = 0; i < n; ++i) w += ch[i] + 4.0;
    const double waves = (double)ntiles * n / (double)slots;
    const double sc = w * ntiles / (double)slots + waves;
    const int my = idx++;
    if (ntop == kTop && !(sc < tscore[kTop - 1])) return;
    int pos = ntop < kTop ? ntop++ : kTop - 1;
    while (pos > 0 && sc < tscore[pos - 1]) {
      tscore[pos] = tscore[pos - 1];
      tidx[pos] = tidx[pos - 1];
      tcand[pos] = tcand[pos - 1];
      --pos;
    }
    tscore[pos] = sc;
    tidx[pos] = my;
    tcand[pos] = pc;
  };
  for (int k = 1; k <= nuni; ++k) consider({0, k, 0});
  for (int a = 16; a < nz; a += 8)
    for (int b : kTail) {
      if (b >= a) continue;
      for (int tail = 1; tail <= 4; ++tail) {
        if (a + tail * b > nz) break;
        consider({a, b, tail});
      }
    }
  double best_m = 1e300;
  int best_n = 0;
  auto simulate = [&](const PlanCandidate &pc) {
    const int n = plan_candidate_chunks(nz, pc, ch);
    const double m = layer_makespan(ch, n, ntiles, slots, preroll);
    if (m < best_m - 1e-9) {
      best_m = m;
      best_n = n;
      std::copy(ch, ch + n, out);
    }
  };
  for (int k = 1; k <= nuni; ++k) simulate({0, k, 0});
  for (int r = 0; r < ntop; ++r)
    if (tidx[r] >= nuni) simulate(tcand[r]);
  return best_n;
}

std::vector<int> plan_layers(int nz, long long ntiles, long long slots,
                             double preroll = 4.0) {
  int out[kMaxLayers];
  const int n = plan_layers(nz, ntiles, slots, preroll, out);
  return std::vector<int>(out, out + n);
}

// Eq. 1 coefficients of one grid spacing (kernel parameters).
StencilCoefs make_coefs(double dx, double dy, double dz) {
  StencilCoefs k{};
  const double ix = 1.0 / (dx * dx), iy = 1.0 / (dy * dy), iz = 1.0 / (dz * dz);
  k.c0 = (float)(kW[0] * (ix + iy + iz));
  for (int m = 1; m <= 4; ++m) {
    k.cx[m - 1] = (float)(kW[m] * ix);
    k.cy[m - 1] = (float)(kW[m] * iy);
    k.cz[m - 1] = (float)(kW[m] * iz);
  }
  k.sxi = (float)(ix / 5040.0);
  k.syi = (float)(iy / 5040.0);
  return k;
}

void set_layers(SweepArgs &a, const int *ch, int n) {
  a.nlayers = n;
  a.zl[0] = 0;
  for (int l = 0; l < n; ++l) a.zl[l + 1] = a.zl[l] + ch[l];
}

void set_layers(SweepArgs &a, const std::vector<int> &ch) {
  a.nlayers = (int)ch.size();
  a.zl[0] = 0;
  for (size_t l = 0; l < ch.size(); ++l) a.zl[l + 1] = a.zl[l] + ch[l];
}

double ricker(double t, double f, double t0, double amp) {
  const double pi = 3.14159265358979323846;
  const double a = pi * pi * f * f * (t - t0) * (t - t0);
  return amp * (1.0 - 2.0 * a) * std::exp(-a);
}

bool finite_pos(double v) { return std::isfinite(v) && v > 0.0; }


// 3D tensor map over a (nz, ny, pitch)-pitched field with logical extent
// (nx, ny, nz); elements outside it read as zero (the zero halo).
int encode_map(CUtensorMap *m, const void *base, int nx, int ny, int nz,
               int pitch, int esize, CUtensorMapDataType dtype, int box_x,
               int box_y) {
  auto enc = get_encode();
  if (!enc) return WAVE_ECUDA;
  cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz};
  cuuint64_t strides[2] = {(cuuint64_t)pitch * esize,
                           (cuuint64_t)pitch * esize * (cuuint64_t)ny};
  cuuint32_t box[3] = {(cuuint32_t)box_x, (cuuint32_t)box_y, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = enc(m, dtype, 3, const_cast<void *>(base), dims, strides, box,
                   estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? WAVE_OK : WAVE_ECUDA;
}

// Receivers (x, y, z) on the host -> entries {z, local index in tile, id,
// tile} sorted by (tile, z, id) and per-tile start offsets (ntiles + 1), in
// caller-provided arrays of nrec and ntiles + 1 elements (no allocation:
// the allocation-free entry point fills its fixed scratch image with it).
// A tile is tx x ty points, tiles numbered y-major (tile = ty_index * ntx +
// tx_index); the local index is (y mod ty) * tx + (x mod tx). Returns
// WAVE_EINVAL for a receiver outside the nx*ny*nz interior (the arrays are
// then unspecified).
int fill_receiver_table(const int32_t *xyz, int nrec, int nx, int ny, int nz,
                        int tx, int ty, int ntx, int ntiles, int4 *entries,
                        int *start) {
  std::fill(start, start + (size_t)ntiles + 1, 0);
  for (int r = 0; r < nrec; ++r) {
    const int x = xyz[3 * r], y = xyz[3 * r + 1], z = xyz[3 * r + 2];
    if (x < 0 || x >= nx || y < 0 || y >= ny || z < 0 || z >= nz)
      return WAVE_EINVAL;
    const int t = (y / ty) * ntx + (x / tx);
    entries[r] = make_int4(z, (y % ty) * tx + (x % tx), r, t);
    start[t + 1]++;
  }
  std::sort(entries, entries + nrec, [](const int4 &a, const int4 &b) {
    if (a.w != b.w) return a.w < b.w;
    if (a.x != b.x) return a.x < b.x;
    return a.z < b.z;
  });
  for (int t = 0; t < ntiles; ++t) start[t + 1] += start[t];
  return WAVE_OK;
}

int build_receiver_table(const int32_t *xyz, int nrec, int nx, int ny, int nz,
                         int tx, int ty, int ntx, int ntiles,
                         std::vector<int4> &entries, std::vector<int> &start) {
  entries.resize(nrec);
  start.resize((size_t)ntiles + 1);
  return fill_receiver_table(xyz, nrec, nx, ny, nz, tx, ty, ntx, ntiles,
                             entries.data(), start.data());
}

// ---------------------------------------------------------------------------
// Receiver table built on the device: the same entries {z, local, id, tile},
// sorted by (tile, z, id), and per-tile starts as fill_receiver_table, from
// receivers in device memory, with no copy to the host and no stream
// synchronisation. Receivers outside the interior are left out of the table
// and recorded as kErrBadReceiver in the error word. Four launches:
// per-tile counts, their exclusive scan, a scatter of the keys (z << 32 | id)
// into the tiles' segments, and a sort of each segment (one block per tile).
struct RecGeom {
  int nx, ny, nz;   // interior
  int tx, ty, ntx;  // tile size and tiles along x
  int ntiles;
};

constexpr int kRecScanThreads = 1024;
constexpr int kRecSortThreads = 256;
constexpr int kRecSortShared = 2048;  // segments up to this size sort in shared memory

__device__ __forceinline__ bool rec_point(const int32_t *xyz, long long r,
                                          const RecGeom &g, int &x, int &y,
                                          int &z) {
  x = xyz[3 * r];
  y = xyz[3 * r + 1];
  z = xyz[3 * r + 2];
  return x >= 0 && x < g.nx && y >= 0 && y < g.ny && z >= 0 && z < g.nz;
}

__global__ void rec_count_kernel(const int32_t *xyz, int nrec, RecGeom g,
                                 int *cnt, int *err) {
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < nrec;
       r += (long long)gridDim.x * blockDim.x) {
    int x, y, z;
    if (!rec_point(xyz, r, g, x, y, z)) {
      atomicCAS(err, 0, kErrBadReceiver);
      continue;
    }
    atomicAdd(&cnt[(y / g.ty) * g.ntx + x / g.tx], 1);
  }
}

// One block: start[t] = sum of cnt[0..t), start[ntiles] = total; cnt[t] is
// overwritten with start[t] (the scatter's cursor).
__global__ void __launch_bounds__(kRecScanThreads)
    rec_scan_kernel(int *cnt, int *start, int ntiles) {
  __shared__ int warp_sum[kRecScanThreads / 32];
  const int tid = threadIdx.x;
  const long long per = ((long long)ntiles + kRecScanThreads - 1) / kRecScanThreads;
  const long long b = tid * per;
  const long long e = b + per < (long long)ntiles ? b + per : (long long)ntiles;
  int sum = 0;
  for (long long i = b; i < e; ++i) sum += cnt[i];
  // exclusive scan of the per-thread sums
  int v = sum;
  for (int o = 1; o < 32; o <<= 1) {
    const int n = __shfl_up_sync(0xffffffffu, v, o);
    if ((tid & 31) >= o) v += n;
  }
  if ((tid & 31) == 31) warp_sum[tid >> 5] = v;
  __syncthreads();
  if (tid < 32) {
    int w = warp_sum[tid];
    for (int o = 1; o < 32; o <<= 1) {
      const int n = __shfl_up_sync(0xffffffffu, w, o);
      if (tid >= o) w += n;
    }
    warp_sum[tid] = w;
  }
  __syncthreads();
  int run = v - sum + ((tid >> 5) > 0 ? warp_sum[(tid >> 5) - 1] : 0);
  for (long long i = b; i < e; ++i) {
    const int c = cnt[i];
    start[i] = run;
    cnt[i] = run;
    run += c;
  }
  if (tid == kRecScanThreads - 1) start[ntiles] = warp_sum[31];
}

__global__ void rec_scatter_kernel(const int32_t *xyz, int nrec, RecGeom g,
                                   int *cursor, unsigned long long *keys) {
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < nrec;
       r += (long long)gridDim.x * blockDim.x) {
    int x, y, z;
    if (!rec_point(xyz, r, g, x, y, z)) continue;
    const int pos = atomicAdd(&cursor[(y / g.ty) * g.ntx + x / g.tx], 1);
    keys[pos] = ((unsigned long long)(unsigned)z << 32) | (unsigned long long)r;
  }
}

// Ascending bitonic sort of a[0, n) by one block, for any n: the network of
// the padded power-of-two size N in the form whose every comparator puts the
// smaller key at the lower index (the first stage of each merge compares
// mirror positions), so the padding, +infinity at [n, N), never moves and
// comparators that reach it are skipped.
__device__ void block_bitonic_sort(unsigned long long *a, long long n) {
  long long N = 1;
  while (N < n) N <<= 1;
  for (long long k = 2; k <= N; k <<= 1) {
    for (long long j = k >> 1; j > 0; j >>= 1) {
      for (long long i = threadIdx.x; i < N / 2; i += blockDim.x) {
        const long long blk = i / j, off = i - blk * j;
        long long lo, hi;
        if (j == (k >> 1)) {  // mirror stage of a merge of size k
          lo = blk * k + off;
          hi = blk * k + k - 1 - off;
        } else {
          lo = blk * 2 * j + off;
          hi = lo + j;
        }
        if (hi < n) {
          const unsigned long long p = a[lo], q = a[hi];
          if (q < p) {
            a[lo] = q;
            a[hi] = p;
          }
        }
      }
      __syncthreads();
    }
  }
}

__global__ void __launch_bounds__(kRecSortThreads)
    rec_sort_kernel(const int32_t *xyz, RecGeom g, const int *start,
                    unsigned long long *keys, int4 *entries) {
  __shared__ unsigned long long sk[kRecSortShared];
  for (int t = blockIdx.x; t < g.ntiles; t += gridDim.x) {
    const int s0 = start[t], n = start[t + 1] - s0;
    if (n == 0) continue;
    unsigned long long *a = keys + s0;
    if (n <= kRecSortShared) {
      for (int i = threadIdx.x; i < n; i += blockDim.x) sk[i] = a[i];
      __syncthreads();
      a = sk;
    }
    if (n > 1) block_bitonic_sort(a, n);
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const unsigned long long k = a[i];
      const int r = (int)(k & 0xffffffffu);
      const int x = xyz[3 * (long long)r], y = xyz[3 * (long long)r + 1];
      entries[s0 + i] = make_int4((int)(k >> 32), (y % g.ty) * g.tx + (x % g.tx), r, t);
    }
    __syncthreads();  // sk is reused by the block's next tile
  }
}

// Enqueue the four launches on st. cnt and start hold ntiles + 1 ints, keys
// nrec, entries nrec; err is the device error word. Requires nrec >= 1.
int build_receiver_table_device(const int32_t *xyz, int nrec, const RecGeom &g,
                                int *cnt, int *start, unsigned long long *keys,
                                int4 *entries, int *err, int sms,
                                cudaStream_t st) {
  WAVE_TRY_CUDA(cudaMemsetAsync(cnt, 0, ((size_t)g.ntiles + 1) * sizeof(int), st));
  const int blocks = (int)std::min<long long>(((long long)nrec + 255) / 256, 4ll * sms);
  rec_count_kernel<<<blocks, 256, 0, st>>>(xyz, nrec, g, cnt, err);
  rec_scan_kernel<<<1, kRecScanThreads, 0, st>>>(cnt, start, g.ntiles);
  rec_scatter_kernel<<<blocks, 256, 0, st>>>(xyz, nrec, g, cnt, keys);
  rec_sort_kernel<<<(int)std::min<long long>(g.ntiles, 16ll * sms), kRecSortThreads, 0,
                    st>>>(xyz, g, start, keys, entries);
  WAVE_TRY_CUDA(cudaGetLastError());
  return WAVE_OK;
}

// Receivers within w cells of a face (the CPML shell), as {x, y, z, id} in
// any order, counted in *count (zeroed by the caller).
__global__ void rec_shell_kernel(const int32_t *xyz, int nrec, RecGeom g, int w,
                                 int4 *out, int *count) {
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < nrec;
       r += (long long)gridDim.x * blockDim.x) {
    int x, y, z;
    if (!rec_point(xyz, r, g, x, y, z)) continue;
    if (x < w || x >= g.nx - w || y < w || y >= g.ny - w || z < w || z >= g.nz - w)
      out[atomicAdd(count, 1)] = make_int4(x, y, z, (int)r);
  }
}

}  // namespace
