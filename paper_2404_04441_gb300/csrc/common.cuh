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
#include <queue>
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

// Device error word value: a receiver trace holds a NaN or an infinity.
constexpr int kErrNonFinite = 2;

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

// c = v^2 dt^2 in place, in FP32 arithmetic (FP64 runs at a small fraction
// of the FP32 rate on this part): v^2 = p + e exactly (TwoProduct with an
// FMA, Ogita, Rump and Oishi 2005), dt^2 = dh + dl (the FP64 value split
// into two floats), c = p dh + (p dl + e dh), small terms first: within
// about one unit in the last place of the exact product, and the same on
// every path. n is a multiple of 4 and c is 16-byte aligned (pitched field).
__global__ void velocity_to_c_kernel(float *c, long long n, float dh, float dl) {
  float4 *c4 = reinterpret_cast<float4 *>(c);
  const long long n4 = n / 4;
  auto conv = [&](float v) {
    const float p = v * v;
    const float e = fmaf(v, v, -p);
    return fmaf(p, dh, fmaf(p, dl, e * dh));
  };
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n4;
       i += (long long)gridDim.x * blockDim.x) {
    float4 t = c4[i];
    t.x = conv(t.x);
    t.y = conv(t.y);
    t.z = conv(t.z);
    t.w = conv(t.w);
    c4[i] = t;
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
__device__ __forceinline__ float to_f32(__nv_bfloat16 v) {
  return __bfloat162float(v);
}
__device__ __forceinline__ float to_f32(__half v) { return __half2float(v); }

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
double layer_makespan(const std::vector<int> &chunks, long long ntiles,
                      long long slots, double preroll = 4.0) {
  // finish points of the resident CTAs, in stages of common progress
  std::priority_queue<double, std::vector<double>, std::greater<double>> live;
  size_t layer = 0;
  long long tile = 0;
  auto next = [&](double &len) {
    if (layer >= chunks.size()) return false;
    len = chunks[layer] + preroll;
    if (++tile == ntiles) {
      tile = 0;
      ++layer;
    }
    return true;
  };
  double t = 0.0, prog = 0.0, len = 0.0;
  while ((long long)live.size() < slots && next(len)) live.push(prog + len);
  while (!live.empty()) {
    const double nxt = live.top();
    t += (nxt - prog) * (1.0 + (double)live.size() / (double)slots);
    prog = nxt;
    while (!live.empty() && live.top() <= prog) {
      live.pop();
      if (next(len)) live.push(prog + len);
    }
  }
  return t;
}

// Split nz into at most kMaxLayers z layers: uniform splits and "k equal
// chunks then a tail of small chunks", scored by layer_makespan.
std::vector<int> plan_layers(int nz, long long ntiles, long long slots,
                             double preroll = 4.0) {
  std::vector<std::vector<int>> cands;
  for (int k = 1; k <= std::min(nz, kMaxLayers); ++k) {
    const int zc = (nz + k - 1) / k;
    std::vector<int> ch;
    for (int z = 0; z < nz; z += zc) ch.push_back(std::min(zc, nz - z));
    cands.push_back(ch);
  }
  for (int a = 16; a < nz; a += 8) {
    for (int b : {8, 16, 24, 32, 48, 64}) {
      if (b >= a) continue;
      for (int tail = 1; tail <= 4; ++tail) {
        if (a + tail * b > nz) break;
        std::vector<int> ch;
        int rest = nz - tail * b;
        while (rest >= a) { ch.push_back(a); rest -= a; }
        if (rest > 0) ch.push_back(rest);
        for (int t = 0; t < tail; ++t) ch.push_back(b);
        if ((int)ch.size() <= kMaxLayers) cands.push_back(ch);
      }
    }
  }
  // Cheap pre-filter by a wave model, then simulate the best few.
  std::vector<std::pair<double, size_t>> score;
  for (size_t i = 0; i < cands.size(); ++i) {
    double w = 0;
    for (int c : cands[i]) w += c + 4.0;
    const double waves = (double)ntiles * cands[i].size() / (double)slots;
    score.push_back({w * ntiles / (double)slots + waves, i});
  }
  std::sort(score.begin(), score.end());
  // Simulate the best few by that score and every uniform split (the first
  // candidates): the score counts work, not idle places.
  const size_t nuni = (size_t)std::min(nz, kMaxLayers);
  std::vector<size_t> sim;
  for (size_t i = 0; i < nuni; ++i) sim.push_back(i);
  for (size_t r = 0; r < std::min<size_t>(score.size(), 48); ++r)
    if (score[r].second >= nuni) sim.push_back(score[r].second);
  size_t best = 0;
  double best_m = 1e300;
  for (size_t i : sim) {
    const double m = layer_makespan(cands[i], ntiles, slots, preroll);
    if (m < best_m - 1e-9) {
      best_m = m;
      best = i;
    }
  }
  return cands[best];
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

}  // namespace
