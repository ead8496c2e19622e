// The leapfrog sweep: one kernel launch advances the whole grid by one step.
//
// Each CTA owns a TX x TY tile of interior columns and a range of z planes
// and streams through z (the 2.5D blocking of Sec. 4.1, with the z
// neighbours of a column held in a per-thread register queue as in the
// shifting-register scheme described there). Per plane, one thread issues
// three TMA loads into shared-memory rings:
//   * u at plane j+4, the tile plus a radius-4 halo in x and y; a slot stays
//     resident for five planes, so it serves first as the "front" that feeds
//     the register queue and, four planes later, as the xy plane of Eq. 1;
//   * u_prev and v^2 dt^2 at plane j, the tile only.
// TMA's out-of-bounds zero fill supplies the zero Dirichlet halo, so the
// fields are stored without padding planes (rows are padded to 16 bytes).
// Each thread computes 4 consecutive x points on VY rows, reads the x and y
// neighbours from the xy plane in shared memory and the z neighbours from its
// queue, and writes u_next over u_prev with streaming stores. The Ricker
// source and the receivers are applied in the same pass.
//
// Storage: the wavefields are FP32, BF16 or FP16 (template type T); the
// arithmetic is FP32 in every case and v^2 dt^2 is always FP32. A 16-bit
// field holding time step k carries a power-of-two scale 2^e_k: value =
// stored * 2^e_k. The scale of each newly written field is chosen from the
// largest magnitudes of the two fields it is computed from, with headroom for
// the largest possible growth in one step, so FP16 never overflows; the
// scale factors are exact powers of two, so scaling adds no rounding.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cstdint>
#include <type_traits>

#include "ptx.cuh"

namespace gbw {

constexpr int kR = 4;                // stencil radius (Sec. 4.1: R = 4)
constexpr int kErrTimeout = 1;       // device error word values
constexpr uint64_t kWaitLimitNs = 2000000000ull;

// Per-context state read by every sweep launch (device memory). The fields
// up to `error` are rewritten at each call; the rest persist.
struct StepDesc {
  long long n;            // index of the next step within the current call
  long long step0;        // absolute step number of the call's first step
  const float *wavelet;   // source value per step of the call (or null)
  float *traces;          // nsteps x nrec, row n written by step n (or null)
  const int4 *rec;        // receivers sorted by (tile, z): {z, local, id, 0}
  const int *rec_start;   // per tile: first entry; size ntiles + 1
  int nrec;
  int src_active;
  int sx, sy, sz;
  // Point injection (adjoint sources): row n of inj_val holds the values of
  // step n; entry {z, local, id, tile} adds v^2 dt^2 * inj_val[n][id] at its
  // point; entries sorted by (tile, z) with per-tile starts like receivers.
  const float *inj_val;
  const int4 *inj;
  const int *inj_start;
  int ninj;
  int error;              // first error recorded by a kernel (0 = none)
  // 16-bit storage only: the field holding absolute step k has scale
  // 2^exps[k & 3] and largest magnitude maxbits[k & 3] (bits of a float).
  int exps[4];
  unsigned maxbits[4];
};

constexpr int kMaxLayers = 16;

// Extra work of a sweep (template bit mask), used by the adjoint gradient:
constexpr int kModeStoreD = 1;   // write D = v^2 dt^2 (L u) + source to a.dout
constexpr int kModeInject = 2;   // add the StepDesc's point injections
constexpr int kModeGradAcc = 4;  // (a.ghi, a.glo) += u * a.dsrc, per point

// Eq. 1 coefficients of one grid spacing.
struct StencilCoefs {
  float c0;                   // w0 * (1/dx^2 + 1/dy^2 + 1/dz^2)
  float cx[4], cy[4], cz[4];  // w_m / h_a^2 for m = 1..4
  float sxi, syi;             // 1 / (5040 h_a^2), a = x, y: scale of the
                              // integer weights 5040 w_m (tensor-core sweep)
};

// Eq. 1's off-centre weights times 5040 (the least common multiple of their
// denominators): 8064, -1008, 128, -9. Each is exact in FP16 and in BF16 (at
// most 6 significant bits), so the 16-bit tensor-core sweep multiplies the
// stored wavefield by exact weights and scales the FP32 sums once.
constexpr float kWInt[5] = {0.f, 8064.f, -1008.f, 128.f, -9.f};

struct SweepArgs {
  int nx, ny, nz, px;  // interior sizes; px = row pitch in elements (16 B rows)
  // z layers: CTAs with blockIdx.z == l stream planes [zl[l], zl[l+1]).
  // Layers are launched in order, so large layers first and small ones last
  // shorten the partial last wave of CTAs.
  int nlayers;
  int zl[kMaxLayers + 1];
  int ntx;             // tiles along x (tile id = by * ntx + bx)
  StencilCoefs k;      // coefficients (kernel parameters: constant operands)
  void *unext;         // output: the u_prev buffer, overwritten in place
  StepDesc *desc;
  int koff;            // step offset of this launch within a graph chunk
  float dt2;           // dt^2, used only when the c field holds velocities
  float cmax;          // largest v^2 dt^2 (16-bit storage: growth bound)
  float *dout;         // kModeStoreD: D of this step (field layout)
  const float *dsrc;   // kModeGradAcc: D paired with this step's u
  float *ghi, *glo;    // kModeGradAcc: running sum of u * D as hi + lo (field layout)
};

// Element access per storage type: 4 consecutive elements to/from float4.
template <class T>
struct Elem;

template <>
struct Elem<float> {
  static constexpr int kHaloX = 4;  // box starts 4 elements left (16 B)
  __device__ static __forceinline__ float4 load4(const float *p) {
    return *reinterpret_cast<const float4 *>(p);
  }
  __device__ static __forceinline__ void store4_cs(float *p, float4 v) {
    __stcs(reinterpret_cast<float4 *>(p), v);
  }
};

template <>
struct Elem<__nv_bfloat16> {
  static constexpr int kHaloX = 8;  // 16-byte aligned box start: 8 elements
  __device__ static __forceinline__ float4 load4(const __nv_bfloat16 *p) {
    const uint2 w = *reinterpret_cast<const uint2 *>(p);
    // A bf16 is the upper half of the float with the same bits.
    return make_float4(__uint_as_float(w.x << 16),
                       __uint_as_float(w.x & 0xffff0000u),
                       __uint_as_float(w.y << 16),
                       __uint_as_float(w.y & 0xffff0000u));
  }
  __device__ static __forceinline__ uint2 load_raw(const __nv_bfloat16 *p) {
    return *reinterpret_cast<const uint2 *>(p);
  }
  // Element k (0..3) of a raw 4-element load, as FP32 (exact).
  __device__ static __forceinline__ float unpack(uint2 w, int k) {
    const unsigned x = (k < 2) ? w.x : w.y;
    return (k & 1) ? __uint_as_float(x & 0xffff0000u) : __uint_as_float(x << 16);
  }
  // Element k of a raw load plus an FP32 value, rounded once (the same result
  // as unpack(w, k) + c) in one mixed-precision add.
  __device__ static __forceinline__ float add_to(uint2 w, int k, float c) {
    const unsigned x = (k < 2) ? w.x : w.y;
    float d;
    if (k & 1)
      asm("{\n\t.reg .b16 l, h;\n\tmov.b32 {l, h}, %1;\n\t"
          "add.rn.f32.bf16 %0, h, %2;\n\t}"
          : "=f"(d) : "r"(x), "f"(c));
    else
      asm("{\n\t.reg .b16 l, h;\n\tmov.b32 {l, h}, %1;\n\t"
          "add.rn.f32.bf16 %0, l, %2;\n\t}"
          : "=f"(d) : "r"(x), "f"(c));
    return d;
  }
  __device__ static __forceinline__ void store4_cs(__nv_bfloat16 *p, float4 v) {
    const __nv_bfloat162 a = __floats2bfloat162_rn(v.x, v.y);
    const __nv_bfloat162 b = __floats2bfloat162_rn(v.z, v.w);
    uint2 w;
    w.x = *reinterpret_cast<const unsigned *>(&a);
    w.y = *reinterpret_cast<const unsigned *>(&b);
    __stcs(reinterpret_cast<uint2 *>(p), w);
  }
};

template <>
struct Elem<__half> {
  static constexpr int kHaloX = 8;
  __device__ static __forceinline__ float4 load4(const __half *p) {
    const uint2 w = *reinterpret_cast<const uint2 *>(p);
    const float2 a = __half22float2(*reinterpret_cast<const __half2 *>(&w.x));
    const float2 b = __half22float2(*reinterpret_cast<const __half2 *>(&w.y));
    return make_float4(a.x, a.y, b.x, b.y);
  }
  __device__ static __forceinline__ uint2 load_raw(const __half *p) {
    return *reinterpret_cast<const uint2 *>(p);
  }
  __device__ static __forceinline__ float unpack(uint2 w, int k) {
    const unsigned x = (k < 2) ? w.x : w.y;
    const __half2 h = *reinterpret_cast<const __half2 *>(&x);
    return (k & 1) ? __high2float(h) : __low2float(h);
  }
  __device__ static __forceinline__ float add_to(uint2 w, int k, float c) {
    const unsigned x = (k < 2) ? w.x : w.y;
    float d;
    if (k & 1)
      asm("{\n\t.reg .b16 l, h;\n\tmov.b32 {l, h}, %1;\n\t"
          "add.rn.f32.f16 %0, h, %2;\n\t}"
          : "=f"(d) : "r"(x), "f"(c));
    else
      asm("{\n\t.reg .b16 l, h;\n\tmov.b32 {l, h}, %1;\n\t"
          "add.rn.f32.f16 %0, l, %2;\n\t}"
          : "=f"(d) : "r"(x), "f"(c));
    return d;
  }
  __device__ static __forceinline__ void store4_cs(__half *p, float4 v) {
    const __half2 a = __floats2half2_rn(v.x, v.y);
    const __half2 b = __floats2half2_rn(v.z, v.w);
    uint2 w;
    w.x = *reinterpret_cast<const unsigned *>(&a);
    w.y = *reinterpret_cast<const unsigned *>(&b);
    __stcs(reinterpret_cast<uint2 *>(p), w);
  }
};

template <int TX_, int TY_, int VY_, int PF_, int MINB_, class T_ = float>
struct SweepCfg {
  using T = T_;
  static constexpr int TX = TX_, TY = TY_, VY = VY_, PF = PF_, MINB = MINB_;
  static constexpr bool kScaled = sizeof(T) == 2;
  static constexpr bool kTensor = false;
  static constexpr int HX = Elem<T>::kHaloX;  // box columns left of the tile
  static constexpr int NTX = TX / 4;          // threads along x (4 points each)
  static constexpr int NTY = TY / VY;         // threads along y (VY rows each)
  static constexpr int THREADS = NTX * NTY;
  static constexpr int SU = PF + 5;           // u ring: 5 live planes + prefetch
  static constexpr int SP = PF + 1;           // u_prev / c ring
  static constexpr int NB = PF + 1;           // one barrier per in-flight stage
  static constexpr int UW = TX + 2 * HX;      // u slot row length (elements)
  static constexpr int UH = TY + 2 * kR;
  static constexpr int BOX_U = UW;            // TMA box widths: u with halo,
  static constexpr int BOX_P = TX;            // u_prev and v^2 dt^2 tiles
  static constexpr int U_SLOT = UW * UH;      // elements
  static constexpr int P_SLOT = TX * TY;      // elements
  static constexpr uint32_t U_BYTES = U_SLOT * sizeof(T);
  static constexpr uint32_t UP_BYTES = P_SLOT * sizeof(T);
  static constexpr uint32_t C_BYTES = P_SLOT * 4;
  // Dynamic shared memory; 4 CTAs per SM fit while this stays within
  // 228 KiB / 4 minus the 1 KiB the hardware reserves per CTA.
  static constexpr size_t SMEM_BYTES = (size_t)SU * U_BYTES +
                                       (size_t)SP * (UP_BYTES + C_BYTES) +
                                       C_BYTES + NB * 8;
  static_assert(TX % 4 == 0 && TY % VY == 0, "tile shape");
  static_assert((UW * sizeof(T)) % 16 == 0, "TMA box row: multiple of 16 B");
  static_assert((TX * sizeof(T)) % 16 == 0, "TMA box row: multiple of 16 B");
  static_assert(U_BYTES % 128 == 0 && UP_BYTES % 128 == 0 &&
                    C_BYTES % 128 == 0,
                "slot alignment");
  static_assert(UW <= 256 && UH <= 256, "TMA box limit");
};


// 16-bit storage on the tensor cores: TX x 16 tiles (TX = 32, 64 or 128), one
// warp per block of 8 x-columns by all 16 rows. Same rings as SweepCfg (u
// planes with the halo, u_prev and v^2 dt^2 tiles, a staging plane, one
// barrier per stage in flight), with wider TMA boxes so that the warps'
// shared-memory accesses fall in distinct banks: u rows of TX + 24 elements
// (112, 176 or 304 bytes: the 8 rows of an ldmatrix land on 8 disjoint
// groups of 4 banks), u_prev and v^2 dt^2 rows of TX + 8 (the extra columns
// are the next tile's, read from L2).
// RING_ = 9: the u_prev / v^2 dt^2 ring and the barriers are 9 deep like
// the u ring (the plane loop's unroll), so every slot and barrier parity of
// the loop is a compile-time constant instead of a division by PF + 1 per
// plane; it needs the shared memory of 2 CTAs per SM or fewer.
template <int TX_, int PF_, int MINB_, class T_, int RING_ = 0>
struct TcCfg {
  using T = T_;
  static_assert(sizeof(T) == 2, "16-bit storage only");
  static_assert(TX_ == 32 || TX_ == 64 || TX_ == 128, "tile width");
  static_assert(RING_ == 0 || RING_ == 9, "ring depth: PF + 1, or 9");
  static constexpr bool kScaled = true;
  static constexpr bool kTensor = true;
  static constexpr int TX = TX_, TY = 16, VY = 1, PF = PF_, MINB = MINB_;
  static constexpr int HX = Elem<T>::kHaloX;  // 8: 16-byte aligned box start
  static constexpr int THREADS = 4 * TX;      // one warp per 8 columns
  static constexpr int SU = PF + 5;
  static constexpr int SP = RING_ ? RING_ : PF + 1;
  static constexpr int NB = RING_ ? RING_ : PF + 1;
  static constexpr int UW = TX + 24;      // u slot row (elements): x0-8 .. x0+TX+15
  static constexpr int UH = TY + 2 * kR;
  static constexpr int PW = TX + 8;       // u_prev / v^2 dt^2 slot row
  static constexpr int BOX_U = UW, BOX_P = PW;
  static constexpr int U_SLOT = UW * UH;
  static constexpr int P_SLOT = PW * TY;
  static constexpr uint32_t U_BYTES = U_SLOT * sizeof(T);
  static constexpr uint32_t UP_BYTES = P_SLOT * sizeof(T);
  static constexpr uint32_t C_BYTES = P_SLOT * 4;
  // rings, then one barrier per stage in flight (receivers are recorded
  // by the threads that own the points: no staging plane)
  static constexpr size_t SMEM_BYTES = (size_t)SU * U_BYTES +
                                       (size_t)SP * (UP_BYTES + C_BYTES) + NB * 8;
  static_assert(SU == 9, "the plane loop keeps ring slot = plane mod 9");
  static_assert(U_BYTES % 128 == 0 && UP_BYTES % 128 == 0 && C_BYTES % 128 == 0,
                "slot alignment");
};

// hi + lo += u d without loss: the product exactly as p + e (an FMA gives
// the rounding error of u d), p added to hi with Knuth's TwoSum (hi + p = s
// + err exactly), err + e gathered in lo. A double-float sum of about 48
// significant bits, in FP32 arithmetic.
__device__ __forceinline__ void acc_exact(float &hi, float &lo, float u, float d) {
  const float p = __fmul_rn(u, d);
  const float e = __fmaf_rn(u, d, -p);
  const float s = __fadd_rn(hi, p);
  const float bp = __fsub_rn(s, hi);
  const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(p, bp));
  hi = s;
  lo = __fadd_rn(lo, __fadd_rn(err, e));
}

__device__ __forceinline__ float exp2_int(int k) {
  return ldexpf(1.0f, max(-126, min(127, k)));
}

// kVelocityField = false: tm_c maps v^2 dt^2. true: tm_c maps the velocity
// itself and the kernel forms v^2 dt^2 from it (the allocation-free entry
// point, which has no buffer of its own to hold v^2 dt^2).
//
// sweep_cta is the work of one CTA: tile (bx, by) of the grid, z layer bz.
// tm_u / tm_up / tm_c point to the tensor maps (kernel parameters or global
// memory), co to the coefficients (kept in kernel parameter space, where the
// arithmetic can use them as constant operands), smem_raw to the dynamic
// shared memory.
template <class C, bool kVelocityField, int kMode>
__device__ __forceinline__ void sweep_cta(const CUtensorMap *tm_u,
                                          const CUtensorMap *tm_up,
                                          const CUtensorMap *tm_c,
                                          const SweepArgs &a,
                                          const StencilCoefs &co, int bx,
                                          int by, int bz,
                                          unsigned char *smem_raw, void *unext,
                                          int koff) {
  using T = typename C::T;
  using E = Elem<T>;
  unsigned char *base = smem_raw;  // 128-byte aligned (declaration below)
  T *su = reinterpret_cast<T *>(base);
  T *sp = reinterpret_cast<T *>(base + C::SU * C::U_BYTES);
  float *sc = reinterpret_cast<float *>(base + C::SU * C::U_BYTES +
                                        C::SP * C::UP_BYTES);
  float *sr = sc + C::SP * C::P_SLOT;  // receiver staging (one plane)
  uint64_t *bars = reinterpret_cast<uint64_t *>(sr + C::P_SLOT);

  const int tid = threadIdx.x;
  const int tx = tid % C::NTX;
  const int ty = tid / C::NTX;
  const int x0 = bx * C::TX;
  const int y0 = by * C::TY;
  const int zb = a.zl[bz];
  const int ze = a.zl[bz + 1];
  const int NS = (ze - zb) + 2 * kR;  // stages: 8 to fill the queue, then one per plane

  // Per-call state.
  StepDesc *d = a.desc;
  const long long n = d->n + koff;
  const int nrec = d->nrec;
  const int sx = d->sx - x0, sy = d->sy - y0, sz = d->sz;
  const bool src_here = d->src_active && sx >= 0 && sx < C::TX && sy >= 0 &&
                        sy < C::TY && sz >= zb && sz < ze;
  float wsrc = src_here ? d->wavelet[n] : 0.f;
  int rcur = 0, rend = 0;
  const int4 *rec = d->rec;
  if (nrec > 0) {
    const int tile = by * a.ntx + bx;
    rcur = d->rec_start[tile];
    rend = d->rec_start[tile + 1];
    while (rcur < rend && rec[rcur].x < zb) ++rcur;
  }
  int rz = (rcur < rend) ? rec[rcur].x : 0x7fffffff;  // z of the next receiver
  float *trow = (nrec > 0) ? d->traces + (size_t)n * nrec : nullptr;
  int icur = 0, iend = 0, iz = 0x7fffffff;  // injections (kModeInject)
  const int4 *inj = nullptr;
  const float *irow = nullptr;
  if constexpr ((kMode & kModeInject) != 0) {
    if (d->ninj > 0) {
      const int tile = by * a.ntx + bx;
      inj = d->inj;
      irow = d->inj_val + (size_t)n * d->ninj;
      icur = d->inj_start[tile];
      iend = d->inj_start[tile + 1];
      while (icur < iend && inj[icur].x < zb) ++icur;
      if (icur < iend) iz = inj[icur].x;
    }
  }

  // 16-bit storage: scales of the input fields (absolute steps ab and ab-1)
  // and of the output field (step ab+1). The output scale bounds the new
  // field: |u_next| <= 2|u| + |u_prev| + c |L u| <= 7 max(|u|, |u_prev|) for
  // dt within the stability limit (c |L u| <= 4 max|u|), plus the source;
  // 8 x that bound maps to at most 2^15 in the stored format.
  float s1 = 1.f, s2 = 1.f, so = 1.f;
  long long ab = 0;
  if constexpr (C::kScaled) {
    ab = d->step0 + n;
    const int eu = d->exps[ab & 3], eup = d->exps[(ab + 3) & 3];
    const float mu = __uint_as_float(d->maxbits[ab & 3]);
    const float mup = __uint_as_float(d->maxbits[(ab + 3) & 3]);
    float bound = 8.f * fmaxf(mu, mup);
    if (d->src_active) bound += a.cmax * fabsf(d->wavelet[n]);
    int eo = 0;
    if (bound > 0.f) {
      int e2;
      frexpf(bound, &e2);  // bound <= 2^e2
      eo = e2 - 15;
    }
    s1 = exp2_int(eu - eo);
    s2 = exp2_int(eup - eo);
    so = exp2_int(eo);
    wsrc *= exp2_int(-eo);
    if (bx == 0 && by == 0 && bz == 0 && tid == 0) {
      d->exps[(ab + 1) & 3] = eo;     // read by the next step only
      d->maxbits[(ab + 2) & 3] = 0u;  // accumulated by the next step
    }
  }
  float vmax_out = 0.f;  // largest |output| of this thread (stored units)

  if (tid == 0) {
    prefetch_tensormap(tm_u);
    prefetch_tensormap(tm_up);
    prefetch_tensormap(tm_c);
    for (int b = 0; b < C::NB; ++b) mbar_init(&bars[b], 1);
    fence_barrier_init();
  }
  __syncthreads();

  // Stage s brings u plane zb-4+s and, once s >= 8, u_prev and c of plane
  // zb-8+s (the plane computed at iteration s).
  auto issue = [&](int s) {
    uint64_t *bar = &bars[s % C::NB];
    const int j = zb - 2 * kR + s;
    const bool full = j >= zb;
    mbar_arrive_expect_tx(bar,
                          C::U_BYTES + (full ? C::UP_BYTES + C::C_BYTES : 0));
    tma_load_3d(su + (s % C::SU) * C::U_SLOT, tm_u, bar, x0 - C::HX, y0 - kR,
                j + kR);
    if (full) {
      tma_load_3d(sp + (s % C::SP) * C::P_SLOT, tm_up, bar, x0, y0, j);
      tma_load_3d(sc + (s % C::SP) * C::P_SLOT, tm_c, bar, x0, y0, j);
    }
  };
  if (tid == 0)
    for (int s = 0; s < C::PF && s < NS; ++s) issue(s);

  // q[v][k]: u of this thread's 4 points on row v. The loop below is unrolled
  // by 9, the queue length, so a plane keeps one register for its whole
  // lifetime: plane P = zb-4+s is written into q[v][s % 9] and read back by
  // static index (no shifting moves). With SU == 9 the u ring slot of a
  // stage is likewise s % 9.
  float4 q[C::VY][9];
#pragma unroll
  for (int v = 0; v < C::VY; ++v)
#pragma unroll
    for (int k = 0; k < 9; ++k) q[v][k] = make_float4(0.f, 0.f, 0.f, 0.f);

  const int col = 4 * tx + C::HX;  // smem column of this thread's first point

  // kModeGradAcc: D and the (hi, lo) partial of the next plane to finish,
  // loaded one plane ahead so that their latency overlaps a plane's work
  // instead of stalling its epilogue.
  float4 gd[C::VY], gh[C::VY], gl[C::VY];
  auto grad_load = [&](int jj) {
#pragma unroll
    for (int v = 0; v < C::VY; ++v) {
      const int y = y0 + ty * C::VY + v;
      const int x = x0 + 4 * tx;
      gd[v] = gh[v] = gl[v] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (jj < ze && y < a.ny && x < a.px) {
        const size_t idx = ((size_t)jj * a.ny + y) * a.px + x;
        gd[v] = __ldcs(reinterpret_cast<const float4 *>(a.dsrc + idx));
        gh[v] = *reinterpret_cast<const float4 *>(a.ghi + idx);
        gl[v] = *reinterpret_cast<const float4 *>(a.glo + idx);
      }
    }
  };
  if constexpr ((kMode & kModeGradAcc) != 0) grad_load(zb);

  int s = 0;
  for (int s0 = 0; s0 < NS; s0 += 9) {
#pragma unroll
    for (int p = 0; p < 9; ++p) {
      s = s0 + p;
      if (s >= NS) break;
      // One barrier per plane: it publishes that stage s has landed for
      // every thread (a uniform verdict, so a timeout leaves the loop
      // everywhere) and that every thread is done with plane s-1, whose
      // slots the next issue may overwrite.
      const bool ok =
          mbar_wait_bounded(&bars[s % C::NB], (s / C::NB) & 1, kWaitLimitNs);
      if (__syncthreads_or(!ok)) goto wait_failed;
      if (tid == 0 && s + C::PF < NS) issue(s + C::PF);
      // Front plane (j+4) into the queue.
      const int fslot = (C::SU == 9) ? p : (s % C::SU);
      const T *uf = su + fslot * C::U_SLOT;
#pragma unroll
      for (int v = 0; v < C::VY; ++v)
        q[v][p] = E::load4(uf + (ty * C::VY + v + kR) * C::UW + col);
      const int j = zb - 2 * kR + s;
      if (j < zb) continue;

      const int cslot = (C::SU == 9) ? (p + 5) % 9 : ((s + C::SU - kR) % C::SU);
      const T *uc = su + cslot * C::U_SLOT;  // plane j
      const T *pp = sp + (s % C::SP) * C::P_SLOT;
      const float *pc = sc + (s % C::SP) * C::P_SLOT;
      float4 res[C::VY];
      float4 dres[C::VY];  // kModeStoreD: c (L u) + source
#pragma unroll
      for (int v = 0; v < C::VY; ++v) {
        const int r = ty * C::VY + v + kR;  // smem row of this point row
        // The centre plane j of this thread's points is already in the queue.
        const float4 a1 = q[v][(p + 5) % 9];
        // Packed FP32x2 arithmetic: points (0,1) in `lo`, (2,3) in `hi`.
        // Lane-wise it is the same sequence of IEEE round-to-nearest
        // additions and fused multiply-adds as the scalar form.
        float2 lo = __fmul2_rn(make_float2(co.c0, co.c0), make_float2(a1.x, a1.y));
        float2 hi = __fmul2_rn(make_float2(co.c0, co.c0), make_float2(a1.z, a1.w));
        if constexpr (!C::kScaled) {
          const float4 a0 = E::load4(uc + r * C::UW + col - 4);
          const float4 a2 = E::load4(uc + r * C::UW + col + 4);
          const float xs[12] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y,
                                a1.z, a1.w, a2.x, a2.y, a2.z, a2.w};
#pragma unroll
          for (int m = 1; m <= kR; ++m) {
            const float4 ym = E::load4(uc + (r - m) * C::UW + col);
            const float4 yp = E::load4(uc + (r + m) * C::UW + col);
            const float4 zm = q[v][(p + 5 - m + 9) % 9];
            const float4 zp = q[v][(p + 5 + m) % 9];
            const float2 cx2 = make_float2(co.cx[m - 1], co.cx[m - 1]);
            const float2 cy2 = make_float2(co.cy[m - 1], co.cy[m - 1]);
            const float2 cz2 = make_float2(co.cz[m - 1], co.cz[m - 1]);
            float2 xl, xh;
            if (m % 2 == 0) {  // operands are aligned register pairs
              xl = __fadd2_rn(make_float2(xs[4 - m], xs[5 - m]),
                              make_float2(xs[4 + m], xs[5 + m]));
              xh = __fadd2_rn(make_float2(xs[6 - m], xs[7 - m]),
                              make_float2(xs[6 + m], xs[7 + m]));
            } else {
              xl = make_float2(xs[4 - m] + xs[4 + m], xs[5 - m] + xs[5 + m]);
              xh = make_float2(xs[6 - m] + xs[6 + m], xs[7 - m] + xs[7 + m]);
            }
            lo = __ffma2_rn(cx2, xl, lo);
            hi = __ffma2_rn(cx2, xh, hi);
            lo = __ffma2_rn(cy2, __fadd2_rn(make_float2(ym.x, ym.y),
                                            make_float2(yp.x, yp.y)), lo);
            hi = __ffma2_rn(cy2, __fadd2_rn(make_float2(ym.z, ym.w),
                                            make_float2(yp.z, yp.w)), hi);
            lo = __ffma2_rn(cz2, __fadd2_rn(make_float2(zm.x, zm.y),
                                            make_float2(zp.x, zp.y)), lo);
            hi = __ffma2_rn(cz2, __fadd2_rn(make_float2(zm.z, zm.w),
                                            make_float2(zp.z, zp.w)), hi);
          }
        } else {
          // 16-bit planes: each neighbour pair sum is one mixed-precision add
          // of a stored element to an FP32 value (the other element, taken
          // from the queue or converted once), never a second conversion.
          const uint2 r0 = E::load_raw(uc + r * C::UW + col - 4);
          const uint2 r2 = E::load_raw(uc + r * C::UW + col + 4);
          const float c1[4] = {a1.x, a1.y, a1.z, a1.w};
          // x slot i of this row: 0..3 in r0, 4..7 = centre (FP32), 8..11 in r2
          auto xpair = [&](int i, int j) -> float {
            const bool i32 = i >= 4 && i < 8, j32 = j >= 4 && j < 8;
            const uint2 ri = (i < 4) ? r0 : r2, rj = (j < 4) ? r0 : r2;
            if (i32 && j32) return c1[i - 4] + c1[j - 4];
            if (i32) return E::add_to(rj, j & 3, c1[i - 4]);
            if (j32) return E::add_to(ri, i & 3, c1[j - 4]);
            return E::add_to(ri, i & 3, E::unpack(rj, j & 3));
          };
#pragma unroll
          for (int m = 1; m <= kR; ++m) {
            const uint2 ym = E::load_raw(uc + (r - m) * C::UW + col);
            const uint2 yp = E::load_raw(uc + (r + m) * C::UW + col);
            const float4 zm = q[v][(p + 5 - m + 9) % 9];
            const float4 zp = q[v][(p + 5 + m) % 9];
            const float2 cx2 = make_float2(co.cx[m - 1], co.cx[m - 1]);
            const float2 cy2 = make_float2(co.cy[m - 1], co.cy[m - 1]);
            const float2 cz2 = make_float2(co.cz[m - 1], co.cz[m - 1]);
            const float2 xl = make_float2(xpair(4 - m, 4 + m), xpair(5 - m, 5 + m));
            const float2 xh = make_float2(xpair(6 - m, 6 + m), xpair(7 - m, 7 + m));
            const float2 yl = make_float2(E::add_to(ym, 0, E::unpack(yp, 0)),
                                          E::add_to(ym, 1, E::unpack(yp, 1)));
            const float2 yh = make_float2(E::add_to(ym, 2, E::unpack(yp, 2)),
                                          E::add_to(ym, 3, E::unpack(yp, 3)));
            lo = __ffma2_rn(cx2, xl, lo);
            hi = __ffma2_rn(cx2, xh, hi);
            lo = __ffma2_rn(cy2, yl, lo);
            hi = __ffma2_rn(cy2, yh, hi);
            lo = __ffma2_rn(cz2, __fadd2_rn(make_float2(zm.x, zm.y),
                                            make_float2(zp.x, zp.y)), lo);
            hi = __ffma2_rn(cz2, __fadd2_rn(make_float2(zm.z, zm.w),
                                            make_float2(zp.z, zp.w)), hi);
          }
        }
        const int pofs = (ty * C::VY + v) * C::TX + 4 * tx;
        const float4 upv = E::load4(pp + pofs);
        float4 cv = *reinterpret_cast<const float4 *>(pc + pofs);
        if (kVelocityField) {
          cv.x = cv.x * cv.x * a.dt2;
          cv.y = cv.y * cv.y * a.dt2;
          cv.z = cv.z * cv.z * a.dt2;
          cv.w = cv.w * cv.w * a.dt2;
        }
        const float2 cvl = make_float2(cv.x, cv.y), cvh = make_float2(cv.z, cv.w);
        const float2 ul = make_float2(a1.x, a1.y), uh = make_float2(a1.z, a1.w);
        const float2 pl = make_float2(-upv.x, -upv.y);
        const float2 ph = make_float2(-upv.z, -upv.w);
        float2 ol, oh;
        if constexpr (C::kScaled) {
          // Stored units: u = 2^eu U, u_prev = 2^eup UP, output 2^eo O.
          const float2 s1v = make_float2(s1, s1), s2v = make_float2(s2, s2);
          ol = __ffma2_rn(s1v, __ffma2_rn(cvl, lo, __fadd2_rn(ul, ul)),
                          __fmul2_rn(s2v, pl));
          oh = __ffma2_rn(s1v, __ffma2_rn(cvh, hi, __fadd2_rn(uh, uh)),
                          __fmul2_rn(s2v, ph));
        } else {
          const float2 two = make_float2(2.f, 2.f);
          ol = __ffma2_rn(cvl, lo, __ffma2_rn(two, ul, pl));
          oh = __ffma2_rn(cvh, hi, __ffma2_rn(two, uh, ph));
        }
        float4 o = make_float4(ol.x, ol.y, oh.x, oh.y);
        float4 dv = make_float4(0.f, 0.f, 0.f, 0.f);
        if constexpr ((kMode & kModeStoreD) != 0) {
          const float2 dl = __fmul2_rn(cvl, lo), dh = __fmul2_rn(cvh, hi);
          dv = make_float4(dl.x, dl.y, dh.x, dh.y);
        }
        if (src_here && j == sz && sy == ty * C::VY + v) {
          const int e = sx - 4 * tx;
          if (e == 0) o.x = fmaf(cv.x, wsrc, o.x);
          if (e == 1) o.y = fmaf(cv.y, wsrc, o.y);
          if (e == 2) o.z = fmaf(cv.z, wsrc, o.z);
          if (e == 3) o.w = fmaf(cv.w, wsrc, o.w);
          if constexpr ((kMode & kModeStoreD) != 0) {
            if (e == 0) dv.x = fmaf(cv.x, wsrc, dv.x);
            if (e == 1) dv.y = fmaf(cv.y, wsrc, dv.y);
            if (e == 2) dv.z = fmaf(cv.z, wsrc, dv.z);
            if (e == 3) dv.w = fmaf(cv.w, wsrc, dv.w);
          }
        }
        if constexpr (C::kScaled) {
          vmax_out = fmaxf(vmax_out, fmaxf(fmaxf(fabsf(o.x), fabsf(o.y)),
                                           fmaxf(fabsf(o.z), fabsf(o.w))));
        }
        res[v] = o;
        dres[v] = dv;
      }

      // Point injections on this plane (adjoint sources): stage the plane,
      // add v^2 dt^2 * value per entry (repeated points add up), read back.
      if constexpr ((kMode & kModeInject) != 0) {
        if (j == iz) {
#pragma unroll
          for (int v = 0; v < C::VY; ++v)
            *reinterpret_cast<float4 *>(sr + (ty * C::VY + v) * C::TX + 4 * tx) =
                res[v];
          __syncthreads();
          int last = icur;
          while (last < iend && inj[last].x == j) ++last;
          for (int e = icur + tid; e < last; e += C::THREADS) {
            const int4 r4 = inj[e];
            atomicAdd(&sr[r4.y], pc[r4.y] * irow[r4.z]);
          }
          __syncthreads();
#pragma unroll
          for (int v = 0; v < C::VY; ++v)
            res[v] = *reinterpret_cast<const float4 *>(
                sr + (ty * C::VY + v) * C::TX + 4 * tx);
          __syncthreads();  // the staging plane is free again
          icur = last;
          iz = (icur < iend) ? inj[icur].x : 0x7fffffff;
        }
      }
#pragma unroll
      for (int v = 0; v < C::VY; ++v) {
        const int y = y0 + ty * C::VY + v;
        const int x = x0 + 4 * tx;
        if (y < a.ny && x < a.px) {
          const size_t idx = ((size_t)j * a.ny + y) * a.px + x;
          E::store4_cs(reinterpret_cast<T *>(unext) + idx, res[v]);
          if constexpr ((kMode & kModeStoreD) != 0)
            __stcs(reinterpret_cast<float4 *>(a.dout + idx), dres[v]);
          if constexpr ((kMode & kModeGradAcc) != 0) {
            // This step's u (centre of the queue) times D into the running
            // double-float partial; the host folds it into the FP64 time
            // sum at fixed step boundaries.
            const float4 uc4 = q[v][(p + 5) % 9];
            const float4 d4 = gd[v];
            float4 h = gh[v], l = gl[v];
            acc_exact(h.x, l.x, uc4.x, d4.x);
            acc_exact(h.y, l.y, uc4.y, d4.y);
            acc_exact(h.z, l.z, uc4.z, d4.z);
            acc_exact(h.w, l.w, uc4.w, d4.w);
            *reinterpret_cast<float4 *>(a.ghi + idx) = h;
            *reinterpret_cast<float4 *>(a.glo + idx) = l;
          }
        }
      }
      if constexpr ((kMode & kModeGradAcc) != 0) grad_load(j + 1);

      // Receivers on this plane: stage the plane, then one thread per entry.
      if (j == rz) {
#pragma unroll
        for (int v = 0; v < C::VY; ++v) {
          float4 t = res[v];
          if constexpr (C::kScaled) {
            t.x *= so;
            t.y *= so;
            t.z *= so;
            t.w *= so;
          }
          *reinterpret_cast<float4 *>(sr + (ty * C::VY + v) * C::TX + 4 * tx) =
              t;
        }
        __syncthreads();
        int last = rcur;
        while (last < rend && rec[last].x == j) ++last;
        for (int e = rcur + tid; e < last; e += C::THREADS) {
          const int4 r4 = rec[e];
          trow[r4.z] = sr[r4.y];
        }
        rcur = last;
        rz = (rcur < rend) ? rec[rcur].x : 0x7fffffff;
      }
    }
  }
  if constexpr (C::kScaled) {
    // Largest |u_next| of the step, for the scale of the step after it.
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
      vmax_out = fmaxf(vmax_out, __shfl_xor_sync(0xffffffffu, vmax_out, o));
    if ((tid & 31) == 0 && vmax_out > 0.f)
      atomicMax(&d->maxbits[(ab + 1) & 3], __float_as_uint(vmax_out * so));
  }
  return;

wait_failed:
  {
    // A wait gave up at stage s: record it, then drain the stages still in
    // flight (issued: [0, s + PF)) so no TMA write lands in shared memory
    // after this CTA has exited.
    if (tid == 0) {
      atomicCAS(&a.desc->error, 0, kErrTimeout);
      const int issued = min(NS, s + C::PF);
      for (int t = s; t < issued; ++t)
        if (!mbar_wait_bounded(&bars[t % C::NB], (t / C::NB) & 1, kWaitLimitNs))
          break;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// 16-bit storage with the x and y parts of Eq. 1 on the tensor cores.
//
// In stored units, the y part at output (x, y) is sum_m 5040 w_m (U(y+m) +
// U(y-m)) / (5040 h_y^2). For a warp's block (all 16 rows of the tile by 8
// columns) it is a banded 16 x 24 matrix of the integer weights kWInt times
// the 24 rows of the plane (tile rows -4..19) at those columns: two
// mma.sync m16n8k16 k-steps over plane rows -4..11 and 12..19, the 16-bit
// operands straight from the TMA-staged plane (ldmatrix), FP32
// accumulation. The x part is the plane's 16 rows at columns x-8..x+7 and
// x+8..x+15 times a banded weight matrix, two more k-steps. Every product
// of a stored value and an integer weight is exact in FP32; only the sums
// round. The z part, the centre term and the update stay in FP32 on the
// CUDA cores as in sweep_cta. Each thread owns the four points of its mma
// accumulator: rows g and g+8 of the tile, columns 2c and 2c+1 of its
// warp's block (g = lane / 4, c = lane % 4), i.e. two pairs of adjacent
// points, loaded and stored as 32-bit pairs.

template <class T>
__device__ __forceinline__ unsigned pack_pair(float lo, float hi);
template <>
__device__ __forceinline__ unsigned pack_pair<__half>(float lo, float hi) {
  const __half2 h = __floats2half2_rn(lo, hi);
  return *reinterpret_cast<const unsigned *>(&h);
}
template <>
__device__ __forceinline__ unsigned pack_pair<__nv_bfloat16>(float lo, float hi) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const unsigned *>(&h);
}

template <class T>
__device__ __forceinline__ void mma_16816(float (&d)[4], const unsigned (&a)[4],
                                          unsigned b0, unsigned b1);
template <>
__device__ __forceinline__ void mma_16816<__half>(float (&d)[4], const unsigned (&a)[4],
                                                  unsigned b0, unsigned b1) {
  asm("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, "
      "{%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
template <>
__device__ __forceinline__ void mma_16816<__nv_bfloat16>(float (&d)[4],
                                                         const unsigned (&a)[4],
                                                         unsigned b0, unsigned b1) {
  asm("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, "
      "{%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Four 8 x 8 matrices of 16-bit elements from shared memory (lanes 8j..8j+7
// give the row addresses of matrix j), as stored or transposed.
__device__ __forceinline__ void ldsm_x4(unsigned (&r)[4], uint32_t addr) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(addr)
               : "memory");
}
__device__ __forceinline__ void ldsm_x4_trans(unsigned (&r)[4], uint32_t addr) {
  asm volatile(
      "ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
      : "r"(addr)
      : "memory");
}

// Two 16-bit elements (one 32-bit word) to FP32, low element first.
template <class T>
__device__ __forceinline__ float2 pair_to_f32(unsigned w);
template <>
__device__ __forceinline__ float2 pair_to_f32<__half>(unsigned w) {
  return __half22float2(*reinterpret_cast<const __half2 *>(&w));
}
template <>
__device__ __forceinline__ float2 pair_to_f32<__nv_bfloat16>(unsigned w) {
  return make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xffff0000u));
}

__device__ __forceinline__ float wint(int off) {
  switch (off < 0 ? -off : off) {
    case 1: return 8064.f;   // 5040 w_m, m = 1..4 (kWInt)
    case 2: return -1008.f;
    case 3: return 128.f;
    case 4: return -9.f;
    default: return 0.f;
  }
}

__device__ __forceinline__ float to_f32(__nv_bfloat16 v) {
  return __bfloat162float(v);
}
__device__ __forceinline__ float to_f32(__half v) { return __half2float(v); }

template <class C>
__device__ __forceinline__ void sweep_cta_tc(const CUtensorMap *tm_u,
                                             const CUtensorMap *tm_up,
                                             const CUtensorMap *tm_c,
                                             const SweepArgs &a,
                                             const StencilCoefs &co, int bx,
                                             int by, int bz,
                                             unsigned char *smem_raw,
                                             void *unext, int koff) {
  using T = typename C::T;
  unsigned char *base = smem_raw;
  T *su = reinterpret_cast<T *>(base);
  T *sp = reinterpret_cast<T *>(base + C::SU * C::U_BYTES);
  float *sc = reinterpret_cast<float *>(base + C::SU * C::U_BYTES +
                                        C::SP * C::UP_BYTES);
  uint64_t *bars = reinterpret_cast<uint64_t *>(sc + C::SP * C::P_SLOT);

  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int g = lane >> 2, cq = lane & 3;
  // this thread's points, tile-relative: columns xt, xt+1 of rows g, g+8
  const int xt = 8 * warp + 2 * cq;
  const int x0 = bx * C::TX;
  const int y0 = by * C::TY;
  const int zb = a.zl[bz];
  const int ze = a.zl[bz + 1];
  const int NS = (ze - zb) + 2 * kR;

  StepDesc *d = a.desc;
  const long long n = d->n + koff;
  const int nrec = d->nrec;
  const int sx = d->sx - x0, sy = d->sy - y0, sz = d->sz;
  const bool src_here = d->src_active && sx >= 0 && sx < C::TX && sy >= 0 &&
                        sy < C::TY && sz >= zb && sz < ze;
  float wsrc = src_here ? d->wavelet[n] : 0.f;
  const int src_j = src_here ? sz : -1;  // plane of the source in this CTA
  int rcur = 0, rend = 0;
  const int4 *rec = d->rec;
  if (nrec > 0) {
    const int tile = by * a.ntx + bx;
    rcur = d->rec_start[tile];
    rend = d->rec_start[tile + 1];
    while (rcur < rend && rec[rcur].x < zb) ++rcur;
  }
  int rz = (rcur < rend) ? rec[rcur].x : 0x7fffffff;
  float *trow = (nrec > 0) ? d->traces + (size_t)n * nrec : nullptr;

  // Field scales (see sweep_cta).
  const long long ab = d->step0 + n;
  float s1, s2, so;
  {
    const int eu = d->exps[ab & 3], eup = d->exps[(ab + 3) & 3];
    const float mu = __uint_as_float(d->maxbits[ab & 3]);
    const float mup = __uint_as_float(d->maxbits[(ab + 3) & 3]);
    float bound = 8.f * fmaxf(mu, mup);
    if (d->src_active) bound += a.cmax * fabsf(d->wavelet[n]);
    int eo = 0;
    if (bound > 0.f) {
      int e2;
      frexpf(bound, &e2);
      eo = e2 - 15;
    }
    s1 = exp2_int(eu - eo);
    s2 = exp2_int(eup - eo);
    so = exp2_int(eo);
    wsrc *= exp2_int(-eo);
    if (bx == 0 && by == 0 && bz == 0 && tid == 0) {
      d->exps[(ab + 1) & 3] = eo;
      d->maxbits[(ab + 2) & 3] = 0u;
    }
  }
  float vmax_out = 0.f;

  // Constant mma operands. y: A[m][k] = weight of plane row k (slot row,
  // tile row k - 4) for output row m; k-step 0 takes slot rows 0..15, k-step
  // 1 slot rows 8..23 of which only 16..23 (k >= 8) carry weights. x: B[k][n]
  // = weight of column k of the window for output column n; window 0 starts
  // 8 columns left of the block, window 1 at the block (only k >= 8 used).
  unsigned ya[2][4], xbw[2][2];
#pragma unroll
  for (int ks = 0; ks < 2; ++ks) {
    auto A = [&](int m, int k) {
      return ks == 0 ? wint(k - 4 - m) : (k >= 8 ? wint(k + 4 - m) : 0.f);
    };
    ya[ks][0] = pack_pair<T>(A(g, 2 * cq), A(g, 2 * cq + 1));
    ya[ks][1] = pack_pair<T>(A(g + 8, 2 * cq), A(g + 8, 2 * cq + 1));
    ya[ks][2] = pack_pair<T>(A(g, 2 * cq + 8), A(g, 2 * cq + 9));
    ya[ks][3] = pack_pair<T>(A(g + 8, 2 * cq + 8), A(g + 8, 2 * cq + 9));
    auto B = [&](int k, int nn) {
      return ks == 0 ? wint(k - 8 - nn) : (k >= 8 ? wint(k - nn) : 0.f);
    };
    xbw[ks][0] = pack_pair<T>(B(2 * cq, g), B(2 * cq + 1, g));
    xbw[ks][1] = pack_pair<T>(B(2 * cq + 8, g), B(2 * cq + 9, g));
  }
  // ldmatrix row addresses within a u slot (elements). y (transposed): lane
  // l gives row (l & 7) of matrix l / 8 = slot rows 0..7, 8..15, 8..15,
  // 16..23 at the block's columns. x (as stored): rows (l & 7) + 8 (l/8 odd)
  // of the tile (slot rows + 4) at the window's column 0 or 8.
  const int lj = lane >> 3;
  const int off_y = (8 * ((lj + 1) >> 1) + (lane & 7)) * C::UW + C::HX + 8 * warp;
  const int off_x0 = ((lane & 7) + 8 * (lj & 1) + kR) * C::UW + 8 * warp +
                     8 * (lj >> 1);               // window 0: block column - 8
  const int off_x1 = off_x0 + C::HX;              // window 1: block column
  // shared-space addresses: the u ring's ldmatrix rows of this lane (slot 0)
  // and the barriers, so that a plane's addresses are these plus constants
  const uint32_t su_s = smem_addr(su), bars_s = smem_addr(bars);
  constexpr uint32_t es = sizeof(T);
  const uint32_t ly_s = su_s + es * off_y, lx0_s = su_s + es * off_x0,
                 lx1_s = su_s + es * off_x1;
  // the thread's points in a u slot and in a tile slot (elements)
  const int ua = (g + kR) * C::UW + C::HX + xt, ub = ua + 8 * C::UW;
  const int pa = g * C::PW + xt, pb = pa + 8 * C::PW;
  // their indices within the tile (receiver table entries) and in the
  // output field (elements of plane 0), with their bounds
  const int la = g * C::TX + xt, lb = la + 8 * C::TX;
  const size_t plane_stride = (size_t)a.ny * a.px;
  const size_t oa = (size_t)(y0 + g) * a.px + (x0 + xt);
  const size_t ob = oa + 8 * (size_t)a.px;
  // the thread's two output rows at plane zb, advanced one plane per plane
  T *outa = reinterpret_cast<T *>(unext) + (size_t)zb * plane_stride + oa;
  T *outb = reinterpret_cast<T *>(unext) + (size_t)zb * plane_stride + ob;
  const bool in_x = x0 + xt < a.px;
  const bool wa = in_x && y0 + g < a.ny, wb = in_x && y0 + g + 8 < a.ny;

  if (tid == 0) {
    prefetch_tensormap(tm_u);
    prefetch_tensormap(tm_up);
    prefetch_tensormap(tm_c);
    for (int b = 0; b < C::NB; ++b) mbar_init(&bars[b], 1);
    fence_barrier_init();
  }
  __syncthreads();

  // Stage t brings u plane zb-4+t (slot t % 9) and, once t >= 8, u_prev and
  // v^2 dt^2 of plane zb-8+t (the plane computed at iteration t). slot:
  // t % 9, passed as a constant from the unrolled loop (the ring slots and
  // barriers are t % 9 when SP == NB == 9).
  auto issue = [&](int t, int slot9) {
    const int bslot = C::NB == 9 ? slot9 : t % C::NB;
    const int pslot = C::SP == 9 ? slot9 : t % C::SP;
    uint64_t *bar = &bars[bslot];
    const int j = zb - 2 * kR + t;
    const bool full = j >= zb;
    mbar_arrive_expect_tx(bar,
                          C::U_BYTES + (full ? C::UP_BYTES + C::C_BYTES : 0));
    tma_load_3d(su + slot9 * C::U_SLOT, tm_u, bar, x0 - C::HX, y0 - kR, j + kR);
    if (full) {
      tma_load_3d(sp + pslot * C::P_SLOT, tm_up, bar, x0, y0, j);
      tma_load_3d(sc + pslot * C::P_SLOT, tm_c, bar, x0, y0, j);
    }
  };
  if (tid == 0)
    for (int t = 0; t < C::PF && t < NS; ++t) issue(t, t);

  // q[k]: u of the thread's points (row g: x, y; row g+8: z, w)
  float4 q[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) q[k] = make_float4(0.f, 0.f, 0.f, 0.f);

  int s = 0;
  const int ns_issue = NS - C::PF;  // stages s below it issue stage s + PF
  uint32_t par9 = 0;  // barrier parity of this round of 9 stages (NB == 9)
  for (int s0 = 0; s0 < NS; s0 += 9, par9 ^= 1u) {
#pragma unroll
    for (int p = 0; p < 9; ++p) {
      s = s0 + p;
      if (s >= NS) break;
      // One barrier per plane: stage s has landed for every thread (a
      // uniform verdict, so a timeout leaves the loop everywhere) and every
      // thread is done with plane s-1, whose slots the next issue reuses.
      const bool ok =
          C::NB == 9 ? mbar_wait_bounded_s(bars_s + 8u * p, par9, kWaitLimitNs)
                     : mbar_wait_bounded(&bars[s % C::NB], (s / C::NB) & 1, kWaitLimitNs);
      if (__syncthreads_or(!ok)) goto wait_failed;
      if (tid == 0 && s < ns_issue) issue(s + C::PF, (p + C::PF) % 9);
      {
        const T *uf = su + p * C::U_SLOT;  // SU == 9: slot of stage s is s % 9
        const float2 fa = pair_to_f32<T>(*reinterpret_cast<const unsigned *>(uf + ua));
        const float2 fb = pair_to_f32<T>(*reinterpret_cast<const unsigned *>(uf + ub));
        q[p] = make_float4(fa.x, fa.y, fb.x, fb.y);
      }
      const int j = zb - 2 * kR + s;
      // j >= zb, i.e. s >= 8: every stage after the first 8 (s0 is a
      // multiple of 9, so only the first round holds the queue's fill)
      if (p == 8 || s0 != 0) {
        const T *uc = su + ((p + 5) % 9) * C::U_SLOT;  // plane j
        const int pslot = C::SP == 9 ? p : s % C::SP;
        const T *pp = sp + pslot * C::P_SLOT;
        const float *pc = sc + pslot * C::P_SLOT;
        // x and y parts on the tensor cores (integer weights, stored units)
        float dyv[4] = {0.f, 0.f, 0.f, 0.f}, dxv[4] = {0.f, 0.f, 0.f, 0.f};
        {
          unsigned r[4];
          const uint32_t cofs = ((p + 5) % 9) * C::U_BYTES;  // plane j's slot
          ldsm_x4_trans(r, ly_s + cofs);
          mma_16816<T>(dyv, ya[0], r[0], r[1]);
          mma_16816<T>(dyv, ya[1], r[2], r[3]);
          ldsm_x4(r, lx0_s + cofs);
          mma_16816<T>(dxv, r, xbw[0][0], xbw[0][1]);
          ldsm_x4(r, lx1_s + cofs);
          mma_16816<T>(dxv, r, xbw[1][0], xbw[1][1]);
        }
        const float2 upa = pair_to_f32<T>(*reinterpret_cast<const unsigned *>(pp + pa));
        const float2 upb = pair_to_f32<T>(*reinterpret_cast<const unsigned *>(pp + pb));
        const float2 cvl = *reinterpret_cast<const float2 *>(pc + pa);
        const float2 cvh = *reinterpret_cast<const float2 *>(pc + pb);

        const float4 a1 = q[(p + 5) % 9];  // centre plane j
        float2 lo = __fmul2_rn(make_float2(co.c0, co.c0), make_float2(a1.x, a1.y));
        float2 hi = __fmul2_rn(make_float2(co.c0, co.c0), make_float2(a1.z, a1.w));
#pragma unroll
        for (int m = 1; m <= kR; ++m) {
          const float4 zm = q[(p + 5 - m + 9) % 9];
          const float4 zp = q[(p + 5 + m) % 9];
          const float2 cz2 = make_float2(co.cz[m - 1], co.cz[m - 1]);
          lo = __ffma2_rn(cz2, __fadd2_rn(make_float2(zm.x, zm.y), make_float2(zp.x, zp.y)), lo);
          hi = __ffma2_rn(cz2, __fadd2_rn(make_float2(zm.z, zm.w), make_float2(zp.z, zp.w)), hi);
        }
        const float2 sy2 = make_float2(co.syi, co.syi), sx2 = make_float2(co.sxi, co.sxi);
        lo = __ffma2_rn(sy2, make_float2(dyv[0], dyv[1]), lo);
        hi = __ffma2_rn(sy2, make_float2(dyv[2], dyv[3]), hi);
        lo = __ffma2_rn(sx2, make_float2(dxv[0], dxv[1]), lo);
        hi = __ffma2_rn(sx2, make_float2(dxv[2], dxv[3]), hi);

        const float2 ul = make_float2(a1.x, a1.y), uh = make_float2(a1.z, a1.w);
        const float2 s1v = make_float2(s1, s1), s2v = make_float2(s2, s2);
        float2 ol = __ffma2_rn(s1v, __ffma2_rn(cvl, lo, __fadd2_rn(ul, ul)),
                               __fmul2_rn(s2v, make_float2(-upa.x, -upa.y)));
        float2 oh = __ffma2_rn(s1v, __ffma2_rn(cvh, hi, __fadd2_rn(uh, uh)),
                               __fmul2_rn(s2v, make_float2(-upb.x, -upb.y)));
        if (j == src_j) {
          const int e = sx - xt;
          if (sy == g) {
            if (e == 0) ol.x = fmaf(cvl.x, wsrc, ol.x);
            if (e == 1) ol.y = fmaf(cvl.y, wsrc, ol.y);
          }
          if (sy == g + 8) {
            if (e == 0) oh.x = fmaf(cvh.x, wsrc, oh.x);
            if (e == 1) oh.y = fmaf(cvh.y, wsrc, oh.y);
          }
        }
        vmax_out = fmaxf(vmax_out, fmaxf(fmaxf(fabsf(ol.x), fabsf(ol.y)),
                                         fmaxf(fabsf(oh.x), fabsf(oh.y))));
        if (wa) __stcs(reinterpret_cast<unsigned *>(outa), pack_pair<T>(ol.x, ol.y));
        if (wb) __stcs(reinterpret_cast<unsigned *>(outb), pack_pair<T>(oh.x, oh.y));
        outa += plane_stride;
        outb += plane_stride;
        // Receivers on this plane: each thread records the entries at its
        // own points (no staging, so no barrier across the warps).
        if (j == rz) {
          int e = rcur;
          for (; e < rend; ++e) {
            const int4 r4 = rec[e];
            if (r4.x != j) break;
            const int da = r4.y - la, db = r4.y - lb;
            if (da == 0) trow[r4.z] = ol.x * so;
            if (da == 1) trow[r4.z] = ol.y * so;
            if (db == 0) trow[r4.z] = oh.x * so;
            if (db == 1) trow[r4.z] = oh.y * so;
          }
          rcur = e;
          rz = (rcur < rend) ? rec[rcur].x : 0x7fffffff;
        }
      }
    }
  }
  {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
      vmax_out = fmaxf(vmax_out, __shfl_xor_sync(0xffffffffu, vmax_out, o));
    if ((tid & 31) == 0 && vmax_out > 0.f)
      atomicMax(&d->maxbits[(ab + 1) & 3], __float_as_uint(vmax_out * so));
  }
  return;

wait_failed:
  {
    // A wait gave up at stage s: record it, then drain the stages still in
    // flight (issued: [0, s + PF)) so no TMA write lands in shared memory
    // after this CTA has exited.
    if (tid == 0) {
      atomicCAS(&a.desc->error, 0, kErrTimeout);
      const int issued = min(NS, s + C::PF);
      for (int t = s; t < issued; ++t)
        if (!mbar_wait_bounded(&bars[t % C::NB], (t / C::NB) & 1, kWaitLimitNs))
          break;
    }
    __syncthreads();
  }
}

// One step of one grid: CTA (blockIdx.x, .y) is a tile, blockIdx.z a z layer.
template <class C, bool kVelocityField = false, int kMode = 0>
__global__ void __launch_bounds__(C::THREADS, C::MINB)
    wave_sweep_kernel(const __grid_constant__ CUtensorMap tm_u,
                      const __grid_constant__ CUtensorMap tm_up,
                      const __grid_constant__ CUtensorMap tm_c,
                      const SweepArgs a) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  // The adjoint-gradient modes are launched back to back without graphs and
  // allow programmatic dependent launch: the next sweep's grid may be
  // scheduled once every CTA of this one has started, and this grid reads
  // nothing until the previous one has completed and its writes are visible
  // (no-ops for an ordinary launch). The plain sweep runs in graphs, where
  // the same scheme measured slower (1024 x 1024 x 512: 407 against 416
  // Gpts/s), and does not use it.
  if constexpr (kMode != 0) {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
  }
  if constexpr (C::kTensor) {
    static_assert(!kVelocityField && kMode == 0, "16-bit sweeps: forward only");
    sweep_cta_tc<C>(&tm_u, &tm_up, &tm_c, a, a.k, blockIdx.x, blockIdx.y,
                    blockIdx.z, smem_raw, a.unext, a.koff);
  } else {
    sweep_cta<C, kVelocityField, kMode>(&tm_u, &tm_up, &tm_c, a, a.k, blockIdx.x,
                                        blockIdx.y, blockIdx.z, smem_raw, a.unext,
                                        a.koff);
  }
}

// One shot of a batch (device memory, 128-byte aligned): its tensor maps for
// both buffer parities, its arguments, and where its CTAs start.
struct alignas(128) BatchShot {
  CUtensorMap halo[2];  // u halo box over buf[0] / buf[1]
  CUtensorMap tile[2];  // u_prev tile box over buf[0] / buf[1]
  CUtensorMap cmap;     // v^2 dt^2 tile box
  SweepArgs args;       // unext and koff are not used: passed per launch
  void *buf[2];         // buf[0] holds the shot's step 0
  long long b0;         // batch step at which the shot takes its step 0
  int nsteps;           // the shot's step count: later batch steps skip it
  int cta_begin;        // first linear CTA index of this shot
  int ntx, nty;         // tiles; args.nlayers layers
};

__device__ __forceinline__ void tensormap_acquire(const CUtensorMap *m) {
  asm volatile(
      "fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(
          reinterpret_cast<uint64_t>(m))
      : "memory");
}

// One step of every shot of a batch: the 1D grid is the concatenation of the
// shots' CTA grids (shot i owns [cta_begin_i, cta_begin_{i+1})). Batch step k
// is step k - b0 of each shot; each shot's buffers alternate from its own
// step 0, so a shot computes exactly what the single-grid kernel computes.
// All shots of one launch share the grid spacing, whose coefficients come as
// a kernel parameter.
template <class C>
__global__ void __launch_bounds__(C::THREADS, C::MINB)
    wave_sweep_batched_kernel(const BatchShot *__restrict__ shots, int nshots,
                              long long k, const StencilCoefs co) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int lin = blockIdx.x;
  int lo = 0, hi = nshots - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (shots[mid].cta_begin <= lin) lo = mid; else hi = mid - 1;
  }
  const BatchShot &sh = shots[lo];
  const int local = lin - sh.cta_begin;
  const int per_layer = sh.ntx * sh.nty;
  const int bz = local / per_layer;
  const int rem = local - bz * per_layer;
  const int by = rem / sh.ntx;
  const int bx = rem - by * sh.ntx;
  const long long n = k - sh.b0;  // the shot's own step
  if (n >= sh.nsteps) return;     // finished inside this group of steps
  const int cur = (int)(n & 1);   // buffer holding the shot's u
  // The shot's arguments are read in place from the table (uniform loads
  // through the read-only path): a shared copy would add static shared
  // memory and leave room for only 3 FP32 CTAs per SM instead of 4. Thread 0
  // issues every TMA load of the CTA, so its acquire orders them after the
  // host's copy of the table.
  if (threadIdx.x == 0) {
    tensormap_acquire(&sh.halo[cur]);
    tensormap_acquire(&sh.tile[cur ^ 1]);
    tensormap_acquire(&sh.cmap);
  }
  if constexpr (C::kTensor)
    sweep_cta_tc<C>(&sh.halo[cur], &sh.tile[cur ^ 1], &sh.cmap, sh.args, co, bx, by,
                    bz, smem_raw, sh.buf[cur ^ 1], (int)n);
  else
    sweep_cta<C, false, 0>(&sh.halo[cur], &sh.tile[cur ^ 1], &sh.cmap, sh.args, co, bx,
                           by, bz, smem_raw, sh.buf[cur ^ 1], (int)n);
}

}  // namespace gbw
