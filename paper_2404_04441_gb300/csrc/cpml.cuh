// CPML absorbing layer for the second-order equation (the paper's CPML-like
// boundary, Sec. 2, after Komatitsch and Martin 2007; it prints no equations).
//
// From complex-frequency-shifted stretching of each axis,
//     u_tt = v^2 sum_a ( d_aa u + d_a psi_a + zeta_a ),
//     psi_a^n  = b_a psi_a^{n-1}  + a_a D1_a u^n,
//     zeta_a^n = b_a zeta_a^{n-1} + a_a ( D2_a u^n + D1_a psi_a^n ),
// b = exp(-(d + alpha) dt), a = d / (d + alpha) (b - 1), D2_a the axis part of
// Eq. 1 and D1_a the 8th-order central first derivative. psi_a and zeta_a are
// non-zero only in the two slabs of npml cells at the faces normal to a and
// are stored there.
//
// The leapfrog update with the layer is the plain update plus
//     C * sum_a ( D1_a psi_a^n + zeta_a^n ),
// and the axis-a term is non-zero only within w = npml + 4 cells of the two
// faces normal to a. So the sweep runs unchanged over the whole grid, and
// afterwards one kernel per axis walks every line along that axis through its
// two end segments of w cells (one segment of the whole line when the two would
// overlap): it updates psi_a and zeta_a from u^n (which the sweep does not
// overwrite) and adds the axis term to u^{n+1}. The three axis kernels run
// one after another, so corner points are updated by each axis in turn with
// no race. Receivers within w of a face are then re-recorded.
#pragma once

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdlib>

#include "common.cuh"
#include "sweep.cuh"

namespace gbw {

struct CpmlGeom {
  int nx, ny, nz;
  int px;   // row pitch of v^2 dt^2 (floats)
  int pxu;  // row pitch of the wavefields (elements; px for FP32 storage)
  int npml, w;         // layer cells; correction width npml + 4
  float *psi[3], *zeta[3];           // slab storage per axis
  const float *bprof[3], *aprof[3];  // per-axis b, a (length n_a)
  float c2[3][5];  // D2 weights / h_a^2 (index 0: centre)
  float c1[3][5];  // D1 weights / h_a (index 1..4)
};

// The layer's profile along one axis of n cells (npml layer cells at each
// end), computed in FP64 and stored FP32: b = exp(-(d + alpha) dt) and
// a = d / (d + alpha) (b - 1), with d = d0 xi^2, d0 = 3 vmax ln(1/R) /
// (2 npml h), alpha = pi f_cps (1 - xi) and xi in (0, 1] the depth into the
// layer (1 at the face); b = 1 and a = 0 outside the layer.
inline void cpml_profile(int n, int npml, double R, double f_cps, double vmax, double h,
                         double dt, float *b, float *a) {
  const double pi = 3.14159265358979323846;
  const double d0 = 3.0 * vmax * std::log(1.0 / R) / (2.0 * npml * h);
  for (int i = 0; i < n; ++i) {
    double xi = 0.0;
    if (i < npml) xi = (double)(npml - i) / npml;
    if (i >= n - npml) xi = std::max(xi, (double)(i - (n - npml - 1)) / npml);
    if (xi <= 0.0) {
      b[i] = 1.f;
      a[i] = 0.f;
      continue;
    }
    const double dd = d0 * xi * xi, al = pi * f_cps * (1.0 - xi);
    const double bb = std::exp(-(dd + al) * dt);
    b[i] = (float)bb;
    a[i] = (float)(dd + al > 0.0 ? dd / (dd + al) * (bb - 1.0) : 0.0);
  }
}

// The layer's D2 (Eq. 1's axis part) and D1 weights along axis ax of
// spacing h.
inline void cpml_axis_coefs(CpmlGeom &g, int ax, double h) {
  g.c2[ax][0] = (float)(kW[0] / (h * h));
  g.c1[ax][0] = 0.f;
  for (int m = 1; m <= 4; ++m) {
    g.c2[ax][m] = (float)(kW[m] / (h * h));
    g.c1[ax][m] = (float)(kW1[m] / h);
  }
}

// Whether an axis of n cells takes the unrolled segment kernels: a layer of
// 8 or 16 cells, two disjoint end segments (n >= 2 (npml + 4)), and 32-bit
// per-position offsets (fstep, sstep: the axis's field and slab steps);
// GBWAVE_CPML_GENERIC=1 keeps the line walks everywhere (the two forms give
// bitwise equal results).
inline bool cpml_seg_fits(int npml, int n, long long fstep, long long sstep) {
  const char *gen = std::getenv("GBWAVE_CPML_GENERIC");
  return (npml == 8 || npml == 16) && n >= 2 * (npml + 4) &&
         (long long)(npml + 3) * fstep <= INT32_MAX &&
         (long long)(npml - 1) * sstep <= INT32_MAX && !(gen && std::atoi(gen) == 1);
}

// Slab storage, cell-major: cell in [0, 2 npml) counts the low slab's npml
// cells, then the high slab's; the x slabs hold ((cell nz + z) ny + y), the y
// slabs ((cell nz + z) nx + x), the z slabs ((cell ny + y) nx + x), so that
// adjacent lines (adjacent threads) are adjacent in memory.
__device__ __forceinline__ bool cpml_in_slab(int i, int n, int npml) {
  return i < npml || i >= n - npml;
}

__device__ __forceinline__ int cpml_cell(int i, int n, int npml) {
  return i < npml ? i : i - (n - 2 * npml);
}

constexpr int kCpmlChunk = 4;  // positions per batch of loads

// Wavefield elements in the layer kernels. FP32 fields are used as stored.
// 16-bit fields (BF16 / FP16 storage) hold value / 2^e, e the exponent of
// the time step the field holds (StepDesc::exps, chosen by the sweep that
// wrote it): a read converts exactly and multiplies by 2^e, a write
// multiplies by 2^-e (exact) and rounds once to the format, as the sweep's
// stores do. v^2 dt^2, psi and zeta stay FP32.
template <class T>
__device__ __forceinline__ float cpml_get(const T *p, float s) {
  if constexpr (std::is_same<T, float>::value) return *p;
  else return to_f32(*p) * s;
}

template <class T>
__device__ __forceinline__ void cpml_put(T *p, float v, float inv) {
  if constexpr (std::is_same<T, float>::value) *p = v;
  else if constexpr (std::is_same<T, __half>::value) *p = __float2half_rn(v * inv);
  else *p = __float2bfloat16_rn(v * inv);
}

// Four consecutive elements from p (16 bytes for FP32, 8 for 16-bit; p
// aligned to that).
template <class T>
__device__ __forceinline__ void cpml_get4(const T *p, float s, float *v) {
  if constexpr (std::is_same<T, float>::value) {
    const float4 t = *reinterpret_cast<const float4 *>(p);
    v[0] = t.x;
    v[1] = t.y;
    v[2] = t.z;
    v[3] = t.w;
  } else {
    const uint2 w = *reinterpret_cast<const uint2 *>(p);
    const T *e = reinterpret_cast<const T *>(&w);
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] = to_f32(e[k]) * s;
  }
}

template <class T>
__device__ __forceinline__ void cpml_put4(T *p, const float *v, float inv) {
  if constexpr (std::is_same<T, float>::value) {
    *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
  } else {
    uint2 w;
    T *e = reinterpret_cast<T *>(&w);
#pragma unroll
    for (int k = 0; k < 4; ++k) cpml_put(e + k, v[k], inv);
    *reinterpret_cast<uint2 *>(p) = w;
  }
}

// Scales of one step's fields (16-bit storage): 2^e of u^n and of u^{n+1},
// 2^-e of u^{n+1}, for absolute step step0 + n + koff; and the running
// maximum of |u^{n+1}| that the next step's scale is chosen from (the
// corrected shell values enter it). FP32: all ones, nothing read.
template <class T>
struct CpmlScale {
  float su = 1.f, so = 1.f, inv_so = 1.f;
  unsigned *maxbits = nullptr;
  __device__ __forceinline__ void init(const StepDesc *d, int koff) {
    if constexpr (!std::is_same<T, float>::value) {
      const long long ab = d->step0 + d->n + koff;
      su = exp2_int(d->exps[ab & 3]);
      const int eo = d->exps[(ab + 1) & 3];
      so = exp2_int(eo);
      inv_so = exp2_int(-eo);
      maxbits = const_cast<unsigned *>(&d->maxbits[(ab + 1) & 3]);
    }
  }
  // the largest |value| the warp's remaining lanes wrote (lanes past the
  // last line have returned), into the running maximum: non-negative floats
  // order as their bit patterns
  __device__ __forceinline__ void commit(float vmax) const {
    if constexpr (!std::is_same<T, float>::value) {
      const unsigned m = __activemask();
      const unsigned r = __reduce_max_sync(m, __float_as_uint(vmax));
      if ((threadIdx.x & 31) == __ffs(m) - 1 && r != 0u) atomicMax(maxbits, r);
    }
  }
};

// Four consecutive values of an x row from position p (p a multiple of 4,
// the row 16-byte aligned with its padding up to a multiple of 4 in
// bounds); positions outside [0, n) read as zero.
template <class T>
__device__ __forceinline__ void cpml_row4(const T *row, int p, int n, float *v, float s) {
  if (p < 0 || p >= n) {
    v[0] = v[1] = v[2] = v[3] = 0.f;
    return;
  }
  float t[4];
  cpml_get4(row + p, s, t);
  v[0] = t[0];
  v[1] = p + 1 < n ? t[1] : 0.f;
  v[2] = p + 2 < n ? t[2] : 0.f;
  v[3] = p + 3 < n ? t[3] : 0.f;
}

// One kernel per axis AX (0 = x, 1 = y, 2 = z): one thread per line along
// AX, adjacent lines (adjacent y for x, adjacent x for y and z) in adjacent
// threads. A thread walks its line's end segments, positions i0 .. i1-1
// ([0, w) and [n - w, n), or [0, n) when they would overlap), with register
// windows of u^n (positions i-4 .. i+F+7) and psi^n (i-4 .. i+F+3), F
// positions per batch: at position i it computes psi(k), k = i + 4, in the
// slab cells of the segment's own range i0 .. i1 + 3 (exactly the segment's
// slab cells, so each is updated once per step), then, for i0 <= i < i1,
// zeta^n(i) in the slab cells and u^{n+1}(i) += C (D1 psi^n + zeta^n). The
// walk starts at or before i0 - 4, where the psi used by the corrections is
// zero (before the grid, or between the slabs). The loads of the next batch
// are in flight while the current one is computed. x rows are walked in
// batches aligned to 4 positions and moved as float4 (a row is contiguous
// in one thread); y and z lines are coalesced across the threads.
// kStoreD (the gradient's recompute): the same correction C (D1 psi + zeta)
// is also added to dout, the step's forward increment D = u^{n+1} - 2u^n +
// u^{n-1} stored by the sweep (field layout).
// T: the wavefields' storage (float, or 16-bit with the step's scales read
// from d at absolute step step0 + n + koff). The walk of line t (index
// across the lines) in row q of lines (z for x and y lines, y for z lines).
template <int AX, class T, bool kStoreD>
__device__ __forceinline__ void cpml_line_walk(const CpmlGeom &g, int t, int q,
                                               const T *__restrict__ u, T *__restrict__ unext,
                                               const float *__restrict__ c,
                                               float *__restrict__ dout, const StepDesc *d,
                                               int koff) {
  static_assert(!kStoreD || std::is_same<T, float>::value, "D is stored for FP32 only");
  constexpr int F = kCpmlChunk;
  int n;
  // field offset and stride (pitch pxu), v^2 dt^2 offset and stride (px),
  // slab offset and stride
  long long ub, us, cb, cs, sb, ss;
  if (AX == 0) {
    if (t >= g.ny) return;
    n = g.nx;
    ub = ((long long)q * g.ny + t) * g.pxu;
    us = 1;
    cb = ((long long)q * g.ny + t) * g.px;
    cs = 1;
    sb = (long long)q * g.ny + t;
    ss = (long long)g.nz * g.ny;
  } else {
    if (t >= g.nx) return;
    n = AX == 1 ? g.ny : g.nz;
    ub = AX == 1 ? (long long)q * g.ny * g.pxu + t : (long long)q * g.pxu + t;
    us = AX == 1 ? (long long)g.pxu : (long long)g.ny * g.pxu;
    cb = AX == 1 ? (long long)q * g.ny * g.px + t : (long long)q * g.px + t;
    cs = AX == 1 ? (long long)g.px : (long long)g.ny * g.px;
    sb = (long long)q * g.nx + t;
    ss = AX == 1 ? (long long)g.nz * g.nx : (long long)g.ny * g.nx;
  }
  if constexpr (std::is_same<T, float>::value) {  // FP32 storage: pxu == px
    cb = ub;
    cs = us;
  }
  CpmlScale<T> sc;
  sc.init(d, koff);
  float vmax = 0.f;
  const T *__restrict__ ul = u + ub;
  const float *__restrict__ cl = c + cb;
  T *__restrict__ nl = unext + ub;
  float *__restrict__ dl = kStoreD ? dout + ub : nullptr;
  float *__restrict__ psi = g.psi[AX] + sb;
  float *__restrict__ zeta = g.zeta[AX] + sb;
  const float *bp = g.bprof[AX];
  const float *ap = g.aprof[AX];
  const int npml = g.npml, w = g.w;
  const bool two = n >= 2 * w;
  for (int sg = 0; sg < (two ? 2 : 1); ++sg) {
    const int i0 = (two && sg == 1) ? n - w : 0;
    const int i1 = two ? (sg == 0 ? w : n) : n;
    // Batch of positions i .. i+F-1: u(i+8+f), psi^{n-1}(i+4+f), zeta^{n-1},
    // C and u^{n+1} at i+f.
    float nw[F], npp[F], nzp[F], ncc[F], nun[F];
    auto load = [&](int i) {
      if (AX == 0) {
        cpml_row4(ul, i + 8, n, nw, sc.su);
        if (i + F > i0 && i < i1) {
          cpml_row4(cl, i, n, ncc, 1.f);
          cpml_row4(nl, i, n, nun, sc.so);
        } else {
#pragma unroll
          for (int f = 0; f < F; ++f) ncc[f] = nun[f] = 0.f;
        }
      }
#pragma unroll
      for (int f = 0; f < F; ++f) {
        const int k = i + 4 + f;
        npp[f] = (k >= 0 && k < n && k < i1 + 4 && cpml_in_slab(k, n, npml))
                     ? psi[cpml_cell(k, n, npml) * ss] : 0.f;
        const int p = i + f;
        const bool act = p >= i0 && p < i1;
        nzp[f] = (act && cpml_in_slab(p, n, npml)) ? zeta[cpml_cell(p, n, npml) * ss] : 0.f;
        if (AX != 0) {
          const int kw = i + 8 + f;
          nw[f] = (kw < n) ? cpml_get(ul + kw * us, sc.su) : 0.f;
          ncc[f] = act ? cl[p * cs] : 0.f;
          nun[f] = act ? cpml_get(nl + p * us, sc.so) : 0.f;
        }
      }
    };
    float W[12 + F];  // W[m] = u(i - 4 + m)
    float P[8 + F];   // P[m] = psi(i - 4 + m)
    int i = AX == 0 ? ((i0 - 4) & ~3) : i0 - 4;
    if (AX == 0) {
#pragma unroll
      for (int m = 0; m < 12; m += 4) cpml_row4(ul, i - 4 + m, n, W + m, sc.su);
    } else {
#pragma unroll
      for (int m = 0; m < 12; ++m) {
        const int k = i - 4 + m;
        W[m] = (k >= 0 && k < n) ? cpml_get(ul + k * us, sc.su) : 0.f;
      }
    }
#pragma unroll
    for (int m = 0; m < 8; ++m) P[m] = 0.f;
    load(i);
    for (; i < i1; i += F) {
      float pp[F], zp[F], cc[F], un[F];
#pragma unroll
      for (int f = 0; f < F; ++f) {
        W[12 + f] = nw[f];
        pp[f] = npp[f];
        zp[f] = nzp[f];
        cc[f] = ncc[f];
        un[f] = nun[f];
      }
      if (i + F < i1) load(i + F);
#pragma unroll
      for (int f = 0; f < F; ++f) {  // psi(i + 4 + f) from u(i + f .. i + f + 8)
        const int k = i + 4 + f;
        float v = 0.f;
        if (k >= 0 && k < n && k < i1 + 4 && cpml_in_slab(k, n, npml)) {
          float d1 = 0.f;
#pragma unroll
          for (int m = 1; m <= kR; ++m) d1 = fmaf(g.c1[AX][m], W[8 + f + m] - W[8 + f - m], d1);
          v = fmaf(__ldg(bp + k), pp[f], __ldg(ap + k) * d1);
          psi[cpml_cell(k, n, npml) * ss] = v;
        }
        P[8 + f] = v;
      }
      float out[F];
#pragma unroll
      for (int f = 0; f < F; ++f) {  // u^{n+1}(i + f) += C (D1 psi + zeta)
        const int p = i + f;
        out[f] = un[f];
        if (p < i0 || p >= i1) continue;
        float d1p = 0.f;
#pragma unroll
        for (int m = 1; m <= kR; ++m) d1p = fmaf(g.c1[AX][m], P[4 + f + m] - P[4 + f - m], d1p);
        float corr = d1p;
        if (cpml_in_slab(p, n, npml)) {
          float d2 = g.c2[AX][0] * W[4 + f];
#pragma unroll
          for (int m = 1; m <= kR; ++m) d2 = fmaf(g.c2[AX][m], W[4 + f + m] + W[4 + f - m], d2);
          const float zt = fmaf(__ldg(bp + p), zp[f], __ldg(ap + p) * (d2 + d1p));
          zeta[cpml_cell(p, n, npml) * ss] = zt;
          corr += zt;
        }
        out[f] = fmaf(cc[f], corr, un[f]);
        vmax = fmaxf(vmax, fabsf(out[f]));
        if (AX != 0) cpml_put(nl + p * us, out[f], sc.inv_so);
        if constexpr (kStoreD) dl[p * us] = fmaf(cc[f], corr, dl[p * us]);
      }
      // x: the whole aligned batch in one store (positions outside the
      // segment keep the value just read, which a 16-bit write reproduces
      // exactly; this thread owns the row)
      if (AX == 0 && i + F > i0 && i < i1) cpml_put4(nl + i, out, sc.inv_so);
#pragma unroll
      for (int m = 0; m < 12; ++m) W[m] = W[m + F];
#pragma unroll
      for (int m = 0; m < 8; ++m) P[m] = P[m + F];
    }
  }
  sc.commit(vmax);
}

template <int AX, class T, bool kStoreD = false>
__global__ void __launch_bounds__(128)
    cpml_line_kernel(CpmlGeom g, const T *__restrict__ u, T *__restrict__ unext,
                     const float *__restrict__ c, float *__restrict__ dout,
                     const StepDesc *d, int koff) {
  cpml_line_walk<AX, T, kStoreD>(g, blockIdx.x * blockDim.x + threadIdx.x, blockIdx.y, u,
                                 unext, c, dout, d, koff);
}


// Discrete adjoint of the layer (the gradient's backward steps), in the
// form the sweep runs it, p = C q. After the plain adjoint sweep has written
// p^k = 2p^{k+1} - p^{k+2} + C L p^{k+1} (+ injections), for each axis a:
//     nu_a^k = p^{k+1} + B_a nu_a^{k+1}              (slab cells)
//     mu_a^k = -D1_a (p^{k+1} + A_a nu_a^k) + B_a mu_a^{k+1}
//     p^k   += C ( D2_a (A_a nu_a^k) - D1_a (A_a mu_a^k) )
// (D2_a symmetric and D1_a antisymmetric with the zero halo). A nu and A mu
// vanish outside the slabs, so the correction reaches w = npml + 4 cells
// from each face, as in the forward. One thread per line, the same end
// segments; the walk starts 8 positions before a segment: at position i it
// forms nu (and g = p + A nu) at i + 8, mu at i + 4 (from g at i .. i + 8)
// and, inside the segment, the correction at i. Each slab cell is updated
// by the segment that owns it (the whole line when the segments overlap).
template <int AX>
__global__ void __launch_bounds__(128)
    cpml_adjoint_line_kernel(CpmlGeom g, const float *__restrict__ p1,
                             float *__restrict__ p0, const float *__restrict__ c,
                             float *__restrict__ nus, float *__restrict__ mus) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int q = blockIdx.y;
  int n;
  long long ub, us, sb, ss;
  if (AX == 0) {
    if (t >= g.ny) return;
    n = g.nx;
    ub = ((long long)q * g.ny + t) * g.px;
    us = 1;
    sb = (long long)q * g.ny + t;
    ss = (long long)g.nz * g.ny;
  } else {
    if (t >= g.nx) return;
    n = AX == 1 ? g.ny : g.nz;
    ub = AX == 1 ? (long long)q * g.ny * g.px + t : (long long)q * g.px + t;
    us = AX == 1 ? (long long)g.px : (long long)g.ny * g.px;
    sb = (long long)q * g.nx + t;
    ss = AX == 1 ? (long long)g.nz * g.nx : (long long)g.ny * g.nx;
  }
  const float *__restrict__ pl = p1 + ub;
  const float *__restrict__ cl = c + ub;
  float *__restrict__ ol = p0 + ub;
  float *__restrict__ nu = nus + sb;
  float *__restrict__ mu = mus + sb;
  const float *bp = g.bprof[AX];
  const float *ap = g.aprof[AX];
  const int npml = g.npml, w = g.w;
  const bool two = n >= 2 * w;
  for (int sg = 0; sg < (two ? 2 : 1); ++sg) {
    const int i0 = (two && sg == 1) ? n - w : 0;
    const int i1 = two ? (sg == 0 ? w : n) : n;
    // slab cells this segment updates
    auto owned = [&](int k) {
      if (k < 0 || k >= n || !cpml_in_slab(k, n, npml)) return false;
      return !two || (sg == 0 ? k < npml : k >= n - npml);
    };
    float G[9];    // g = p + A nu at positions i .. i+8
    float AN[13];  // A nu at i-4 .. i+8
    float AM[9];   // A mu at i-4 .. i+4
#pragma unroll
    for (int m = 0; m < 9; ++m) G[m] = AM[m] = 0.f;
#pragma unroll
    for (int m = 0; m < 13; ++m) AN[m] = 0.f;
    for (int i = i0 - 8; i < i1; ++i) {
      // nu and g at i + 8
      const int k8 = i + 8;
      float pv = 0.f, an = 0.f;
      if (k8 >= 0 && k8 < n) {
        pv = pl[k8 * us];
        if (cpml_in_slab(k8, n, npml)) {
          const long long cell = cpml_cell(k8, n, npml) * ss;
          const float nv = fmaf(__ldg(bp + k8), nu[cell], pv);
          if (owned(k8)) nu[cell] = nv;
          an = __fmul_rn(__ldg(ap + k8), nv);
        }
      }
      G[8] = __fadd_rn(pv, an);  // rounded as written (no contraction)
      AN[12] = an;
      // mu at i + 4 from g at i .. i + 8
      const int k4 = i + 4;
      float am = 0.f;
      if (k4 >= 0 && k4 < n && cpml_in_slab(k4, n, npml)) {
        float d1 = 0.f;
#pragma unroll
        for (int m = 1; m <= kR; ++m) d1 = fmaf(g.c1[AX][m], G[4 + m] - G[4 - m], d1);
        const long long cell = cpml_cell(k4, n, npml) * ss;
        const float mv = fmaf(__ldg(bp + k4), mu[cell], -d1);
        if (owned(k4)) mu[cell] = mv;
        am = __fmul_rn(__ldg(ap + k4), mv);
      }
      AM[8] = am;
      // correction at i
      if (i >= i0) {
        float d2 = g.c2[AX][0] * AN[4];
        float d1 = 0.f;
#pragma unroll
        for (int m = 1; m <= kR; ++m) {
          d2 = fmaf(g.c2[AX][m], AN[4 + m] + AN[4 - m], d2);
          d1 = fmaf(g.c1[AX][m], AM[4 + m] - AM[4 - m], d1);
        }
        const float corr = d2 - d1;
        if (corr != 0.f) ol[i * us] = fmaf(cl[i * us], corr, ol[i * us]);
      }
#pragma unroll
      for (int m = 0; m < 8; ++m) G[m] = G[m + 1];
#pragma unroll
      for (int m = 0; m < 12; ++m) AN[m] = AN[m + 1];
#pragma unroll
      for (int m = 0; m < 8; ++m) AM[m] = AM[m + 1];
    }
  }
}

// Unrolled segment kernels for layers of NPML = 8 or 16 cells, on axes
// where the two end segments are disjoint (n >= 2 w): one thread per line
// end (blockIdx.z: 0 the low face, 1 the high face), so the two segments of
// a line run in parallel. Positions are counted from the face, j = 0 .. w-1
// (i = j, or i = n-1-j at the high face); mirroring flips the sign of D1,
// which the kernels fold into the order of each difference, so every
// operation rounds exactly as in the line walks above (the results are
// bitwise equal). With NPML fixed the whole segment is unrolled: u^n is read
// at the w positions the layer needs (psi reaches u up to npml + 3 cells from
// the face), psi and zeta at the npml slab cells, C and u^{n+1} at the w
// correction points, with no per-position predicates; the profile values
// travel in the kernel's parameters (constant operands of the FMAs).
template <int NPML>
struct CpmlSideProf {
  float b[2][NPML], a[2][NPML];  // [face][j], j counted from the face
};

// Profile values of an axis of n cells (b, a along the axis) by face and
// depth from the face.
template <int NPML>
inline void cpml_side_prof(const float *b, const float *a, int n, CpmlSideProf<NPML> &pf) {
  for (int j = 0; j < NPML; ++j)
    for (int sd = 0; sd < 2; ++sd) {
      const int i = sd ? n - 1 - j : j;
      pf.b[sd][j] = b[i];
      pf.a[sd][j] = a[i];
    }
}

// Segment addressing shared by the unrolled kernels: line offset of
// position j (field layout) and of slab cell j (slab layout).
// The per-position steps are 32-bit (the host takes these kernels only
// where (w - 1) times the field step and (npml - 1) times the slab step fit
// in an int), which keeps one register per offset instead of a 64-bit
// address for each of the segment's loads and stores.
struct CpmlSeg {
  long long u0;  // field offset of j = 0 (pitch pxu)
  long long c0;  // v^2 dt^2 offset of j = 0 (pitch px)
  long long s0;  // slab offset of j = 0
  int ustep;     // per-position field step
  int cstep;     // per-position v^2 dt^2 step
  int sstep;     // per-cell slab step
  int n;
};

// t: index across the lines, q: row of lines (z for x and y lines, y for
// z lines).
template <int AX, int NPML>
__device__ __forceinline__ bool cpml_seg_setup(const CpmlGeom &g, int side, int t, int q,
                                               CpmlSeg &sg) {
  long long ub, us, cb, cs, sb, ss;
  if (AX == 0) {
    if (t >= g.ny) return false;
    sg.n = g.nx;
    ub = ((long long)q * g.ny + t) * g.pxu;
    us = 1;
    cb = ((long long)q * g.ny + t) * g.px;
    cs = 1;
    sb = (long long)q * g.ny + t;
    ss = (long long)g.nz * g.ny;
  } else {
    if (t >= g.nx) return false;
    sg.n = AX == 1 ? g.ny : g.nz;
    ub = AX == 1 ? (long long)q * g.ny * g.pxu + t : (long long)q * g.pxu + t;
    us = AX == 1 ? (long long)g.pxu : (long long)g.ny * g.pxu;
    cb = AX == 1 ? (long long)q * g.ny * g.px + t : (long long)q * g.px + t;
    cs = AX == 1 ? (long long)g.px : (long long)g.ny * g.px;
    sb = (long long)q * g.nx + t;
    ss = AX == 1 ? (long long)g.nz * g.nx : (long long)g.ny * g.nx;
  }
  // the high face's slab cell of position j is 2 npml - 1 - j
  sg.u0 = side ? ub + (long long)(sg.n - 1) * us : ub;
  sg.ustep = (int)(side ? -us : us);
  sg.c0 = side ? cb + (long long)(sg.n - 1) * cs : cb;
  sg.cstep = (int)(side ? -cs : cs);
  sg.s0 = side ? sb + (long long)(2 * NPML - 1) * ss : sb;
  sg.sstep = (int)(side ? -ss : ss);
  return true;
}

// W = NPML + 4 values of a field along the segment, v[j] = f(position j)
// (base: offset of j = 0, step: per position), times s (16-bit fields).
// x lines are rows: read as 4-element vectors when the segment starts on a
// vector boundary (the low face always; the high face when n is a multiple
// of 4).
template <int AX, int W, int SIDE, class T>
__device__ __forceinline__ void cpml_seg_load(const T *f, long long base, int step, int n,
                                              float s, float *v) {
  if (AX == 0 && (SIDE == 0 || (n & 3) == 0)) {
    const T *r = SIDE == 0 ? f + base : f + base - (W - 1);
#pragma unroll
    for (int k = 0; k < W; k += 4) {
      float e[4];
      cpml_get4(r + k, s, e);
#pragma unroll
      for (int m = 0; m < 4; ++m) v[SIDE == 0 ? k + m : W - 1 - (k + m)] = e[m];
    }
  } else {
    const T *r = f + base;
#pragma unroll
    for (int j = 0; j < W; ++j) v[j] = cpml_get(r + j * step, s);
  }
}

template <int AX, int W, int SIDE, class T>
__device__ __forceinline__ void cpml_seg_store(T *f, long long base, int step, int n,
                                               float inv, const float *v) {
  if (AX == 0 && (SIDE == 0 || (n & 3) == 0)) {
    T *r = SIDE == 0 ? f + base : f + base - (W - 1);
#pragma unroll
    for (int k = 0; k < W; k += 4) {
      float e[4];
#pragma unroll
      for (int m = 0; m < 4; ++m) e[m] = v[SIDE == 0 ? k + m : W - 1 - (k + m)];
      cpml_put4(r + k, e, inv);
    }
  } else {
    T *r = f + base;
#pragma unroll
    for (int j = 0; j < W; ++j) cpml_put(r + j * step, v[j], inv);
  }
}

// Window value v[k], zero outside [0, N) (k is a compile-time constant
// after unrolling, so the test costs nothing).
template <int N>
__device__ __forceinline__ float cpml_seg_at(const float *v, int k) {
  return (k >= 0 && k < N) ? v[k] : 0.f;
}

// D1 at position j of a window v (zero outside [0, N)), as the line walks
// round it: sum over m of c1_m (f(i+m) - f(i-m)), i the grid position, which
// at the high face is v(j-m) - v(j+m).
template <int SIDE, int N>
__device__ __forceinline__ float cpml_seg_d1(const float *v, int j, const float *c1) {
  float d = 0.f;
#pragma unroll
  for (int m = 1; m <= kR; ++m) {
    const float hi = cpml_seg_at<N>(v, j + m);
    const float lo = cpml_seg_at<N>(v, j - m);
    d = fmaf(c1[m], SIDE == 0 ? hi - lo : lo - hi, d);
  }
  return d;
}

template <int N>
__device__ __forceinline__ float cpml_seg_d2(const float *v, int j, const float *c2) {
  float d = c2[0] * cpml_seg_at<N>(v, j);
#pragma unroll
  for (int m = 1; m <= kR; ++m)
    d = fmaf(c2[m], cpml_seg_at<N>(v, j + m) + cpml_seg_at<N>(v, j - m), d);
  return d;
}

template <int AX, int NPML, class T, bool kStoreD, int SIDE>
__device__ __forceinline__ void cpml_seg_forward(const CpmlGeom &g, const CpmlSideProf<NPML> &pf,
                                                 int t, int q, const T *__restrict__ u,
                                                 T *__restrict__ unext,
                                                 const float *__restrict__ c,
                                                 float *__restrict__ dout,
                                                 const StepDesc *d, int koff) {
  constexpr int W = NPML + 4;
  CpmlSeg sg;
  if (!cpml_seg_setup<AX, NPML>(g, SIDE, t, q, sg)) return;
  CpmlScale<T> sc;
  sc.init(d, koff);
  float *psi = g.psi[AX] + sg.s0;
  float *zeta = g.zeta[AX] + sg.s0;
  // Two phases, each issuing all of its loads before its first store (the
  // slabs and the fields are not known to be distinct, so a load after a
  // store waits for it): u^n, psi and zeta -> the new psi, zeta and the
  // corrections; then C, u^{n+1} (and D) -> u^{n+1} (and D) updated. The
  // second phase's loads wait behind the slab stores once per thread, and
  // the live set stays about half of what one phase would hold.
  float U[W], PS[NPML], ZT[NPML], CORR[W];
  cpml_seg_load<AX, W, SIDE>(u, sg.u0, sg.ustep, sg.n, sc.su, U);
#pragma unroll
  for (int j = 0; j < NPML; ++j) {
    PS[j] = psi[j * sg.sstep];
    ZT[j] = zeta[j * sg.sstep];
  }
#pragma unroll
  for (int j = 0; j < NPML; ++j) {
    const float d1 = cpml_seg_d1<SIDE, W>(U, j, g.c1[AX]);
    PS[j] = fmaf(pf.b[SIDE][j], PS[j], pf.a[SIDE][j] * d1);
  }
#pragma unroll
  for (int j = 0; j < W; ++j) {
    const float d1p = cpml_seg_d1<SIDE, NPML>(PS, j, g.c1[AX]);
    CORR[j] = d1p;
    if (j < NPML) {
      const float d2 = cpml_seg_d2<W>(U, j, g.c2[AX]);
      ZT[j] = fmaf(pf.b[SIDE][j], ZT[j], pf.a[SIDE][j] * (d2 + d1p));
      CORR[j] += ZT[j];
    }
  }
#pragma unroll
  for (int j = 0; j < NPML; ++j) {
    psi[j * sg.sstep] = PS[j];
    zeta[j * sg.sstep] = ZT[j];
  }
  float CC[W], UN[W], DO[kStoreD ? W : 1];
  if constexpr (std::is_same<T, float>::value)  // FP32 storage: pxu == px
    cpml_seg_load<AX, W, SIDE>(c, sg.u0, sg.ustep, sg.n, 1.f, CC);
  else
    cpml_seg_load<AX, W, SIDE>(c, sg.c0, sg.cstep, sg.n, 1.f, CC);
  cpml_seg_load<AX, W, SIDE>(unext, sg.u0, sg.ustep, sg.n, sc.so, UN);
  if constexpr (kStoreD) cpml_seg_load<AX, W, SIDE>(dout, sg.u0, sg.ustep, sg.n, 1.f, DO);
  float vmax = 0.f;
#pragma unroll
  for (int j = 0; j < W; ++j) {
    UN[j] = fmaf(CC[j], CORR[j], UN[j]);
    vmax = fmaxf(vmax, fabsf(UN[j]));
    if constexpr (kStoreD) DO[j] = fmaf(CC[j], CORR[j], DO[j]);
  }
  cpml_seg_store<AX, W, SIDE>(unext, sg.u0, sg.ustep, sg.n, sc.inv_so, UN);
  if constexpr (kStoreD) cpml_seg_store<AX, W, SIDE>(dout, sg.u0, sg.ustep, sg.n, 1.f, DO);
  sc.commit(vmax);
}

// T: the wavefields' storage (float, or 16-bit with the step's scales read
// from d at absolute step step0 + n + koff); D is stored for FP32 only.
template <int AX, int NPML, class T, bool kStoreD = false>
__global__ void __launch_bounds__(128)
    cpml_seg_kernel(CpmlGeom g, CpmlSideProf<NPML> pf, const T *__restrict__ u,
                    T *__restrict__ unext, const float *__restrict__ c,
                    float *__restrict__ dout, const StepDesc *d, int koff) {
  static_assert(!kStoreD || std::is_same<T, float>::value, "D is stored for FP32 only");
  const int t = blockIdx.x * blockDim.x + threadIdx.x, q = blockIdx.y;
  if (blockIdx.z == 0)
    cpml_seg_forward<AX, NPML, T, kStoreD, 0>(g, pf, t, q, u, unext, c, dout, d, koff);
  else
    cpml_seg_forward<AX, NPML, T, kStoreD, 1>(g, pf, t, q, u, unext, c, dout, d, koff);
}

// The adjoint's segment form (cpml_adjoint_line_kernel, unrolled): nu and
// g = p^{k+1} + A nu at the w positions, mu at the slab cells, then
// p^k += C (D2 (A nu) - D1 (A mu)) over the segment.
template <int AX, int NPML, int SIDE>
__device__ __forceinline__ void cpml_seg_adjoint(const CpmlGeom &g, const CpmlSideProf<NPML> &pf,
                                                 const float *__restrict__ p1,
                                                 float *__restrict__ p0,
                                                 const float *__restrict__ c,
                                                 float *__restrict__ nus,
                                                 float *__restrict__ mus) {
  constexpr int W = NPML + 4;
  CpmlSeg sg;
  if (!cpml_seg_setup<AX, NPML>(g, SIDE, blockIdx.x * blockDim.x + threadIdx.x, blockIdx.y,
                                sg))
    return;
  float *nu = nus + sg.s0;
  float *mu = mus + sg.s0;
  // two phases as in the forward: p^{k+1}, nu, mu -> nu, mu and the
  // corrections; then C, p^k -> p^k updated
  float P[W], G[W], NU[NPML], MU[NPML], AN[NPML], AM[NPML], CORR[W];
  cpml_seg_load<AX, W, SIDE>(p1, sg.u0, sg.ustep, sg.n, 1.f, P);
#pragma unroll
  for (int j = 0; j < NPML; ++j) {
    NU[j] = nu[j * sg.sstep];
    MU[j] = mu[j * sg.sstep];
  }
#pragma unroll
  for (int j = 0; j < W; ++j) {
    G[j] = P[j];
    if (j < NPML) {
      NU[j] = fmaf(pf.b[SIDE][j], NU[j], P[j]);
      AN[j] = __fmul_rn(pf.a[SIDE][j], NU[j]);
      G[j] = __fadd_rn(P[j], AN[j]);  // as the line walk: no contraction
    }
  }
#pragma unroll
  for (int j = 0; j < NPML; ++j) {
    const float d1 = cpml_seg_d1<SIDE, W>(G, j, g.c1[AX]);
    MU[j] = fmaf(pf.b[SIDE][j], MU[j], -d1);
    AM[j] = __fmul_rn(pf.a[SIDE][j], MU[j]);
  }
#pragma unroll
  for (int j = 0; j < W; ++j) {
    // A nu and A mu are zero past the slab
    const float d2 = cpml_seg_d2<NPML>(AN, j, g.c2[AX]);
    const float d1 = cpml_seg_d1<SIDE, NPML>(AM, j, g.c1[AX]);
    CORR[j] = d2 - d1;
  }
#pragma unroll
  for (int j = 0; j < NPML; ++j) {
    nu[j * sg.sstep] = NU[j];
    mu[j * sg.sstep] = MU[j];
  }
  float CC[W], PO[W];
  cpml_seg_load<AX, W, SIDE>(c, sg.u0, sg.ustep, sg.n, 1.f, CC);  // FP32: pxu == px
  cpml_seg_load<AX, W, SIDE>(p0, sg.u0, sg.ustep, sg.n, 1.f, PO);
#pragma unroll
  for (int j = 0; j < W; ++j) PO[j] = fmaf(CC[j], CORR[j], PO[j]);
  cpml_seg_store<AX, W, SIDE>(p0, sg.u0, sg.ustep, sg.n, 1.f, PO);
}

template <int AX, int NPML>
__global__ void __launch_bounds__(128)
    cpml_seg_adjoint_kernel(CpmlGeom g, CpmlSideProf<NPML> pf, const float *__restrict__ p1,
                            float *__restrict__ p0, const float *__restrict__ c,
                            float *__restrict__ nus, float *__restrict__ mus) {
  if (blockIdx.z == 0)
    cpml_seg_adjoint<AX, NPML, 0>(g, pf, p1, p0, c, nus, mus);
  else
    cpml_seg_adjoint<AX, NPML, 1>(g, pf, p1, p0, c, nus, mus);
}

// Receivers within w of a face: {x, y, z, receiver id}, recorded from the
// field after the three axis passes (16-bit: the stored value times its
// scale).
template <class T>
__global__ void cpml_record_kernel(CpmlGeom g, const T *__restrict__ unext,
                                   const StepDesc *d, const int4 *srec,
                                   const int *nsrec, int koff) {
  const int nr = *nsrec;
  if (nr == 0) return;
  const long long n = d->n + koff;
  CpmlScale<T> sc;
  sc.init(d, koff);
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nr;
       t += gridDim.x * blockDim.x) {
    const int4 e = srec[t];
    d->traces[(size_t)n * d->nrec + e.w] =
        cpml_get(unext + ((size_t)e.z * g.ny + e.y) * g.pxu + e.x, sc.so);
  }
}

// One served shot's layer in the shot server's batched layer launches: its
// geometry and slabs, fields, descriptor, shell receivers, step bookkeeping
// (batch step b0 is the shot's step 0, as in the batched sweep), and its
// first block in each axis launch (a 1D grid that concatenates the shots'
// blocks: ceil(lines across / 128) per row of lines).
struct CpmlBatchShot {
  CpmlGeom g;
  void *buf[2];  // buf[0] holds the shot's step 0
  const float *c;
  const StepDesc *desc;
  const int4 *srec;  // receivers within w of a face: {x, y, z, id}
  int nsrec;
  long long b0;
  int nsteps;
  int blk_begin[3];
  // per axis: 0 for the line walk, or 8 / 16 for the unrolled segment form
  // (both faces' segments in blocks of their own), with its profile values
  int seg[3];
  CpmlSideProf<16> p16[3];
  CpmlSideProf<8> p8[3];
};

__device__ __forceinline__ int cpml_batch_find(const CpmlBatchShot *shots, int nshots, int ax,
                                               int blk) {
  int lo = 0, hi = nshots - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (shots[mid].blk_begin[ax] <= blk) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// The axis-AX pass of batch step k over every shot of the table, each in
// its form (shots outside their steps return at once): a shot's blocks are
// rows x ceil(lines across / 128) for the line walk, twice that for the
// segment form (the low face's blocks, then the high face's).
template <int AX, class T>
__global__ void __launch_bounds__(128, 3)
    cpml_line_batched_kernel(const CpmlBatchShot *__restrict__ shots, int nshots, long long k) {
  const CpmlBatchShot &sh = shots[cpml_batch_find(shots, nshots, AX, blockIdx.x)];
  const long long n = k - sh.b0;
  if (n < 0 || n >= sh.nsteps) return;
  const int cur = (int)(n & 1);
  const int across = AX == 0 ? sh.g.ny : sh.g.nx;
  const int rows = AX == 2 ? sh.g.ny : sh.g.nz;
  const int bpr = (across + 127) / 128;  // blocks per row of lines
  int local = blockIdx.x - sh.blk_begin[AX];
  const T *u = static_cast<const T *>(sh.buf[cur]);
  T *un = static_cast<T *>(sh.buf[cur ^ 1]);
  const int form = sh.seg[AX];
  const int side = (form != 0 && local >= rows * bpr) ? 1 : 0;
  local -= side * rows * bpr;
  const int q = local / bpr;
  const int t = (local - q * bpr) * 128 + threadIdx.x;
  // the shot's profile values staged in shared memory (block-uniform form),
  // read with immediate offsets where the single-grid kernels take them as
  // constant operands
  __shared__ CpmlSideProf<16> s16;
  __shared__ CpmlSideProf<8> s8;
  if (form == 16) {
    constexpr int NV = sizeof(CpmlSideProf<16>) / 4;
    for (int i = threadIdx.x; i < NV; i += blockDim.x)
      reinterpret_cast<float *>(&s16)[i] = reinterpret_cast<const float *>(&sh.p16[AX])[i];
    __syncthreads();
    if (side == 0)
      cpml_seg_forward<AX, 16, T, false, 0>(sh.g, s16, t, q, u, un, sh.c, nullptr, sh.desc,
                                            (int)n);
    else
      cpml_seg_forward<AX, 16, T, false, 1>(sh.g, s16, t, q, u, un, sh.c, nullptr, sh.desc,
                                            (int)n);
  } else if (form == 8) {
    constexpr int NV = sizeof(CpmlSideProf<8>) / 4;
    for (int i = threadIdx.x; i < NV; i += blockDim.x)
      reinterpret_cast<float *>(&s8)[i] = reinterpret_cast<const float *>(&sh.p8[AX])[i];
    __syncthreads();
    if (side == 0)
      cpml_seg_forward<AX, 8, T, false, 0>(sh.g, s8, t, q, u, un, sh.c, nullptr, sh.desc,
                                           (int)n);
    else
      cpml_seg_forward<AX, 8, T, false, 1>(sh.g, s8, t, q, u, un, sh.c, nullptr, sh.desc,
                                           (int)n);
  } else {
    cpml_line_walk<AX, T, false>(sh.g, t, q, u, un, sh.c, nullptr, sh.desc, (int)n);
  }
}

// Shell receivers of batch step k: blocks_per_shot blocks per shot (a
// receiver plane inside the layer puts all of a shot's receivers here).
template <class T>
__global__ void cpml_record_batched_kernel(const CpmlBatchShot *__restrict__ shots, long long k,
                                           int blocks_per_shot) {
  const CpmlBatchShot &sh = shots[blockIdx.x / blocks_per_shot];
  const int part = blockIdx.x % blocks_per_shot;
  const long long n = k - sh.b0;
  if (n < 0 || n >= sh.nsteps || sh.nsrec == 0) return;
  const StepDesc *d = sh.desc;
  CpmlScale<T> sc;
  sc.init(d, (int)n);
  const T *un = static_cast<const T *>(sh.buf[(n & 1) ^ 1]);
  for (int r = part * blockDim.x + threadIdx.x; r < sh.nsrec;
       r += blocks_per_shot * blockDim.x) {
    const int4 e = sh.srec[r];
    d->traces[(size_t)(d->n + n) * d->nrec + e.w] =
        cpml_get(un + ((size_t)e.z * sh.g.ny + e.y) * sh.g.pxu + e.x, sc.so);
  }
}

}  // namespace gbw
