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

#include <cstdint>

#include "sweep.cuh"

namespace gbw {

struct CpmlGeom {
  int nx, ny, nz, px;  // grid and row pitch of the fields (floats)
  int npml, w;         // layer cells; correction width npml + 4
  float *psi[3], *zeta[3];           // slab storage per axis
  const float *bprof[3], *aprof[3];  // per-axis b, a (length n_a)
  float c2[3][5];  // D2 weights / h_a^2 (index 0: centre)
  float c1[3][5];  // D1 weights / h_a (index 1..4)
};

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

// Four consecutive values of an x row from position p (p a multiple of 4,
// the row 16-byte aligned with its padding up to a multiple of 4 in
// bounds); positions outside [0, n) read as zero.
__device__ __forceinline__ void cpml_row4(const float *row, int p, int n, float *v) {
  if (p < 0 || p >= n) {
    v[0] = v[1] = v[2] = v[3] = 0.f;
    return;
  }
  const float4 t = *reinterpret_cast<const float4 *>(row + p);
  v[0] = t.x;
  v[1] = p + 1 < n ? t.y : 0.f;
  v[2] = p + 2 < n ? t.z : 0.f;
  v[3] = p + 3 < n ? t.w : 0.f;
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
template <int AX, bool kStoreD = false>
__global__ void __launch_bounds__(128)
    cpml_line_kernel(CpmlGeom g, const float *__restrict__ u,
                     float *__restrict__ unext, const float *__restrict__ c,
                     float *__restrict__ dout = nullptr) {
  constexpr int F = kCpmlChunk;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int q = blockIdx.y;  // z for x and y lines, y for z lines
  int n;
  long long ub, us, sb, ss;  // u offset and stride; slab offset and stride
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
  const float *__restrict__ ul = u + ub;
  const float *__restrict__ cl = c + ub;
  float *__restrict__ nl = unext + ub;
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
        cpml_row4(ul, i + 8, n, nw);
        if (i + F > i0 && i < i1) {
          cpml_row4(cl, i, n, ncc);
          cpml_row4(nl, i, n, nun);
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
          nw[f] = (kw < n) ? ul[kw * us] : 0.f;
          ncc[f] = act ? cl[p * us] : 0.f;
          nun[f] = act ? nl[p * us] : 0.f;
        }
      }
    };
    float W[12 + F];  // W[m] = u(i - 4 + m)
    float P[8 + F];   // P[m] = psi(i - 4 + m)
    int i = AX == 0 ? ((i0 - 4) & ~3) : i0 - 4;
    if (AX == 0) {
#pragma unroll
      for (int m = 0; m < 12; m += 4) cpml_row4(ul, i - 4 + m, n, W + m);
    } else {
#pragma unroll
      for (int m = 0; m < 12; ++m) {
        const int k = i - 4 + m;
        W[m] = (k >= 0 && k < n) ? ul[k * us] : 0.f;
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
        if (AX != 0) nl[p * us] = out[f];
        if constexpr (kStoreD) dl[p * us] = fmaf(cc[f], corr, dl[p * us]);
      }
      // x: the whole aligned batch in one store (positions outside the
      // segment keep the value just read; this thread owns the row)
      if (AX == 0 && i + F > i0 && i < i1)
        *reinterpret_cast<float4 *>(nl + i) = make_float4(out[0], out[1], out[2], out[3]);
#pragma unroll
      for (int m = 0; m < 12; ++m) W[m] = W[m + F];
#pragma unroll
      for (int m = 0; m < 8; ++m) P[m] = P[m + F];
    }
  }
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
          an = __ldg(ap + k8) * nv;
        }
      }
      G[8] = pv + an;
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
        am = __ldg(ap + k4) * mv;
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

// Receivers within w of a face: {x, y, z, receiver id}.
__global__ void cpml_record_kernel(CpmlGeom g, const float *__restrict__ unext,
                                   const StepDesc *d, const int4 *srec,
                                   const int *nsrec, int koff) {
  const int nr = *nsrec;
  if (nr == 0) return;
  const long long n = d->n + koff;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nr;
       t += gridDim.x * blockDim.x) {
    const int4 e = srec[t];
    d->traces[(size_t)n * d->nrec + e.w] =
        unext[((size_t)e.z * g.ny + e.y) * g.px + e.x];
  }
}

}  // namespace gbw
