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
// afterwards one kernel per axis walks every line along that axis through
// its two end segments of w cells (one segment of the whole line when the
// two would overlap): it updates psi_a and zeta_a from u^n (which the sweep
// does not overwrite) and adds the axis term to u^{n+1}. The three axis
// kernels run one after another, so corner points are updated by each axis
// in turn with no race. Receivers within w of a face are then re-recorded.
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

// Slab storage: the x slabs hold ((z ny + y) 2npml + cell), the y slabs
// ((cell nz + z) nx + x), the z slabs ((cell ny + y) nx + x), where cell in
// [0, 2 npml) counts the low slab's npml cells, then the high slab's.
__device__ __forceinline__ bool cpml_in_slab(int i, int n, int npml) {
  return i < npml || i >= n - npml;
}

__device__ __forceinline__ int cpml_cell(int i, int n, int npml) {
  return i < npml ? i : i - (n - 2 * npml);
}

// y (AX = 1) and z (AX = 2): one thread per line, x across the threads of a
// warp (coalesced), walking the line with register windows of u^n
// (positions i-4 .. i+8) and psi^n (i-4 .. i+4); psi(i+4) is computed as it
// enters the window, so each slab cell's psi is computed once per step.
template <int AX>
__global__ void __launch_bounds__(128)
    cpml_line_kernel(CpmlGeom g, const float *__restrict__ u,
                     float *__restrict__ unext, const float *__restrict__ c) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int o = blockIdx.y;  // z for the y lines, y for the z lines
  if (x >= g.nx) return;
  const int n = AX == 1 ? g.ny : g.nz;
  const long long us = AX == 1 ? (long long)g.px : (long long)g.ny * g.px;
  const long long ub = AX == 1 ? (long long)o * g.ny * g.px + x
                               : (long long)o * g.px + x;
  const long long ss = AX == 1 ? (long long)g.nz * g.nx : (long long)g.ny * g.nx;
  float *psi = g.psi[AX] + (long long)o * g.nx + x;
  float *zeta = g.zeta[AX] + (long long)o * g.nx + x;
  const float *bp = g.bprof[AX];
  const float *ap = g.aprof[AX];
  const int npml = g.npml, w = g.w;
  const int nseg = n >= 2 * w ? 2 : 1;
  for (int s = 0; s < nseg; ++s) {
    const int i0 = (nseg == 2 && s == 1) ? n - w : 0;
    const int i1 = nseg == 1 ? n : (s == 0 ? w : n);
    // Start 4 positions early so psi(i0 .. i0+3) enter the window; psi at
    // i0-8 .. i0-1 is zero (before the grid, or between the slabs).
    int i = i0 - 4;
    float U[13], P[9];
#pragma unroll
    for (int m = 0; m < 13; ++m) {
      const int k = i - 4 + m;
      U[m] = (k >= 0 && k < n) ? u[ub + k * us] : 0.f;
    }
#pragma unroll
    for (int m = 0; m < 9; ++m) P[m] = 0.f;
    for (; i < i1; ++i) {
      const int k = i + 4;  // psi(k) from U(k-4 .. k+4) = U[4 .. 12]
      float pk = 0.f;
      if (k < n && cpml_in_slab(k, n, npml)) {
        float d1 = 0.f;
#pragma unroll
        for (int m = 1; m <= kR; ++m) d1 = fmaf(g.c1[AX][m], U[8 + m] - U[8 - m], d1);
        float *pp = psi + (long long)cpml_cell(k, n, npml) * ss;
        pk = fmaf(bp[k], *pp, ap[k] * d1);
        *pp = pk;
      }
      P[8] = pk;
      if (i >= i0) {
        float d1p = 0.f;
#pragma unroll
        for (int m = 1; m <= kR; ++m) d1p = fmaf(g.c1[AX][m], P[4 + m] - P[4 - m], d1p);
        float corr = d1p;
        if (cpml_in_slab(i, n, npml)) {
          float d2 = g.c2[AX][0] * U[4];
#pragma unroll
          for (int m = 1; m <= kR; ++m) d2 = fmaf(g.c2[AX][m], U[4 + m] + U[4 - m], d2);
          float *zp = zeta + (long long)cpml_cell(i, n, npml) * ss;
          const float zt = fmaf(bp[i], *zp, ap[i] * (d2 + d1p));
          *zp = zt;
          corr += zt;
        }
        const long long off = ub + i * us;
        unext[off] = fmaf(c[off], corr, unext[off]);
      }
#pragma unroll
      for (int m = 0; m < 12; ++m) U[m] = U[m + 1];
      const int kn = i + 9;
      U[12] = (kn < n) ? u[ub + kn * us] : 0.f;
#pragma unroll
      for (int m = 0; m < 8; ++m) P[m] = P[m + 1];
    }
  }
}

// x: one warp per row (y, z), lanes across the row's cells; psi of the row's
// slab cells first, then (after the warp's stores are visible) the
// corrections of its end segments.
__global__ void __launch_bounds__(256)
    cpml_x_kernel(CpmlGeom g, const float *__restrict__ u,
                  float *__restrict__ unext, const float *__restrict__ c) {
  const int lane = threadIdx.x & 31;
  const int y = blockIdx.x * 8 + (threadIdx.x >> 5);
  const int z = blockIdx.y;
  if (y >= g.ny) return;
  const int n = g.nx, npml = g.npml, w = g.w;
  const long long row = ((long long)z * g.ny + y) * g.px;
  const float *ur = u + row;
  const float *cr = c + row;
  float *unr = unext + row;
  float *psi = g.psi[0] + ((long long)z * g.ny + y) * (2 * npml);
  float *zeta = g.zeta[0] + ((long long)z * g.ny + y) * (2 * npml);
  const float *bp = g.bprof[0];
  const float *ap = g.aprof[0];
  auto U = [&](int k) { return (k >= 0 && k < n) ? ur[k] : 0.f; };
  for (int j = lane; j < 2 * npml; j += 32) {
    const int i = j < npml ? j : n - 2 * npml + j;
    float d1 = 0.f;
#pragma unroll
    for (int m = 1; m <= kR; ++m) d1 = fmaf(g.c1[0][m], U(i + m) - U(i - m), d1);
    psi[j] = fmaf(bp[i], psi[j], ap[i] * d1);
  }
  __syncwarp();
  auto P = [&](int k) {
    return (k >= 0 && k < n && cpml_in_slab(k, n, npml)) ? psi[cpml_cell(k, n, npml)] : 0.f;
  };
  const bool two = n >= 2 * w;
  const int ncorr = two ? 2 * w : n;
  for (int q = lane; q < ncorr; q += 32) {
    const int i = (two && q >= w) ? n - 2 * w + q : q;
    float d1p = 0.f;
#pragma unroll
    for (int m = 1; m <= kR; ++m) d1p = fmaf(g.c1[0][m], P(i + m) - P(i - m), d1p);
    float corr = d1p;
    if (cpml_in_slab(i, n, npml)) {
      float d2 = g.c2[0][0] * ur[i];
#pragma unroll
      for (int m = 1; m <= kR; ++m) d2 = fmaf(g.c2[0][m], U(i + m) + U(i - m), d2);
      float *zp = zeta + cpml_cell(i, n, npml);
      const float zt = fmaf(bp[i], *zp, ap[i] * (d2 + d1p));
      *zp = zt;
      corr += zt;
    }
    unr[i] = fmaf(cr[i], corr, unr[i]);
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
