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
// are stored there. Points farther than npml + 4 cells from every face see
// no layer term, so the standard sweep computes them exactly; the points of
// the "shell" (closer than npml + 4 to some face) are recomputed here.
//
// Per step, on the context's stream:
//   1. cpml_psi_kernel   psi_a^n in every slab point, from u^n;
//   2. cpml_shell_kernel u^{n+1} of every shell point into a compact buffer
//                        (with zeta_a^n and the point source), before the
//                        sweep overwrites u_prev;
//   3. the sweep         (every point, in place);
//   4. cpml_commit_kernel the shell values over the sweep's, and the traces
//                        of receivers in the shell.
#pragma once

#include <cstdint>

#include "sweep.cuh"

namespace gbw {

struct CpmlGeom {
  int nx, ny, nz, px;  // grid and row pitch of the fields (floats)
  int npml, w;         // layer cells; shell width npml + 4
  // Shell enumeration: region Z (z in zlist, every y, x), region Y (z in
  // zmid, y in ylist, every x), region X (z in zmid, y in ymid, x in xlist).
  const int *zlist, *zmid, *ylist, *ymid, *xlist;
  int nzl, nzm, nyl, nym, nxl;
  long long cz, cy, cx;  // points per region
  float *psi[3], *zeta[3];       // slab storage per axis
  const float *bprof[3], *aprof[3];  // per-axis b, a (length n_a)
  float c2[3][5];  // D2 weights / h_a^2 (index 0: centre)
  float c1[3][5];  // D1 weights / h_a (index 1..4)
  float *sbuf;     // u^{n+1} of the shell points
};

__device__ __forceinline__ bool cpml_in_slab(int c, int n, int npml) {
  return c < npml || c >= n - npml;
}

__device__ __forceinline__ int cpml_slab_cell(int c, int n, int npml) {
  return c < npml ? c : npml + (c - (n - npml));  // side * npml + cell
}

// Slab storage index of point (x, y, z) for axis ax (the point must be in
// that axis's slab): x slab ((z ny + y) 2npml + cell), y slab ((cell nz + z)
// nx + x), z slab ((cell ny + y) nx + x).
__device__ __forceinline__ size_t cpml_slab_index(const CpmlGeom &g, int ax,
                                                  int x, int y, int z) {
  if (ax == 0)
    return ((size_t)z * g.ny + y) * (2 * g.npml) +
           cpml_slab_cell(x, g.nx, g.npml);
  if (ax == 1)
    return ((size_t)cpml_slab_cell(y, g.ny, g.npml) * g.nz + z) * g.nx + x;
  return ((size_t)cpml_slab_cell(z, g.nz, g.npml) * g.ny + y) * g.nx + x;
}

__device__ __forceinline__ float cpml_u(const float *u, const CpmlGeom &g,
                                        int x, int y, int z) {
  if (x < 0 || x >= g.nx || y < 0 || y >= g.ny || z < 0 || z >= g.nz) return 0.f;
  return u[((size_t)z * g.ny + y) * g.px + x];
}

__device__ __forceinline__ float cpml_psi_at(const CpmlGeom &g, int ax, int x,
                                             int y, int z) {
  const int n[3] = {g.nx, g.ny, g.nz};
  const int c[3] = {x, y, z};
  if (c[ax] < 0 || c[ax] >= n[ax] || !cpml_in_slab(c[ax], n[ax], g.npml))
    return 0.f;
  return g.psi[ax][cpml_slab_index(g, ax, x, y, z)];
}

// 1. psi_a^n = b psi_a^{n-1} + a D1_a u^n over the three slab sets.
__global__ void cpml_psi_kernel(CpmlGeom g, const float *__restrict__ u) {
  const long long nxs = 2ll * g.npml * g.ny * g.nz;
  const long long nys = 2ll * g.npml * g.nz * g.nx;
  const long long nzs = 2ll * g.npml * g.ny * g.nx;
  const long long total = nxs + nys + nzs;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
       t < total; t += (long long)gridDim.x * blockDim.x) {
    int ax, x, y, z, cell;
    if (t < nxs) {
      ax = 0;
      cell = (int)(t % (2 * g.npml));
      const long long yz = t / (2 * g.npml);
      y = (int)(yz % g.ny);
      z = (int)(yz / g.ny);
      x = cell < g.npml ? cell : g.nx - 2 * g.npml + cell;
    } else if (t < nxs + nys) {
      ax = 1;
      const long long r = t - nxs;
      x = (int)(r % g.nx);
      const long long q = r / g.nx;
      z = (int)(q % g.nz);
      cell = (int)(q / g.nz);
      y = cell < g.npml ? cell : g.ny - 2 * g.npml + cell;
    } else {
      ax = 2;
      const long long r = t - nxs - nys;
      x = (int)(r % g.nx);
      const long long q = r / g.nx;
      y = (int)(q % g.ny);
      cell = (int)(q / g.ny);
      z = cell < g.npml ? cell : g.nz - 2 * g.npml + cell;
    }
    const int dx = ax == 0, dy = ax == 1, dz = ax == 2;
    float d1 = 0.f;
#pragma unroll
    for (int m = 1; m <= kR; ++m)
      d1 = fmaf(g.c1[ax][m],
                cpml_u(u, g, x + m * dx, y + m * dy, z + m * dz) -
                    cpml_u(u, g, x - m * dx, y - m * dy, z - m * dz),
                d1);
    const int c = ax == 0 ? x : (ax == 1 ? y : z);
    float *p = g.psi[ax] + cpml_slab_index(g, ax, x, y, z);
    *p = fmaf(g.bprof[ax][c], *p, g.aprof[ax][c] * d1);
  }
}

__device__ __forceinline__ bool cpml_shell_point(const CpmlGeom &g,
                                                 long long t, int &x, int &y,
                                                 int &z) {
  const long long plane = (long long)g.nx * g.ny;
  if (t < g.cz) {
    z = g.zlist[t / plane];
    const long long r = t % plane;
    y = (int)(r / g.nx);
    x = (int)(r % g.nx);
    return true;
  }
  t -= g.cz;
  if (t < g.cy) {
    const long long row = (long long)g.nyl * g.nx;
    z = g.zmid[t / row];
    const long long r = t % row;
    y = g.ylist[r / g.nx];
    x = (int)(r % g.nx);
    return true;
  }
  t -= g.cy;
  if (t < g.cx) {
    const long long row = (long long)g.nym * g.nxl;
    z = g.zmid[t / row];
    const long long r = t % row;
    y = g.ymid[r / g.nxl];
    x = g.xlist[r % g.nxl];
    return true;
  }
  return false;
}

// 2. u^{n+1} of the shell points (zeta_a^n updated in the slabs).
__global__ void cpml_shell_kernel(CpmlGeom g, const float *__restrict__ u,
                                  const float *__restrict__ up,
                                  const float *__restrict__ c, StepDesc *d,
                                  int koff) {
  const long long total = g.cz + g.cy + g.cx;
  const long long n = d->n + koff;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
       t < total; t += (long long)gridDim.x * blockDim.x) {
    int x, y, z;
    cpml_shell_point(g, t, x, y, z);
    const int pc[3] = {x, y, z};
    const int nn[3] = {g.nx, g.ny, g.nz};
    const float uc = cpml_u(u, g, x, y, z);
    float sum = 0.f;
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
      const int dx = ax == 0, dy = ax == 1, dz = ax == 2;
      float d2 = g.c2[ax][0] * uc;
      float d1p = 0.f;
#pragma unroll
      for (int m = 1; m <= kR; ++m) {
        d2 = fmaf(g.c2[ax][m],
                  cpml_u(u, g, x + m * dx, y + m * dy, z + m * dz) +
                      cpml_u(u, g, x - m * dx, y - m * dy, z - m * dz),
                  d2);
        d1p = fmaf(g.c1[ax][m],
                   cpml_psi_at(g, ax, x + m * dx, y + m * dy, z + m * dz) -
                       cpml_psi_at(g, ax, x - m * dx, y - m * dy, z - m * dz),
                   d1p);
      }
      float zt = 0.f;
      if (cpml_in_slab(pc[ax], nn[ax], g.npml)) {
        float *zp = g.zeta[ax] + cpml_slab_index(g, ax, x, y, z);
        zt = fmaf(g.bprof[ax][pc[ax]], *zp, g.aprof[ax][pc[ax]] * (d2 + d1p));
        *zp = zt;
      }
      sum += d2 + d1p + zt;
    }
    const size_t idx = ((size_t)z * g.ny + y) * g.px + x;
    const float cv = c[idx];
    float un = fmaf(cv, sum, 2.f * uc - up[idx]);
    if (d->src_active && x == d->sx && y == d->sy && z == d->sz)
      un = fmaf(cv, d->wavelet[n], un);
    g.sbuf[t] = un;
  }
}

// 4. Shell values over the sweep's; receivers in the shell re-recorded.
__global__ void cpml_commit_kernel(CpmlGeom g, float *__restrict__ unext,
                                   const StepDesc *d, const int2 *srec,
                                   const int *nsrec, int koff) {
  const long long total = g.cz + g.cy + g.cx;
  const int nr = *nsrec;
  const long long n = d->n + koff;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
       t < total + nr; t += (long long)gridDim.x * blockDim.x) {
    if (t < total) {
      int x, y, z;
      cpml_shell_point(g, t, x, y, z);
      unext[((size_t)z * g.ny + y) * g.px + x] = g.sbuf[t];
    } else {
      const int2 e = srec[t - total];
      d->traces[(size_t)n * d->nrec + e.y] = g.sbuf[e.x];
    }
  }
}

}  // namespace gbw
