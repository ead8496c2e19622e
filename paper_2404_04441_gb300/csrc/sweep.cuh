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
// fields are stored without padding planes (rows are padded to 4 floats).
// Each thread computes 4 consecutive x points (float4) on VY rows, reads the
// x and y neighbours from the xy plane in shared memory and the z neighbours
// from its queue, and writes u_next over u_prev with 128-bit streaming
// stores. The Ricker source and the receivers are applied in the same pass.
#pragma once

#include <cuda.h>
#include <cstdint>

#include "ptx.cuh"

namespace gbw {

constexpr int kR = 4;                // stencil radius (Sec. 4.1: R = 4)
constexpr int kErrTimeout = 1;       // device error word values
constexpr uint64_t kWaitLimitNs = 2000000000ull;

// Per-call state read by every sweep launch (device memory, one per context).
struct StepDesc {
  long long n;            // index of the next step within the current call
  const float *wavelet;   // source value per step of the call (or null)
  float *traces;          // nsteps x nrec, row n written by step n (or null)
  const int4 *rec;        // receivers sorted by (tile, z): {z, local, id, 0}
  const int *rec_start;   // per tile: first entry; size ntiles + 1
  int nrec;
  int src_active;
  int sx, sy, sz;
  int error;              // first error recorded by a kernel (0 = none)
};

constexpr int kMaxLayers = 16;

struct SweepArgs {
  int nx, ny, nz, px;  // interior sizes; px = row pitch in floats (mult. of 4)
  // z layers: CTAs with blockIdx.z == l stream planes [zl[l], zl[l+1]).
  // Layers are launched in order, so large layers first and small ones last
  // shorten the partial last wave of CTAs.
  int nlayers;
  int zl[kMaxLayers + 1];
  int ntx;             // tiles along x (tile id = by * ntx + bx)
  float c0;            // w0 * (1/dx^2 + 1/dy^2 + 1/dz^2)
  float cx[4], cy[4], cz[4];  // w_m / h_a^2 for m = 1..4
  float *unext;        // output: the u_prev buffer, overwritten in place
  StepDesc *desc;
  int koff;            // step offset of this launch within a graph chunk
  float dt2;           // dt^2, used only when the c field holds velocities
};

template <int TX_, int TY_, int VY_, int PF_, int MINB_>
struct SweepCfg {
  static constexpr int TX = TX_, TY = TY_, VY = VY_, PF = PF_, MINB = MINB_;
  static constexpr int NTX = TX / 4;       // threads along x (4 points each)
  static constexpr int NTY = TY / VY;      // threads along y (VY rows each)
  static constexpr int THREADS = NTX * NTY;
  static constexpr int SU = PF + 5;        // u ring: 5 live planes + prefetch
  static constexpr int SP = PF + 1;        // u_prev / c ring
  static constexpr int NB = PF + 1;        // one barrier per in-flight stage
  static constexpr int UW = TX + 2 * kR;   // u slot row length (floats)
  static constexpr int UH = TY + 2 * kR;
  static constexpr int U_SLOT = UW * UH;   // floats
  static constexpr int P_SLOT = TX * TY;
  static constexpr uint32_t U_BYTES = U_SLOT * 4;
  static constexpr uint32_t P_BYTES = P_SLOT * 4;
  static constexpr size_t SMEM_BYTES =
      128 + (size_t)(SU * U_SLOT + 2 * SP * P_SLOT + P_SLOT) * 4 + NB * 8;
  static_assert(TX % 4 == 0 && TY % VY == 0, "tile shape");
  static_assert((UW * 4) % 16 == 0, "TMA box row must be a multiple of 16 B");
  static_assert(U_BYTES % 128 == 0 && P_BYTES % 128 == 0, "slot alignment");
  static_assert(UW <= 256 && UH <= 256, "TMA box limit");
};

// kVelocityField = false: tm_c maps v^2 dt^2. true: tm_c maps the velocity
// itself and the kernel forms v^2 dt^2 from it (the allocation-free entry
// point, which has no buffer of its own to hold v^2 dt^2).
template <class C, bool kVelocityField = false>
__global__ void __launch_bounds__(C::THREADS, C::MINB)
    wave_sweep_kernel(const __grid_constant__ CUtensorMap tm_u,
                      const __grid_constant__ CUtensorMap tm_up,
                      const __grid_constant__ CUtensorMap tm_c,
                      const SweepArgs a) {
  extern __shared__ unsigned char smem_raw[];
  float *su = reinterpret_cast<float *>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
  float *sp = su + C::SU * C::U_SLOT;
  float *sc = sp + C::SP * C::P_SLOT;
  float *sr = sc + C::SP * C::P_SLOT;  // receiver staging (one plane)
  uint64_t *bars = reinterpret_cast<uint64_t *>(sr + C::P_SLOT);

  const int tid = threadIdx.x;
  const int tx = tid % C::NTX;
  const int ty = tid / C::NTX;
  const int x0 = blockIdx.x * C::TX;
  const int y0 = blockIdx.y * C::TY;
  const int zb = a.zl[blockIdx.z];
  const int ze = a.zl[blockIdx.z + 1];
  const int NS = (ze - zb) + 2 * kR;  // stages: 8 to fill the queue, then one per plane

  // Per-call state.
  const StepDesc *d = a.desc;
  const long long n = d->n + a.koff;
  const int nrec = d->nrec;
  const int sx = d->sx - x0, sy = d->sy - y0, sz = d->sz;
  const bool src_here = d->src_active && sx >= 0 && sx < C::TX && sy >= 0 &&
                        sy < C::TY && sz >= zb && sz < ze;
  const float wsrc = src_here ? d->wavelet[n] : 0.f;
  int rcur = 0, rend = 0;
  const int4 *rec = d->rec;
  if (nrec > 0) {
    const int tile = blockIdx.y * a.ntx + blockIdx.x;
    rcur = d->rec_start[tile];
    rend = d->rec_start[tile + 1];
    while (rcur < rend && rec[rcur].x < zb) ++rcur;
  }
  int rz = (rcur < rend) ? rec[rcur].x : 0x7fffffff;  // z of the next receiver
  float *trow = (nrec > 0) ? d->traces + (size_t)n * nrec : nullptr;

  if (tid == 0) {
    prefetch_tensormap(&tm_u);
    prefetch_tensormap(&tm_up);
    prefetch_tensormap(&tm_c);
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
    mbar_arrive_expect_tx(bar, C::U_BYTES + (full ? 2 * C::P_BYTES : 0));
    tma_load_3d(su + (s % C::SU) * C::U_SLOT, &tm_u, bar, x0 - kR, y0 - kR,
                j + kR);
    if (full) {
      tma_load_3d(sp + (s % C::SP) * C::P_SLOT, &tm_up, bar, x0, y0, j);
      tma_load_3d(sc + (s % C::SP) * C::P_SLOT, &tm_c, bar, x0, y0, j);
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

  const int col = 4 * tx + kR;  // smem column of this thread's first point
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
      const float *uf = su + fslot * C::U_SLOT;
#pragma unroll
      for (int v = 0; v < C::VY; ++v)
        q[v][p] = lds4(uf + (ty * C::VY + v + kR) * C::UW + col);
      const int j = zb - 2 * kR + s;
      if (j < zb) continue;

      const int cslot = (C::SU == 9) ? (p + 5) % 9 : ((s + C::SU - kR) % C::SU);
      const float *uc = su + cslot * C::U_SLOT;  // plane j
      const float *pp = sp + (s % C::SP) * C::P_SLOT;
      const float *pc = sc + (s % C::SP) * C::P_SLOT;
      float4 res[C::VY];
#pragma unroll
      for (int v = 0; v < C::VY; ++v) {
        const int r = ty * C::VY + v + kR;  // smem row of this point row
        const float4 a0 = lds4(uc + r * C::UW + col - 4);
        const float4 a1 = lds4(uc + r * C::UW + col);
        const float4 a2 = lds4(uc + r * C::UW + col + 4);
        const float xs[12] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y,
                              a1.z, a1.w, a2.x, a2.y, a2.z, a2.w};
        float acc[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) acc[e] = a.c0 * xs[4 + e];
#pragma unroll
        for (int m = 1; m <= kR; ++m) {
          const float4 ym = lds4(uc + (r - m) * C::UW + col);
          const float4 yp = lds4(uc + (r + m) * C::UW + col);
          const float4 zm = q[v][(p + 5 - m + 9) % 9];
          const float4 zp = q[v][(p + 5 + m) % 9];
          const float cxm = a.cx[m - 1], cym = a.cy[m - 1], czm = a.cz[m - 1];
          acc[0] = fmaf(cxm, xs[4 - m] + xs[4 + m], acc[0]);
          acc[1] = fmaf(cxm, xs[5 - m] + xs[5 + m], acc[1]);
          acc[2] = fmaf(cxm, xs[6 - m] + xs[6 + m], acc[2]);
          acc[3] = fmaf(cxm, xs[7 - m] + xs[7 + m], acc[3]);
          acc[0] = fmaf(cym, ym.x + yp.x, acc[0]);
          acc[1] = fmaf(cym, ym.y + yp.y, acc[1]);
          acc[2] = fmaf(cym, ym.z + yp.z, acc[2]);
          acc[3] = fmaf(cym, ym.w + yp.w, acc[3]);
          acc[0] = fmaf(czm, zm.x + zp.x, acc[0]);
          acc[1] = fmaf(czm, zm.y + zp.y, acc[1]);
          acc[2] = fmaf(czm, zm.z + zp.z, acc[2]);
          acc[3] = fmaf(czm, zm.w + zp.w, acc[3]);
        }
        const int pofs = (ty * C::VY + v) * C::TX + 4 * tx;
        const float4 upv = lds4(pp + pofs);
        float4 cv = lds4(pc + pofs);
        if (kVelocityField) {
          cv.x = cv.x * cv.x * a.dt2;
          cv.y = cv.y * cv.y * a.dt2;
          cv.z = cv.z * cv.z * a.dt2;
          cv.w = cv.w * cv.w * a.dt2;
        }
        float4 o;
        o.x = fmaf(cv.x, acc[0], fmaf(2.f, xs[4], -upv.x));
        o.y = fmaf(cv.y, acc[1], fmaf(2.f, xs[5], -upv.y));
        o.z = fmaf(cv.z, acc[2], fmaf(2.f, xs[6], -upv.z));
        o.w = fmaf(cv.w, acc[3], fmaf(2.f, xs[7], -upv.w));
        if (src_here && j == sz && sy == ty * C::VY + v) {
          const int e = sx - 4 * tx;
          if (e == 0) o.x = fmaf(cv.x, wsrc, o.x);
          if (e == 1) o.y = fmaf(cv.y, wsrc, o.y);
          if (e == 2) o.z = fmaf(cv.z, wsrc, o.z);
          if (e == 3) o.w = fmaf(cv.w, wsrc, o.w);
        }
        res[v] = o;
        const int y = y0 + ty * C::VY + v;
        const int x = x0 + 4 * tx;
        if (y < a.ny && x < a.px)
          __stcs(reinterpret_cast<float4 *>(a.unext + ((size_t)j * a.ny + y) *
                                                          a.px + x),
                 o);
      }

      // Receivers on this plane: stage the plane, then one thread per entry.
      if (j == rz) {
#pragma unroll
        for (int v = 0; v < C::VY; ++v)
          *reinterpret_cast<float4 *>(sr + (ty * C::VY + v) * C::TX + 4 * tx) =
              res[v];
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

}  // namespace gbw
