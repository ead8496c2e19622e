/*
 * gbwave shot server: continuous batching of independent seismic shots on
 * one GPU.
 *
 * The paper studies one grid stepped by one kernel per time step (Sec. 4)
 * and overlaps small kernels on two streams to keep the GPU busy (Sec. 5.1,
 * "fine-grained concurrent kernels"). This server keeps the GPU busy with
 * many grids instead: every time step is one launch whose CTAs cover the
 * tiles of all resident shots, each shot advancing by one step of the
 * update declared in wave.h (Eq. 1 Laplacian, leapfrog, Ricker source,
 * receivers). Shots of different sizes and step counts join as memory and
 * slots free up and leave when done, at step boundaries; each shot's
 * arithmetic is that of wave_propagate, so its traces are the same
 * alone or in any mix.
 *
 * Threading: serve_create starts one engine thread that owns all GPU work
 * (admission, launches, completion). serve_submit / serve_poll /
 * serve_wait / serve_stats may be called from any thread.
 *
 * Memory: each admitted shot holds its wavefields (2 fields, FP32 or 16-bit),
 * v^2 dt^2 (FP32), and its tables (source wavelet, receiver table, and a
 * trace staging buffer when `traces` is host memory); a shot with the CPML
 * layer also holds the layer's memory variables (psi, zeta in FP32 slabs of
 * 2 npml cells per axis) and profiles, the profile set from that shot's
 * largest velocity and time step. After each batched step, the layered
 * shots of a storage type take their layer passes in one launch per axis
 * and their shell receivers in one more. Admission is first in,
 * first out: the head request waits until its bytes fit in the budget next to
 * the resident shots, a slot is free, and one batched step over the resident
 * shots and it would launch no more than six waves of CTAs (four per SM),
 * unless nothing is resident (so every admissible request runs eventually).
 */
#ifndef GBWAVE_WAVE_SERVE_H
#define GBWAVE_WAVE_SERVE_H

#include "wave.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct serve_ctx serve_ctx; /* opaque */

typedef struct {
  wave_grid grid;       /* interior points */
  wave_spacing spacing; /* metres */
  double dt;            /* seconds; <= 0 selects 0.5 * wave_cfl_dt of the model */
  const float *velocity;/* nx*ny*nz float32 m/s, host or device; read when the
                           request is admitted: keep it valid until the request
                           completes */
  int storage;          /* WAVE_STORAGE_F32 / BF16 / F16 */
  wave_shot shot;       /* Ricker source (required) */
  int nsteps;           /* >= 1 */
  const int32_t *rec_xyz; /* nrec*3 int32 (x, y, z), host or device; read at
                             admission */
  int nrec;             /* >= 0 */
  float *traces;        /* nsteps*nrec float32, host or device, caller-owned;
                           complete when the request completes */
  int npml;             /* CPML layer cells per face (wave_set_cpml's layer);
                           0: none, else 2 npml <= nx, ny, nz and ny, nz <=
                           65535 */
  double reflection;    /* the layer's target reflection, 0 < R < 1 */
  double f_cps;         /* the layer's frequency shift (Hz, >= 0) */
} wave_request;

typedef struct {
  int status;       /* WAVE_OK, WAVE_EBUSY (queued or running), or an error */
  uint64_t ticket;
  double submit_s;  /* times in seconds since serve_create (steady clock) */
  double start_s;   /* admitted (-1 if not yet) */
  double done_s;    /* completed (-1 if not yet) */
  double dt;        /* time step used (0 until admitted) */
  int64_t steps_done;
} wave_result;

typedef struct {
  int64_t submitted, completed, failed, queued, resident;
  size_t bytes_resident;    /* device bytes held by resident shots */
  size_t bytes_peak;        /* largest bytes_resident seen */
  int resident_peak;        /* largest number of resident shots seen */
  int64_t batch_steps;      /* launches of the batched step (per storage type) */
  double point_steps;       /* sum over shots of grid points x steps done */
  double busy_s;            /* engine time with at least one resident shot */
} serve_stats_t;

/*
 * Start a server.
 *   hbm_budget_bytes  device bytes the resident shots may hold (> 0)
 *   max_slots         most shots resident at once (1 .. 4096)
 *   stream            cudaStream_t for all the server's work; NULL: the
 *                     server creates its own non-blocking stream
 * The current device at this call is the server's device.
 */
int serve_create(size_t hbm_budget_bytes, int max_slots, void *stream,
                 serve_ctx **out);

/*
 * Queue a request. Checks sizes, positions and pointers at once
 * (WAVE_EINVAL), and that the request's device bytes fit the budget at all
 * (WAVE_ETOOBIG); velocity and receivers are read at admission, where bad
 * values fail the request (status WAVE_EINVAL or WAVE_EUNSTABLE).
 *   ticket  receives the request's id (> 0)
 */
int serve_submit(serve_ctx *s, const wave_request *req, uint64_t *ticket);

/*
 * State of a request without waiting: WAVE_EBUSY while queued or running,
 * otherwise the request's final status; *out (if not NULL) is filled either
 * way. WAVE_EINVAL for an unknown ticket.
 */
int serve_poll(serve_ctx *s, uint64_t ticket, wave_result *out);

/* As serve_poll, but waits up to timeout_s seconds (< 0: no limit). */
int serve_wait(serve_ctx *s, uint64_t ticket, double timeout_s, wave_result *out);

int serve_get_stats(serve_ctx *s, serve_stats_t *out);

/*
 * Stop accepting requests, finish every queued and resident request, stop
 * the engine and free the server. NULL is a no-op.
 */
void serve_destroy(serve_ctx *s);

#ifdef __cplusplus
}
#endif

#endif /* GBWAVE_WAVE_SERVE_H */
