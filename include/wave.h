/*
 * gbwave: time-stepped 3D acoustic wave propagation on one GB300 (sm_103a).
 *
 * The operation (Sec. 2, Eq. 1; Sec. 4.1 for R = 4 and the x-innermost
 * layout): at every interior grid point and every time step,
 *
 *     L u = sum_{a in x,y,z} (1/h_a^2) ( w0 u + sum_{m=1..4} w_m (u(+m e_a) + u(-m e_a)) )
 *     u_next = 2 u - u_prev + v^2 dt^2 L u                 (second-order leapfrog)
 *
 * with w = (-205/72, 8/5, -1/5, 8/315, -1/560) (Eq. 1's c_am = w_m / h_a^2;
 * its m = 0 term counts the centre twice, c_a0 = w0 / (2 h_a^2)). Points
 * outside the interior read as zero (zero Dirichlet halo of width 4); an
 * absorbing CPML layer like the paper's (Sec. 2) can be switched on per
 * context with wave_set_cpml. After the update of
 * step n a Ricker point source adds v^2 dt^2 s(t_n) at the source point,
 * t_n = n dt, s(t) = amp (1 - 2 pi^2 f^2 (t-t0)^2) exp(-pi^2 f^2 (t-t0)^2),
 * and every receiver records u_next at its point.
 *
 * Conventions shared by every entry point:
 *  - Grids are interior points only, x fastest, then y, then z (z = depth).
 *    Dense user arrays are nx*ny*nz float32 with index (k*ny + j)*nx + i.
 *  - Pointers may be host or device memory; the library asks the CUDA runtime
 *    which (cudaPointerGetAttributes). A call that reads a host buffer has
 *    finished reading it when it returns; a call that writes a host buffer
 *    returns after the data is there (it synchronizes the context's stream).
 *    Calls that touch device buffers only are asynchronous on that stream.
 *  - The caller owns every buffer it passes; the context owns the wavefields
 *    and its internal tables and frees them in wave_destroy.
 *  - All work is enqueued on the stream given to wave_create (a cudaStream_t,
 *    NULL = the legacy default stream). A context is not thread-safe;
 *    separate contexts are independent.
 *  - Functions return WAVE_OK (0) or a negative status; none aborts. Inputs
 *    are validated before anything is launched.
 *  - Device-side waits are bounded: a kernel whose copy pipeline stalls for
 *    about two seconds records WAVE_ETIMEOUT, which the next synchronizing
 *    call (wave_synchronize, wave_get_field to host, ...) returns. Such a
 *    recorded error (also WAVE_ENAN) stays until wave_reset or
 *    wave_set_state replaces the state.
 */
#ifndef GBWAVE_WAVE_H
#define GBWAVE_WAVE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  WAVE_OK = 0,
  WAVE_EINVAL = -1,    /* bad argument (sizes, positions, pointers, NaN or v <= 0) */
  WAVE_ENOMEM = -2,    /* device allocation failed */
  WAVE_ECUDA = -3,     /* a CUDA runtime/driver call failed */
  WAVE_EUNSTABLE = -4, /* dt above the leapfrog stability limit (wave_cfl_dt) */
  WAVE_ETIMEOUT = -5,  /* a bounded device wait gave up */
  WAVE_EBUSY = -6,     /* result not ready yet */
  WAVE_ENAN = -7,      /* a receiver trace holds a NaN or an infinity (checked
                          after every wave_propagate, noalloc call and served
                          shot; reported by the next synchronizing call) */
  WAVE_ENOTSUP = -8,   /* option not supported by this build */
  WAVE_ETOOBIG = -9    /* request exceeds the fixed scratch of wave_propagate_noalloc */
};

/*
 * Storage precision of the two wavefields (argument of wave_create). The
 * arithmetic is FP32 in every mode and v^2 dt^2 is stored FP32, so a step
 * moves 16 bytes per point in F32 mode and 10 in the 16-bit modes. In the
 * 16-bit modes each field carries a power-of-two scale chosen on the device
 * when the field is written (from the largest magnitudes of the two fields
 * it is computed from, with headroom for the largest growth one stable step
 * allows), so FP16 cannot overflow and scaling adds no rounding. The values
 * read back (wave_get_field, traces) are FP32 = stored value x scale. The
 * rounding of u to 16 bits every step accumulates: measured against the FP64
 * oracle on 128^3 x 500 steps, FP16 stays near 1e-2 relative L2 while BF16
 * (8-bit mantissa) drifts to tens of percent.
 */
enum { WAVE_STORAGE_F32 = 0, WAVE_STORAGE_BF16 = 1, WAVE_STORAGE_F16 = 2 };

typedef struct wave_ctx wave_ctx; /* opaque; owns the device wavefields */

typedef struct {
  int32_t nx, ny, nz; /* interior points per axis, each >= 1 */
} wave_grid;

typedef struct {
  double dx, dy, dz; /* grid spacing in metres, each > 0 */
} wave_spacing;

typedef struct {
  int32_t sx, sy, sz; /* source point, inside the interior */
  double f_peak;      /* Ricker peak frequency in Hz (> 0) */
  double t0;          /* Ricker delay in seconds; t0 < 0 selects 1 / f_peak */
  double amp;         /* Ricker amplitude */
} wave_shot;

/*
 * Largest stable time step of the scheme for velocities up to vmax:
 * dt_max = 2 / (vmax sqrt(S (1/dx^2 + 1/dy^2 + 1/dz^2))), S = |w0| + 2 sum |w_m|
 * (von Neumann analysis of the leapfrog recurrence on the highest mode of
 * Eq. 1). Returns a negative value for invalid arguments.
 * Defined by: Eq. 1 (the stencil) with the second-order time update of the
 * wave equation of Sec. 2.
 */
double wave_cfl_dt(const wave_spacing *h, double vmax);

/*
 * Create a context for one grid and velocity model.
 *   g, h      grid size and spacing (read during the call)
 *   dt        time step in seconds; must be in (0, wave_cfl_dt(h, max v)]
 *   velocity  nx*ny*nz float32 velocities in m/s, dense, x fastest; host or
 *             device; every value finite and > 0. The context keeps
 *             v^2 dt^2 (FP32), not the pointer.
 *   storage   WAVE_STORAGE_F32, WAVE_STORAGE_BF16 or WAVE_STORAGE_F16
 *             (other values: WAVE_ENOTSUP)
 *   stream    cudaStream_t all work of this context is enqueued on
 *   out       receives the new context (NULL on failure)
 * The wavefields start at zero, step counter 0. Returns WAVE_EINVAL,
 * WAVE_EUNSTABLE, WAVE_ENOMEM, WAVE_ENOTSUP or WAVE_ECUDA on failure.
 * Defined by: Sec. 2 (the acoustic isotropic medium the stencil is applied
 * to) and Sec. 4.1 (the grid as one flat array, x innermost).
 */
int wave_create(const wave_grid *g, const wave_spacing *h, double dt,
                const float *velocity, int storage, void *stream,
                wave_ctx **out);

/*
 * As wave_create, with the model given as the squared velocity m = v^2
 * (m^2/s^2, nx*ny*nz float32, every value finite and > 0): the variable
 * wave_adjoint / wave_gradient differentiate with respect to. The context
 * keeps c = m dt^2 (one product, no square root taken and squared again),
 * and the stability limit uses vmax = sqrt(max m).
 */
int wave_create_m(const wave_grid *g, const wave_spacing *h, double dt,
                  const float *m, int storage, void *stream, wave_ctx **out);

/*
 * As wave_create, but the call returns before the velocity model has been
 * read. Reading it, validating it and converting it to v^2 dt^2 run on a
 * stream of the context's own in 32 depth slabs, overlapped with the first
 * steps of a propagation from rest: on a host model the transfer (bound by
 * the host link) is then hidden behind the stepping instead of preceding it.
 *  - While the context is still at rest (zero fields, nothing stepped, no
 *    wave_set_state), a wave_propagate with a source waits before its step k
 *    only for the slabs that reach depth sz + 4k: the stencil of Eq. 1 moves
 *    the field by at most R = 4 planes per step (Sec. 4.1), so every deeper
 *    plane still holds zero and computes zero whatever its v^2 dt^2 (which
 *    starts at zero). Any other call that steps or needs the model waits
 *    for all of it first. Results are identical to those of wave_create.
 *  - The caller's velocity buffer must stay valid and unchanged until a
 *    synchronizing call on this context has returned (wave_synchronize, a
 *    wave_propagate or wave_get_field with a host destination, wave_set_cpml,
 *    wave_adjoint, wave_gradient) or the context is destroyed.
 *  - Velocities that are not finite and positive (WAVE_EINVAL) and a dt
 *    above the stability limit (WAVE_EUNSTABLE) are reported by that
 *    synchronizing call and by every later synchronizing call (wave_reset
 *    does not clear them); what was computed before is meaningless.
 *  - The deferral applies to FP32 storage when the GPU can read the model
 *    where it lies: device memory, pinned host memory, or pageable host
 *    memory on systems whose GPU uses the host's page tables. Otherwise the
 *    call behaves exactly like wave_create.
 */
int wave_create_async(const wave_grid *g, const wave_spacing *h, double dt,
                      const float *velocity, int storage, void *stream,
                      wave_ctx **out);

/*
 * Advance nsteps (>= 0) leapfrog steps with no source and no receivers.
 * Defined by: Eq. 1 applied at every interior point once per time step
 * (Sec. 2), the update u_next = 2u - u_prev + v^2 dt^2 L u.
 */
int wave_step(wave_ctx *ctx, int nsteps);

/*
 * Advance nsteps (>= 0) steps with the Ricker source of *shot (NULL: no
 * source) and record receivers.
 *   rec_xyz  nrec*3 int32 receiver points (x, y, z), host or device; each
 *            inside the interior (WAVE_EINVAL otherwise); may repeat
 *   traces   nsteps*nrec float32, host or device, caller-owned; row n holds
 *            the receivers after step n of this call (time (step0+n+1) dt,
 *            step0 = the context's step counter at entry)
 * The source time of the call's step n is t = (step0 + n) dt.
 * Defined by: Eq. 1 and the per-step update of Sec. 2; the paper does not
 * state the source or the receivers: a Ricker point source injected after
 * each update and receivers recording the updated field are the readings
 * taken here.
 */
int wave_propagate(wave_ctx *ctx, const wave_shot *shot, int nsteps,
                   const int32_t *rec_xyz, int nrec, float *traces);

/*
 * Copy a wavefield out as nx*ny*nz float32 (dense, x fastest).
 *   which  0 = u at the current step, 1 = u at the previous step
 * 16-bit storage: the values are expanded to FP32 with the field's scale (a
 * host destination is staged through a temporary device buffer).
 * Defined by: the wavefield of Sec. 2 in the layout of Sec. 4.1.
 */
int wave_get_field(const wave_ctx *ctx, int which, float *out);

/*
 * Replace the state: u (current step) and u_prev (previous step), each
 * nx*ny*nz float32 dense (host or device), and the step counter.
 * 16-bit storage: each field is rounded to the storage format with a
 * power-of-two scale that maps its largest magnitude to at most 2^14
 * (host inputs are staged through temporary device buffers; the call
 * synchronizes). Non-finite values return WAVE_EINVAL.
 * Defined by: the two time levels the leapfrog update of Sec. 2 carries.
 */
int wave_set_state(wave_ctx *ctx, const float *u, const float *u_prev,
                   int64_t step);

/* Current step counter (number of steps taken since creation/reset/set_state;
 * the iteration count of the time loop of Sec. 2). */
int wave_get_step(const wave_ctx *ctx, int64_t *step);

/* Zero both wavefields and the step counter (the time loop of Sec. 2 from rest). */
int wave_reset(wave_ctx *ctx);

/*
 * Absorbing boundary: a convolutional PML (CPML) of npml cells inside every
 * face of the grid, in place of the bare zero halo (the paper's domain is
 * surrounded by a CPML-like layer after Komatitsch and Martin 2007, Sec. 2).
 * Second-order form from complex-frequency-shifted coordinate stretching:
 *   u_tt = v^2 sum_a (d_aa u + d_a psi_a + zeta_a),
 *   psi_a^n = b psi_a^{n-1} + a D1_a u^n,
 *   zeta_a^n = b zeta_a^{n-1} + a (D2_a u^n + D1_a psi_a^n),
 *   b = exp(-(d + alpha) dt), a = d / (d + alpha) (b - 1),
 * with D2_a the axis part of Eq. 1, D1_a the 8th-order central first
 * derivative (4/5, -1/5, 4/105, -1/280), and per axis the profile
 * d = d0 xi^2, d0 = 3 vmax ln(1/reflection) / (2 npml h_a), alpha =
 * pi f_cps (1 - xi), xi in (0, 1] the depth into the layer (1 at the face).
 *   npml        layer cells per face; 0 switches the layer off; otherwise
 *               1 <= npml and 2 npml <= nx, ny, nz
 *   reflection  target reflection coefficient, 0 < reflection < 1
 *   f_cps       frequency shift (Hz, >= 0), typically the source's peak
 * ny, nz <= 65535 only (WAVE_ENOTSUP otherwise). With 16-bit storage the
 * layer's passes read and write the stored fields through the step's
 * power-of-two scales (one more rounding to the format per pass at the
 * shell points); psi and zeta stay FP32. The
 * layer's memory variables start at zero here and are zeroed by wave_reset
 * and wave_set_state. The
 * source and receivers may lie in the layer. wave_adjoint / wave_gradient
 * differentiate the run with the layer (its profile held fixed).
 */
int wave_set_cpml(wave_ctx *ctx, int npml, double reflection, double f_cps);

/* Wait for the context's stream; return any error a kernel recorded. No
 * counterpart in the paper (error reporting of this library). */
int wave_synchronize(wave_ctx *ctx);

/* Free everything the context owns (waits for its stream first). NULL is a
 * no-op. No counterpart in the paper. */
void wave_destroy(wave_ctx *ctx);

/* Static message for a status code. No counterpart in the paper. */
const char *wave_strerror(int status);

/*
 * Launch geometry of the stencil sweep for this context (for reports and
 * benchmarks): CTA tile in x and y, z planes per CTA, grid size, resident
 * CTAs per SM. Any output pointer may be NULL. The blocking itself follows
 * the 2.5D streaming scheme of Sec. 4.1 (xy tile plus halo, z streamed).
 */
int wave_get_launch_info(const wave_ctx *ctx, int *tile_x, int *tile_y,
                         int *z_chunk, int *grid_ctas, int *ctas_per_sm);

/*
 * Diagnostic of the bounded device wait used by every kernel of this
 * library: launches one thread that waits on a shared-memory barrier nothing
 * arrives on, with a limit of limit_ns nanoseconds (clamped to 1 ms .. 10 s).
 * Synchronizes the stream. Returns WAVE_ETIMEOUT when the wait gave up as
 * designed, WAVE_ECUDA if it reported completion or a CUDA call failed.
 * No counterpart in the paper (failure detection of this library).
 */
int wave_selftest_wait(int64_t limit_ns, void *stream);

/*
 * Gradient of a trace objective with respect to m = v^2 at every point: the
 * discrete adjoint of wave_propagate from rest (u = u_prev = 0, step 0).
 *
 * With the forward recursion u^{n+1} = 2u^n - u^{n-1} + C L u^n + C_s w_n
 * (C = m dt^2, Eq. 1 for L) and traces d^n = R u^{n+1}, the adjoint field
 * q^k = 2q^{k+1} - q^{k+2} + L(C q^{k+1}) + R^T r^{k-1} runs backwards from
 * zero, r^n = dJ/dd^n, and dJ/dm = (1/m) sum_n q^{n+1} (u^{n+1} - 2u^n +
 * u^{n-1}): the back-propagated residual correlated with the forward second
 * time difference. The library runs p = C q, which obeys the forward update
 * with the residuals injected at the receivers, on the same sweep kernel;
 * the forward fields come from checkpoints every ckpt_every steps, one
 * segment recomputed at a time; the time sum is accumulated in FP64 (each
 * block of 256 steps, counted from step 0, is first summed as an FP32
 * double-float pair of about 48 significant bits, then added to the FP64
 * sum).
 * With the CPML layer (wave_set_cpml) the forward map includes the memory
 * variables and the adjoint is that of the whole layered update: per axis
 * a, with A = the profile's a, B = its b and p^{N+1} = nu^{N+1} = mu^{N+1}
 * = 0, each backward step k forms nu^k = p^{k+1} + B nu^{k+1} and mu^k =
 * -D1_a (p^{k+1} + A nu^k) + B mu^{k+1} in the slabs and adds
 * C (D2_a (A nu^k) - D1_a (A mu^k)) to p^k; u^{n+1} - 2u^n + u^{n-1}
 * includes the layer's term, and the checkpoints also hold psi and zeta.
 * The profile (which depends on the largest velocity) is held fixed.
 * Device memory then also holds (2 ceil(nsteps/ckpt_every) + 2) times the
 * memory-variable slabs (2 npml (ny nz + nz nx + ny nx) floats each).
 *
 *   shot         Ricker source of the forward run (NULL: none)
 *   rec_xyz      nrec*3 int32 receivers (host or device), as wave_propagate
 *   resid        nsteps*nrec float32 dJ/dtraces (host or device)
 *   ckpt_every   steps per checkpoint segment (>= 1); device memory holds
 *                2 * ceil(nsteps/ckpt_every) + 2 * ckpt_every + 6 float32
 *                fields (ckpt_every + 8 when one segment covers nsteps; the
 *                FP64 time sum counts as two), plus the traces
 *   grad_v2      nx*ny*nz float32 output (host or device), dense, x fastest
 *   traces       optional nsteps*nrec float32 output of the forward traces
 * FP32 storage and the default kernel variant only (else WAVE_ENOTSUP). The
 * call synchronizes; it leaves the context reset (zero fields, step 0).
 * Defined by: the discrete adjoint of the update of Eq. 1 and Sec. 2 (the
 * paper computes no gradient; this is the exact derivative of the discrete
 * forward map).
 */
int wave_adjoint(wave_ctx *ctx, const wave_shot *shot, int nsteps,
                 const int32_t *rec_xyz, int nrec, const float *resid,
                 int ckpt_every, float *grad_v2, float *traces);

/*
 * The L2 trace misfit J = 1/2 sum_{n,r} (d^n_r - observed^n_r)^2 of a run
 * from rest and its gradient dJ/d(v^2) (wave_adjoint with resid = d -
 * observed). The residual and the misfit sum are formed on the GPU, the sum
 * in FP64. observed: nsteps*nrec float32, host or device; misfit: host.
 * Defined by: as wave_adjoint.
 */
int wave_gradient(wave_ctx *ctx, const wave_shot *shot, int nsteps,
                  const int32_t *rec_xyz, int nrec, const float *observed,
                  int ckpt_every, double *misfit, float *grad_v2,
                  float *traces);

/*
 * Allocation-free propagation. The paper has no counterpart to this entry
 * point; it exists for callers that must not allocate device memory: code
 * running inside an application whose memory pool already owns the whole
 * GPU (a cudaMalloc there fails or fragments the pool), plugins held to a
 * fixed memory budget, and services that forbid allocation once they have
 * started. It runs the same leapfrog sweep as wave_propagate, but on buffers
 * the caller owns, and keeps its small tables (step descriptor, receiver
 * table, source wavelet) in one fixed array of WAVE_NOALLOC_SCRATCH_BYTES
 * that the library declares statically: every GPU that loads the library
 * holds that array until the process exits. It calls no cudaMalloc, no
 * cudaFree and no allocating library routine; its own host-side work (the
 * z-layer plan, the table image, staged host receivers) uses fixed static
 * storage, so the call allocates no host heap either (the CUDA runtime's
 * internal bookkeeping aside).
 *
 *   g, h, dt     as for wave_create; nx must be a multiple of 4 (rows of the
 *                caller's dense arrays must start on 16-byte boundaries)
 *   velocity     device, nx*ny*nz float32 m/s, dense, 16-byte aligned
 *   u, u_prev    device, nx*ny*nz float32 each, dense, 16-byte aligned; the
 *                state at steps step0 and step0-1 on entry. The sweep writes
 *                each new step over the older buffer, so on return the
 *                newest step is in u if *newest == 0 and in u_prev if
 *                *newest == 1 (nsteps odd); the other buffer holds the step
 *                before it
 *   shot         Ricker source or NULL; source time of step n is (step0+n) dt
 *   rec_xyz      nrec*3 int32, host or device; traces: device, nsteps*nrec
 *
 * Limits: the tables must fit the array: 512 + (16 * nrec) +
 * (4 * nsteps rounded up to 256, if shot) + (4 * (tiles + 1) rounded up to
 * 256, if nrec > 0) bytes, tiles = ceil(nx/64) * ceil(ny/16); otherwise the
 * call returns WAVE_ETOOBIG before launching anything. With 4 MiB this is,
 * for example, 65536 receivers and 100000 steps on a 1024 x 1024 grid.
 *
 * The first call on each device finds the array's device address
 * (cudaGetSymbolAddress) and sets the kernel's shared-memory limit, with that
 * device current; make that first call before any stream capture. First
 * calls from several host threads are serialised by a lock. The address is
 * kept for the life of the process: after cudaDeviceReset the library has
 * to be unloaded and loaded again before this entry point is used. Every
 * call shares the one array and overwrites what the last call left there;
 * calls whose work overlaps on the GPU (other streams, other host threads)
 * race on it, so serialize them. The call validates the velocities
 * (finite, > 0, dt within wave_cfl_dt) and synchronizes the stream before
 * it returns, so a timed-out device wait comes back as WAVE_ETIMEOUT.
 */
#define WAVE_NOALLOC_SCRATCH_BYTES (4u << 20)

int wave_propagate_noalloc(const wave_grid *g, const wave_spacing *h, double dt,
                           const float *velocity, float *u, float *u_prev,
                           const wave_shot *shot, int64_t step0, int nsteps,
                           const int32_t *rec_xyz, int nrec, float *traces,
                           void *stream, int *newest);

#ifdef __cplusplus
}
#endif

#endif /* GBWAVE_WAVE_H */
