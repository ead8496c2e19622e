/*
 * FP64 CPU oracle for the time-stepped 3D acoustic wave update.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path may link, load or
 * call this file; only the tests, the package smoke check and the CPU
 * baseline leg of the benchmark do. It shares no code, header, table or
 * constant with the CUDA library.
 *
 * What it computes (plain definition, no blocking, no fusion):
 *
 *   Eq. 1 (Sec. 2): the 25-point, radius-4 star approximation of the
 *   Laplacian,
 *       L u(i,j,k) = sum_{m=0..4} c_xm [u(i+m,j,k) + u(i-m,j,k)]
 *                               + c_ym [u(i,j+m,k) + u(i,j-m,k)]
 *                               + c_zm [u(i,j,k+m) + u(i,j,k-m)]
 *   with c_am = w_m / h_a^2 for m >= 1. The m = 0 term of Eq. 1 adds the
 *   centre twice, so c_a0 = w_0 / (2 h_a^2). The w_m are the 8th-order
 *   central second-derivative weights (-205/72, 8/5, -1/5, 8/315, -1/560);
 *   the paper calls them only "discretization parameters" and gives R = 4
 *   (Sec. 4.1).
 *
 *   Sec. 2 applies Eq. 1 at every grid point once per time iteration to
 *   advance the acoustic isotropic wave equation u_tt = v^2 lap(u). The
 *   paper does not print the time update; the oracle uses the second-order
 *   leapfrog
 *       u_next = 2 u - u_prev + v^2 dt^2 L u,
 *   then adds the point source  u_next[src] += v^2[src] dt^2 s(t_n),
 *   t_n = (step0 + n) dt, with the Ricker wavelet
 *       s(t) = amp (1 - 2 pi^2 f^2 (t - t0)^2) exp(-pi^2 f^2 (t - t0)^2),
 *   then records  traces[n][r] = u_next[rec_r], then rotates the fields.
 *
 *   Boundary: points outside the nx*ny*nz interior read as zero (zero
 *   Dirichlet halo of width R = 4). The paper's CPML layer (Sec. 2, Sec. 4.1)
 *   is not part of this path. A periodic mode wraps indices instead; it exists
 *   only so the tests can check dispersion and energy on Fourier modes.
 *
 * Layout: x fastest, then y, then z (Sec. 4.1 stores the grid as a flat 1D
 * array with X innermost); index (k*ny + j)*nx + i.
 *
 * Pins (tests/test_oracle_pins.py): weights from an exact rational solve,
 * polynomial exactness up to degree 9 and the predicted degree-10 error,
 * 8th-order convergence, the exact discrete dispersion relation, second
 * order in time against a manufactured standing wave, the stability limit,
 * discrete energy conservation, mirror symmetry, Ricker closed-form values,
 * and a dense-matrix brute force on tiny grids. tests/test_oracle_mutants.py
 * plants single mistakes in copies of this file and checks that the pins
 * reject each one.
 */
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_R 4

static const double ORACLE_W[ORACLE_R + 1] = {
    -205.0 / 72.0, 8.0 / 5.0, -1.0 / 5.0, 8.0 / 315.0, -1.0 / 560.0};

/* Number of OpenMP threads the parallel loops run with. */
int oracle_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void oracle_weights(double *w) {
  for (int m = 0; m <= ORACLE_R; m++) w[m] = ORACLE_W[m];
}

/* Value of u at (i,j,k); zero outside the interior unless periodic. */
static double oracle_at(const double *u, int nx, int ny, int nz, int i, int j,
                        int k, int periodic) {
  if (periodic) {
    i = ((i % nx) + nx) % nx;
    j = ((j % ny) + ny) % ny;
    k = ((k % nz) + nz) % nz;
  } else if (i < 0 || i >= nx || j < 0 || j >= ny || k < 0 || k >= nz) {
    return 0.0;
  }
  return u[((size_t)k * ny + j) * nx + i];
}

/* The Eq. 1 coefficients c_am for one axis of spacing h. */
static void oracle_axis_coeffs(double h, double *c) {
  c[0] = ORACLE_W[0] / (2.0 * h * h);
  for (int m = 1; m <= ORACLE_R; m++) c[m] = ORACLE_W[m] / (h * h);
}

/* Eq. 1 at one point. */
static double oracle_lap_point(const double *u, int nx, int ny, int nz,
                               int i, int j, int k, const double *cx,
                               const double *cy, const double *cz,
                               int periodic) {
  double s = 0.0;
  for (int m = 0; m <= ORACLE_R; m++) {
    s += cx[m] * (oracle_at(u, nx, ny, nz, i + m, j, k, periodic) +
                  oracle_at(u, nx, ny, nz, i - m, j, k, periodic));
    s += cy[m] * (oracle_at(u, nx, ny, nz, i, j + m, k, periodic) +
                  oracle_at(u, nx, ny, nz, i, j - m, k, periodic));
    s += cz[m] * (oracle_at(u, nx, ny, nz, i, j, k + m, periodic) +
                  oracle_at(u, nx, ny, nz, i, j, k - m, periodic));
  }
  return s;
}

/* out = L u over the whole interior (Eq. 1). */
void oracle_laplacian(int nx, int ny, int nz, double dx, double dy, double dz,
                      const double *u, double *out, int periodic) {
  double cx[ORACLE_R + 1], cy[ORACLE_R + 1], cz[ORACLE_R + 1];
  oracle_axis_coeffs(dx, cx);
  oracle_axis_coeffs(dy, cy);
  oracle_axis_coeffs(dz, cz);
#pragma omp parallel for schedule(static)
  for (int k = 0; k < nz; k++)
    for (int j = 0; j < ny; j++)
      for (int i = 0; i < nx; i++)
        out[((size_t)k * ny + j) * nx + i] =
            oracle_lap_point(u, nx, ny, nz, i, j, k, cx, cy, cz, periodic);
}

/* Ricker wavelet with peak frequency f, centred at t0, amplitude amp. */
double oracle_ricker(double t, double f, double t0, double amp) {
  const double pi = 3.14159265358979323846;
  double a = pi * pi * f * f * (t - t0) * (t - t0);
  return amp * (1.0 - 2.0 * a) * exp(-a);
}

/*
 * Leapfrog stability limit of the scheme (von Neumann). The Fourier symbol
 * of L is  -sum_a (1/h_a^2) (-w0 - 2 sum_m w_m cos(m theta_a));  its largest
 * magnitude is reached at theta_a = pi on every axis, where it equals
 * S * sum_a 1/h_a^2 with S = |w0| + 2 sum_m |w_m| (the weights alternate in
 * sign). The recurrence u_next = 2u - u_prev - v^2 dt^2 K u stays bounded
 * while v^2 dt^2 K <= 4, so dt_max = 2 / (vmax sqrt(S sum_a 1/h_a^2)).
 */
double oracle_cfl_dt(double dx, double dy, double dz, double vmax) {
  double s = fabs(ORACLE_W[0]);
  for (int m = 1; m <= ORACLE_R; m++) s += 2.0 * fabs(ORACLE_W[m]);
  double inv = 1.0 / (dx * dx) + 1.0 / (dy * dy) + 1.0 / (dz * dz);
  return 2.0 / (vmax * sqrt(s * inv));
}

/*
 * Advance the state (u, u_prev) by nsteps leapfrog steps.
 *
 *   vel       nx*ny*nz velocities (m/s)
 *   u, u_prev nx*ny*nz fields at steps step0 and step0-1; on return they
 *             hold steps step0+nsteps and step0+nsteps-1
 *   src       if has_source, the Ricker source at (sx,sy,sz) with peak
 *             frequency f, delay t0 and amplitude amp; if wavelet is not
 *             NULL it replaces the Ricker values: s(t_n) = wavelet[n]
 *   rec       nrec*3 int32 (x,y,z) receiver positions; traces is nsteps*nrec
 *   periodic  wrap indices instead of the zero halo (tests only)
 *
 * Returns 0, or -1 on invalid input or allocation failure.
 */
int oracle_propagate(int nx, int ny, int nz, double dx, double dy, double dz,
                     double dt, const double *vel, double *u, double *u_prev,
                     int64_t step0, int nsteps, int has_source, int sx, int sy,
                     int sz, double f, double t0, double amp,
                     const double *wavelet, const int32_t *rec, int nrec,
                     double *traces, int periodic) {
  if (nx < 1 || ny < 1 || nz < 1 || nsteps < 0 || nrec < 0) return -1;
  if (has_source && (sx < 0 || sx >= nx || sy < 0 || sy >= ny || sz < 0 || sz >= nz))
    return -1;
  for (int r = 0; r < nrec; r++)
    if (rec[3 * r] < 0 || rec[3 * r] >= nx || rec[3 * r + 1] < 0 ||
        rec[3 * r + 1] >= ny || rec[3 * r + 2] < 0 || rec[3 * r + 2] >= nz)
      return -1;
  size_t n = (size_t)nx * ny * nz;
  double *c = (double *)malloc(n * sizeof(double));
  double *unext = (double *)malloc(n * sizeof(double));
  if (!c || !unext) {
    free(c);
    free(unext);
    return -1;
  }
  for (size_t p = 0; p < n; p++) c[p] = vel[p] * vel[p] * dt * dt;
  double cx[ORACLE_R + 1], cy[ORACLE_R + 1], cz[ORACLE_R + 1];
  oracle_axis_coeffs(dx, cx);
  oracle_axis_coeffs(dy, cy);
  oracle_axis_coeffs(dz, cz);

  for (int s = 0; s < nsteps; s++) {
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; k++)
      for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
          size_t p = ((size_t)k * ny + j) * nx + i;
          double lap =
              oracle_lap_point(u, nx, ny, nz, i, j, k, cx, cy, cz, periodic);
          unext[p] = 2.0 * u[p] - u_prev[p] + c[p] * lap;
        }
    if (has_source) {
      size_t ps = ((size_t)sz * ny + sy) * nx + sx;
      double t = (double)(step0 + s) * dt;
      double w = wavelet ? wavelet[s] : oracle_ricker(t, f, t0, amp);
      unext[ps] += c[ps] * w;
    }
    for (int r = 0; r < nrec; r++) {
      size_t pr = ((size_t)rec[3 * r + 2] * ny + rec[3 * r + 1]) * nx +
                  rec[3 * r + 0];
      traces[(size_t)s * nrec + r] = unext[pr];
    }
    /* rotate: u_prev <- u, u <- u_next (copies keep the caller's buffers) */
    memcpy(u_prev, u, n * sizeof(double));
    memcpy(u, unext, n * sizeof(double));
  }
  free(c);
  free(unext);
  return 0;
}

/*
 * Gradient of a receiver misfit with respect to the squared velocity m = v^2
 * (the discrete adjoint of oracle_propagate from rest, zero halo).
 *
 * The forward recursion from u^0 = u^-1 = 0 is
 *     u^{n+1} = 2 u^n - u^{n-1} + C (L u^n) + C_s w_n e_s,   C = m dt^2,
 * the traces are d^n = R u^{n+1} (n = 0..N-1), and the caller passes
 * resid[n][r] = dJ/dd^n_r (for J = 1/2 sum |d - d_obs|^2 this is d - d_obs).
 * Setting the derivative of the Lagrangian with respect to each u^k to zero
 * gives the adjoint recursion, run backwards from q^{N+1} = q^{N+2} = 0:
 *     q^k = 2 q^{k+1} - q^{k+2} + L^T (C q^{k+1}) + R^T resid^{k-1},
 * and the derivative with respect to m_i (through C and the source term)
 *     g_i = (1/m_i) sum_{n=0}^{N-1} q^{n+1}_i (u^{n+1} - 2 u^n + u^{n-1})_i,
 * the adjoint field correlated with the forward second time difference.
 * L is symmetric with the zero halo (Eq. 1 is a symmetric star), so L^T = L.
 * All forward fields are kept in memory: small grids only.
 *
 * Returns 0, or -1 on invalid input or allocation failure.
 */
int oracle_gradient(int nx, int ny, int nz, double dx, double dy, double dz,
                    double dt, const double *vel, int nsteps, int sx, int sy,
                    int sz, double f, double t0, double amp, const int32_t *rec,
                    int nrec, const double *resid, double *grad) {
  if (nx < 1 || ny < 1 || nz < 1 || nsteps < 1 || nrec < 0) return -1;
  if (sx < 0 || sx >= nx || sy < 0 || sy >= ny || sz < 0 || sz >= nz) return -1;
  for (int r = 0; r < nrec; r++)
    if (rec[3 * r] < 0 || rec[3 * r] >= nx || rec[3 * r + 1] < 0 ||
        rec[3 * r + 1] >= ny || rec[3 * r + 2] < 0 || rec[3 * r + 2] >= nz)
      return -1;
  const size_t n = (size_t)nx * ny * nz;
  /* u[k] holds u^{k-1}, k = 0..nsteps+1 */
  double *u = (double *)calloc(n * (size_t)(nsteps + 2), sizeof(double));
  double *c = (double *)malloc(n * sizeof(double));
  double *q0 = (double *)calloc(n, sizeof(double)); /* q^{k+2} */
  double *q1 = (double *)calloc(n, sizeof(double)); /* q^{k+1} */
  double *q2 = (double *)calloc(n, sizeof(double)); /* q^k */
  double *cq = (double *)malloc(n * sizeof(double));
  double *lap = (double *)malloc(n * sizeof(double));
  if (!u || !c || !q0 || !q1 || !q2 || !cq || !lap) {
    free(u); free(c); free(q0); free(q1); free(q2); free(cq); free(lap);
    return -1;
  }
  for (size_t p = 0; p < n; p++) c[p] = vel[p] * vel[p] * dt * dt;
  /* forward: u^{n+1} from u^n, u^{n-1}; keep every field */
  for (int s = 0; s < nsteps; s++) {
    const double *um = u + (size_t)s * n;       /* u^{s-1} */
    const double *uc = u + (size_t)(s + 1) * n; /* u^s */
    double *un = u + (size_t)(s + 2) * n;       /* u^{s+1} */
    oracle_laplacian(nx, ny, nz, dx, dy, dz, uc, lap, 0);
    for (size_t p = 0; p < n; p++) un[p] = 2.0 * uc[p] - um[p] + c[p] * lap[p];
    size_t ps = ((size_t)sz * ny + sy) * nx + sx;
    un[ps] += c[ps] * oracle_ricker(s * dt, f, t0, amp);
  }
  for (size_t p = 0; p < n; p++) grad[p] = 0.0;
  /* adjoint: q^k for k = N .. 1 */
  for (int k = nsteps; k >= 1; k--) {
    for (size_t p = 0; p < n; p++) cq[p] = c[p] * q1[p];
    oracle_laplacian(nx, ny, nz, dx, dy, dz, cq, lap, 0);
    for (size_t p = 0; p < n; p++) q2[p] = 2.0 * q1[p] - q0[p] + lap[p];
    for (int r = 0; r < nrec; r++) {
      size_t pr = ((size_t)rec[3 * r + 2] * ny + rec[3 * r + 1]) * nx + rec[3 * r];
      q2[pr] += resid[(size_t)(k - 1) * nrec + r];
    }
    /* term n = k - 1: q^k (u^k - 2 u^{k-1} + u^{k-2}) */
    const double *a = u + (size_t)(k + 1) * n, *b = u + (size_t)k * n,
                 *d = u + (size_t)(k - 1) * n;
    for (size_t p = 0; p < n; p++)
      grad[p] += q2[p] * (a[p] - 2.0 * b[p] + d[p]);
    double *t = q0; q0 = q1; q1 = q2; q2 = t;
  }
  for (size_t p = 0; p < n; p++) grad[p] /= vel[p] * vel[p];
  free(u); free(c); free(q0); free(q1); free(q2); free(cq); free(lap);
  return 0;
}

/*
 * Convolutional PML (CPML) around the grid, for the second-order equation.
 *
 * The paper surrounds its domain with a CPML-like layer after Komatitsch and
 * Martin (2007) (Sec. 2, Sec. 4.1) without printing its equations. This
 * restatement follows from complex-frequency-shifted coordinate stretching
 * of each axis, s_a = 1 + d_a / (alpha_a + i omega): with
 * 1/s_a = 1 + chi_a, chi_a(t) = -d_a exp(-(d_a + alpha_a) t) for t > 0,
 *     u_tt = v^2 sum_a ( d_aa u + d_a psi_a + zeta_a ),
 *     psi_a  = chi_a * d_a u,   zeta_a = chi_a * ( d_aa u + d_a psi_a ),
 * and the recursive convolution of Komatitsch and Martin (2007) gives per
 * step  psi^n = b psi^{n-1} + a (d_a u)^n  (same for zeta) with
 *     b = exp(-(d + alpha) dt),  a = d / (d + alpha) (b - 1).
 * Discretised: d_aa by the axis part of Eq. 1, d_a by the 8th-order central
 * first derivative (weights 4/5, -1/5, 4/105, -1/280), zero outside the grid.
 * Step n: psi_a^n from u^n; then zeta_a^n from u^n and psi_a^n; then
 *     u^{n+1} = 2u^n - u^{n-1} + v^2 dt^2 sum_a (D2_a u^n + D1_a psi_a^n + zeta_a^n),
 * then source and receivers as in oracle_propagate.
 * Profiles (readings, the paper gives none): layer of npml cells on every
 * face; xi = depth into the layer / npml in (0, 1] (1 at the outer cell);
 * d = d0 xi^2 with d0 = 3 vmax ln(1/R) / (2 npml h_a); alpha = pi f_cps (1 -
 * xi) inside the layer; d = alpha = 0 (b = 1, a = 0) elsewhere.
 */
static const double ORACLE_W1[ORACLE_R + 1] = {0.0, 4.0 / 5.0, -1.0 / 5.0,
                                               4.0 / 105.0, -1.0 / 280.0};

void oracle_first_weights(double *w) {
  for (int m = 0; m <= ORACLE_R; m++) w[m] = ORACLE_W1[m];
}

/* b and a of one axis of n cells (spacing h). */
void oracle_cpml_profile(int n, int npml, double h, double dt, double vmax,
                         double R, double fcps, double *b, double *a) {
  const double pi = 3.14159265358979323846;
  const double L = npml * h;
  const double d0 = (npml > 0) ? 3.0 * vmax * log(1.0 / R) / (2.0 * L) : 0.0;
  for (int i = 0; i < n; i++) {
    double xi = 0.0;
    if (i < npml) xi = (double)(npml - i) / npml;
    if (i >= n - npml) {
      double xr = (double)(i - (n - npml - 1)) / npml;
      if (xr > xi) xi = xr;
    }
    if (xi <= 0.0) {
      b[i] = 1.0;
      a[i] = 0.0;
      continue;
    }
    const double d = d0 * xi * xi;
    const double al = pi * fcps * (1.0 - xi);
    b[i] = exp(-(d + al) * dt);
    a[i] = (d + al > 0.0) ? d / (d + al) * (b[i] - 1.0) : 0.0;
  }
}

/* axis part of Eq. 1 (second derivative) and the first derivative of f at
 * (i,j,k) along axis ax (0 = x, 1 = y, 2 = z), zero outside the grid */
static double oracle_d2(const double *f, int nx, int ny, int nz, int i, int j,
                        int k, int ax, double h) {
  int di = ax == 0, dj = ax == 1, dk = ax == 2;
  double s = ORACLE_W[0] * oracle_at(f, nx, ny, nz, i, j, k, 0);
  for (int m = 1; m <= ORACLE_R; m++)
    s += ORACLE_W[m] * (oracle_at(f, nx, ny, nz, i + m * di, j + m * dj, k + m * dk, 0) +
                        oracle_at(f, nx, ny, nz, i - m * di, j - m * dj, k - m * dk, 0));
  return s / (h * h);
}

static double oracle_d1(const double *f, int nx, int ny, int nz, int i, int j,
                        int k, int ax, double h) {
  int di = ax == 0, dj = ax == 1, dk = ax == 2;
  double s = 0.0;
  for (int m = 1; m <= ORACLE_R; m++)
    s += ORACLE_W1[m] * (oracle_at(f, nx, ny, nz, i + m * di, j + m * dj, k + m * dk, 0) -
                         oracle_at(f, nx, ny, nz, i - m * di, j - m * dj, k - m * dk, 0));
  return s / h;
}

/*
 * oracle_propagate with the CPML above (zero halo beyond it). psi and zeta
 * are 3 arrays each of nx*ny*nz (axis x, y, z), in/out, zero to start.
 * vmax sets d0 (pass the model's largest velocity).
 */
int oracle_propagate_cpml(int nx, int ny, int nz, double dx, double dy,
                          double dz, double dt, const double *vel, double *u,
                          double *u_prev, double *psi, double *zeta,
                          int64_t step0, int nsteps, int npml, double R,
                          double fcps, double vmax, int has_source, int sx,
                          int sy, int sz, double f, double t0, double amp,
                          const int32_t *rec, int nrec, double *traces) {
  if (nx < 1 || ny < 1 || nz < 1 || nsteps < 0 || nrec < 0 || npml < 0 ||
      !(R > 0.0 && R <= 1.0))
    return -1;
  if (has_source && (sx < 0 || sx >= nx || sy < 0 || sy >= ny || sz < 0 || sz >= nz))
    return -1;
  for (int r = 0; r < nrec; r++)
    if (rec[3 * r] < 0 || rec[3 * r] >= nx || rec[3 * r + 1] < 0 ||
        rec[3 * r + 1] >= ny || rec[3 * r + 2] < 0 || rec[3 * r + 2] >= nz)
      return -1;
  const size_t n = (size_t)nx * ny * nz;
  const int dims[3] = {nx, ny, nz};
  const double hs[3] = {dx, dy, dz};
  double *b[3], *a[3];
  double *c = (double *)malloc(n * sizeof(double));
  double *unext = (double *)malloc(n * sizeof(double));
  int ok = c && unext;
  for (int ax = 0; ax < 3; ax++) {
    b[ax] = (double *)malloc(dims[ax] * sizeof(double));
    a[ax] = (double *)malloc(dims[ax] * sizeof(double));
    ok = ok && b[ax] && a[ax];
  }
  if (!ok) {
    free(c); free(unext);
    for (int ax = 0; ax < 3; ax++) { free(b[ax]); free(a[ax]); }
    return -1;
  }
  for (int ax = 0; ax < 3; ax++)
    oracle_cpml_profile(dims[ax], npml, hs[ax], dt, vmax, R, fcps, b[ax], a[ax]);
  for (size_t p = 0; p < n; p++) c[p] = vel[p] * vel[p] * dt * dt;
  for (int s = 0; s < nsteps; s++) {
    /* psi_a^n from u^n */
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; k++)
      for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
          const size_t p = ((size_t)k * ny + j) * nx + i;
          const int idx[3] = {i, j, k};
          for (int ax = 0; ax < 3; ax++)
            psi[ax * n + p] = b[ax][idx[ax]] * psi[ax * n + p] +
                              a[ax][idx[ax]] *
                                  oracle_d1(u, nx, ny, nz, i, j, k, ax, hs[ax]);
        }
    /* zeta_a^n and u^{n+1} */
#pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; k++)
      for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) {
          const size_t p = ((size_t)k * ny + j) * nx + i;
          const int idx[3] = {i, j, k};
          double sum = 0.0;
          for (int ax = 0; ax < 3; ax++) {
            const double d2 = oracle_d2(u, nx, ny, nz, i, j, k, ax, hs[ax]);
            const double d1p =
                oracle_d1(psi + ax * n, nx, ny, nz, i, j, k, ax, hs[ax]);
            zeta[ax * n + p] = b[ax][idx[ax]] * zeta[ax * n + p] +
                               a[ax][idx[ax]] * (d2 + d1p);
            sum += d2 + d1p + zeta[ax * n + p];
          }
          unext[p] = 2.0 * u[p] - u_prev[p] + c[p] * sum;
        }
    if (has_source) {
      size_t ps = ((size_t)sz * ny + sy) * nx + sx;
      unext[ps] += c[ps] * oracle_ricker((double)(step0 + s) * dt, f, t0, amp);
    }
    for (int r = 0; r < nrec; r++) {
      size_t pr = ((size_t)rec[3 * r + 2] * ny + rec[3 * r + 1]) * nx + rec[3 * r];
      traces[(size_t)s * nrec + r] = unext[pr];
    }
    memcpy(u_prev, u, n * sizeof(double));
    memcpy(u, unext, n * sizeof(double));
  }
  free(c); free(unext);
  for (int ax = 0; ax < 3; ax++) { free(b[ax]); free(a[ax]); }
  return 0;
}

/*
 * Discrete adjoint gradient dJ/dm (m = v^2) of oracle_propagate_cpml from
 * rest, the layer held fixed (its profile uses the given vmax, not the
 * model, so b and a do not depend on m).
 *
 * Forward, step n = 0 .. N-1 (psi^-1 = zeta^-1 = 0, u^0 = u^-1 = 0):
 *     psi_a^n  = B_a psi_a^{n-1}  + A_a D1_a u^n
 *     zeta_a^n = B_a zeta_a^{n-1} + A_a (D2_a u^n + D1_a psi_a^n)
 *     u^{n+1}  = 2u^n - u^{n-1} + C sum_a (D2_a u^n + D1_a psi_a^n + zeta_a^n)
 *                + C s_n e_src,     d^n = R u^{n+1},   C = m dt^2
 * (B_a, A_a the diagonal per-axis b and a). With multipliers q^{n+1} for the
 * u equation, mu_a^n for psi and nu_a^n for zeta, setting the derivative of
 * the Lagrangian J - sum (multiplier . residual) with respect to every state
 * to zero gives, for k = N .. 1 (q^{N+1} = q^{N+2} = 0, mu^N = nu^N = 0):
 *     nu_a^k = C q^{k+1} + B_a nu_a^{k+1}
 *     mu_a^k = D1_a^T (C q^{k+1} + A_a nu_a^k) + B_a mu_a^{k+1}
 *     q^k    = 2q^{k+1} - q^{k+2}
 *              + sum_a [D2_a^T (C q^{k+1} + A_a nu_a^k) + D1_a^T A_a mu_a^k]
 *              + R^T r^{k-1},        r^n = dJ/dd^n,
 * and dJ/dm = (1/m) sum_n q^{n+1} (u^{n+1} - 2u^n + u^{n-1}) as without the
 * layer. With the zero halo D2_a is symmetric and D1_a antisymmetric, so
 * D2_a^T = D2_a and D1_a^T = -D1_a. Every forward field is kept.
 */
int oracle_gradient_cpml(int nx, int ny, int nz, double dx, double dy,
                         double dz, double dt, const double *vel, int nsteps,
                         int npml, double R, double fcps, double vmax, int sx,
                         int sy, int sz, double f, double t0, double amp,
                         const int32_t *rec, int nrec, const double *resid,
                         double *grad) {
  if (nx < 1 || ny < 1 || nz < 1 || nsteps < 1 || nrec < 0 || npml < 0 ||
      !(R > 0.0 && R <= 1.0))
    return -1;
  if (sx < 0 || sx >= nx || sy < 0 || sy >= ny || sz < 0 || sz >= nz) return -1;
  for (int r = 0; r < nrec; r++)
    if (rec[3 * r] < 0 || rec[3 * r] >= nx || rec[3 * r + 1] < 0 ||
        rec[3 * r + 1] >= ny || rec[3 * r + 2] < 0 || rec[3 * r + 2] >= nz)
      return -1;
  const size_t n = (size_t)nx * ny * nz;
  const int dims[3] = {nx, ny, nz};
  const double hs[3] = {dx, dy, dz};
  /* u[k] holds u^{k-1}, k = 0..nsteps+1 */
  double *u = (double *)calloc(n * (size_t)(nsteps + 2), sizeof(double));
  double *c = (double *)malloc(n * sizeof(double));
  double *psi = (double *)calloc(3 * n, sizeof(double));
  double *zeta = (double *)calloc(3 * n, sizeof(double));
  double *mu = (double *)calloc(3 * n, sizeof(double));
  double *nu = (double *)calloc(3 * n, sizeof(double));
  double *q0 = (double *)calloc(n, sizeof(double)); /* q^{k+2} */
  double *q1 = (double *)calloc(n, sizeof(double)); /* q^{k+1} */
  double *q2 = (double *)calloc(n, sizeof(double)); /* q^k */
  double *g = (double *)malloc(3 * n * sizeof(double)); /* C q + A nu, per axis */
  double *am = (double *)malloc(3 * n * sizeof(double)); /* A mu, per axis */
  double *b[3], *a[3];
  int ok = u && c && psi && zeta && mu && nu && q0 && q1 && q2 && g && am;
  for (int ax = 0; ax < 3; ax++) {
    b[ax] = (double *)malloc(dims[ax] * sizeof(double));
    a[ax] = (double *)malloc(dims[ax] * sizeof(double));
    ok = ok && b[ax] && a[ax];
  }
  if (ok) {
    for (int ax = 0; ax < 3; ax++)
      oracle_cpml_profile(dims[ax], npml, hs[ax], dt, vmax, R, fcps, b[ax], a[ax]);
    for (size_t p = 0; p < n; p++) c[p] = vel[p] * vel[p] * dt * dt;
    /* forward, keeping every u */
    for (int s = 0; s < nsteps; s++) {
      const double *um = u + (size_t)s * n, *uc = u + (size_t)(s + 1) * n;
      double *un = u + (size_t)(s + 2) * n;
#pragma omp parallel for schedule(static)
      for (int k = 0; k < nz; k++)
        for (int j = 0; j < ny; j++)
          for (int i = 0; i < nx; i++) {
            const size_t p = ((size_t)k * ny + j) * nx + i;
            const int idx[3] = {i, j, k};
            for (int ax = 0; ax < 3; ax++)
              psi[ax * n + p] = b[ax][idx[ax]] * psi[ax * n + p] +
                                a[ax][idx[ax]] * oracle_d1(uc, nx, ny, nz, i, j, k, ax, hs[ax]);
          }
#pragma omp parallel for schedule(static)
      for (int k = 0; k < nz; k++)
        for (int j = 0; j < ny; j++)
          for (int i = 0; i < nx; i++) {
            const size_t p = ((size_t)k * ny + j) * nx + i;
            const int idx[3] = {i, j, k};
            double sum = 0.0;
            for (int ax = 0; ax < 3; ax++) {
              const double d2 = oracle_d2(uc, nx, ny, nz, i, j, k, ax, hs[ax]);
              const double d1p = oracle_d1(psi + ax * n, nx, ny, nz, i, j, k, ax, hs[ax]);
              zeta[ax * n + p] = b[ax][idx[ax]] * zeta[ax * n + p] +
                                 a[ax][idx[ax]] * (d2 + d1p);
              sum += d2 + d1p + zeta[ax * n + p];
            }
            un[p] = 2.0 * uc[p] - um[p] + c[p] * sum;
          }
      const size_t ps = ((size_t)sz * ny + sy) * nx + sx;
      un[ps] += c[ps] * oracle_ricker(s * dt, f, t0, amp);
    }
    for (size_t p = 0; p < n; p++) grad[p] = 0.0;
    /* adjoint, k = N .. 1 */
    for (int kk = nsteps; kk >= 1; kk--) {
      const int last = kk == nsteps; /* mu^N = nu^N = 0 */
#pragma omp parallel for schedule(static)
      for (int k = 0; k < nz; k++)
        for (int j = 0; j < ny; j++)
          for (int i = 0; i < nx; i++) {
            const size_t p = ((size_t)k * ny + j) * nx + i;
            const int idx[3] = {i, j, k};
            const double cq = c[p] * q1[p];
            for (int ax = 0; ax < 3; ax++) {
              if (!last) nu[ax * n + p] = cq + b[ax][idx[ax]] * nu[ax * n + p];
              g[ax * n + p] = cq + a[ax][idx[ax]] * nu[ax * n + p];
            }
          }
      if (!last) {
#pragma omp parallel for schedule(static)
        for (int k = 0; k < nz; k++)
          for (int j = 0; j < ny; j++)
            for (int i = 0; i < nx; i++) {
              const size_t p = ((size_t)k * ny + j) * nx + i;
              const int idx[3] = {i, j, k};
              for (int ax = 0; ax < 3; ax++)
                mu[ax * n + p] = -oracle_d1(g + ax * n, nx, ny, nz, i, j, k, ax, hs[ax]) +
                                 b[ax][idx[ax]] * mu[ax * n + p];
            }
      }
#pragma omp parallel for schedule(static)
      for (int k = 0; k < nz; k++)
        for (int j = 0; j < ny; j++)
          for (int i = 0; i < nx; i++) {
            const size_t p = ((size_t)k * ny + j) * nx + i;
            const int idx[3] = {i, j, k};
            for (int ax = 0; ax < 3; ax++)
              am[ax * n + p] = a[ax][idx[ax]] * mu[ax * n + p];
          }
#pragma omp parallel for schedule(static)
      for (int k = 0; k < nz; k++)
        for (int j = 0; j < ny; j++)
          for (int i = 0; i < nx; i++) {
            const size_t p = ((size_t)k * ny + j) * nx + i;
            double sum = 0.0;
            for (int ax = 0; ax < 3; ax++)
              sum += oracle_d2(g + ax * n, nx, ny, nz, i, j, k, ax, hs[ax]) -
                     oracle_d1(am + ax * n, nx, ny, nz, i, j, k, ax, hs[ax]);
            q2[p] = 2.0 * q1[p] - q0[p] + sum;
          }
      for (int r = 0; r < nrec; r++) {
        const size_t pr = ((size_t)rec[3 * r + 2] * ny + rec[3 * r + 1]) * nx + rec[3 * r];
        q2[pr] += resid[(size_t)(kk - 1) * nrec + r];
      }
      /* term n = kk - 1: q^kk (u^kk - 2 u^{kk-1} + u^{kk-2}) */
      const double *ua = u + (size_t)(kk + 1) * n, *ub = u + (size_t)kk * n,
                   *ud = u + (size_t)(kk - 1) * n;
      for (size_t p = 0; p < n; p++) grad[p] += q2[p] * (ua[p] - 2.0 * ub[p] + ud[p]);
      double *t = q0; q0 = q1; q1 = q2; q2 = t;
    }
    for (size_t p = 0; p < n; p++) grad[p] /= vel[p] * vel[p];
  }
  free(u); free(c); free(psi); free(zeta); free(mu); free(nu);
  free(q0); free(q1); free(q2); free(g); free(am);
  for (int ax = 0; ax < 3; ax++) { free(b[ax]); free(a[ax]); }
  return ok ? 0 : -1;
}
