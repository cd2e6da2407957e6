/*
 * FP64 CPU oracle for periodic tricubic B-spline particle interpolation.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * statement of what the GPU library computes.  Only the test suite, the smoke
 * check and the CPU-baseline leg of the benchmark load it.  It shares no code,
 * header, table or constant with the CUDA library, and the CUDA library never
 * calls it.
 *
 * Every function follows the definitions of Buaria & Yeung (arXiv 2005.13193):
 *   - Sec. 2.2, Eq. (spline): g+ = sum_{i,j,k=1..4} b_i(x') c_j(y') d_k(z') S_pqr,
 *     p = alpha+i-2, q = beta+j-2, r = gamma+k-2, x' = (x+ - x_alpha)/dx.
 *   - Sec. 2.2: along each grid line of N points, N+3 coefficients from a
 *     tridiagonal system with periodicity in space (Ahlberg), solved by the
 *     Thomas algorithm (Sec. 2.2, Table 1 discussion), directions x, z, y.
 *   - Sec. 2.2: positions outside [0, L0) use their periodic "shadow" image.
 *   - Sec. 2.1 / Sec. 4.3: second-order Runge-Kutta particle advance.
 *
 * Readings where the paper is silent (the 1D basis is only referenced):
 *   - basis = uniform cubic B-spline, b(t) = [(1-t)^3, 3t^3-6t^2+4,
 *     -3t^3+3t^2+3t+1, t^3]/6, which is the only basis consistent with the
 *     1/6, 4/6, 1/6 interpolation system and the N+3 storage;
 *   - 0-based padded storage P = a + i (i = 0..3 for the four basis functions,
 *     a = cell index in [0, N)); padded P holds node (P-1) mod N, i.e. one
 *     ghost below and two above, matching the three-deep halo of Sec. 3;
 *   - the solve has N unknowns per line (periodic); N+3 is storage only;
 *   - RK2 is Heun's predictor-corrector; positions stay unwrapped.
 *
 * Compiled with -ffp-contract=off so that every multiply and add rounds as
 * written; cell indices are then bit-identical to any other IEEE-754
 * evaluation of the same expressions.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORA_OK 0
#define ORA_ERR_ARG 1
#define ORA_ERR_NONFINITE 2
#define ORA_ERR_NOMEM 3

/* |x * N/L| >= 2^50 is rejected (an implementation limit the paper does not
 * set): the cell index and the fraction are then exact in FP64 arithmetic. */
#define ORA_MAX_ABS_S 1125899906842624.0

int ora_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void ora_set_num_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

/* ------------------------------------------------------------------------ */
/* Cyclic tridiagonal solve (Sec. 2.2: tridiagonal system with periodicity,  */
/* Thomas algorithm).  Solves (1/6) c[j-1] + (4/6) c[j] + (1/6) c[j+1] = g[j] */
/* for j = 0..n-1, indices mod n.                                            */
/*                                                                          */
/* The periodic matrix A is the tridiagonal T plus the two corner entries.  */
/* Write A = T' + u v^T with u = (gam, 0, .., 0, alpha)^T and               */
/* v = (1, 0, .., 0, beta/gam)^T, where alpha = A[n-1][0] and               */
/* beta = A[0][n-1]; T' is T with its first diagonal entry reduced by gam   */
/* and its last by alpha*beta/gam.  Sherman-Morrison then gives             */
/* A^-1 g = y - (v.y / (1 + v.z)) z  with  T' y = g,  T' z = u.             */
/* Both tridiagonal solves use the Thomas algorithm.  Requires n >= 3.      */
/* ------------------------------------------------------------------------ */

/* Thomas algorithm for constant off-diagonals `off` and diagonal d[0..n-1]. */
static void thomas(int n, double off, const double* d, const double* r,
                   double* x, double* cp, double* dp) {
  cp[0] = off / d[0];
  dp[0] = r[0] / d[0];
  for (int i = 1; i < n; ++i) {
    double m = d[i] - off * cp[i - 1];
    cp[i] = off / m;
    dp[i] = (r[i] - off * dp[i - 1]) / m;
  }
  x[n - 1] = dp[n - 1];
  for (int i = n - 2; i >= 0; --i) x[i] = dp[i] - cp[i] * x[i + 1];
}

/* work must hold 6*n doubles. */
static int cyclic_solve_line(int n, const double* g, double* c, double* work) {
  if (n < 3) return ORA_ERR_ARG;
  const double off = 1.0 / 6.0, diag = 4.0 / 6.0;
  const double alpha = off, beta = off;
  const double gam = -diag;
  double* d = work;
  double* y = work + n;
  double* z = work + 2 * n;
  double* u = work + 3 * n;
  double* cp = work + 4 * n;
  double* dp = work + 5 * n;
  for (int i = 0; i < n; ++i) { d[i] = diag; u[i] = 0.0; }
  d[0] = diag - gam;
  d[n - 1] = diag - alpha * beta / gam;
  u[0] = gam;
  u[n - 1] = alpha;
  thomas(n, off, d, g, y, cp, dp);
  thomas(n, off, d, u, z, cp, dp);
  double vy = y[0] + (beta / gam) * y[n - 1];
  double vz = z[0] + (beta / gam) * z[n - 1];
  double f = vy / (1.0 + vz);
  for (int i = 0; i < n; ++i) c[i] = y[i] - f * z[i];
  return ORA_OK;
}

int ora_cyclic_solve(int n, const double* g, double* c) {
  if (n < 3) return ORA_ERR_ARG;
  double* work = (double*)malloc(sizeof(double) * 6 * (size_t)n);
  if (!work) return ORA_ERR_NOMEM;
  int rc = cyclic_solve_line(n, g, c, work);
  free(work);
  return rc;
}

/* Solve every line of a[nz][ny][nx] along one axis (0 = x, 1 = y, 2 = z). */
static int solve_axis(const int32_t n[3], double* a, int axis) {
  const int64_t nx = n[0], ny = n[1], nz = n[2];
  const int64_t len = n[axis];
  const int64_t stride = axis == 0 ? 1 : (axis == 1 ? nx : nx * ny);
  const int64_t nlines = nx * ny * nz / len;
  int err = ORA_OK;
#pragma omp parallel
  {
    double* buf = (double*)malloc(sizeof(double) * 8 * (size_t)len);
    if (!buf) {
#pragma omp atomic write
      err = ORA_ERR_NOMEM;
    } else {
      double* g = buf + 6 * len;
      double* c = buf + 7 * len;
#pragma omp for schedule(static)
      for (int64_t l = 0; l < nlines; ++l) {
        /* base index of line l: enumerate the two other axes */
        int64_t base;
        if (axis == 0) {
          base = l * nx;
        } else if (axis == 1) {
          int64_t x = l % nx, z = l / nx;
          base = z * nx * ny + x;
        } else {
          base = l; /* l = y*nx + x */
        }
        for (int64_t i = 0; i < len; ++i) g[i] = a[base + i * stride];
        cyclic_solve_line((int)len, g, c, buf);
        for (int64_t i = 0; i < len; ++i) a[base + i * stride] = c[i];
      }
      free(buf);
    }
  }
  return err;
}

/* Periodic padding: padded index P in [0, n+2] holds node (P-1) mod n. */
static int64_t pad_source(int64_t P, int64_t n) {
  int64_t m = (P - 1) % n;
  return m < 0 ? m + n : m;
}

/*
 * Spline coefficients (Sec. 2.2, "Operation 1"): for each component solve
 * along x, then z, then y (the paper's order), then store the N+3 padded
 * coefficients per axis.
 *   field: [ncomp][nz][ny][nx]          (x fastest)
 *   coef : [ncomp][nz+3][ny+3][nx+3]
 */
int ora_spline_coeffs(const int32_t n[3], int ncomp, const double* field,
                      double* coef) {
  if (n[0] < 3 || n[1] < 3 || n[2] < 3 || ncomp < 1) return ORA_ERR_ARG;
  const int64_t nx = n[0], ny = n[1], nz = n[2];
  const int64_t mx = nx + 3, my = ny + 3, mz = nz + 3;
  const int64_t vol = nx * ny * nz;
  double* a = (double*)malloc(sizeof(double) * (size_t)vol);
  if (!a) return ORA_ERR_NOMEM;
  for (int c = 0; c < ncomp; ++c) {
    memcpy(a, field + (int64_t)c * vol, sizeof(double) * (size_t)vol);
    int rc = solve_axis(n, a, 0);
    if (!rc) rc = solve_axis(n, a, 2);
    if (!rc) rc = solve_axis(n, a, 1);
    if (rc) { free(a); return rc; }
    double* out = coef + (int64_t)c * mx * my * mz;
#pragma omp parallel for schedule(static)
    for (int64_t Pz = 0; Pz < mz; ++Pz)
      for (int64_t Py = 0; Py < my; ++Py)
        for (int64_t Px = 0; Px < mx; ++Px) {
          int64_t z = pad_source(Pz, nz), y = pad_source(Py, ny),
                  x = pad_source(Px, nx);
          out[(Pz * my + Py) * mx + Px] = a[(z * ny + y) * nx + x];
        }
  }
  free(a);
  return ORA_OK;
}

/* ------------------------------------------------------------------------ */
/* Operation 2: cell index, local coordinate and basis (Sec. 2.2).          */
/* ------------------------------------------------------------------------ */

/* Cell a = floor(x * N/L) mod N (periodic shadow), t = x*N/L - floor(x*N/L). */
static int locate(double x, double inv_h, int64_t n, int64_t* cell, double* t) {
  if (!isfinite(x)) return ORA_ERR_NONFINITE;
  double s = x * inv_h;
  if (!(fabs(s) < ORA_MAX_ABS_S)) return ORA_ERR_NONFINITE;
  double a = floor(s);
  *t = s - a;
  int64_t m = ((int64_t)a) % n;
  if (m < 0) m += n;
  *cell = m;
  return ORA_OK;
}

/* Uniform cubic B-spline basis on the four nodes a-1, a, a+1, a+2. */
static void basis(double t, double b[4]) {
  double s = 1.0 - t;
  b[0] = s * s * s / 6.0;
  b[1] = (3.0 * t * t * t - 6.0 * t * t + 4.0) / 6.0;
  b[2] = (-3.0 * t * t * t + 3.0 * t * t + 3.0 * t + 1.0) / 6.0;
  b[3] = t * t * t / 6.0;
}

/* d b / d t. */
static void dbasis(double t, double d[4]) {
  double s = 1.0 - t;
  d[0] = -3.0 * s * s / 6.0;
  d[1] = (9.0 * t * t - 12.0 * t) / 6.0;
  d[2] = (-9.0 * t * t + 6.0 * t + 3.0) / 6.0;
  d[3] = 3.0 * t * t / 6.0;
}

/* Exposed for tests: basis values and derivatives at t. */
void ora_basis(double t, double* b, double* db) {
  basis(t, b);
  dbasis(t, db);
}

/* Exposed for tests: cell index and local coordinate of one coordinate. */
int ora_locate(double x, double L, int n, int64_t* cell, double* t) {
  double inv_h = (double)n / L;
  return locate(x, inv_h, n, cell, t);
}

/*
 * Operation 3 (Sec. 2.2, Eq. (spline)): 64-term sum per component, and the
 * spatial derivatives from the same stencil with b'(t)/h.
 *   coef: [ncomp][nz+3][ny+3][nx+3]; pos: [3][np]; vel: [ncomp][np];
 *   grad (optional): [ncomp][3][np], grad[c][d] = d u_c / d x_d.
 * Returns ORA_ERR_NONFINITE (and writes NaN) for a non-finite position.
 */
static int interp_one(const int32_t n[3], const double inv_h[3], int ncomp,
                      const double* coef, const double x[3], double* u,
                      double (*du)[3]) {
  int64_t cell[3];
  double t[3], b[3][4], db[3][4];
  for (int d = 0; d < 3; ++d) {
    int rc = locate(x[d], inv_h[d], n[d], &cell[d], &t[d]);
    if (rc) return rc;
    basis(t[d], b[d]);
    dbasis(t[d], db[d]);
  }
  const int64_t mx = n[0] + 3, my = n[1] + 3, mz = n[2] + 3;
  for (int c = 0; c < ncomp; ++c) {
    const double* C = coef + (int64_t)c * mx * my * mz;
    double acc = 0.0, gx = 0.0, gy = 0.0, gz = 0.0;
    for (int k = 0; k < 4; ++k)
      for (int j = 0; j < 4; ++j)
        for (int i = 0; i < 4; ++i) {
          double s = C[((cell[2] + k) * my + cell[1] + j) * mx + cell[0] + i];
          acc += b[0][i] * b[1][j] * b[2][k] * s;
          gx += db[0][i] * b[1][j] * b[2][k] * s;
          gy += b[0][i] * db[1][j] * b[2][k] * s;
          gz += b[0][i] * b[1][j] * db[2][k] * s;
        }
    u[c] = acc;
    if (du) {
      du[c][0] = gx * inv_h[0];
      du[c][1] = gy * inv_h[1];
      du[c][2] = gz * inv_h[2];
    }
  }
  return ORA_OK;
}

static void inv_spacing(const int32_t n[3], const double L[3], double inv_h[3]) {
  for (int d = 0; d < 3; ++d) inv_h[d] = (double)n[d] / L[d];
}

int ora_interp(const int32_t n[3], const double L[3], int ncomp,
               const double* coef, int64_t np, const double* pos, double* vel,
               double* grad) {
  if (ncomp < 1 || ncomp > 8) return ORA_ERR_ARG;
  double inv_h[3];
  inv_spacing(n, L, inv_h);
  int err = ORA_OK;
#pragma omp parallel for schedule(static)
  for (int64_t p = 0; p < np; ++p) {
    double x[3] = {pos[p], pos[np + p], pos[2 * np + p]};
    double u[8], du[8][3];
    int rc = interp_one(n, inv_h, ncomp, coef, x, u, grad ? du : NULL);
    if (rc) {
#pragma omp atomic write
      err = rc;
      for (int c = 0; c < ncomp; ++c) u[c] = NAN;
      for (int c = 0; c < ncomp; ++c)
        for (int d = 0; d < 3; ++d) du[c][d] = NAN;
    }
    for (int c = 0; c < ncomp; ++c) vel[(int64_t)c * np + p] = u[c];
    if (grad)
      for (int c = 0; c < ncomp; ++c)
        for (int d = 0; d < 3; ++d)
          grad[((int64_t)c * 3 + d) * np + p] = du[c][d];
  }
  return err;
}

/* ------------------------------------------------------------------------ */
/* Second derivatives of the interpolant (the spline is twice continuously  */
/* differentiable, Sec. 2.2): d2 b_i / dt2 = (1-t), 3t-2, 1-3t, t for       */
/* i = 0..3, and each derivative along axis d brings a factor n_d/L_d.      */
/*   hess: [ncomp][6][np] in the order xx, yy, zz, xy, xz, yz.              */
/* ------------------------------------------------------------------------ */
static void ddbasis(double t, double d2[4]) {
  d2[0] = 1.0 - t;
  d2[1] = 3.0 * t - 2.0;
  d2[2] = 1.0 - 3.0 * t;
  d2[3] = t;
}

int ora_interp_hessian(const int32_t n[3], const double L[3], int ncomp,
                       const double* coef, int64_t np, const double* pos, double* hess) {
  if (ncomp < 1 || ncomp > 8) return ORA_ERR_ARG;
  double inv_h[3];
  inv_spacing(n, L, inv_h);
  const int64_t mx = n[0] + 3, my = n[1] + 3, mz = n[2] + 3;
  int err = ORA_OK;
#pragma omp parallel for schedule(static)
  for (int64_t p = 0; p < np; ++p) {
    int64_t cell[3];
    double t[3], b[3][4], db[3][4], d2[3][4];
    int bad = 0;
    for (int d = 0; d < 3; ++d) {
      if (locate(pos[d * np + p], inv_h[d], n[d], &cell[d], &t[d])) bad = 1;
      basis(t[d], b[d]);
      dbasis(t[d], db[d]);
      ddbasis(t[d], d2[d]);
    }
    for (int c = 0; c < ncomp; ++c) {
      double h[6] = {0, 0, 0, 0, 0, 0};
      if (!bad) {
        const double* C = coef + (int64_t)c * mx * my * mz;
        for (int k = 0; k < 4; ++k)
          for (int j = 0; j < 4; ++j)
            for (int i = 0; i < 4; ++i) {
              const double s = C[((cell[2] + k) * my + cell[1] + j) * mx + cell[0] + i];
              h[0] += d2[0][i] * b[1][j] * b[2][k] * s;
              h[1] += b[0][i] * d2[1][j] * b[2][k] * s;
              h[2] += b[0][i] * b[1][j] * d2[2][k] * s;
              h[3] += db[0][i] * db[1][j] * b[2][k] * s;
              h[4] += db[0][i] * b[1][j] * db[2][k] * s;
              h[5] += b[0][i] * db[1][j] * db[2][k] * s;
            }
        h[0] *= inv_h[0] * inv_h[0];
        h[1] *= inv_h[1] * inv_h[1];
        h[2] *= inv_h[2] * inv_h[2];
        h[3] *= inv_h[0] * inv_h[1];
        h[4] *= inv_h[0] * inv_h[2];
        h[5] *= inv_h[1] * inv_h[2];
      }
      for (int e = 0; e < 6; ++e) hess[((int64_t)c * 6 + e) * np + p] = bad ? NAN : h[e];
    }
    if (bad) {
#pragma omp atomic write
      err = ORA_ERR_NONFINITE;
    }
  }
  return err;
}

/* Lagrangian acceleration of fluid particles (Sec. 2.1: particles move with */
/* the local fluid velocity): a = du/dt + (u . grad) u, the time derivative */
/* taken as (u(x, t+dt) - u(x, t)) / dt from two fields when coef_np1 is    */
/* given (else zero), the convective term from the field at t.  acc [3][np]. */
int ora_lagrangian_accel(const int32_t n[3], const double L[3], const double* coef_n,
                         const double* coef_np1, double dt_field, int64_t np,
                         const double* pos, double* acc) {
  double inv_h[3];
  inv_spacing(n, L, inv_h);
  int err = ORA_OK;
#pragma omp parallel for schedule(static)
  for (int64_t p = 0; p < np; ++p) {
    double x[3] = {pos[p], pos[np + p], pos[2 * np + p]};
    double u[8], du[8][3], u1[8];
    int rc = interp_one(n, inv_h, 3, coef_n, x, u, du);
    if (!rc && coef_np1) rc = interp_one(n, inv_h, 3, coef_np1, x, u1, NULL);
    for (int c = 0; c < 3; ++c) {
      double a = du[c][0] * u[0] + du[c][1] * u[1] + du[c][2] * u[2];
      if (coef_np1) a += (u1[c] - u[c]) / dt_field;
      acc[(int64_t)c * np + p] = rc ? NAN : a;
    }
    if (rc) {
#pragma omp atomic write
      err = rc;
    }
  }
  return err;
}

/* ------------------------------------------------------------------------ */
/* Binning: the single-device reading of the dynamic particle-to-process    */
/* mapping by instantaneous position (Sec. 3).  Bricks of B cells per axis, */
/* bin = (bz*nBy + by)*nBx + bx; stable counting sort.                      */
/* ------------------------------------------------------------------------ */
int ora_bin(const int32_t n[3], const double L[3], const int32_t brick[3],
            int64_t np, const double* pos, int32_t* bin_of,
            int32_t* bin_offsets, int64_t* perm) {
  int64_t nb[3];
  for (int d = 0; d < 3; ++d) {
    if (brick[d] < 1 || n[d] < 3) return ORA_ERR_ARG;
    nb[d] = (n[d] + brick[d] - 1) / brick[d];
  }
  double inv_h[3];
  inv_spacing(n, L, inv_h);
  int64_t nbins = nb[0] * nb[1] * nb[2];
  int64_t* count = (int64_t*)calloc((size_t)nbins + 1, sizeof(int64_t));
  if (!count) return ORA_ERR_NOMEM;
  int err = ORA_OK;
  for (int64_t p = 0; p < np; ++p) {
    int64_t cell[3], bb[3];
    double t;
    int bad = 0;
    for (int d = 0; d < 3; ++d) {
      if (locate(pos[d * np + p], inv_h[d], n[d], &cell[d], &t)) bad = 1;
      bb[d] = cell[d] / brick[d];
    }
    if (bad) { err = ORA_ERR_NONFINITE; bb[0] = bb[1] = bb[2] = 0; }
    int64_t bin = (bb[2] * nb[1] + bb[1]) * nb[0] + bb[0];
    bin_of[p] = (int32_t)bin;
    count[bin + 1] += 1;
  }
  for (int64_t b = 0; b < nbins; ++b) count[b + 1] += count[b];
  for (int64_t b = 0; b <= nbins; ++b) bin_offsets[b] = (int32_t)count[b];
  for (int64_t p = 0; p < np; ++p) perm[count[bin_of[p]]++] = p;
  free(count);
  return err;
}

/* ------------------------------------------------------------------------ */
/* Adjoint.  The map field -> u(x_p) is  u = W pad(S_y S_z S_x field)  with */
/* W the basis weights.  Its transpose is  S_x S_z S_y fold(W^T g)  because */
/* every per-axis matrix A is symmetric (A^T = A), and fold (adding each    */
/* padded slot into the node it copies) is the transpose of pad.            */
/*   g_vel: [ncomp][np]; g_pos: [3][np] = sum_c g_c du_c/dx_d;              */
/*   g_field: [ncomp][nz][ny][nx].                                          */
/* ------------------------------------------------------------------------ */
int ora_interp_backward(const int32_t n[3], const double L[3], int ncomp,
                        const double* coef, int64_t np, const double* pos,
                        const double* g_vel, double* g_pos, double* g_field) {
  if (ncomp < 1 || ncomp > 8) return ORA_ERR_ARG;
  double inv_h[3];
  inv_spacing(n, L, inv_h);
  const int64_t nx = n[0], ny = n[1], nz = n[2];
  const int64_t mx = nx + 3, my = ny + 3, mz = nz + 3;
  int err = ORA_OK;
  if (g_pos) {
    if (!coef) return ORA_ERR_ARG;
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < np; ++p) {
      double x[3] = {pos[p], pos[np + p], pos[2 * np + p]};
      double u[8], du[8][3];
      int rc = interp_one(n, inv_h, ncomp, coef, x, u, du);
      for (int d = 0; d < 3; ++d) {
        double s = 0.0;
        for (int c = 0; c < ncomp; ++c) s += g_vel[(int64_t)c * np + p] * du[c][d];
        g_pos[(int64_t)d * np + p] = rc ? NAN : s;
      }
      if (rc) {
#pragma omp atomic write
        err = rc;
      }
    }
  }
  if (g_field) {
    int64_t pvol = mx * my * mz, vol = nx * ny * nz;
    double* G = (double*)calloc((size_t)(ncomp * pvol), sizeof(double));
    if (!G) return ORA_ERR_NOMEM;
    /* scatter: transpose of the 64-term weighted sum */
    for (int64_t p = 0; p < np; ++p) {
      int64_t cell[3];
      double t[3], b[3][4];
      int bad = 0;
      for (int d = 0; d < 3; ++d) {
        if (locate(pos[d * np + p], inv_h[d], n[d], &cell[d], &t[d])) bad = 1;
        basis(t[d], b[d]);
      }
      if (bad) { err = ORA_ERR_NONFINITE; continue; }
      for (int c = 0; c < ncomp; ++c) {
        double gc = g_vel[(int64_t)c * np + p];
        double* Gc = G + c * pvol;
        for (int k = 0; k < 4; ++k)
          for (int j = 0; j < 4; ++j)
            for (int i = 0; i < 4; ++i)
              Gc[((cell[2] + k) * my + cell[1] + j) * mx + cell[0] + i] +=
                  b[0][i] * b[1][j] * b[2][k] * gc;
      }
    }
    /* fold: transpose of the periodic padding */
    for (int c = 0; c < ncomp; ++c) {
      double* out = g_field + c * vol;
      const double* Gc = G + c * pvol;
      memset(out, 0, sizeof(double) * (size_t)vol);
      for (int64_t Pz = 0; Pz < mz; ++Pz)
        for (int64_t Py = 0; Py < my; ++Py)
          for (int64_t Px = 0; Px < mx; ++Px) {
            int64_t z = pad_source(Pz, nz), y = pad_source(Py, ny),
                    x = pad_source(Px, nx);
            out[(z * ny + y) * nx + x] += Gc[(Pz * my + Py) * mx + Px];
          }
      /* transposed solves: the per-axis matrices are symmetric */
      int rc = solve_axis(n, out, 1);
      if (!rc) rc = solve_axis(n, out, 2);
      if (!rc) rc = solve_axis(n, out, 0);
      if (rc) { free(G); return rc; }
    }
    free(G);
  }
  return err;
}

/* ------------------------------------------------------------------------ */
/* Second-order Runge-Kutta particle advance (Sec. 2.1; Sec. 4.3), read as  */
/* Heun's method:  u1 = u(x^n, t^n);  x* = x^n + dt u1;                     */
/* u2 = u(x*, t^n+1);  x^n+1 = x^n + (dt/2)(u1 + u2).                       */
/* coef_np1 == NULL means a frozen field (coef_n used for both stages).     */
/* vel_out (optional, [3][np]) receives u1, the velocity at x^n.            */
/* ------------------------------------------------------------------------ */
int ora_rk2_step(const int32_t n[3], const double L[3], const double* coef_n,
                 const double* coef_np1, int64_t np, double* pos, double dt,
                 double* vel_out) {
  double inv_h[3];
  inv_spacing(n, L, inv_h);
  const double* cn1 = coef_np1 ? coef_np1 : coef_n;
  int err = ORA_OK;
#pragma omp parallel for schedule(static)
  for (int64_t p = 0; p < np; ++p) {
    double x[3] = {pos[p], pos[np + p], pos[2 * np + p]};
    double u1[3], u2[3], xs[3];
    int rc = interp_one(n, inv_h, 3, coef_n, x, u1, NULL);
    for (int d = 0; d < 3; ++d) xs[d] = x[d] + dt * u1[d];
    if (!rc) rc = interp_one(n, inv_h, 3, cn1, xs, u2, NULL);
    if (rc) {
#pragma omp atomic write
      err = rc;
      for (int d = 0; d < 3; ++d) { u1[d] = NAN; u2[d] = NAN; }
    }
    for (int d = 0; d < 3; ++d) {
      pos[(int64_t)d * np + p] = x[d] + (dt / 2.0) * (u1[d] + u2[d]);
      if (vel_out) vel_out[(int64_t)d * np + p] = u1[d];
    }
  }
  return err;
}

/* ------------------------------------------------------------------------ */
/* Windowed coefficients for grids too large for host memory.               */
/* The inverse of the periodic 1/6,4/6,1/6 matrix is the circulant with     */
/* entries G_N(d) = sqrt(3) (r^d + r^(N-d)) / (1 - r^N), r = sqrt(3) - 2,   */
/* 0 <= d < N.  Since |r|^25 < 5e-15, the coefficient at a node is, to FP64 */
/* rounding, the separable sum of G over |d| <= W (W = 24) of field values. */
/* ora_interp_windowed evaluates Eq. (spline) with coefficients obtained    */
/* this way from a single-precision field [3][nz][ny][nx].                  */
/* ------------------------------------------------------------------------ */
#define ORA_WIN 24

static double green(int64_t d, int64_t n) {
  const double r = sqrt(3.0) - 2.0;
  int64_t m = d % n;
  if (m < 0) m += n;
  return sqrt(3.0) * (pow(r, (double)m) + pow(r, (double)(n - m))) /
         (1.0 - pow(r, (double)n));
}

void ora_green(int64_t n, int64_t d, double* out) { *out = green(d, n); }

/* ------------------------------------------------------------------------ */
/* Truncated-inverse coefficients: the periodic solve of Sec. 2.2 written as */
/* the convolution with the inverse's entries G_N (above), kept for |d| <= K */
/* only:  c_j = sum_{d=-K..K} G_N(d) g_{(j+d) mod N}  along x, then y, then  */
/* z, then the same N+3 padding as ora_spline_coeffs.  With 2K + 1 = N (N    */
/* odd) every residue appears once and the result is the exact solve's.     */
/* Requires 1 <= K and 2K + 1 <= N on every axis.                           */
/* ------------------------------------------------------------------------ */
static void fir_axis(const int64_t n[3], int axis, int K, const double* in, double* out) {
  const int64_t N = n[axis];
  const int64_t stride = axis == 0 ? 1 : (axis == 1 ? n[0] : n[0] * n[1]);
  const int64_t vol = n[0] * n[1] * n[2];
  double* g = (double*)malloc(sizeof(double) * (size_t)(2 * K + 1));
  for (int d = -K; d <= K; ++d) g[d + K] = green(d, N);
#pragma omp parallel for schedule(static)
  for (int64_t idx = 0; idx < vol; ++idx) {
    const int64_t j = (idx / stride) % N;
    const int64_t base = idx - j * stride;
    double acc = 0.0;
    for (int d = -K; d <= K; ++d) {
      int64_t m = (j + d) % N;
      if (m < 0) m += N;
      acc += g[d + K] * in[base + m * stride];
    }
    out[idx] = acc;
  }
  free(g);
}

int ora_spline_coeffs_truncated(const int32_t n[3], int ncomp, int K, const double* field,
                                double* coef) {
  if (ncomp < 1 || K < 1) return ORA_ERR_ARG;
  for (int d = 0; d < 3; ++d)
    if (n[d] < 3 || 2 * K + 1 > n[d]) return ORA_ERR_ARG;
  const int64_t nn[3] = {n[0], n[1], n[2]};
  const int64_t nx = n[0], ny = n[1], nz = n[2];
  const int64_t mx = nx + 3, my = ny + 3, mz = nz + 3;
  const int64_t vol = nx * ny * nz;
  double* a = (double*)malloc(sizeof(double) * (size_t)vol);
  double* b = (double*)malloc(sizeof(double) * (size_t)vol);
  if (!a || !b) { free(a); free(b); return ORA_ERR_NOMEM; }
  for (int c = 0; c < ncomp; ++c) {
    fir_axis(nn, 0, K, field + (int64_t)c * vol, a);
    fir_axis(nn, 1, K, a, b);
    fir_axis(nn, 2, K, b, a);
    double* out = coef + (int64_t)c * mx * my * mz;
#pragma omp parallel for schedule(static)
    for (int64_t Pz = 0; Pz < mz; ++Pz)
      for (int64_t Py = 0; Py < my; ++Py)
        for (int64_t Px = 0; Px < mx; ++Px) {
          int64_t z = pad_source(Pz, nz), y = pad_source(Py, ny),
                  x = pad_source(Px, nx);
          out[(Pz * my + Py) * mx + Px] = a[(z * ny + y) * nx + x];
        }
  }
  free(a);
  free(b);
  return ORA_OK;
}

int ora_interp_windowed(const int32_t n[3], const double L[3],
                        const float* field, int64_t np, const double* pos,
                        double* vel) {
  for (int d = 0; d < 3; ++d)
    if (n[d] < 2 * ORA_WIN + 2) return ORA_ERR_ARG;
  double inv_h[3];
  inv_spacing(n, L, inv_h);
  const int64_t nx = n[0], ny = n[1], nz = n[2];
  const int64_t vol = nx * ny * nz;
  enum { W = ORA_WIN, S = 2 * ORA_WIN + 1 };
  double gw[3][S];
  for (int d = 0; d < 3; ++d)
    for (int e = -W; e <= W; ++e) gw[d][e + W] = green(e, n[d]);
  int err = ORA_OK;
#pragma omp parallel
  {
    /* rows[z][y][i]: x-filtered field for the 4 needed x nodes */
    double* rows = (double*)malloc(sizeof(double) * (S + 3) * (S + 3) * 4);
    double* cols = (double*)malloc(sizeof(double) * (S + 3) * 4 * 4);
#pragma omp for schedule(dynamic, 16)
    for (int64_t p = 0; p < np; ++p) {
      int64_t cell[3];
      double t[3], b[3][4];
      int bad = 0;
      for (int d = 0; d < 3; ++d) {
        if (locate(pos[d * np + p], inv_h[d], n[d], &cell[d], &t[d])) bad = 1;
        basis(t[d], b[d]);
      }
      if (bad || !rows || !cols) {
#pragma omp atomic write
        err = bad ? ORA_ERR_NONFINITE : ORA_ERR_NOMEM;
        for (int c = 0; c < 3; ++c) vel[c * np + p] = NAN;
        continue;
      }
      /* stencil node for basis i along axis d: cell + i - 1 */
      for (int c = 0; c < 3; ++c) {
        const float* F = field + c * vol;
        /* filter along x: rows over z, y in the window around the stencil */
        for (int zz = 0; zz < S + 3; ++zz)
          for (int yy = 0; yy < S + 3; ++yy) {
            int64_t z = ((cell[2] - 1 - W + zz) % nz + nz) % nz;
            int64_t y = ((cell[1] - 1 - W + yy) % ny + ny) % ny;
            const float* row = F + (z * ny + y) * nx;
            for (int i = 0; i < 4; ++i) {
              double s = 0.0;
              for (int e = -W; e <= W; ++e) {
                int64_t x = ((cell[0] - 1 + i + e) % nx + nx) % nx;
                s += gw[0][e + W] * (double)row[x];
              }
              rows[(zz * (S + 3) + yy) * 4 + i] = s;
            }
          }
        /* filter along y */
        for (int zz = 0; zz < S + 3; ++zz)
          for (int j = 0; j < 4; ++j)
            for (int i = 0; i < 4; ++i) {
              double s = 0.0;
              for (int e = -W; e <= W; ++e)
                s += gw[1][e + W] * rows[(zz * (S + 3) + (j + W + e)) * 4 + i];
              cols[(zz * 4 + j) * 4 + i] = s;
            }
        /* filter along z, then the 64-term sum */
        double acc = 0.0;
        for (int k = 0; k < 4; ++k)
          for (int j = 0; j < 4; ++j)
            for (int i = 0; i < 4; ++i) {
              double s = 0.0;
              for (int e = -W; e <= W; ++e)
                s += gw[2][e + W] * cols[((k + W + e) * 4 + j) * 4 + i];
              acc += b[0][i] * b[1][j] * b[2][k] * s;
            }
        vel[c * np + p] = acc;
      }
    }
    free(rows);
    free(cols);
  }
  return err;
}
