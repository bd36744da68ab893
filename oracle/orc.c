/*
 * FP64 CPU oracle for the coupled D3Q19 BGK lattice Boltzmann step with the
 * Ota-Suzuki-Inamuro multi-direct-forcing immersed boundary loop
 * (Beny & Latt, "Efficient LBM on GPUs for dense moving objects using
 * immersed boundary condition", arXiv:1904.02108).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain definition that the
 * CUDA library is checked against.  Only the test-suite, the smoke check and
 * the CPU-baseline leg of the benchmark may load it.  It shares no code, no
 * header and no table with the CUDA library.
 *
 * Every loop runs in the order the paper states the method, in double
 * precision, with no blocking or fusion.  Readings of places where the paper
 * is silent or garbled are marked "Reading:".
 *
 * Layout: cell n = (z*ny + y)*nx + x; populations f[i*N + n]; Eulerian
 * vectors U[c*N + n] (c = 0,1,2); Lagrangian vectors v[3*k + c].
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define Q 19

/* D3Q19 velocity set (Sec. 2): one rest vector, six axis vectors and twelve
 * face diagonals such as [1,-1,0]. */
static const int E[Q][3] = {
    {0, 0, 0},
    {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},  {0, -1, 0}, {0, 0, 1},  {0, 0, -1},
    {1, 1, 0},  {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0},
    {1, 0, 1},  {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
    {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1},
};

/* Lattice weights t_i of Eq. 3 for D3Q19: 1/3 (rest), 1/18 (axis), 1/36
 * (diagonal). */
static double weight(int i) {
  if (i == 0) return 1.0 / 3.0;
  if (i <= 6) return 1.0 / 18.0;
  return 1.0 / 36.0;
}

static long wrap(long a, long n) {
  long r = a % n;
  return r < 0 ? r + n : r;
}

void orc_velocity_set(int *e, double *t) {
  for (int i = 0; i < Q; i++) {
    for (int c = 0; c < 3; c++) e[3 * i + c] = E[i][c];
    t[i] = weight(i);
  }
}

/* Eq. 3 with the density factor.  Reading: Eq. 3 is printed without rho, but
 * step 4 of the Sec. 2 summary evaluates Eq(i, rho, U^G); mass conservation
 * needs the factor. */
double orc_equilibrium(int i, double rho, const double U[3]) {
  double eu = E[i][0] * U[0] + E[i][1] * U[1] + E[i][2] * U[2];
  double uu = U[0] * U[0] + U[1] * U[1] + U[2] * U[2];
  return rho * weight(i) * (1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * uu);
}

/* Populations at equilibrium for given rho (NULL: 1) and U (NULL: 0). */
void orc_init_equilibrium(int nx, int ny, int nz, const double *rho,
                          const double *U, double *f) {
  long N = (long)nx * ny * nz;
  for (long n = 0; n < N; n++) {
    double r = rho ? rho[n] : 1.0;
    double u[3] = {0.0, 0.0, 0.0};
    if (U)
      for (int c = 0; c < 3; c++) u[c] = U[c * N + n];
    for (int i = 0; i < Q; i++) f[i * N + n] = orc_equilibrium(i, r, u);
  }
}

/* Eq. 1: rho = sum_i f_i, U = (1/rho) sum_i e_i f_i on every cell. */
void orc_moments(int nx, int ny, int nz, const double *f, double *rho,
                 double *U) {
  long N = (long)nx * ny * nz;
#pragma omp parallel for schedule(static)
  for (long n = 0; n < N; n++) {
    double r = 0.0, m[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < Q; i++) {
      double fi = f[i * N + n];
      r += fi;
      for (int c = 0; c < 3; c++) m[c] += E[i][c] * fi;
    }
    if (rho) rho[n] = r;
    for (int c = 0; c < 3; c++) U[c * N + n] = m[c] / r;
  }
}

/* Steps 3-5 of the Sec. 2 summary: U^G = U + tau*G, then the BGK relaxation
 * of Eq. 2 towards Eq(i, rho, U^G).  G may be NULL (no force). */
void orc_collide(int nx, int ny, int nz, double tau, double *f,
                 const double *rho, const double *U, const double *G) {
  long N = (long)nx * ny * nz;
#pragma omp parallel for schedule(static)
  for (long n = 0; n < N; n++) {
    double uG[3];
    for (int c = 0; c < 3; c++)
      uG[c] = U[c * N + n] + (G ? tau * G[c * N + n] : 0.0);
    for (int i = 0; i < Q; i++) {
      double fi = f[i * N + n];
      f[i * N + n] = fi + (orc_equilibrium(i, rho[n], uG) - fi) / tau;
    }
  }
}

/* Eq. 4: f_i(X + e_i, t+1) = f_i(X, t).  Reading: the paper states no
 * boundary; the domain is periodic in all three directions. */
void orc_stream(int nx, int ny, int nz, const double *fin, double *fout) {
  long N = (long)nx * ny * nz;
#pragma omp parallel for schedule(static)
  for (long z = 0; z < nz; z++)
    for (long y = 0; y < ny; y++)
      for (long x = 0; x < nx; x++) {
        long n = (z * ny + y) * nx + x;
        for (int i = 0; i < Q; i++) {
          long xd = wrap(x + E[i][0], nx), yd = wrap(y + E[i][1], ny),
               zd = wrap(z + E[i][2], nz);
          fout[i * N + (zd * ny + yd) * nx + xd] = fin[i * N + n];
        }
      }
}

/* Sec. 3 weighting function w(r), support |r| < 2.
 * kernel 0: cosine four-point kernel (1 + cos(pi r / 2)) / 4.
 * kernel 1: Peskin's four-point kernel.  Reading: the second branch is
 * printed as sqrt(1 - 7 + 12|r| - 4r^2); the Peskin kernel has
 * sqrt(-7 + 12|r| - 4r^2) there, which is also the only form that is
 * continuous at |r| = 1 and vanishes at |r| = 2. */
double orc_delta(int kernel, double r) {
  double a = fabs(r);
  if (a >= 2.0) return 0.0;
  if (kernel == 0) return 0.25 * (1.0 + cos(M_PI * a / 2.0));
  if (a <= 1.0) return (3.0 - 2.0 * a + sqrt(1.0 + 4.0 * a - 4.0 * a * a)) / 8.0;
  double q = -7.0 + 12.0 * a - 4.0 * a * a;
  if (q < 0.0) q = 0.0; /* rounding at a -> 2 */
  return (5.0 - 2.0 * a - sqrt(q)) / 8.0;
}

/* The 5x5x5 neighbourhood round(x)-2 .. round(x)+2 of Alg. 2, with the
 * product weight w(|x-X|) w(|y-Y|) w(|z-Z|).  Cells outside |r| < 2 carry
 * weight zero.  Indices wrap periodically. */
typedef struct {
  long idx[125];
  double w[125];
} stencil_t;

static void stencil(int nx, int ny, int nz, int kernel, const double *xk,
                    stencil_t *st) {
  long r0 = lround(xk[0]), r1 = lround(xk[1]), r2 = lround(xk[2]);
  double wx[5], wy[5], wz[5];
  for (int a = 0; a < 5; a++) {
    wx[a] = orc_delta(kernel, xk[0] - (double)(r0 - 2 + a));
    wy[a] = orc_delta(kernel, xk[1] - (double)(r1 - 2 + a));
    wz[a] = orc_delta(kernel, xk[2] - (double)(r2 - 2 + a));
  }
  int m = 0;
  for (int c = 0; c < 5; c++)
    for (int b = 0; b < 5; b++)
      for (int a = 0; a < 5; a++) {
        long X = r0 - 2 + a, Y = r1 - 2 + b, Z = r2 - 2 + c;
        st->idx[m] = (wrap(Z, nz) * ny + wrap(Y, ny)) * nx + wrap(X, nx);
        st->w[m] = wx[a] * wy[b] * wz[c];
        m++;
      }
}

/* Interpolation, fluid -> surface (Sec. 3, Alg. 1):
 * u(k) = sum_X U(X) w(|x_k - X|) w(|y_k - Y|) w(|z_k - Z|). */
void orc_interpolate(int nx, int ny, int nz, int kernel, const double *U,
                     long np, const double *x, double *u) {
  long N = (long)nx * ny * nz;
#pragma omp parallel for schedule(static)
  for (long k = 0; k < np; k++) {
    stencil_t st;
    stencil(nx, ny, nz, kernel, x + 3 * k, &st);
    double acc[3] = {0.0, 0.0, 0.0};
    for (int m = 0; m < 125; m++)
      for (int c = 0; c < 3; c++) acc[c] += U[c * N + st.idx[m]] * st.w[m];
    for (int c = 0; c < 3; c++) u[3 * k + c] = acc[c];
  }
}

/* Spreading, surface -> fluid (Sec. 3, Alg. 2):
 * F(X) += sum_k v(k) w(|x_k - X|) w(|y_k - Y|) w(|z_k - Z|).
 * Accumulates into F; points are visited in index order. */
void orc_spread(int nx, int ny, int nz, int kernel, long np, const double *x,
                const double *v, double *F) {
  long N = (long)nx * ny * nz;
  for (long k = 0; k < np; k++) {
    stencil_t st;
    stencil(nx, ny, nz, kernel, x + 3 * k, &st);
    for (int m = 0; m < 125; m++)
      for (int c = 0; c < 3; c++) F[c * N + st.idx[m]] += v[3 * k + c] * st.w[m];
  }
}

/* Rigid-body kinematics of Alg. 1: x(t) = M(t) [x_rest, 1] with M(t) the 4x4
 * affine map of a rotation by phi(t) = phase_b + omega_b t about the z axis
 * through centre_b, and the surface velocity u_k = x(t) - x(t-1).
 * Reading: u_k is the backward difference printed in Alg. 1, with x(t-1)
 * taken from M(t-1) (also at t = 0). */
static void affine_rotation_z(const double *c, double phi, double M[4][4]) {
  double cs = cos(phi), sn = sin(phi);
  double R[3][3] = {{cs, -sn, 0.0}, {sn, cs, 0.0}, {0.0, 0.0, 1.0}};
  for (int a = 0; a < 3; a++) {
    double t = c[a];
    for (int b = 0; b < 3; b++) {
      M[a][b] = R[a][b];
      t -= R[a][b] * c[b];
    }
    M[a][3] = t;
  }
  M[3][0] = M[3][1] = M[3][2] = 0.0;
  M[3][3] = 1.0;
}

void orc_kinematics(long np, const double *xrest, const int *body,
                    const double *centre, const double *omega,
                    const double *phase, long t, double *x, double *ut) {
  for (long k = 0; k < np; k++) {
    int b = body[k];
    double Mt[4][4], Mp[4][4];
    affine_rotation_z(centre + 3 * b, phase[b] + omega[b] * (double)t, Mt);
    affine_rotation_z(centre + 3 * b, phase[b] + omega[b] * (double)(t - 1), Mp);
    double h[4] = {xrest[3 * k], xrest[3 * k + 1], xrest[3 * k + 2], 1.0};
    for (int a = 0; a < 3; a++) {
      double xa = 0.0, xp = 0.0;
      for (int b2 = 0; b2 < 4; b2++) {
        xa += Mt[a][b2] * h[b2];
        xp += Mp[a][b2] * h[b2];
      }
      x[3 * k + a] = xa;
      if (ut) ut[3 * k + a] = xa - xp;
    }
  }
}

static double norm_field(long N, const double *F) {
  double s = 0.0;
  for (long n = 0; n < 3 * N; n++) s += F[n] * F[n];
  return sqrt(s);
}

static double norm_points(long np, const double *v) {
  double s = 0.0;
  for (long n = 0; n < 3 * np; n++) s += v[n] * v[n];
  return sqrt(s);
}

/* Denominators of the residuals: den = ||S[s u_t]|| (Eulerian) and
 * den_pt = ||u_t|| (pointwise); where one vanishes, the same norm of the
 * zero-start increment (s (u_t - I[U0]), resp. u_t - I[U0]), then 1. */
static void residual_denominators(int nx, int ny, int nz, int kernel, const double *U0,
                                  long np, const double *x, const double *ut,
                                  const double *s, double *den_out, double *den_pt_out) {
  long N = (long)nx * ny * nz;
  double *tmp = malloc(sizeof(double) * 3 * N);
  double *un = malloc(sizeof(double) * 3 * np);
  double *v = malloc(sizeof(double) * 3 * np);
  for (long k = 0; k < np; k++)
    for (int c = 0; c < 3; c++) v[3 * k + c] = s[k] * ut[3 * k + c];
  memset(tmp, 0, sizeof(double) * 3 * N);
  orc_spread(nx, ny, nz, kernel, np, x, v, tmp);
  double den = norm_field(N, tmp);
  double den_pt = norm_points(np, ut);
  if (den == 0.0 || den_pt == 0.0) {
    orc_interpolate(nx, ny, nz, kernel, U0, np, x, un);
    for (long k = 0; k < np; k++)
      for (int c = 0; c < 3; c++)
        v[3 * k + c] = ut[3 * k + c] - un[3 * k + c];
    if (den_pt == 0.0) den_pt = norm_points(np, v);
    for (long k = 0; k < np; k++)
      for (int c = 0; c < 3; c++) v[3 * k + c] *= s[k];
    if (den == 0.0) {
      memset(tmp, 0, sizeof(double) * 3 * N);
      orc_spread(nx, ny, nz, kernel, np, x, v, tmp);
      den = norm_field(N, tmp);
    }
    if (den == 0.0) den = 1.0;
    if (den_pt == 0.0) den_pt = 1.0;
  }
  *den_out = den;
  *den_pt_out = den_pt;
  free(tmp);
  free(un);
  free(v);
}

/* The multi-direct-forcing fixed point of Sec. 3.
 *
 *   U_0 = U0 + S[du_init]               (du_init = 0 in the paper)
 *   for n = 0, 1, ...:
 *     u_n(k)  = I[U_n](k)
 *     g_n(k)  = u_k - u_n(k)
 *     du(k)  += g_n(k) s(k)
 *     U_{n+1} = U_n + S[g_n s]          (literal: U_n + S[g_n])
 *   G = S[du]
 *
 * Readings: the first estimate includes g_0 (the text's du = 0 + g_0 s, not
 * the algorithm listing's du = 0); the Eulerian update carries s(k) like the
 * Lagrangian one, so that U_N = U0 + G (literal = 1 restores the printed form
 * without s).  Residual eps_n = ||S[s g_n]|| / ||S[s u_t]|| (both over the
 * lattice, FP64); if the denominator vanishes, ||S[s (u_t - I[U0])]|| is used,
 * then 1.  Pointwise residual ||g_n|| / ||u_t|| with the same fallback.
 *
 * n_iter > 0: exactly n_iter iterations.  n_iter == 0: iterate until
 * eps_n <= tol or max_iter iterations.  Returns the number of iterations.
 * eps, eps_pt: arrays of at least (n_iter or max_iter) entries, or NULL.
 */
int orc_ibm(int nx, int ny, int nz, int kernel, const double *U0, long np,
            const double *x, const double *ut, const double *s, int n_iter,
            double tol, int max_iter, int literal, const double *du_init,
            double *du, double *G, double *eps, double *eps_pt) {
  long N = (long)nx * ny * nz;
  double *Un = malloc(sizeof(double) * 3 * N);
  double *inc = malloc(sizeof(double) * 3 * N);
  double *tmp = malloc(sizeof(double) * 3 * N);
  double *un = malloc(sizeof(double) * 3 * np);
  double *v = malloc(sizeof(double) * 3 * np);
  memcpy(Un, U0, sizeof(double) * 3 * N);
  for (long n = 0; n < 3 * np; n++) du[n] = du_init ? du_init[n] : 0.0;
  if (du_init) orc_spread(nx, ny, nz, kernel, np, x, du_init, Un);

  double den, den_pt;
  residual_denominators(nx, ny, nz, kernel, U0, np, x, ut, s, &den, &den_pt);

  int n = 0;
  for (;;) {
    orc_interpolate(nx, ny, nz, kernel, Un, np, x, un);
    for (long k = 0; k < np; k++)
      for (int c = 0; c < 3; c++) {
        double g = ut[3 * k + c] - un[3 * k + c];
        du[3 * k + c] += g * s[k];
        v[3 * k + c] = literal ? g : g * s[k];
      }
    memset(inc, 0, sizeof(double) * 3 * N);
    orc_spread(nx, ny, nz, kernel, np, x, v, inc);
    for (long m = 0; m < 3 * N; m++) Un[m] += inc[m];
    double e;
    if (literal) {
      for (long k = 0; k < np; k++)
        for (int c = 0; c < 3; c++) v[3 * k + c] *= s[k];
      memset(tmp, 0, sizeof(double) * 3 * N);
      orc_spread(nx, ny, nz, kernel, np, x, v, tmp);
      e = norm_field(N, tmp) / den;
    } else {
      e = norm_field(N, inc) / den;
    }
    double gp = 0.0;
    for (long k = 0; k < np; k++)
      for (int c = 0; c < 3; c++) {
        double g = ut[3 * k + c] - un[3 * k + c];
        gp += g * g;
      }
    if (eps) eps[n] = e;
    if (eps_pt) eps_pt[n] = sqrt(gp) / den_pt;
    n++;
    if (n_iter > 0) {
      if (n >= n_iter) break;
    } else if (e <= tol || n >= max_iter) {
      break;
    }
  }
  memset(G, 0, sizeof(double) * 3 * N);
  orc_spread(nx, ny, nz, kernel, np, x, du, G);
  free(Un);
  free(inc);
  free(tmp);
  free(un);
  free(v);
  return n;
}

/* Conjugate gradients on the same fixed point (not in the paper; a Krylov
 * replacement for the loop above).
 *
 * On the lattice, the loop above is Richardson's iteration with unit step,
 * G_{n+1} = G_n + (c - B G_n), on the linear system
 *
 *   B G = c,   B = S diag(s) I,   c = S[s (u_t - I[U0])],
 *
 * whose residual c - B G_n = S[s g_n] is the one eps measures.  B is
 * symmetric positive semi-definite (S is the adjoint of I) and c lies in its
 * range, so conjugate gradients apply even where A = I S is singular (points
 * closer than the kernel resolves: the point-space system A du = b is then
 * inconsistent, and CG on it diverges).  Hestenes-Stiefel CG on B G = c:
 *
 *   R_0 = c - B G_0,  P_0 = R_0
 *   for n = 0, 1, ...:
 *     eps_n   = ||R_n|| / ||S[s u_t]||
 *     alpha_n = (R_n . R_n) / (P_n . B P_n)
 *     G_{n+1} = G_n + alpha_n P_n,   R_{n+1} = R_n - alpha_n B P_n
 *     beta_n  = (R_{n+1} . R_{n+1}) / (R_n . R_n),   P_{n+1} = R_{n+1} + beta_n P_n
 *
 * Every iterate is a spread of point values, so the oracle carries those
 * instead: G_n = S[du_n], R_n = S[s r_n] with r_n = u_t - I[U0 + G_n], and
 * P_n = S[p_n]; then B P_n = S[s y_n] with y_n = I[P_n], P_n . B P_n =
 * sum_k s(k) |y_n(k)|^2, and the updates read
 *
 *   du += alpha_n p_n,   r_{n+1} = r_n - alpha_n y_n,   p_{n+1} = s r_{n+1} + beta_n p_n,
 *
 * with R . R = ||S[s r]||^2 spread anew each iteration.  Where R_n . R_n or
 * P_n . B P_n is not positive (an exact solution) alpha_n = 0, and beta_n = 0
 * when R_n . R_n is 0.  Iteration counts, n_iter, tol, max_iter, the
 * denominators and the pointwise residual ||r_n|| / ||u_t|| are as in
 * orc_ibm; u_interp (NULL or [np][3]) receives u_t - r_n of the last
 * iteration, the velocity interpolated from its iterate. */
int orc_ibm_cg(int nx, int ny, int nz, int kernel, const double *U0, long np,
               const double *x, const double *ut, const double *s, int n_iter,
               double tol, int max_iter, const double *du_init, double *du, double *G,
               double *eps, double *eps_pt, double *u_interp) {
  long N = (long)nx * ny * nz;
  long M = 3 * np;
  double *F = malloc(sizeof(double) * 3 * N);
  double *r = malloc(sizeof(double) * M);
  double *v = malloc(sizeof(double) * M);
  double *p = malloc(sizeof(double) * M);
  double *y = malloc(sizeof(double) * M);
  double den, den_pt;
  residual_denominators(nx, ny, nz, kernel, U0, np, x, ut, s, &den, &den_pt);

  for (long m = 0; m < M; m++) du[m] = du_init ? du_init[m] : 0.0;
  memcpy(F, U0, sizeof(double) * 3 * N);
  if (du_init) orc_spread(nx, ny, nz, kernel, np, x, du, F);
  orc_interpolate(nx, ny, nz, kernel, F, np, x, y);
  for (long k = 0; k < np; k++)
    for (int c = 0; c < 3; c++) {
      long m = 3 * k + c;
      r[m] = ut[m] - y[m];
      v[m] = s[k] * r[m];
      p[m] = v[m];
    }
  memset(F, 0, sizeof(double) * 3 * N);
  orc_spread(nx, ny, nz, kernel, np, x, v, F);
  double rr = norm_field(N, F);
  rr *= rr;

  int n = 0;
  for (;;) {
    if (eps) eps[n] = sqrt(rr) / den;
    if (eps_pt) eps_pt[n] = norm_points(np, r) / den_pt;
    if (u_interp)
      for (long m = 0; m < M; m++) u_interp[m] = ut[m] - r[m];

    memset(F, 0, sizeof(double) * 3 * N);
    orc_spread(nx, ny, nz, kernel, np, x, p, F);
    orc_interpolate(nx, ny, nz, kernel, F, np, x, y);
    double pbp = 0.0;
    for (long k = 0; k < np; k++)
      for (int c = 0; c < 3; c++) pbp += s[k] * y[3 * k + c] * y[3 * k + c];
    double alpha = (rr > 0.0 && pbp > 0.0) ? rr / pbp : 0.0;
    for (long k = 0; k < np; k++)
      for (int c = 0; c < 3; c++) {
        long m = 3 * k + c;
        du[m] += alpha * p[m];
        r[m] -= alpha * y[m];
        v[m] = s[k] * r[m];
      }
    memset(F, 0, sizeof(double) * 3 * N);
    orc_spread(nx, ny, nz, kernel, np, x, v, F);
    double rr_next = norm_field(N, F);
    rr_next *= rr_next;
    double beta = rr > 0.0 ? rr_next / rr : 0.0;
    for (long m = 0; m < M; m++) p[m] = v[m] + beta * p[m];
    double e = sqrt(rr) / den;
    rr = rr_next;

    n++;
    if (n_iter > 0) {
      if (n >= n_iter) break;
    } else if (e <= tol || n >= max_iter) {
      break;
    }
  }
  memset(G, 0, sizeof(double) * 3 * N);
  orc_spread(nx, ny, nz, kernel, np, x, du, G);
  free(F);
  free(r);
  free(v);
  free(p);
  free(y);
  return n;
}

/* Global sums of the populations: mass sum_X sum_i f_i and momentum
 * sum_X sum_i e_i f_i.  out[0] = mass, out[1..3] = momentum. */
void orc_sums(int nx, int ny, int nz, const double *f, double *out) {
  long N = (long)nx * ny * nz;
  double m = 0.0, p[3] = {0.0, 0.0, 0.0};
  for (int i = 0; i < Q; i++)
    for (long n = 0; n < N; n++) {
      double fi = f[i * N + n];
      m += fi;
      for (int c = 0; c < 3; c++) p[c] += E[i][c] * fi;
    }
  out[0] = m;
  for (int c = 0; c < 3; c++) out[c + 1] = p[c];
}

/* One full time step in the order of the Sec. 2 summary:
 *   1. rho, U from Eq. 1 (U0 below);
 *   2. G = immersedBoundary(object, U) by orc_ibm (np > 0; solver 0) or
 *      by orc_ibm_cg (solver 1);
 *      plus an optional uniform body force gbody (a test hook, not in the
 *      paper);
 *   3-5. U^G = U + tau G, equilibrium, BGK collision;
 *   6. streaming.
 * f holds the populations in and out; ftmp is scratch of the same size.
 * rho, U0, G receive the step's fields (rho, G may be NULL).
 * Returns the number of IBM iterations (0 without points). */
int orc_step(int nx, int ny, int nz, double tau, int kernel, double *f,
             double *ftmp, long np, const double *x, const double *ut,
             const double *s, int n_iter, double tol, int max_iter,
             int literal, const double *du_init, double *du,
             const double *gbody, double *rho, double *U0, double *G,
             double *eps, double *eps_pt, int solver) {
  long N = (long)nx * ny * nz;
  double *r = rho ? rho : malloc(sizeof(double) * N);
  double *g = G ? G : malloc(sizeof(double) * 3 * N);
  orc_moments(nx, ny, nz, f, r, U0);
  int iters = 0;
  if (np > 0 && solver == 1)
    iters = orc_ibm_cg(nx, ny, nz, kernel, U0, np, x, ut, s, n_iter, tol,
                       max_iter, du_init, du, g, eps, eps_pt, NULL);
  else if (np > 0)
    iters = orc_ibm(nx, ny, nz, kernel, U0, np, x, ut, s, n_iter, tol,
                    max_iter, literal, du_init, du, g, eps, eps_pt);
  else
    memset(g, 0, sizeof(double) * 3 * N);
  if (gbody)
    for (int c = 0; c < 3; c++)
      for (long n = 0; n < N; n++) g[c * N + n] += gbody[c];
  orc_collide(nx, ny, nz, tau, f, r, U0, g);
  orc_stream(nx, ny, nz, f, ftmp);
  memcpy(f, ftmp, sizeof(double) * Q * N);
  if (!rho) free(r);
  if (!G) free(g);
  return iters;
}

/* ---- per-point MLP of the learned warm start (not in the paper) ----------
 * y = W3 s(W2 s(W1 x + b1) + b2) + b3 with s(v) = v / (1 + exp(-v)) (SiLU),
 * x in R^16, hidden widths 64 and 64, y in R^3.  Parameters are one flat
 * vector P = [W1 (64x16, row-major: out x in), b1 (64), W2 (64x64), b2 (64),
 * W3 (3x64), b3 (3)], 5443 values.  Plain FP64 loops, no blocking. */
#define MLP_IN 16
#define MLP_H 64
#define MLP_OUT 3
#define MLP_NPARAM (MLP_H * MLP_IN + MLP_H + MLP_H * MLP_H + MLP_H + MLP_OUT * MLP_H + MLP_OUT)

static double silu(double v) { return v / (1.0 + exp(-v)); }
static double silu_grad(double v) {
  double sg = 1.0 / (1.0 + exp(-v));
  return sg * (1.0 + v * (1.0 - sg));
}

int orc_mlp_nparam(void) { return MLP_NPARAM; }

/* Forward pass of one sample; a1, a2 receive the pre-activations (may be
 * NULL). */
static void mlp_one(const double *P, const double *x, double *y, double *a1, double *a2) {
  const double *W1 = P, *b1 = W1 + MLP_H * MLP_IN, *W2 = b1 + MLP_H, *b2 = W2 + MLP_H * MLP_H,
               *W3 = b2 + MLP_H, *b3 = W3 + MLP_OUT * MLP_H;
  double h1[MLP_H], h2[MLP_H], z1[MLP_H], z2[MLP_H];
  for (int o = 0; o < MLP_H; o++) {
    double v = b1[o];
    for (int i = 0; i < MLP_IN; i++) v += W1[o * MLP_IN + i] * x[i];
    z1[o] = v;
    h1[o] = silu(v);
  }
  for (int o = 0; o < MLP_H; o++) {
    double v = b2[o];
    for (int i = 0; i < MLP_H; i++) v += W2[o * MLP_H + i] * h1[i];
    z2[o] = v;
    h2[o] = silu(v);
  }
  for (int o = 0; o < MLP_OUT; o++) {
    double v = b3[o];
    for (int i = 0; i < MLP_H; i++) v += W3[o * MLP_H + i] * h2[i];
    y[o] = v;
  }
  if (a1) memcpy(a1, z1, sizeof z1);
  if (a2) memcpy(a2, z2, sizeof z2);
}

void orc_mlp_forward(long n, const double *P, const double *x, double *y) {
  for (long k = 0; k < n; k++) mlp_one(P, x + MLP_IN * k, y + MLP_OUT * k, NULL, NULL);
}

/* Loss L = (1/n) sum_k 0.5 |y_k - t_k|^2 and its gradient dL/dP (chain rule
 * through the three layers, accumulated over the samples in order). */
double orc_mlp_loss_grad(long n, const double *P, const double *x, const double *t,
                         double *grad) {
  const double *W1 = P, *b1 = W1 + MLP_H * MLP_IN, *W2 = b1 + MLP_H, *b2 = W2 + MLP_H * MLP_H,
               *W3 = b2 + MLP_H;
  (void)b1;
  (void)b2;
  double *gW1 = grad, *gb1 = gW1 + MLP_H * MLP_IN, *gW2 = gb1 + MLP_H,
         *gb2 = gW2 + MLP_H * MLP_H, *gW3 = gb2 + MLP_H, *gb3 = gW3 + MLP_OUT * MLP_H;
  if (grad) memset(grad, 0, sizeof(double) * MLP_NPARAM);
  double loss = 0.0;
  for (long k = 0; k < n; k++) {
    const double *xk = x + MLP_IN * k;
    double y[MLP_OUT], z1[MLP_H], z2[MLP_H], h1[MLP_H], h2[MLP_H];
    mlp_one(P, xk, y, z1, z2);
    for (int o = 0; o < MLP_H; o++) {
      h1[o] = silu(z1[o]);
      h2[o] = silu(z2[o]);
    }
    double dy[MLP_OUT];
    for (int o = 0; o < MLP_OUT; o++) {
      double e = y[o] - t[MLP_OUT * k + o];
      loss += 0.5 * e * e / (double)n;
      dy[o] = e / (double)n;
    }
    if (!grad) continue;
    double dh2[MLP_H], dz2[MLP_H], dh1[MLP_H], dz1[MLP_H];
    for (int o = 0; o < MLP_OUT; o++) {
      gb3[o] += dy[o];
      for (int i = 0; i < MLP_H; i++) gW3[o * MLP_H + i] += dy[o] * h2[i];
    }
    for (int i = 0; i < MLP_H; i++) {
      double v = 0.0;
      for (int o = 0; o < MLP_OUT; o++) v += W3[o * MLP_H + i] * dy[o];
      dh2[i] = v;
      dz2[i] = v * silu_grad(z2[i]);
    }
    for (int o = 0; o < MLP_H; o++) {
      gb2[o] += dz2[o];
      for (int i = 0; i < MLP_H; i++) gW2[o * MLP_H + i] += dz2[o] * h1[i];
    }
    for (int i = 0; i < MLP_H; i++) {
      double v = 0.0;
      for (int o = 0; o < MLP_H; o++) v += W2[o * MLP_H + i] * dz2[o];
      dh1[i] = v;
      dz1[i] = v * silu_grad(z1[i]);
    }
    for (int o = 0; o < MLP_H; o++) {
      gb1[o] += dz1[o];
      for (int i = 0; i < MLP_IN; i++) gW1[o * MLP_IN + i] += dz1[o] * xk[i];
    }
  }
  return loss;
}

/* ---- inputs and initial guess of the learned warm start (not in the paper)
 *
 * Features of point k for the per-point MLP above, in this order:
 *   0-2   u_i(k) = I[U0 + S[du_prev]](k): the velocity interpolated on the
 *         lattice with the previous step's correction already spread on it
 *         (the first estimate U_0 of the Sec. 3 loop when it starts from
 *         du_prev), divided by vscale;
 *   3-5   u_k / vscale, the surface velocity of the point (Alg. 1);
 *   6-8   du_prev(k) / vscale (zero when du_prev is NULL);
 *   9     local point density: over the 4x4x4 bricks that the point's support
 *         touches, the mean number of supports touching each brick, per cell
 *         of a brick (divided by 64);
 *   10-11 distance from the body's rotation axis (the z line through its
 *         centre) and axial offset z - z_c, divided by lscale (0 without
 *         bodies);
 *   12    |omega_b| r / vscale, the speed of rigid rotation at that radius;
 *   13-15 (u_k - u_i(k)) / vscale, the slip the fixed point has to remove.
 *
 * Reading: the support of a point is the block of four cells per axis,
 * floor(x) - 1 .. floor(x) + 2 (wrapped), at which the kernel's taps sit (the
 * 5-wide window of Alg. 2 contains them; its fifth tap has weight 0).  A
 * brick is touched when one of those cells lies in it.
 * body: [np] body of each point (NULL: 0); centre [nb][3], omega [nb]; nb = 0
 * means no bodies.  feat: [np][16]. */
static long brick_of_cell(long X, long Y, long Z, int nx, int ny, int nz) {
  long bx = wrap(X, nx) / 4, by = wrap(Y, ny) / 4, bz = wrap(Z, nz) / 4;
  return (bz * (ny / 4) + by) * (nx / 4) + bx;
}

/* The distinct bricks touched by the support of a point at xk (at most 8). */
static int touched_bricks(int nx, int ny, int nz, const double *xk, long out[8]) {
  long f0 = (long)floor(xk[0]), f1 = (long)floor(xk[1]), f2 = (long)floor(xk[2]);
  int m = 0;
  for (long c = -1; c <= 2; c++)
    for (long b = -1; b <= 2; b++)
      for (long a = -1; a <= 2; a++) {
        long br = brick_of_cell(f0 + a, f1 + b, f2 + c, nx, ny, nz);
        int seen = 0;
        for (int j = 0; j < m; j++) seen |= out[j] == br;
        if (!seen) out[m++] = br;
      }
  return m;
}

void orc_mlp_features(int nx, int ny, int nz, int kernel, const double *U0, long np,
                      const double *x, const double *ut, const double *du_prev,
                      const int *body, int nb, const double *centre, const double *omega,
                      double vscale, double lscale, double *feat) {
  long N = (long)nx * ny * nz;
  long nbrick = (long)(nx / 4) * (ny / 4) * (nz / 4);
  double *Uf = malloc(sizeof(double) * 3 * N);
  double *ui = malloc(sizeof(double) * 3 * np);
  long *touch = malloc(sizeof(long) * 8 * np);
  int *ntouch = malloc(sizeof(int) * np);
  long *count = calloc(nbrick, sizeof(long));

  /* u_i = I[U0 + S[du_prev]] */
  memcpy(Uf, U0, sizeof(double) * 3 * N);
  if (du_prev) orc_spread(nx, ny, nz, kernel, np, x, du_prev, Uf);
  orc_interpolate(nx, ny, nz, kernel, Uf, np, x, ui);

  /* supports touching each brick */
  for (long k = 0; k < np; k++) {
    ntouch[k] = touched_bricks(nx, ny, nz, x + 3 * k, touch + 8 * k);
    for (int j = 0; j < ntouch[k]; j++) count[touch[8 * k + j]]++;
  }

  for (long k = 0; k < np; k++) {
    double *o = feat + 16 * k;
    double dens = 0.0;
    for (int j = 0; j < ntouch[k]; j++) dens += (double)count[touch[8 * k + j]];
    dens /= 64.0 * ntouch[k];
    double r = 0.0, dz = 0.0, speed = 0.0;
    if (nb > 0) {
      int b = body ? body[k] : 0;
      double ex = x[3 * k] - centre[3 * b], ey = x[3 * k + 1] - centre[3 * b + 1];
      r = sqrt(ex * ex + ey * ey);
      dz = x[3 * k + 2] - centre[3 * b + 2];
      speed = fabs(omega[b]) * r;
    }
    for (int c = 0; c < 3; c++) {
      o[c] = ui[3 * k + c] / vscale;
      o[3 + c] = ut[3 * k + c] / vscale;
      o[6 + c] = du_prev ? du_prev[3 * k + c] / vscale : 0.0;
      o[13 + c] = (ut[3 * k + c] - ui[3 * k + c]) / vscale;
    }
    o[9] = dens;
    o[10] = r / lscale;
    o[11] = dz / lscale;
    o[12] = speed / vscale;
  }
  free(Uf);
  free(ui);
  free(touch);
  free(ntouch);
  free(count);
}

/* The learned initial guess of the fixed point: du_init = du_prev + V MLP(x)
 * with x the features above (V = vscale); du_prev NULL counts as zero. */
void orc_learned_init(long np, const double *P, const double *feat, const double *du_prev,
                      double vscale, double *du_init) {
  double *y = malloc(sizeof(double) * MLP_OUT * np);
  orc_mlp_forward(np, P, feat, y);
  for (long k = 0; k < np; k++)
    for (int c = 0; c < 3; c++)
      du_init[3 * k + c] = (du_prev ? du_prev[3 * k + c] : 0.0) + vscale * y[3 * k + c];
  free(y);
}
