/*
 * acat_oracle.c -- plain, slow FP64 CPU oracle of the ACAT method
 * (Carrillo, Macca, Pares, Russo, Zorio, "An order-adaptive compact
 * approximation Taylor method for systems of conservation laws",
 * arXiv 2007.01416).
 *
 * TEST INFRASTRUCTURE. This is the correctness reference for the CUDA
 * library and shares no code with it. Only the test suite, the package smoke
 * check and the benchmark's CPU-baseline leg may load it; the library never
 * does. It is compiled with -ffp-contract=off so that every product and sum is
 * rounded as written.
 *
 * Pins (tests/test_oracle_*.py): Fornberg weights against exact rational
 * Vandermonde solves; the CAT2 closed form (Eqs. 2.16-2.17) and its 2D form
 * (Eqs. 4.3-4.4); exact reduction of CAT2p to the (2p+1)-point Lax-Wendroff
 * scheme for linear flux (Sec. 2.2); order 2p on smooth solutions; discrete
 * conservation; constant data and jumps for the indicators (Sec. 3.2); their
 * homothetic invariance; the limiter fallback at a jump; Riemann problems
 * against an exact solver.
 */
#include "acat_oracle.h"

#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Differentiation weights gamma^{k,q}_{p,r} on the 2p nodes r = -p+1..p
 * (Eq. 2.10), computed by Fornberg's recursive algorithm (Fornberg 1988,
 * "Generation of finite difference formulas on arbitrarily spaced grids";
 * cited in Sec. 2.1 and Sec. 5). w[r + p - 1] receives gamma^{k,q}_{p,r}. */
static int fornberg_nodes(int n, const double *x, int k, double q, double *w) {
  if (n < 1 || n > OR_MAXN + 1 || k < 0 || k >= n) return -1;
  double c[OR_MAXN + 1][OR_MAXN + 1]; /* c[node][derivative order] */
  memset(c, 0, sizeof c);
  double c1 = 1.0, c4 = x[0] - q;
  c[0][0] = 1.0;
  for (int i = 1; i < n; i++) {
    const int mn = i < k ? i : k;
    double c2 = 1.0, c5 = c4;
    c4 = x[i] - q;
    for (int j = 0; j < i; j++) {
      const double c3 = x[i] - x[j];
      c2 = c2 * c3;
      if (j == i - 1) {
        for (int m = mn; m >= 1; m--) c[i][m] = c1 * (m * c[i - 1][m - 1] - c5 * c[i - 1][m]) / c2;
        c[i][0] = -c1 * c5 * c[i - 1][0] / c2;
      }
      for (int m = mn; m >= 1; m--) c[j][m] = (c4 * c[j][m] - m * c[j][m - 1]) / c3;
      c[j][0] = c4 * c[j][0] / c3;
    }
    c1 = c2;
  }
  for (int r = 0; r < n; r++) w[r] = c[r][k];
  return 0;
}

int or_fornberg(int p, int k, double q, double *w) {
  double x[OR_MAXN];
  if (p < 1 || p > OR_MAXP) return -1;
  for (int r = 0; r < 2 * p; r++) x[r] = (double)(r - p + 1);
  return fornberg_nodes(2 * p, x, k, q, w);
}

/* Weights gamma^{0,1/2}_{p,r} of the flux formula A^{0,1/2}_{p,0} in Eq. 2.14
 * (and Eqs. 4.5-4.6). They are the weights for which Eq. 2.11 holds at k = 1:
 *   D^1_{p,i} = (A^{0,1/2}_{p,i} - A^{0,1/2}_{p,i-1}) / dx,
 * with D^1_p the centred (2p+1)-point first-derivative formula of Eq. 2.5
 * (weights delta^1_{p,j}, j = -p..p, Fornberg on the nodes -p..p). Matching
 * the coefficient of f_{i+l} gives gamma_{l} - gamma_{l+1} = delta_l, i.e.
 * gamma_m = -sum_{l=-p}^{m-1} delta_l, m = -p+1..p. This is the reading under
 * which CAT2p reduces to the (2p+1)-point Lax-Wendroff scheme for linear flux
 * and has order 2p, as Sec. 2.2 states; the 2p-point Lagrange midpoint
 * interpolant differs from it for p >= 2 and gives a second-order update. */
int or_flux_weights(int p, double *w) {
  double x[OR_MAXN + 1], d[OR_MAXN + 1];
  if (p < 1 || p > OR_MAXP) return -1;
  for (int r = 0; r <= 2 * p; r++) x[r] = (double)(r - p);
  if (fornberg_nodes(2 * p + 1, x, 1, 0.0, d)) return -1;
  double s = 0.0;
  for (int m = 0; m < 2 * p; m++) {
    s = s - d[m];
    w[m] = s;
  }
  return 0;
}

int or_nvars(const or_params *P) {
  switch (P->flux) {
  case OR_EULER1D: return 3;
  case OR_EULER2D: return 4;
  default: return 1;
  }
}

long or_bc_map(int bc, long i, long n);
long or_bc_map(int bc, long i, long n) {
  if (bc == OR_PERIODIC) {
    long r = i % n;
    return r < 0 ? r + n : r;
  }
  return i < 0 ? 0 : (i >= n ? n - 1 : i);
}

/* Weight tables used by one step (filled once per call from or_fornberg). */
typedef struct {
  double g1[OR_MAXP + 1][OR_MAXN][OR_MAXN]; /* [p][j][r] gamma^{1,j}_{p,r}     */
  double gk[OR_MAXP + 1][OR_MAXN][OR_MAXN]; /* [p][k][r] gamma^{k,0}_{p,r}     */
  double gh[OR_MAXP + 1][OR_MAXN];          /* [p][r]    gamma^{0,1/2}_{p,r}
                                               (flux weights, or_flux_weights) */
  double gd[OR_MAXP + 1][OR_MAXN];          /* [p][r]    gamma^{2p-1,1/2}_{p,r} */
} or_tables;

static void or_fill_tables(or_tables *T, int Pmax) {
  memset(T, 0, sizeof *T);
  for (int p = 1; p <= Pmax; p++) {
    const int n = 2 * p;
    for (int j = 0; j < n; j++) or_fornberg(p, 1, (double)(j - p + 1), T->g1[p][j]);
    for (int k = 0; k < n; k++) or_fornberg(p, k, 0.0, T->gk[p][k]);
    or_flux_weights(p, T->gh[p]);
    or_fornberg(p, n - 1, 0.5, T->gd[p]);
  }
}

/* Smoothness indicator psi^p of one component (Eqs. 3.8-3.12).
 * q[ic] is u_i, the cell left of the interface, q[ic + j] is u_{i+j}. */
static double or_psi_p(const or_params *P, const or_tables *T, int p, const double *q, int ic) {
  double IL = 0.0, IR = 0.0;
  for (int j = -p + 1; j <= -1; j++) {
    const double d = q[ic + 1 + j] - q[ic + j];
    IL = IL + d * d;
  }
  IL = IL + P->eps;
  for (int j = 1; j <= p - 1; j++) {
    const double d = q[ic + 1 + j] - q[ic + j];
    IR = IR + d * d;
  }
  IR = IR + P->eps;
  const double Ip = IL * IR / (IL + IR);
  double S = 0.0;
  for (int j = -p + 1; j <= p; j++) S = S + T->gd[p][j + p - 1] * q[ic + j];
  double fact = 1.0;
  if (P->tau_factorial)
    for (int m = 2; m <= 2 * p - 1; m++) fact = fact * m;
  const double D = fact * S;
  const double tau = D * D;
  return Ip / (Ip + tau);
}

/* Modified indicator psi~^2 of one component (Sec. 3.2, the variant for
 * critical points at the midpoints x_{i-1/2}, x_{i+3/2}): the two splits of
 * the three differences of S_2 into lateral weights that keep the central
 * difference,
 *   I^1_L = d_{-1}^2 + eps,          I^1_R = d_0^2 + d_1^2 + eps,
 *   I^2_L = d_{-1}^2 + d_0^2 + eps,  I^2_R = d_1^2 + eps,
 * with d_j = f_{i+1+j} - f_{i+j}; I^j = I^j_L I^j_R / (I^j_L + I^j_R); and
 * psi~^2 = max(I^1 / (I^1 + tau_2), I^2 / (I^2 + tau_2)), tau_2 as in
 * Eq. 3.12. The maximum is taken as (a > b ? a : b). */
static double or_psi2_mod(const or_params *P, const or_tables *T, const double *q, int ic) {
  const double dm = q[ic] - q[ic - 1], d0 = q[ic + 1] - q[ic], dp = q[ic + 2] - q[ic + 1];
  const double I1L = dm * dm + P->eps, I1R = (d0 * d0 + dp * dp) + P->eps;
  const double I2L = (dm * dm + d0 * d0) + P->eps, I2R = dp * dp + P->eps;
  const double I1 = I1L * I1R / (I1L + I1R), I2 = I2L * I2R / (I2L + I2R);
  double S = 0.0;
  for (int j = -1; j <= 2; j++) S = S + T->gd[2][j + 1] * q[ic + j];
  const double fact = P->tau_factorial ? 6.0 : 1.0; /* (2p-1)! at p = 2 */
  const double D = fact * S;
  const double tau = D * D;
  const double a = I1 / (I1 + tau), b = I2 / (I2 + tau);
  return a > b ? a : b;
}

/* Admissible set and selected order (Eqs. 3.2-3.3; systems: minimum over the
 * components, Sec. 3.4). Returns p_s = max A, or 1 when A is empty. */
static int or_select(const or_params *P, const or_tables *T, const double *line, int LW,
                     int ic, int unused, double *psi) {
  (void)unused;
  const int s = or_nvars(P);
  const double thr = 1.0 - P->psi_tol;
  int ps = 1;
  for (int p = 2; p <= P->P; p++) {
    double m = 0.0;
    for (int c = 0; c < s; c++) {
      const double v = (p == 2 && P->psi2_mod) ? or_psi2_mod(P, T, line + c * LW, ic)
                                               : or_psi_p(P, T, p, line + c * LW, ic);
      if (c == 0 || v < m) m = v;
    }
    if (psi) psi[p] = m;
    if (m >= thr) ps = p;
  }
  return ps;
}

/* ---- instantiate the generic core for double and double complex -------- */
#define R double
#define RE(x) (x)
#define SQRT_R(x) sqrt(x)
#define SFX _d
#include "acat_oracle_impl.h"
#undef R
#undef RE
#undef SQRT_R
#undef SFX

#define R double complex
#define RE(x) creal(x)
#define SQRT_R(x) csqrt(x)
#define SFX _z
#include "acat_oracle_impl.h"
#undef R
#undef RE
#undef SQRT_R
#undef SFX

/* ---- public entry points -------------------------------------------------- */
void or_flux_x(const or_params *P, const double *u, double *f) { flux_x_d(P, u, f); }
void or_flux_y(const or_params *P, const double *u, double *f) { flux_y_d(P, u, f); }

/* The physical flux f(u_i) of every cell of a 1D state (SoA in and out). */
void or_cell_flux_1d(const or_params *P, const double *u, double *f) {
  const int s = or_nvars(P);
  const long N = P->nx;
  for (long i = 0; i < N; i++) {
    double q[OR_MAXS], g[OR_MAXS];
    for (int c = 0; c < s; c++) q[c] = u[c * N + i];
    flux_x_d(P, q, g);
    for (int c = 0; c < s; c++) f[c * N + i] = g[c];
  }
}

/* dt = CFL dx / s^max (1D; Sec. 5.1-5.3 state the CFL number). */
double or_dt_1d(const or_params *P, const double *u) {
  const int s = or_nvars(P);
  const long N = P->nx;
  const double dx = (P->x1 - P->x0) / (double)N;
  double smax = 0.0;
  for (long i = 0; i < N; i++) {
    double q[OR_MAXS];
    for (int c = 0; c < s; c++) q[c] = u[c * N + i];
    const double a = speed_d(P, q, 0);
    if (!(a <= smax)) smax = a; /* propagates NaN */
  }
  if (!(smax > 0.0) || isnan(smax) || isinf(smax)) return -1.0;
  return P->cfl * dx / smax;
}

/* dt = CFL/2 min(dx / s^max_x, dy / s^max_y) (Sec. 5.5). */
double or_dt_2d(const or_params *P, const double *u) {
  const int s = or_nvars(P);
  const long NX = P->nx, NY = P->ny, NC = NX * NY;
  const double dx = (P->x1 - P->x0) / (double)NX, dy = (P->y1 - P->y0) / (double)NY;
  double sx = 0.0, sy = 0.0;
  for (long i = 0; i < NC; i++) {
    double q[OR_MAXS];
    for (int c = 0; c < s; c++) q[c] = u[c * NC + i];
    const double a = speed_d(P, q, 0), b = speed_d(P, q, 1);
    if (!(a <= sx)) sx = a;
    if (!(b <= sy)) sy = b;
  }
  if (isnan(sx) || isnan(sy) || isinf(sx) || isinf(sy) || !(sx > 0.0 || sy > 0.0)) return -1.0;
  const double tx = sx > 0.0 ? dx / sx : INFINITY, ty = sy > 0.0 ? dy / sy : INFINITY;
  return (P->cfl / 2.0) * (tx < ty ? tx : ty);
}

static int or_check(const or_params *P) {
  if (P->P < 1 || P->P > OR_MAXP) return -1;
  if (P->flux < OR_LINEAR || P->flux > OR_EULER2D) return -1;
  if (P->nx < 2 || P->ny < 1) return -1;
  return 0;
}

int or_cat_flux_1d(const or_params *P, int p, const double *us, double dt, double dx, double *F) {
  if (p < 1 || p > OR_MAXP) return -1;
  or_tables T;
  or_fill_tables(&T, p);
  cat_flux_1d_d(P, &T, p, us, dt, dx, F);
  return 0;
}

int or_cat_flux_2d(const or_params *P, int p, const double *ub, double dt, double dx, double dy,
                   double *F, double *G) {
  if (p < 1 || p > OR_MAXP) return -1;
  or_tables T;
  or_fill_tables(&T, p);
  cat_flux_2d_d(P, &T, p, ub, dt, dx, dy, F, G);
  return 0;
}

/* The fluxes of the rectangular block S_{p1,p2} (Sec. 4, end). */
int or_cat_flux_2d_rect(const or_params *P, int p1, int p2, const double *ub, double dt, double dx,
                        double dy, double *F, double *G) {
  if (p1 < 1 || p1 > OR_MAXP || p2 < 1 || p2 > OR_MAXP) return -1;
  or_tables T;
  or_fill_tables(&T, p1 > p2 ? p1 : p2);
  cat_flux_2d_rect_d(P, &T, p1, p2, ub, dt, dx, dy, F, G);
  return 0;
}

/* One 1D step. *dt_io > 0 imposes dt; otherwise the CFL dt is computed and
 * returned there. orders: nx+1 codes; psi: (nx+1) x P values psi^1..psi^P
 * (psi^1 the limiter, psi^p the indicators); flux: (nx+1) x s. */
int or_step_1d(const or_params *P, const double *u, double *u_out, double *dt_io,
               int8_t *orders, double *psi, double *flux) {
  if (or_check(P)) return -1;
  double dt = *dt_io;
  if (!(dt > 0.0)) {
    dt = or_dt_1d(P, u);
    if (!(dt > 0.0)) return -2;
    *dt_io = dt;
  }
  return step_1d_d(P, u, u_out, dt, orders, psi, flux);
}

/* Fluxes at selected interfaces only (interface m between cells m-1, m). */
int or_fluxes_1d_at(const or_params *P, const double *u, double dt, int n, const int32_t *ifaces,
                    double *F, int8_t *orders) {
  if (or_check(P)) return -1;
  const int s = or_nvars(P), G = P->P > 2 ? P->P : 2;
  const double dx = (P->x1 - P->x0) / (double)P->nx;
  or_tables T;
  or_fill_tables(&T, P->P);
#pragma omp parallel for schedule(dynamic, 8)
  for (int q = 0; q < n; q++) {
    double line[OR_MAXS * 2 * OR_MAXP];
    gather_line_1d_d(P, u, (long)ifaces[q] - 1, G, line);
    int o = iface_1d_d(P, &T, line, line, G, dt, dx, F + (long)q * s, NULL);
    if (orders) orders[q] = (int8_t)o;
  }
  return 0;
}

/* u^{n+1} at selected cells only (Eq. 2.12 with the fluxes of its two
 * interfaces); out[q*s + c]. */
int or_step_1d_cells(const or_params *P, const double *u, double dt, int n, const int32_t *cells,
                     double *out) {
  if (or_check(P)) return -1;
  const int s = or_nvars(P), G = P->P > 2 ? P->P : 2;
  const long N = P->nx;
  const double dx = (P->x1 - P->x0) / (double)N;
  or_tables T;
  or_fill_tables(&T, P->P);
  const double lam = dt / dx;
#pragma omp parallel for schedule(dynamic, 8)
  for (int q = 0; q < n; q++) {
    const long i = cells[q];
    double line[OR_MAXS * 2 * OR_MAXP], fl[OR_MAXS], fr[OR_MAXS];
    gather_line_1d_d(P, u, i - 1, G, line);
    iface_1d_d(P, &T, line, line, G, dt, dx, fl, NULL);
    gather_line_1d_d(P, u, i, G, line);
    iface_1d_d(P, &T, line, line, G, dt, dx, fr, NULL);
    for (int c = 0; c < s; c++) out[(long)q * s + c] = u[c * N + i] + lam * (fl[c] - fr[c]);
  }
  return 0;
}

/* Complex-step evaluation of one 1D step at fixed dt (all branches are taken
 * on the real parts). */
int or_step_1d_z(const or_params *P, const double *u_re, const double *u_im, double dt,
                 double *out_re, double *out_im) {
  if (or_check(P)) return -1;
  const long M = (long)P->nx * or_nvars(P);
  double complex *a = malloc(sizeof(double complex) * (size_t)M);
  double complex *b = malloc(sizeof(double complex) * (size_t)M);
  if (!a || !b) { free(a); free(b); return -3; }
  for (long q = 0; q < M; q++) a[q] = u_re[q] + I * u_im[q];
  int rc = step_1d_z(P, a, b, dt, NULL, NULL, NULL);
  for (long q = 0; q < M; q++) { out_re[q] = creal(b[q]); out_im[q] = cimag(b[q]); }
  free(a);
  free(b);
  return rc;
}

int or_step_2d(const or_params *P, const double *u, double *u_out, double *dt_io, int8_t *ord_x,
               int8_t *ord_y) {
  if (or_check(P)) return -1;
  double dt = *dt_io;
  if (!(dt > 0.0)) {
    dt = or_dt_2d(P, u);
    if (!(dt > 0.0)) return -2;
    *dt_io = dt;
  }
  return step_2d_d(P, u, u_out, dt, ord_x, ord_y);
}

/* u^{n+1} at selected cells (cx[q], cy[q]) only; out[q*s + c]. */
int or_step_2d_cells(const or_params *P, const double *u, double dt, int n, const int32_t *cx,
                     const int32_t *cy, double *out) {
  if (or_check(P)) return -1;
  const int s = or_nvars(P);
  const long NX = P->nx, NY = P->ny;
  const double dx = (P->x1 - P->x0) / (double)NX, dy = (P->y1 - P->y0) / (double)NY;
  or_tables T;
  or_fill_tables(&T, P->P);
  const double lx = dt / dx, ly = dt / dy;
#pragma omp parallel for schedule(dynamic, 4)
  for (int q = 0; q < n; q++) {
    const long x = cx[q], y = cy[q];
    double fl[OR_MAXS], fr[OR_MAXS], gb[OR_MAXS], gt[OR_MAXS];
    iface_2d_d(P, &T, u, x - 1, y, 0, dt, dx, dy, fl);
    iface_2d_d(P, &T, u, x, y, 0, dt, dx, dy, fr);
    iface_2d_d(P, &T, u, x, y - 1, 1, dt, dx, dy, gb);
    iface_2d_d(P, &T, u, x, y, 1, dt, dx, dy, gt);
    for (int c = 0; c < s; c++) {
      const double u0 = u[((long)c * NY + y) * NX + x];
      out[(long)q * s + c] = u0 + lx * (fl[c] - fr[c]) + ly * (gb[c] - gt[c]);
    }
  }
  return 0;
}

void or_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

int or_get_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
