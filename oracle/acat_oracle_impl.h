/*
 * acat_oracle_impl.h -- generic core of the ACAT CPU oracle.
 *
 * TEST INFRASTRUCTURE (see acat_oracle.h). Included twice by acat_oracle.c:
 *   R = double          (SFX _d)  the oracle proper;
 *   R = double complex  (SFX _z)  the same step evaluated on complex states,
 *                                 used for complex-step derivatives. Every
 *                                 discrete choice (order, limiter piece,
 *                                 upwind side, component minimum, Rusanov
 *                                 maximum) is taken on real parts, so a
 *                                 complex perturbation differentiates the step
 *                                 with those choices frozen.
 * Macros expected: R, RE(x), SQRT_R(x), SFX.
 *
 * Everything follows the paper in its own notation and order; nothing is
 * blocked, fused or rescaled.
 */

#define CAT_(a, b) a##b
#define CAT(a, b) CAT_(a, b)
#define FN(name) CAT(name, SFX)

static R FN(rabs)(R x) { return RE(x) < 0.0 ? -x : x; }

/* x-flux f(u) and y-flux g(u): Sec. 5 (Eq. 5.1 linear transport, Eq. 5.13
 * its 2D form, Eq. 5.5 Burgers, Eqs. 5.6-5.9 1D Euler with the ideal-gas law,
 * Eqs. 5.15-5.16 2D Euler). */
static void FN(flux_x)(const or_params *P, const R *u, R *f) {
  switch (P->flux) {
  case OR_LINEAR: f[0] = P->adv[0] * u[0]; break;
  case OR_BURGERS: f[0] = 0.5 * u[0] * u[0]; break;
  case OR_EULER1D: {
    R rho = u[0], m = u[1], E = u[2];
    R v = m / rho;
    R p = (P->gamma - 1.0) * (E - 0.5 * rho * v * v);
    f[0] = m;
    f[1] = m * v + p;
    f[2] = v * (E + p);
  } break;
  default: {
    R rho = u[0], mx = u[1], my = u[2], E = u[3];
    R v = mx / rho, w = my / rho;
    R p = (P->gamma - 1.0) * (E - 0.5 * rho * (v * v + w * w));
    f[0] = mx;
    f[1] = mx * v + p;
    f[2] = mx * w;
    f[3] = v * (E + p);
  } break;
  }
}

static void FN(flux_y)(const or_params *P, const R *u, R *g) {
  switch (P->flux) {
  case OR_LINEAR: g[0] = P->adv[1] * u[0]; break;
  case OR_BURGERS: g[0] = 0.5 * u[0] * u[0]; break;
  case OR_EULER2D: {
    R rho = u[0], mx = u[1], my = u[2], E = u[3];
    R v = mx / rho, w = my / rho;
    R p = (P->gamma - 1.0) * (E - 0.5 * rho * (v * v + w * w));
    g[0] = my;
    g[1] = my * v;
    g[2] = my * w + p;
    g[3] = w * (E + p);
  } break;
  default: g[0] = 0.0; g[1] = 0.0; g[2] = 0.0; break;
  }
}

/* Spectral radius of the flux Jacobian in direction dir (0: x, 1: y):
 * |a| for transport, |u| for Burgers, |v| + c with c = sqrt(gamma p / rho)
 * for Euler (Sec. 5.5, definition of s^max). */
static R FN(speed)(const or_params *P, const R *u, int dir) {
  switch (P->flux) {
  case OR_LINEAR: return fabs(P->adv[dir]);
  case OR_BURGERS: return FN(rabs)(u[0]);
  case OR_EULER1D: {
    R rho = u[0], m = u[1], E = u[2];
    R v = m / rho;
    R p = (P->gamma - 1.0) * (E - 0.5 * rho * v * v);
    return FN(rabs)(v) + SQRT_R(P->gamma * p / rho);
  }
  default: {
    R rho = u[0], mx = u[1], my = u[2], E = u[3];
    R v = mx / rho, w = my / rho;
    R p = (P->gamma - 1.0) * (E - 0.5 * rho * (v * v + w * w));
    R vn = dir == 0 ? v : w;
    return FN(rabs)(vn) + SQRT_R(P->gamma * p / rho);
  }
  }
}

static void FN(flux_dir)(const or_params *P, const R *u, R *f, int dir) {
  if (dir == 0) FN(flux_x)(P, u, f); else FN(flux_y)(P, u, f);
}

/* ---------------------------------------------------------------------------
 * CAT2p numerical flux, 1D (Sec. 2.2: Eq. 2.14 with the local approximations
 * of Eq. 2.15 built by the three-step recursion that follows it).
 *   us[c*2p + r] holds u^n_{i+j}, node j = r - p + 1, j = -p+1..p.
 * ------------------------------------------------------------------------- */
static void FN(cat_flux_1d)(const or_params *P, const or_tables *T, int p,
                            const R *us, double dt, double dx, R *F) {
  const int n = 2 * p, s = or_nvars(P);
  R ft[OR_MAXS][OR_MAXN];               /* f~^{(k-1)}_{i,j}                 */
  R nf[OR_MAXS][OR_MAXN];
  R ut[OR_MAXN][OR_MAXS][OR_MAXN];      /* u~^{(l)}_{i,j}, l = 1..2p-1       */
  R st[OR_MAXS], fr[OR_MAXS];

  /* step 1: f~^{(0)}_{i,j} = f(u^n_{i+j}) */
  for (int j = 0; j < n; j++) {
    for (int c = 0; c < s; c++) st[c] = us[c * n + j];
    FN(flux_x)(P, st, fr);
    for (int c = 0; c < s; c++) ft[c][j] = fr[c];
  }
  /* k = 1 term of Eq. 2.14: dt^0/1! A^{0,1/2}_{p,0}(f~^{(0)}) */
  for (int c = 0; c < s; c++) {
    R a = 0.0;
    for (int j = 0; j < n; j++) a = a + T->gh[p][j] * ft[c][j];
    F[c] = a;
  }
  double dtk = 1.0, kfact = 1.0;
  for (int k = 2; k <= n; k++) {
    /* (a) u~^{(k-1)}_{i,j} = -A^{1,j}_{p,0}(f~^{(k-2)}_{i,*}, dx) */
    for (int j = 0; j < n; j++)
      for (int c = 0; c < s; c++) {
        R a = 0.0;
        for (int r = 0; r < n; r++) a = a + T->g1[p][j][r] * ft[c][r];
        ut[k - 1][c][j] = -(a / dx);
      }
    dtk = dtk * dt;          /* dt^(k-1) */
    kfact = kfact * k;       /* k!       */
    /* (b) f~^{k-1,n+r}_{i,j} = f(u^n_{i+j} + sum_l (r dt)^l / l! u~^{(l)}_{i,j})
     * (c) f~^{(k-1)}_{i,j}  = A^{k-1,0}_{p,n}(f~^{k-1,*}_{i,j}, dt)          */
    for (int j = 0; j < n; j++) {
      R acc[OR_MAXS];
      for (int c = 0; c < s; c++) acc[c] = 0.0;
      for (int rr = 0; rr < n; rr++) {
        const double rdt = (double)(rr - p + 1) * dt;
        for (int c = 0; c < s; c++) {
          R v = us[c * n + j];
          double pw = 1.0, lf = 1.0;
          for (int l = 1; l <= k - 1; l++) {
            pw = pw * rdt;
            lf = lf * l;
            v = v + (pw / lf) * ut[l][c][j];
          }
          st[c] = v;
        }
        FN(flux_x)(P, st, fr);
        for (int c = 0; c < s; c++) acc[c] = acc[c] + T->gk[p][k - 1][rr] * fr[c];
      }
      for (int c = 0; c < s; c++) nf[c][j] = acc[c] / dtk;
    }
    for (int c = 0; c < s; c++)
      for (int j = 0; j < n; j++) ft[c][j] = nf[c][j];
    /* term k of Eq. 2.14: dt^{k-1}/k! A^{0,1/2}_{p,0}(f~^{(k-1)}) */
    for (int c = 0; c < s; c++) {
      R a = 0.0;
      for (int j = 0; j < n; j++) a = a + T->gh[p][j] * ft[c][j];
      F[c] = F[c] + (dtk / kfact) * a;
    }
  }
}

/* ---------------------------------------------------------------------------
 * CAT2p numerical fluxes, 2D (Sec. 4: the recursion on the block anchored at
 * the corner x_{i+1/2}, Eqs. 4.5-4.6), on the rectangular block S_{p1,p2}:
 * 2 p1 nodes in x (j1 = -p1+1..p1), 2 p2 nodes in y (j2 = -p2+1..p2).
 *   ub[(c*2p2 + b)*2p1 + a] holds u^n_{i+j}, j = (a - p1 + 1, b - p2 + 1).
 * x-derivatives take the 2 p1-point weights of the rows, y-derivatives the
 * 2 p2-point weights of the columns. The time derivatives take the 2 pm time
 * nodes r = -pm+1..pm, pm = max(p1, p2), and the recursion runs to k = 2 pm.
 * F^{p1} is taken along the row j2 = 0 with the sum to k = 2 p1, G^{p2} along
 * the column j1 = 0 with the sum to k = 2 p2. With p1 = p2 = p this is the
 * square block S_p of the paper, operation for operation.
 * ------------------------------------------------------------------------- */
static void FN(cat_flux_2d_rect)(const or_params *P, const or_tables *T, int p1, int p2,
                                 const R *ub, double dt, double dx, double dy,
                                 R *F, R *G) {
  const int n1 = 2 * p1, n2 = 2 * p2, s = or_nvars(P);
  const int pm = p1 > p2 ? p1 : p2, n = 2 * pm;
  const int z1 = p1 - 1, z2 = p2 - 1, zt = pm - 1; /* local indices of j1 = 0, j2 = 0, r = 0 */
  R ft[OR_MAXS][OR_MAXN][OR_MAXN], gt[OR_MAXS][OR_MAXN][OR_MAXN]; /* [c][b][a] */
  R nf[OR_MAXS][OR_MAXN][OR_MAXN], ng[OR_MAXS][OR_MAXN][OR_MAXN];
  R ut[OR_MAXN][OR_MAXS][OR_MAXN][OR_MAXN];
  R st[OR_MAXS], fr[OR_MAXS], gr[OR_MAXS];
  (void)zt;

  for (int b = 0; b < n2; b++)
    for (int a = 0; a < n1; a++) {
      for (int c = 0; c < s; c++) st[c] = ub[(c * n2 + b) * n1 + a];
      FN(flux_x)(P, st, fr);
      FN(flux_y)(P, st, gr);
      for (int c = 0; c < s; c++) { ft[c][b][a] = fr[c]; gt[c][b][a] = gr[c]; }
    }
  for (int c = 0; c < s; c++) {
    R a1 = 0.0, a2 = 0.0;
    for (int l = 0; l < n1; l++) a1 = a1 + T->gh[p1][l] * ft[c][z2][l];
    for (int l = 0; l < n2; l++) a2 = a2 + T->gh[p2][l] * gt[c][l][z1];
    F[c] = a1;
    G[c] = a2;
  }
  double dtk = 1.0, kfact = 1.0;
  for (int k = 2; k <= n; k++) {
    /* (a) u~^{(k-1)} = -A^{1,j1}_{p1,0}(f~^{(k-2)}_{(*,j2)}, dx)
     *                  -A^{1,j2}_{p2,0}(g~^{(k-2)}_{(j1,*)}, dy)          */
    for (int b = 0; b < n2; b++)
      for (int a = 0; a < n1; a++)
        for (int c = 0; c < s; c++) {
          R sx = 0.0, sy = 0.0;
          for (int l = 0; l < n1; l++) sx = sx + T->g1[p1][a][l] * ft[c][b][l];
          for (int l = 0; l < n2; l++) sy = sy + T->g1[p2][b][l] * gt[c][l][a];
          ut[k - 1][c][b][a] = -(sx / dx) - (sy / dy);
        }
    dtk = dtk * dt;
    kfact = kfact * k;
    /* (b), (c) for f and g, time nodes r = -pm+1..pm */
    for (int b = 0; b < n2; b++)
      for (int a = 0; a < n1; a++) {
        R af[OR_MAXS], ag[OR_MAXS];
        for (int c = 0; c < s; c++) { af[c] = 0.0; ag[c] = 0.0; }
        for (int rr = 0; rr < n; rr++) {
          const double rdt = (double)(rr - pm + 1) * dt;
          for (int c = 0; c < s; c++) {
            R v = ub[(c * n2 + b) * n1 + a];
            double pw = 1.0, lf = 1.0;
            for (int l = 1; l <= k - 1; l++) {
              pw = pw * rdt;
              lf = lf * l;
              v = v + (pw / lf) * ut[l][c][b][a];
            }
            st[c] = v;
          }
          FN(flux_x)(P, st, fr);
          FN(flux_y)(P, st, gr);
          for (int c = 0; c < s; c++) {
            af[c] = af[c] + T->gk[pm][k - 1][rr] * fr[c];
            ag[c] = ag[c] + T->gk[pm][k - 1][rr] * gr[c];
          }
        }
        for (int c = 0; c < s; c++) {
          nf[c][b][a] = af[c] / dtk;
          ng[c][b][a] = ag[c] / dtk;
        }
      }
    for (int c = 0; c < s; c++)
      for (int b = 0; b < n2; b++)
        for (int a = 0; a < n1; a++) { ft[c][b][a] = nf[c][b][a]; gt[c][b][a] = ng[c][b][a]; }
    for (int c = 0; c < s; c++) {
      if (k <= n1) {
        R a1 = 0.0;
        for (int l = 0; l < n1; l++) a1 = a1 + T->gh[p1][l] * ft[c][z2][l];
        F[c] = F[c] + (dtk / kfact) * a1;
      }
      if (k <= n2) {
        R a2 = 0.0;
        for (int l = 0; l < n2; l++) a2 = a2 + T->gh[p2][l] * gt[c][l][z1];
        G[c] = G[c] + (dtk / kfact) * a2;
      }
    }
  }
}

/* The square block S_p of Eqs. 4.5-4.6. */
static void FN(cat_flux_2d)(const or_params *P, const or_tables *T, int p,
                            const R *ub, double dt, double dx, double dy,
                            R *F, R *G) {
  FN(cat_flux_2d_rect)(P, T, p, p, ub, dt, dx, dy, F, G);
}

/* ---------------------------------------------------------------------------
 * Flux limiter psi^1 (Sec. 3.1). line[c*LW + q] holds the cells along the
 * direction, with q = ic the cell i left of the interface.
 * Scalar laws: Roe intermediate speed chooses r^- or r^+ (Eq. 3.6);
 * systems: min(psi(r^+), psi(r^-)) per component, then min over components
 * (Eq. 3.7 and Sec. 3.4). The superbee limiter is used (Sec. 5).
 * ------------------------------------------------------------------------- */
static R FN(ratio)(R upw, R loc) {
  if (RE(loc) == 0.0) {
    if (RE(upw) == 0.0) return 1.0;
    return RE(upw) > 0.0 ? (R)INFINITY : (R)(-INFINITY);
  }
  return upw / loc;
}

static R FN(superbee)(R r) {
  R a = RE(2.0 * r) < 1.0 ? 2.0 * r : (R)1.0; /* min(2r, 1) */
  R b = RE(r) < 2.0 ? r : (R)2.0;             /* min(r, 2)  */
  R m = RE(a) > RE(b) ? a : b;                /* max        */
  return RE(m) > 0.0 ? m : (R)0.0;            /* max(0, .)  */
}

static R FN(psi1)(const or_params *P, const R *line, int LW, int ic, int dir) {
  const int s = or_nvars(P);
  if (s == 1 && P->limiter_form == 0) {
    R um = line[ic - 1], u0 = line[ic], u1 = line[ic + 1], u2 = line[ic + 2];
    /* Roe speed a_{i+1/2}; its sign only picks the upwind side */
    double a;
    double r0 = RE(u0), r1 = RE(u1);
    if (r0 != r1) {
      double f0, f1;
      if (P->flux == OR_LINEAR) { f0 = P->adv[dir] * r0; f1 = P->adv[dir] * r1; }
      else { f0 = 0.5 * r0 * r0; f1 = 0.5 * r1 * r1; }
      a = (f1 - f0) / (r1 - r0);
    } else {
      a = (P->flux == OR_LINEAR) ? P->adv[dir] : r0;
    }
    R upw = (a > 0.0) ? u0 - um : u2 - u1;
    return FN(superbee)(FN(ratio)(upw, u1 - u0));
  }
  R best = 2.0;
  for (int c = 0; c < s; c++) {
    const R *q = line + c * LW;
    R loc = q[ic + 1] - q[ic];
    R pm = FN(superbee)(FN(ratio)(q[ic] - q[ic - 1], loc));
    R pp = FN(superbee)(FN(ratio)(q[ic + 2] - q[ic + 1], loc));
    R v = RE(pp) < RE(pm) ? pp : pm;
    if (RE(v) < RE(best)) best = v;
  }
  return best;
}

/* Smallest and largest eigenvalue of the flux Jacobian in direction dir:
 * a (transport), u (Burgers), v_n -/+ c (Euler). */
static void FN(eig_bounds)(const or_params *P, const R *u, int dir, R *lmin, R *lmax) {
  switch (P->flux) {
  case OR_LINEAR: *lmin = *lmax = P->adv[dir]; return;
  case OR_BURGERS: *lmin = *lmax = u[0]; return;
  case OR_EULER1D: {
    R rho = u[0], m = u[1], E = u[2];
    R v = m / rho;
    R p = (P->gamma - 1.0) * (E - 0.5 * rho * v * v);
    R c = SQRT_R(P->gamma * p / rho);
    *lmin = v - c;
    *lmax = v + c;
    return;
  }
  default: {
    R rho = u[0], mx = u[1], my = u[2], E = u[3];
    R v = mx / rho, w = my / rho;
    R p = (P->gamma - 1.0) * (E - 0.5 * rho * (v * v + w * w));
    R vn = dir == 0 ? v : w;
    R c = SQRT_R(P->gamma * p / rho);
    *lmin = vn - c;
    *lmax = vn + c;
    return;
  }
  }
}

/* Robust first-order flux F^lo of Eq. 3.4 (left unspecified there), between
 * the states ul, ur in direction dir; h = dx or dy. lo_flux selects
 *   0: Rusanov (local Lax-Friedrichs), 1/2 (f_l + f_r) - 1/2 alpha (u_r - u_l),
 *      alpha the larger spectral radius of the two states (the default reading);
 *   1: global Lax-Friedrichs, the same with alpha = h / dt;
 *   2: HLL with the wave-speed bounds s_l = min of the two states' smallest
 *      eigenvalues, s_r = max of their largest:
 *      f_l if s_l >= 0, f_r if s_r <= 0, otherwise
 *      (s_r f_l - s_l f_r + s_l s_r (u_r - u_l)) / (s_r - s_l).
 * The LF and HLL schemes are the first-order comparisons of Sec. 5. */
static void FN(flux_lo)(const or_params *P, const R *ul, const R *ur, int dir, double dt, double h,
                        R *F) {
  const int s = or_nvars(P);
  R fl[OR_MAXS], fq[OR_MAXS];
  FN(flux_dir)(P, ul, fl, dir);
  FN(flux_dir)(P, ur, fq, dir);
  if (P->lo_flux == 2) {
    R al, bl, ar, br;
    FN(eig_bounds)(P, ul, dir, &al, &bl);
    FN(eig_bounds)(P, ur, dir, &ar, &br);
    R sl = RE(ar) < RE(al) ? ar : al;
    R sr = RE(br) > RE(bl) ? br : bl;
    if (RE(sl) >= 0.0) {
      for (int c = 0; c < s; c++) F[c] = fl[c];
    } else if (RE(sr) <= 0.0) {
      for (int c = 0; c < s; c++) F[c] = fq[c];
    } else {
      for (int c = 0; c < s; c++)
        F[c] = (sr * fl[c] - sl * fq[c] + sl * sr * (ur[c] - ul[c])) / (sr - sl);
    }
    return;
  }
  R alpha;
  if (P->lo_flux == 1) {
    alpha = h / dt;
  } else {
    R al = FN(speed)(P, ul, dir), ar = FN(speed)(P, ur, dir);
    alpha = RE(ar) > RE(al) ? ar : al;
  }
  for (int c = 0; c < s; c++) F[c] = 0.5 * (fl[c] + fq[c]) - 0.5 * alpha * (ur[c] - ul[c]);
}

/* 1D interface between cells i and i+1: order selection (Eqs. 3.2-3.3 with
 * the indicators of Eqs. 3.8-3.12 and Sec. 3.4), then CAT2p_s or FL-CAT2
 * (Eq. 3.4). line[c*LW + q]: cells i-G+1..i+G, cell i at q = G-1. */
static int FN(iface_1d)(const or_params *P, const or_tables *T, const R *line,
                        const double *line_re, int G, double dt, double dx,
                        R *F, double *psi) {
  const int s = or_nvars(P), LW = 2 * G, ic = G - 1;
  const int ps = or_select(P, T, line_re, LW, ic, 1, psi);
  if (ps >= 2) {
    R us[OR_MAXS * OR_MAXN];
    const int n = 2 * ps;
    for (int c = 0; c < s; c++)
      for (int r = 0; r < n; r++) us[c * n + r] = line[c * LW + ic - ps + 1 + r];
    FN(cat_flux_1d)(P, T, ps, us, dt, dx, F);
    if (psi) psi[1] = RE(FN(psi1)(P, line, LW, ic, 0));
    return ps;
  }
  R us[OR_MAXS * 2], F1[OR_MAXS], Flo[OR_MAXS], ul[OR_MAXS], ur[OR_MAXS];
  for (int c = 0; c < s; c++) {
    us[c * 2 + 0] = line[c * LW + ic];
    us[c * 2 + 1] = line[c * LW + ic + 1];
    ul[c] = line[c * LW + ic];
    ur[c] = line[c * LW + ic + 1];
  }
  FN(cat_flux_1d)(P, T, 1, us, dt, dx, F1);
  FN(flux_lo)(P, ul, ur, 0, dt, dx, Flo);
  R w = FN(psi1)(P, line, LW, ic, 0);
  if (psi) psi[1] = RE(w);
  for (int c = 0; c < s; c++) F[c] = w * F1[c] + (1.0 - w) * Flo[c];
  return 1;
}

static void FN(gather_line_1d)(const or_params *P, const R *u, long i, int G, R *line) {
  const int s = or_nvars(P), LW = 2 * G;
  const long N = P->nx;
  for (int c = 0; c < s; c++)
    for (int q = 0; q < LW; q++) line[c * LW + q] = u[c * N + or_bc_map(P->bc, i - G + 1 + q, N)];
}

/* One ACAT2P step, 1D (Eq. 3.19, conservative form Eq. 2.12). */
static int FN(step_1d)(const or_params *P, const R *u, R *u_out, double dt,
                       int8_t *orders, double *psi, R *flux) {
  const int s = or_nvars(P), G = P->P > 2 ? P->P : 2;
  const long N = P->nx;
  const double dx = (P->x1 - P->x0) / (double)N;
  or_tables T;
  or_fill_tables(&T, P->P);
  R *F = (R *)malloc(sizeof(R) * (size_t)(N + 1) * (size_t)s);
  if (!F) return -3;
#pragma omp parallel for schedule(dynamic, 64)
  for (long m = 0; m <= N; m++) {
    R line[OR_MAXS * 2 * OR_MAXP];
    double line_re[OR_MAXS * 2 * OR_MAXP];
    double ps[OR_MAXP + 1];
    FN(gather_line_1d)(P, u, m - 1, G, line);
    for (int q = 0; q < s * 2 * G; q++) line_re[q] = RE(line[q]);
    int o = FN(iface_1d)(P, &T, line, line_re, G, dt, dx, F + m * s, psi ? ps : NULL);
    if (orders) orders[m] = (int8_t)o;
    if (psi)
      for (int p = 1; p <= P->P; p++) psi[m * P->P + (p - 1)] = ps[p];
  }
  const double lam = dt / dx;
  for (int c = 0; c < s; c++)
    for (long i = 0; i < N; i++)
      u_out[c * N + i] = u[c * N + i] + lam * (F[i * s + c] - F[(i + 1) * s + c]);
  if (flux)
    for (long q = 0; q < (N + 1) * s; q++) flux[q] = F[q];
  free(F);
  return 0;
}

/* 2D: gather the line through (x, y) along dir, G cells either side of the
 * interface, and the 2p x 2p block anchored at (x, y). */
static void FN(gather_line_2d)(const or_params *P, const R *u, long x, long y, int dir,
                               int G, R *line) {
  const int s = or_nvars(P), LW = 2 * G;
  const long NX = P->nx, NY = P->ny;
  for (int c = 0; c < s; c++)
    for (int q = 0; q < LW; q++) {
      long xx = dir == 0 ? x - G + 1 + q : x, yy = dir == 0 ? y : y - G + 1 + q;
      line[c * LW + q] = u[((long)c * NY + or_bc_map(P->bc, yy, NY)) * NX + or_bc_map(P->bc, xx, NX)];
    }
}

static void FN(gather_block_2d_rect)(const or_params *P, const R *u, long x, long y, int p1, int p2, R *ub) {
  const int s = or_nvars(P), n1 = 2 * p1, n2 = 2 * p2;
  const long NX = P->nx, NY = P->ny;
  for (int c = 0; c < s; c++)
    for (int b = 0; b < n2; b++)
      for (int a = 0; a < n1; a++)
        ub[(c * n2 + b) * n1 + a] =
            u[((long)c * NY + or_bc_map(P->bc, y - p2 + 1 + b, NY)) * NX + or_bc_map(P->bc, x - p1 + 1 + a, NX)];
}

static void FN(gather_block_2d)(const or_params *P, const R *u, long x, long y, int p, R *ub) {
  FN(gather_block_2d_rect)(P, u, x, y, p, p, ub);
}

/* 2D interface flux anchored at cell (x, y): dir 0 gives F at (x+1/2, y),
 * dir 1 gives G at (x, y+1/2): orders from the dimension-by-dimension
 * admissible sets A_1, A_2 of Sec. 4, FL-CAT2 per direction from the 2D CAT2
 * flux (Eqs. 4.3-4.4) blended as in Eqs. 4.7-4.8. */
static int FN(iface_2d)(const or_params *P, const or_tables *T, const R *u, long x, long y,
                        int dir, double dt, double dx, double dy, R *out) {
  const int s = or_nvars(P), G = P->P > 2 ? P->P : 2, LW = 2 * G, ic = G - 1;
  R line[OR_MAXS * 2 * OR_MAXP];
  double line_re[OR_MAXS * 2 * OR_MAXP];
  FN(gather_line_2d)(P, u, x, y, dir, G, line);
  for (int q = 0; q < s * LW; q++) line_re[q] = RE(line[q]);
  const int ps = or_select(P, T, line_re, LW, ic, 1, NULL);
  R ub[OR_MAXS * OR_MAXN * OR_MAXN], F[OR_MAXS], Gf[OR_MAXS];
  if (ps >= 2) {
    if (P->rect_2d) {
      /* the other direction's order at the same anchor (1 on FL-CAT2) gives
       * the block's extent across this direction */
      R oline[OR_MAXS * 2 * OR_MAXP];
      double oline_re[OR_MAXS * 2 * OR_MAXP];
      FN(gather_line_2d)(P, u, x, y, 1 - dir, G, oline);
      for (int q = 0; q < s * LW; q++) oline_re[q] = RE(oline[q]);
      const int po = or_select(P, T, oline_re, LW, ic, 1, NULL);
      const int p1 = dir == 0 ? ps : po, p2 = dir == 0 ? po : ps;
      FN(gather_block_2d_rect)(P, u, x, y, p1, p2, ub);
      FN(cat_flux_2d_rect)(P, T, p1, p2, ub, dt, dx, dy, F, Gf);
    } else {
      FN(gather_block_2d)(P, u, x, y, ps, ub);
      FN(cat_flux_2d)(P, T, ps, ub, dt, dx, dy, F, Gf);
    }
    for (int c = 0; c < s; c++) out[c] = dir == 0 ? F[c] : Gf[c];
    return ps;
  }
  FN(gather_block_2d)(P, u, x, y, 1, ub);
  FN(cat_flux_2d)(P, T, 1, ub, dt, dx, dy, F, Gf);
  R ul[OR_MAXS], ur[OR_MAXS], lo[OR_MAXS];
  for (int c = 0; c < s; c++) { ul[c] = line[c * LW + ic]; ur[c] = line[c * LW + ic + 1]; }
  FN(flux_lo)(P, ul, ur, dir, dt, dir == 0 ? dx : dy, lo);
  R w = FN(psi1)(P, line, LW, ic, dir);
  for (int c = 0; c < s; c++) out[c] = w * (dir == 0 ? F[c] : Gf[c]) + (1.0 - w) * lo[c];
  return 1;
}

/* One 2D ACAT2P step (Eq. 4.9). */
static int FN(step_2d)(const or_params *P, const R *u, R *u_out, double dt,
                       int8_t *ordx, int8_t *ordy) {
  const int s = or_nvars(P);
  const long NX = P->nx, NY = P->ny;
  const double dx = (P->x1 - P->x0) / (double)NX, dy = (P->y1 - P->y0) / (double)NY;
  or_tables T;
  or_fill_tables(&T, P->P);
  R *Fx = (R *)malloc(sizeof(R) * (size_t)(NX + 1) * (size_t)NY * (size_t)s);
  R *Gy = (R *)malloc(sizeof(R) * (size_t)NX * (size_t)(NY + 1) * (size_t)s);
  if (!Fx || !Gy) { free(Fx); free(Gy); return -3; }
#pragma omp parallel for schedule(dynamic, 16)
  for (long y = 0; y < NY; y++)
    for (long m = 0; m <= NX; m++) {
      int o = FN(iface_2d)(P, &T, u, m - 1, y, 0, dt, dx, dy, Fx + (y * (NX + 1) + m) * s);
      if (ordx) ordx[y * (NX + 1) + m] = (int8_t)o;
    }
#pragma omp parallel for schedule(dynamic, 16)
  for (long m = 0; m <= NY; m++)
    for (long x = 0; x < NX; x++) {
      int o = FN(iface_2d)(P, &T, u, x, m - 1, 1, dt, dx, dy, Gy + (m * NX + x) * s);
      if (ordy) ordy[m * NX + x] = (int8_t)o;
    }
  const double lx = dt / dx, ly = dt / dy;
  for (int c = 0; c < s; c++)
    for (long y = 0; y < NY; y++)
      for (long x = 0; x < NX; x++) {
        R fl = Fx[(y * (NX + 1) + x) * s + c], fr = Fx[(y * (NX + 1) + x + 1) * s + c];
        R gb = Gy[(y * NX + x) * s + c], gt = Gy[((y + 1) * NX + x) * s + c];
        const long q = ((long)c * NY + y) * NX + x;
        u_out[q] = u[q] + lx * (fl - fr) + ly * (gb - gt);
      }
  free(Fx);
  free(Gy);
  return 0;
}

#undef FN
