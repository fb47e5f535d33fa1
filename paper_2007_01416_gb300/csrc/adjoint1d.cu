// adjoint1d.cu -- hand-written adjoint (transposed Jacobian) of one 1D ACAT
// step, FP64 and FP32 (compensated state and cotangent).
//
// The step u^{n+1} = u^n + lambda (F_{i-1/2} - F_{i+1/2}) is differentiated
// with its discrete choices frozen at u^n: the selected order of every
// interface, and for FL-CAT2 interfaces the superbee piece, the upwind side
// (scalar laws) or the (component, side) attaining the limiter minimum
// (systems) and the cell attaining the Rusanov maximum. dt is a constant (the
// value the forward step used). The adjoint kernel recomputes the forward
// quantities from u^n with the forward's own code, so the frozen choices are
// exactly the forward's.
//
// Given ubar^{n+1}, interface m (between cells m-1 and m) receives
// Fbar_m = lambda (ubar_m - ubar_{m-1}) (cells outside 0..N-1 contribute
// nothing); each interface then propagates Fbar_m back through its flux:
//   - CAT2p: a reverse sweep of the local recursion (Sec. 2.2) with one lane
//     per stencil node, the forward's U^(k) kept in registers and the Taylor
//     arguments recomputed in the forward's order; the spatial derivative is
//     transposed with shuffles (lane j gathers sum_i gamma^{1,i}_j Ubar_i);
//   - FL-CAT2: the blend, the CAT2 recursion, Rusanov and the limiter, on one
//     lane.
// Each interface writes the cotangent of every stencil node to a scratch
// array, and a gather kernel sums, for every cell, the contributions of all
// (interface, node) pairs whose position maps to it through the boundary
// condition (the adjoint of the ghost fill), in a fixed order.
#include "phys1d.cuh"

namespace {

// out += J_f(u)^T y and the gradient of the spectral radius.
template <int FLUX>
struct Jac;

template <>
struct Jac<ACAT_FLUX_LINEAR> {
  template <typename R>
  __device__ static void jt(const R *, const R *y, R *out, R a, R) {
    out[0] += a * y[0];
  }
  __device__ static void grad_speed(const double *, double, double *g) { g[0] = 0.0; }
  // gradients of the smallest and largest eigenvalue (HLL wave-speed bounds)
  __device__ static void grad_eig(const double *, double, double *gmin, double *gmax) { gmin[0] = gmax[0] = 0.0; }
};

template <>
struct Jac<ACAT_FLUX_BURGERS> {
  template <typename R>
  __device__ static void jt(const R *u, const R *y, R *out, R, R) {
    out[0] += u[0] * y[0];
  }
  __device__ static void grad_speed(const double *u, double, double *g) { g[0] = u[0] < 0.0 ? -1.0 : 1.0; }
  __device__ static void grad_eig(const double *, double, double *gmin, double *gmax) { gmin[0] = gmax[0] = 1.0; }
};

template <>
struct Jac<ACAT_FLUX_EULER1D> {
  // f = (m, m v + p, v (E + p)), v = m / rho, p = (gamma - 1)(E - m v / 2):
  // df1 = ((gm1 - 2) v^2 / 2, (2 - gm1) v, gm1),
  // df2 = (v (gm1 v^2 / 2 - H), H - gm1 v^2, gamma v), H = (E + p) / rho.
  template <typename R>
  __device__ static void jt(const R *u, const R *y, R *out, R, R gm1) {
    const R ri = recip(u[0]);  // FP64: within an ulp of 1/rho; float: the hardware approximation
    const R v = u[1] * ri;
    const R p = gm1 * (u[2] - R(0.5) * u[1] * v);
    const R H = (u[2] + p) * ri;
    out[0] += y[1] * (R(0.5) * (gm1 - R(2)) * v * v) + y[2] * (v * (R(0.5) * gm1 * v * v - H));
    out[1] += y[0] + y[1] * ((R(2) - gm1) * v) + y[2] * (H - gm1 * v * v);
    out[2] += y[1] * gm1 + y[2] * ((R(1) + gm1) * v);
  }
  // s = |v| + c, c = sqrt(gamma p / rho)
  __device__ static void grad_speed(const double *u, double gamma, double *g) {
    const double gm1 = gamma - 1.0;
    const double ri = 1.0 / u[0];
    const double v = u[1] * ri;
    const double p = gm1 * (u[2] - 0.5 * u[1] * v);
    const double c = sqrt(gamma * p * ri);
    const double sg = v < 0.0 ? -1.0 : 1.0;
    const double k = gamma / (2.0 * c) * ri;  // dc = k (dp - p/rho drho)
    g[0] = sg * (-v * ri) + k * (0.5 * gm1 * v * v - p * ri);
    g[1] = sg * ri + k * (-gm1 * v);
    g[2] = k * gm1;
  }
  // v -/+ c: grad v = (-v/rho, 1/rho, 0), grad c = k (gm1 v^2/2 - p/rho, -gm1 v, gm1)
  __device__ static void grad_eig(const double *u, double gamma, double *gmin, double *gmax) {
    const double gm1 = gamma - 1.0;
    const double ri = 1.0 / u[0];
    const double v = u[1] * ri;
    const double p = gm1 * (u[2] - 0.5 * u[1] * v);
    const double c = sqrt(gamma * p * ri);
    const double k = gamma / (2.0 * c) * ri;
    const double gv[3] = {-v * ri, ri, 0.0};
    const double gc[3] = {k * (0.5 * gm1 * v * v - p * ri), k * (-gm1 * v), k * gm1};
#pragma unroll
    for (int q = 0; q < 3; q++) {
      gmin[q] = gv[q] - gc[q];
      gmax[q] = gv[q] + gc[q];
    }
  }
};

// Reverse sweep of the CAT2p flux of one interface (lane l <-> node
// j = l - p + 1). Fbar: cotangent of the interface flux. ubar: cotangent of
// this lane's node.
template <int p, int FLUX, typename R>
__device__ __forceinline__ void cat_flux_adj(const R *q, int cs, int l, int base, R lam, R adv, R gm1,
                                             const R *Fbar, R *ubar) {
  using TB = Tab<R>;
  constexpr int S = Phys<FLUX>::S;
  constexpr int n = 2 * p;
  const unsigned mask = ((1u << n) - 1u) << base;
  const int j = l - p + 1;
  R g1r[n], g1c[n];
#pragma unroll
  for (int r = 0; r < n; r++) {
    g1r[r] = TB::g1(p, l, r);  // row: d/dx at node j
    g1c[r] = TB::g1(p, r, l);  // column: weight of node j at node r
  }
  R u[S], f0[S], Uk[n + 1][S];
#pragma unroll
  for (int c = 0; c < S; c++) u[c] = q[c * cs + j];
  Phys<FLUX>::flux(u, f0, adv, gm1);
  // forward recomputation, keeping U^(k)
  {
    R arg[n][S], Fprev[S];
#pragma unroll
    for (int rr = 0; rr < n; rr++)
#pragma unroll
      for (int c = 0; c < S; c++) arg[rr][c] = u[c];
#pragma unroll
    for (int c = 0; c < S; c++) Fprev[c] = f0[c];
#pragma unroll
    for (int k = 2; k <= n; k++) {
      R U[S], acc[S];
#pragma unroll
      for (int c = 0; c < S; c++) U[c] = R(0);
#pragma unroll
      for (int r = 0; r < n; r++)
#pragma unroll
        for (int c = 0; c < S; c++) U[c] = fmar(g1r[r], __shfl_sync(mask, Fprev[c], base + r), U[c]);
#pragma unroll
      for (int c = 0; c < S; c++) {
        U[c] *= -lam;
        Uk[k][c] = U[c];
        acc[c] = TB::gk(p, k - 1, p - 1) * f0[c];
      }
      if (k < n) {
#pragma unroll
        for (int rr = 0; rr < n; rr++) {
          if (rr == p - 1) continue;
          R fr[S];
#pragma unroll
          for (int c = 0; c < S; c++) arg[rr][c] = fmar(TB::taylor(p, rr, k - 1), U[c], arg[rr][c]);
          Phys<FLUX>::flux(arg[rr], fr, adv, gm1);
#pragma unroll
          for (int c = 0; c < S; c++) acc[c] = fmar(TB::gk(p, k - 1, rr), fr[c], acc[c]);
        }
#pragma unroll
        for (int c = 0; c < S; c++) Fprev[c] = acc[c];
      }
    }
  }
  // reverse sweep
  R Fsb[S], f0b[S], argb[n][S], Ub[S];
#pragma unroll
  for (int c = 0; c < S; c++) {
    Fsb[c] = TB::gh(p, l) * Fbar[c];
    f0b[c] = Fsb[c];
    Ub[c] = R(0);
  }
#pragma unroll
  for (int rr = 0; rr < n; rr++)
#pragma unroll
    for (int c = 0; c < S; c++) argb[rr][c] = R(0);
#pragma unroll
  for (int k = n; k >= 2; k--) {
    R accb[S];
#pragma unroll
    for (int c = 0; c < S; c++) accb[c] = TB::invfact(k) * Fsb[c];
    if (k < n) {
      // acc^(k) feeds U^(k+1)_i = -lam sum_r g1[i][r] acc^(k)_r
#pragma unroll
      for (int i = 0; i < n; i++)
#pragma unroll
        for (int c = 0; c < S; c++) accb[c] = fmar(-lam * g1c[i], __shfl_sync(mask, Ub[c], base + i), accb[c]);
    }
#pragma unroll
    for (int c = 0; c < S; c++) f0b[c] = fmar(TB::gk(p, k - 1, p - 1), accb[c], f0b[c]);
#pragma unroll
    for (int rr = 0; rr < n; rr++) {
      if (rr == p - 1) continue;
      R a[S], y[S];
#pragma unroll
      for (int c = 0; c < S; c++) {
        a[c] = u[c];
        y[c] = TB::gk(p, k - 1, rr) * accb[c];
      }
#pragma unroll
      for (int kk = 2; kk <= k; kk++)
#pragma unroll
        for (int c = 0; c < S; c++) a[c] = fmar(TB::taylor(p, rr, kk - 1), Uk[kk][c], a[c]);
      Jac<FLUX>::jt(a, y, argb[rr], adv, gm1);
    }
#pragma unroll
    for (int c = 0; c < S; c++) {
      R s = R(0);
#pragma unroll
      for (int rr = 0; rr < n; rr++)
        if (rr != p - 1) s = fmar(TB::taylor(p, rr, k - 1), argb[rr][c], s);
      Ub[c] = s;  // Ubar of U^(k)
    }
  }
  // U^(2)_i = -lam sum_r g1[i][r] f0_r
#pragma unroll
  for (int i = 0; i < n; i++)
#pragma unroll
    for (int c = 0; c < S; c++) f0b[c] = fmar(-lam * g1c[i], __shfl_sync(mask, Ub[c], base + i), f0b[c]);
#pragma unroll
  for (int c = 0; c < S; c++) {
    R s = R(0);
#pragma unroll
    for (int rr = 0; rr < n; rr++)
      if (rr != p - 1) s += argb[rr][c];
    ubar[c] = s;
  }
  Jac<FLUX>::jt(u, f0b, ubar, adv, gm1);
}

// Derivative of the superbee limiter value with respect to r within the
// piece the forward evaluation took.
__device__ __forceinline__ double superbee_d(double r) {
  const double r2 = __dmul_rn(2.0, r);
  const double a = r2 < 1.0 ? r2 : 1.0, da = r2 < 1.0 ? 2.0 : 0.0;
  const double b = r < 2.0 ? r : 2.0, db = r < 2.0 ? 1.0 : 0.0;
  const double m = a > b ? a : b, dm = a > b ? da : db;
  return m > 0.0 ? dm : 0.0;
}

// psi^1 of a 1D interface and its gradient with respect to the four cells
// i-1, i, i+1, i+2 (grad[node][c], node 0 <-> i-1), frozen as the forward.
template <int FLUX>
__device__ void psi1_grad(const double *q, int cs, int limiter_form, double adv, double *grad) {
  constexpr int S = Phys<FLUX>::S;
#pragma unroll
  for (int k = 0; k < 4 * S; k++) grad[k] = 0.0;
  if (S == 1 && limiter_form == 0) {
    const double um = q[-1], u0 = q[0], u1 = q[1], u2 = q[2];
    double a;
    if (u0 != u1) {
      double f0, f1;
      if (FLUX == ACAT_FLUX_LINEAR) {
        f0 = __dmul_rn(adv, u0);
        f1 = __dmul_rn(adv, u1);
      } else {
        f0 = __dmul_rn(__dmul_rn(0.5, u0), u0);
        f1 = __dmul_rn(__dmul_rn(0.5, u1), u1);
      }
      a = __ddiv_rn(__dsub_rn(f1, f0), __dsub_rn(u1, u0));
    } else {
      a = (FLUX == ACAT_FLUX_LINEAR) ? adv : u0;
    }
    const double loc = __dsub_rn(u1, u0);
    if (loc == 0.0) return;  // r is a constant there
    const bool left = a > 0.0;
    const double upw = left ? __dsub_rn(u0, um) : __dsub_rn(u2, u1);
    const double r = __ddiv_rn(upw, loc);
    const double dw = superbee_d(r);
    const double dup = dw / loc, dlo = -dw * r / loc;
    if (left) {
      grad[1] += dup;
      grad[0] -= dup;
    } else {
      grad[3] += dup;
      grad[2] -= dup;
    }
    grad[2] += dlo;
    grad[1] -= dlo;
    return;
  }
  double best = 2.0;
  int bc = -1, bside = 0;
  double br = 0.0;
#pragma unroll
  for (int c = 0; c < S; c++) {
    const double *p = q + c * cs;
    const double loc = __dsub_rn(p[1], p[0]);
    const double rm = lim_ratio(__dsub_rn(p[0], p[-1]), loc);
    const double rp = lim_ratio(__dsub_rn(p[2], p[1]), loc);
    const double pm = superbee(rm), pp = superbee(rp);
    const double v = pp < pm ? pp : pm;
    const int side = pp < pm ? 1 : 0;
    if (v < best) {
      best = v;
      bc = c;
      bside = side;
      br = side ? rp : rm;
    }
  }
  if (bc < 0) return;
  const double *p = q + bc * cs;
  const double loc = __dsub_rn(p[1], p[0]);
  if (loc == 0.0) return;
  const double dw = superbee_d(br);
  const double dup = dw / loc, dlo = -dw * br / loc;
  if (bside == 0) {  // r- = (u_i - u_{i-1}) / loc
    grad[1 * S + bc] += dup;
    grad[0 * S + bc] -= dup;
  } else {  // r+ = (u_{i+2} - u_{i+1}) / loc
    grad[3 * S + bc] += dup;
    grad[2 * S + bc] -= dup;
  }
  grad[2 * S + bc] += dlo;
  grad[1 * S + bc] -= dlo;
}

// Reverse sweep of the FL-CAT2 flux (Eq. 3.4) on one lane; ub[node][c] for
// the cells i-1..i+2 (node 0 <-> i-1).
template <int FLUX>
__device__ void flcat2_adj(const double *q, int cs, double lam, double adv, double gamma,
                           int limiter_form, int lo_flux, const double *Fbar, double *ub) {
  constexpr int S = Phys<FLUX>::S;
  const double gm1 = gamma - 1.0;
  double u0[S], u1[S], f0[S], f1[S], a0[S], a1[S], t0[S], t1[S];
#pragma unroll
  for (int c = 0; c < S; c++) {
    u0[c] = q[c * cs];
    u1[c] = q[c * cs + 1];
  }
  Phys<FLUX>::flux(u0, f0, adv, gm1);
  Phys<FLUX>::flux(u1, f1, adv, gm1);
  double U[S];
#pragma unroll
  for (int c = 0; c < S; c++) {
    U[c] = -lam * (f1[c] - f0[c]);
    a0[c] = u0[c] + U[c];
    a1[c] = u1[c] + U[c];
  }
  Phys<FLUX>::flux(a0, t0, adv, gm1);
  Phys<FLUX>::flux(a1, t1, adv, gm1);
  bool ok;
  const double s0 = Phys<FLUX>::speed(u0, adv, gamma, ok), s1 = Phys<FLUX>::speed(u1, adv, gamma, ok);
  const bool right = s1 > s0;
  // F^lo: Rusanov (alpha the larger spectral radius), global LF (alpha =
  // 1/lambda, a constant with dt frozen) or HLL (frozen branch and frozen
  // argmin / argmax of the eigenvalue bounds)
  const bool hll = lo_flux == ACAT_LO_HLL, glf = lo_flux == ACAT_LO_GLOBAL_LF;
  const double alpha = glf ? 1.0 / lam : (right ? s1 : s0);
  double n0 = 0.0, x0 = 0.0, n1 = 0.0, x1 = 0.0;
  if (hll) {
    Phys<FLUX>::eig(u0, adv, gamma, n0, x0);
    Phys<FLUX>::eig(u1, adv, gamma, n1, x1);
  }
  const bool lmin1 = n1 < n0, lmax1 = x1 > x0;
  const double sl = lmin1 ? n1 : n0, sr = lmax1 ? x1 : x0;
  const int hcase = !hll ? -1 : (sl >= 0.0 ? 0 : (sr <= 0.0 ? 1 : 2));
  const double w = psi1<FLUX>(q, cs, limiter_form, adv);
  double F1[S], Flo[S];
#pragma unroll
  for (int c = 0; c < S; c++) {
    F1[c] = 0.5 * (f0[c] + f1[c]) + 0.25 * ((t0[c] - f0[c]) + (t1[c] - f1[c]));
    if (hcase == 0) Flo[c] = f0[c];
    else if (hcase == 1) Flo[c] = f1[c];
    else if (hcase == 2) Flo[c] = (sr * f0[c] - sl * f1[c] + sl * sr * (u1[c] - u0[c])) / (sr - sl);
    else Flo[c] = 0.5 * (f0[c] + f1[c]) - 0.5 * alpha * (u1[c] - u0[c]);
  }
#pragma unroll
  for (int k = 0; k < 4 * S; k++) ub[k] = 0.0;
  double wb = 0.0, alb = 0.0, slb = 0.0, srb = 0.0;
  double f0b[S], f1b[S], t0b[S], t1b[S];
#pragma unroll
  for (int c = 0; c < S; c++) {
    wb += Fbar[c] * (F1[c] - Flo[c]);
    const double F1b = w * Fbar[c], Flob = (1.0 - w) * Fbar[c];
    f0b[c] = 0.25 * F1b;
    f1b[c] = 0.25 * F1b;
    t0b[c] = 0.25 * F1b;
    t1b[c] = 0.25 * F1b;
    if (hcase == 0) {
      f0b[c] += Flob;
    } else if (hcase == 1) {
      f1b[c] += Flob;
    } else if (hcase == 2) {
      const double D = sr - sl, du = u1[c] - u0[c];
      f0b[c] += sr / D * Flob;
      f1b[c] -= sl / D * Flob;
      ub[2 * S + c] += sl * sr / D * Flob;
      ub[1 * S + c] -= sl * sr / D * Flob;
      slb += Flob * (-f1[c] + sr * du + Flo[c]) / D;
      srb += Flob * (f0[c] + sl * du - Flo[c]) / D;
    } else {
      f0b[c] += 0.5 * Flob;
      f1b[c] += 0.5 * Flob;
      ub[1 * S + c] += 0.5 * alpha * Flob;
      ub[2 * S + c] -= 0.5 * alpha * Flob;
      alb -= 0.5 * Flob * (u1[c] - u0[c]);
    }
  }
  double a0b[S], a1b[S];
#pragma unroll
  for (int c = 0; c < S; c++) a0b[c] = a1b[c] = 0.0;
  Jac<FLUX>::jt(a0, t0b, a0b, adv, gm1);
  Jac<FLUX>::jt(a1, t1b, a1b, adv, gm1);
#pragma unroll
  for (int c = 0; c < S; c++) {
    ub[1 * S + c] += a0b[c];
    ub[2 * S + c] += a1b[c];
    const double Ubar = a0b[c] + a1b[c];
    f1b[c] -= lam * Ubar;
    f0b[c] += lam * Ubar;
  }
  Jac<FLUX>::jt(u0, f0b, ub + 1 * S, adv, gm1);
  Jac<FLUX>::jt(u1, f1b, ub + 2 * S, adv, gm1);
  if (lo_flux == ACAT_LO_RUSANOV) {
    double gs[S];
    Jac<FLUX>::grad_speed(right ? u1 : u0, gamma, gs);
#pragma unroll
    for (int c = 0; c < S; c++) ub[(right ? 2 : 1) * S + c] += alb * gs[c];
  }
  if (hcase == 2) {
    double gmin[S], gmax[S], gjunk[S];
    Jac<FLUX>::grad_eig(lmin1 ? u1 : u0, gamma, gmin, gjunk);
    Jac<FLUX>::grad_eig(lmax1 ? u1 : u0, gamma, gjunk, gmax);
#pragma unroll
    for (int c = 0; c < S; c++) {
      ub[(lmin1 ? 2 : 1) * S + c] += slb * gmin[c];
      ub[(lmax1 ? 2 : 1) * S + c] += srb * gmax[c];
    }
  }
  double gw[4 * S];
  psi1_grad<FLUX>(q, cs, limiter_form, adv, gw);
#pragma unroll
  for (int k = 0; k < 4 * S; k++) ub[k] += wb * gw[k];
}

// Per-interface cotangents of the stencil nodes: contrib[(m * NS + s) * S + c],
// node j = s - NS/2 + 1.
template <int P, int FLUX>
__device__ __forceinline__ void adj1d_body(const Step1DArgs a, const double *__restrict__ ubar1,
                                           double *__restrict__ contrib) {
  using TL = Tiling<P, NWF>;
  constexpr int S = Phys<FLUX>::S;
  constexpr int NS = 2 * P > 4 ? 2 * P : 4;
  __shared__ double tile[S][TL::TW];
  const double *__restrict__ uin = static_cast<const double *>(a.u_in);
  const long N = a.N;
  const long i0 = (long)blockIdx.x * TL::NI;
  for (int q = threadIdx.x; q < S * TL::TW; q += NWF * 32) {
    const int c = q / TL::TW, k = q - c * TL::TW;
    tile[c][k] = uin[c * N + bc_index(i0 - TL::GH + k, N, a.bc)];
  }
  __syncthreads();
  const double lam = (a.dt_in ? *a.dt_in : a.dt_fixed) / a.dx;
  const double gm1 = a.gamma - 1.0;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int grp = lane / TL::L, l = lane - grp * TL::L;
  const bool valid = grp < TL::GPW;
  const int il = warp * TL::GPW + grp;
  const long m = i0 + il;
  const bool active = valid && m <= N;
  const int ic = il - 1 + TL::GH;
  const FiltConst FC = filt_const(a.epsf, a.rf, a.factf);
  const int ps = select_order<P, S, false>(&tile[0][valid ? ic : 0], nullptr, nullptr, TL::TW, l, grp,
                                           active, valid, FC, a.eps, a.thr, a.fact_tau, a.psi2_mod);
  if (!active) return;
  double Fb[S];
#pragma unroll
  for (int c = 0; c < S; c++) {
    const double right = m <= N - 1 ? ubar1[c * N + m] : 0.0;  // cell m gains +lam F_m
    const double left = m >= 1 ? ubar1[c * N + m - 1] : 0.0;    // cell m-1 loses lam F_m
    Fb[c] = lam * (right - left);
  }
  const int base = grp * TL::L;
  const double *q0 = &tile[0][ic];
  double *out = contrib + m * NS * S;
  if (ps >= 2) {
    double ub[S];
    bool mine = false;
    int pp = 2;
    if (ps == 4) {
      if constexpr (P >= 4) {
        cat_flux_adj<4, FLUX>(q0, TL::TW, l, base, lam, a.adv, gm1, Fb, ub);
        mine = true;
        pp = 4;
      }
    } else if (ps == 3) {
      if constexpr (P >= 3) {
        if (l < 6) {
          cat_flux_adj<3, FLUX>(q0, TL::TW, l, base, lam, a.adv, gm1, Fb, ub);
          mine = true;
        }
        pp = 3;
      }
    } else {
      if constexpr (P >= 2) {
        if (l < 4) {
          cat_flux_adj<2, FLUX>(q0, TL::TW, l, base, lam, a.adv, gm1, Fb, ub);
          mine = true;
        }
        pp = 2;
      }
    }
    if (mine) {
      const int s = (l - pp + 1) + NS / 2 - 1;
#pragma unroll
      for (int c = 0; c < S; c++) out[s * S + c] = ub[c];
    } else if (l < NS) {
      // slots of nodes outside S_pp: zero (lanes 2pp..2P-1 cover them)
      const int k = l - 2 * pp;
      const int s = k < NS / 2 - pp ? k : k + 2 * pp;
      if (s >= 0 && s < NS)
#pragma unroll
        for (int c = 0; c < S; c++) out[s * S + c] = 0.0;
    }
  } else if (l == 0) {
    double ub[4 * S];
    flcat2_adj<FLUX>(q0, TL::TW, lam, a.adv, a.gamma, a.limiter_form, a.lo_flux, Fb, ub);
    for (int s = 0; s < NS; s++) {
      const int node = s - NS / 2 + 1;  // -1..2 carry values
#pragma unroll
      for (int c = 0; c < S; c++) out[s * S + c] = (node >= -1 && node <= 2) ? ub[(node + 1) * S + c] : 0.0;
    }
  }
}

// The launched kernel: the programmatic-launch wait, adj1d_body, the
// release (acat_pdl_wait, acat_pdl_release); the body's early returns
// still reach the release.
template <int P, int FLUX>
__global__ void __launch_bounds__(NWF * 32) k_adj1d(const Step1DArgs a, const double *__restrict__ ubar1,
                                                    double *__restrict__ contrib) {
  acat_pdl_wait();
  adj1d_body<P, FLUX>(a, ubar1, contrib);
  acat_pdl_release();
}

// ubar^n_i = ubar^{n+1}_i + the contributions of every (interface, node)
// whose position maps to cell i through the boundary condition.
template <int P, int S>
__device__ __forceinline__ void adj_gather_body(const Step1DArgs a, const double *__restrict__ ubar1,
                                                const double *__restrict__ contrib,
                                                double *__restrict__ ubar0) {
  constexpr int NS = 2 * P > 4 ? 2 * P : 4;
  constexpr int GA = P > 2 ? P : 2;
  const long N = a.N;
  for (long i = (long)blockIdx.x * NT + threadIdx.x; i < N; i += (long)gridDim.x * NT) {
    double acc[S];
#pragma unroll
    for (int c = 0; c < S; c++) acc[c] = ubar1[c * N + i];
    // positions g that map to i
    long gs[2 * GA + 3];
    int ng = 0;
    if (a.bc == ACAT_BC_PERIODIC) {
      for (long g = i - N; g <= i + N; g += N)
        if (g >= -GA && g <= N - 1 + GA) gs[ng++] = g;
    } else {
      gs[ng++] = i;
      if (i == 0)
        for (long g = -GA; g < 0; g++) gs[ng++] = g;
      if (i == N - 1)
        for (long g = N; g <= N - 1 + GA; g++) gs[ng++] = g;
    }
    for (int t = 0; t < ng; t++) {
      const long g = gs[t];
      for (int s = 0; s < NS; s++) {
        const long m = g + 1 - (s - NS / 2 + 1);
        if (m < 0 || m > N) continue;
#pragma unroll
        for (int c = 0; c < S; c++) acc[c] += contrib[(m * NS + s) * S + c];
      }
    }
#pragma unroll
    for (int c = 0; c < S; c++) ubar0[c * N + i] = acc[c];
  }
}

// The launched kernel: the programmatic-launch wait, adj_gather_body, the
// release (acat_pdl_wait, acat_pdl_release); the body's early returns
// still reach the release.
template <int P, int S>
__global__ void __launch_bounds__(NT) k_adj_gather(const Step1DArgs a, const double *__restrict__ ubar1,
                                                   const double *__restrict__ contrib,
                                                   double *__restrict__ ubar0) {
  acat_pdl_wait();
  adj_gather_body<P, S>(a, ubar1, contrib, ubar0);
  acat_pdl_release();
}

// FP32 adjoint step on the compensated state [hi(S x N); lo(S x N)] with a
// compensated cotangent of the same layout. The order decisions are the FP32
// forward's (taken on hi + lo); Fbar_m = lambda (ubar_m - ubar_{m-1}) is
// formed from the cotangent pairs in float-float; the CAT2p reverse sweep runs
// in float on hi (the Jacobians are evaluated, not differenced, so float
// arguments carry only relative rounding); FL-CAT2 interfaces are
// differentiated in FP64 on hi + lo. Per-interface node cotangents go to a
// float scratch array.
template <int P, int FLUX>
__device__ __forceinline__ void adj1d_f32_body(const Step1DArgs a, const float *__restrict__ ubar1,
                                               float *__restrict__ contrib) {
  using TL = Tiling<P, NWF>;
  constexpr int S = Phys<FLUX>::S;
  constexpr int NS = 2 * P > 4 ? 2 * P : 4;
  __shared__ float thi[S][TL::TW], tlo[S][TL::TW];
  const float *__restrict__ uin = static_cast<const float *>(a.u_in);
  const long N = a.N;
  const long i0 = (long)blockIdx.x * TL::NI;
  for (int q = threadIdx.x; q < S * TL::TW; q += NWF * 32) {
    const int c = q / TL::TW, k = q - c * TL::TW;
    const long g = bc_index(i0 - TL::GH + k, N, a.bc);
    thi[c][k] = uin[c * N + g];
    tlo[c][k] = uin[(S + c) * N + g];
  }
  __syncthreads();
  const double lamd = (a.dt_in ? *a.dt_in : a.dt_fixed) / a.dx;
  const float lam = (float)lamd;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int grp = lane / TL::L, l = lane - grp * TL::L;
  const bool valid = grp < TL::GPW;
  const int il = warp * TL::GPW + grp;
  const long m = i0 + il;
  const bool active = valid && m <= N;
  const int ic = il - 1 + TL::GH;
  const int icv = valid ? ic : 0;
  const FiltConst FC = filt_const(a.epsf, a.rf, a.factf);
  const int ps = select_order<P, S, true>(nullptr, &thi[0][icv], &tlo[0][icv], TL::TW, l, grp, active, valid,
                                          FC, a.eps, a.thr, a.fact_tau, a.psi2_mod);
  if (!active) return;
  // Fbar_m = lambda (ubar_m - ubar_{m-1}), cells outside 0..N-1 contribute nothing
  float Fb[S];
  double Fbd[S];
#pragma unroll
  for (int c = 0; c < S; c++) {
    const float rh = m <= N - 1 ? ubar1[c * N + m] : 0.0f, rl = m <= N - 1 ? ubar1[(S + c) * N + m] : 0.0f;
    const float lh = m >= 1 ? ubar1[c * N + m - 1] : 0.0f, ll = m >= 1 ? ubar1[(S + c) * N + m - 1] : 0.0f;
    const FF d = ff_jump(lh, ll, rh, rl);
    Fbd[c] = lamd * ((double)d.h + (double)d.l);
    Fb[c] = (float)Fbd[c];
  }
  const int base = grp * TL::L;
  float *out = contrib + m * NS * S;
  if (ps >= 2) {
    float ub[S];
    bool mine = false;
    int pp = 2;
    const float *q0 = &thi[0][ic];
    if (ps == 4) {
      if constexpr (P >= 4) {
        cat_flux_adj<4, FLUX, float>(q0, TL::TW, l, base, lam, a.advf, a.gm1f, Fb, ub);
        mine = true;
        pp = 4;
      }
    } else if (ps == 3) {
      if constexpr (P >= 3) {
        if (l < 6) {
          cat_flux_adj<3, FLUX, float>(q0, TL::TW, l, base, lam, a.advf, a.gm1f, Fb, ub);
          mine = true;
        }
        pp = 3;
      }
    } else {
      if constexpr (P >= 2) {
        if (l < 4) {
          cat_flux_adj<2, FLUX, float>(q0, TL::TW, l, base, lam, a.advf, a.gm1f, Fb, ub);
          mine = true;
        }
        pp = 2;
      }
    }
    if (mine) {
      const int s = (l - pp + 1) + NS / 2 - 1;
#pragma unroll
      for (int c = 0; c < S; c++) out[s * S + c] = ub[c];
    } else if (l < NS) {
      const int k = l - 2 * pp;
      const int s = k < NS / 2 - pp ? k : k + 2 * pp;
      if (s >= 0 && s < NS)
#pragma unroll
        for (int c = 0; c < S; c++) out[s * S + c] = 0.0f;
    }
  } else if (l == 0) {
    // cells i-1..i+2 of the interface as FP64 values hi + lo
    double qd[S][4], ub[4 * S];
#pragma unroll
    for (int c = 0; c < S; c++)
#pragma unroll
      for (int k = 0; k < 4; k++) qd[c][k] = (double)thi[c][ic - 1 + k] + (double)tlo[c][ic - 1 + k];
    flcat2_adj<FLUX>(&qd[0][1], 4, lamd, a.adv, a.gamma, a.limiter_form, a.lo_flux, Fbd, ub);
    for (int s = 0; s < NS; s++) {
      const int node = s - NS / 2 + 1;
#pragma unroll
      for (int c = 0; c < S; c++)
        out[s * S + c] = (node >= -1 && node <= 2) ? (float)ub[(node + 1) * S + c] : 0.0f;
    }
  }
}

// The launched kernel: the programmatic-launch wait, adj1d_f32_body, the
// release (acat_pdl_wait, acat_pdl_release); the body's early returns
// still reach the release.
template <int P, int FLUX>
__global__ void __launch_bounds__(NWF * 32) k_adj1d_f32(const Step1DArgs a, const float *__restrict__ ubar1,
                                                        float *__restrict__ contrib) {
  acat_pdl_wait();
  adj1d_f32_body<P, FLUX>(a, ubar1, contrib);
  acat_pdl_release();
}

// Compensated gather: ubar^n = ubar^{n+1} + the float sum of the contributions
// that map to the cell, added to the pair with TwoSum and renormalised.
template <int P, int S>
__device__ __forceinline__ void adj_gather_f32_body(const Step1DArgs a, const float *__restrict__ ubar1,
                                                    const float *__restrict__ contrib,
                                                    float *__restrict__ ubar0) {
  constexpr int NS = 2 * P > 4 ? 2 * P : 4;
  constexpr int GA = P > 2 ? P : 2;
  const long N = a.N;
  for (long i = (long)blockIdx.x * NT + threadIdx.x; i < N; i += (long)gridDim.x * NT) {
    float acc[S];
#pragma unroll
    for (int c = 0; c < S; c++) acc[c] = 0.0f;
    long gs[2 * GA + 3];
    int ng = 0;
    if (a.bc == ACAT_BC_PERIODIC) {
      for (long g = i - N; g <= i + N; g += N)
        if (g >= -GA && g <= N - 1 + GA) gs[ng++] = g;
    } else {
      gs[ng++] = i;
      if (i == 0)
        for (long g = -GA; g < 0; g++) gs[ng++] = g;
      if (i == N - 1)
        for (long g = N; g <= N - 1 + GA; g++) gs[ng++] = g;
    }
    for (int t = 0; t < ng; t++) {
      const long g = gs[t];
      for (int s = 0; s < NS; s++) {
        const long m = g + 1 - (s - NS / 2 + 1);
        if (m < 0 || m > N) continue;
#pragma unroll
        for (int c = 0; c < S; c++) acc[c] += contrib[(m * NS + s) * S + c];
      }
    }
#pragma unroll
    for (int c = 0; c < S; c++) {
      const float h = ubar1[c * N + i], w = ubar1[(S + c) * N + i], d = acc[c];
      const float s = __fadd_rn(h, d);
      const float bp = __fsub_rn(s, h);
      const float e = __fadd_rn(__fsub_rn(h, __fsub_rn(s, bp)), __fsub_rn(d, bp));
      const float w2 = __fadd_rn(w, e);
      const float hn = __fadd_rn(s, w2);
      ubar0[c * N + i] = hn;
      ubar0[(S + c) * N + i] = __fsub_rn(w2, __fsub_rn(hn, s));
    }
  }
}

// The launched kernel: the programmatic-launch wait, adj_gather_f32_body, the
// release (acat_pdl_wait, acat_pdl_release); the body's early returns
// still reach the release.
template <int P, int S>
__global__ void __launch_bounds__(NT) k_adj_gather_f32(const Step1DArgs a, const float *__restrict__ ubar1,
                                                       const float *__restrict__ contrib,
                                                       float *__restrict__ ubar0) {
  acat_pdl_wait();
  adj_gather_f32_body<P, S>(a, ubar1, contrib, ubar0);
  acat_pdl_release();
}

template <int FLUX>
int launch_adj_f32(int P, const Step1DArgs &a, const float *ub1, float *contrib, float *ub0, cudaStream_t st) {
  constexpr int S = Phys<FLUX>::S;
  const long blocks = (a.N + NT - 1) / NT;
  const unsigned g2 = (unsigned)(blocks < 4096 ? blocks : 4096);
  switch (P) {
#define ACAT_ADJ32_CASE(PP)                                                                       \
  case PP: {                                                                                      \
    const unsigned grid = (unsigned)((a.N + Tiling<PP, NWF>::NI) / Tiling<PP, NWF>::NI);          \
    if (int e = acat_launch_dep(k_adj1d_f32<PP, FLUX>, grid, NWF * 32, st, a, ub1, contrib)) return e;  \
    return acat_launch_dep(k_adj_gather_f32<PP, S>, g2, NT, st, a, ub1, (const float *)contrib, ub0); \
  }
    ACAT_ADJ32_CASE(1)
    ACAT_ADJ32_CASE(2)
    ACAT_ADJ32_CASE(3)
    ACAT_ADJ32_CASE(4)
#undef ACAT_ADJ32_CASE
  default: return (int)cudaErrorInvalidValue;
  }
  return (int)cudaGetLastError();
}

template <int FLUX>
int launch_adj_f(int P, const Step1DArgs &a, const double *ub1, double *contrib, double *ub0,
                 cudaStream_t st) {
  constexpr int S = Phys<FLUX>::S;
  const long blocks = (a.N + NT - 1) / NT;
  const unsigned g2 = (unsigned)(blocks < 4096 ? blocks : 4096);
  switch (P) {
#define ACAT_ADJ_CASE(PP)                                                                         \
  case PP: {                                                                                      \
    const unsigned grid = (unsigned)((a.N + Tiling<PP, NWF>::NI) / Tiling<PP, NWF>::NI);          \
    if (int e = acat_launch_dep(k_adj1d<PP, FLUX>, grid, NWF * 32, st, a, ub1, contrib)) return e;     \
    return acat_launch_dep(k_adj_gather<PP, S>, g2, NT, st, a, ub1, (const double *)contrib, ub0);   \
  }
    ACAT_ADJ_CASE(1)
    ACAT_ADJ_CASE(2)
    ACAT_ADJ_CASE(3)
    ACAT_ADJ_CASE(4)
#undef ACAT_ADJ_CASE
  default: return (int)cudaErrorInvalidValue;
  }
  return (int)cudaGetLastError();
}

}  // namespace

int acat_adjoint_slots(int P) { return 2 * P > 4 ? 2 * P : 4; }

int acat_launch_adjoint1d(int P, int flux, int prec, const Step1DArgs &a, const void *ubar1_, void *contrib_,
                          void *ubar0_, void *stream) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (prec == ACAT_PREC_F32) {
    const float *ubar1 = static_cast<const float *>(ubar1_);
    float *contrib = static_cast<float *>(contrib_), *ubar0 = static_cast<float *>(ubar0_);
    switch (flux) {
    case ACAT_FLUX_LINEAR: return launch_adj_f32<ACAT_FLUX_LINEAR>(P, a, ubar1, contrib, ubar0, st);
    case ACAT_FLUX_BURGERS: return launch_adj_f32<ACAT_FLUX_BURGERS>(P, a, ubar1, contrib, ubar0, st);
    case ACAT_FLUX_EULER1D: return launch_adj_f32<ACAT_FLUX_EULER1D>(P, a, ubar1, contrib, ubar0, st);
    }
    return (int)cudaErrorInvalidValue;
  }
  const double *ubar1 = static_cast<const double *>(ubar1_);
  double *contrib = static_cast<double *>(contrib_), *ubar0 = static_cast<double *>(ubar0_);
  switch (flux) {
  case ACAT_FLUX_LINEAR: return launch_adj_f<ACAT_FLUX_LINEAR>(P, a, ubar1, contrib, ubar0, st);
  case ACAT_FLUX_BURGERS: return launch_adj_f<ACAT_FLUX_BURGERS>(P, a, ubar1, contrib, ubar0, st);
  case ACAT_FLUX_EULER1D: return launch_adj_f<ACAT_FLUX_EULER1D>(P, a, ubar1, contrib, ubar0, st);
  }
  return (int)cudaErrorInvalidValue;
}

int acat_upload_tables_adj(const AcatTables *T) { return (int)cudaMemcpyToSymbol(c_tab, T, sizeof *T); }
