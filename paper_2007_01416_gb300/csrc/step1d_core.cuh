// step1d_core.cuh -- device code shared by the single-instance and batched
// 1D steps: the CAT2p and FL-CAT2 fluxes (FP64 and the FP32 delta form), the
// per-step dt, and the tile functions that stage, select orders, compute the
// interface fluxes and update the cells of one tile. Included by step1d.cu
// and batch1d.cu; each translation unit holds its own copy of the weight
// tables in constant memory.
#pragma once
#include <cstring>
#include <type_traits>

#include "phys1d.cuh"

namespace {

// ---------------------------------------------------------------------------
// CAT2p flux of one interface by a group of 2p lanes (lane l <-> node
// j = l - p + 1). q points at cell i (left of the interface) for component 0
// of the shared tile, components `cs` apart. Every lane returns the flux.
// ---------------------------------------------------------------------------
template <int p, int FLUX, typename R>
__device__ __forceinline__ void cat_flux(const R *q, int cs, int l, int base, R lam, R adv, R gm1,
                                         R *Fout) {
  using TB = Tab<R>;
  constexpr int S = Phys<FLUX>::S;
  constexpr int n = 2 * p;
  const unsigned mask = ((1u << n) - 1u) << base;
  const int j = l - p + 1;
  // the node's derivative weights scaled by -lambda once, so that each order's
  // U^(k-1)_j = -lambda sum_r g1[j][r] F_r needs no multiply per component
  R g1r[n];
#pragma unroll
  for (int r = 0; r < n; r++) g1r[r] = TB::g1(p, l, r) * -lam;
  R f0[S], Fsum[S], Fprev[S], arg[n][S];
  {
    R u[S];
#pragma unroll
    for (int c = 0; c < S; c++) u[c] = q[c * cs + j];
    Phys<FLUX>::flux(u, f0, adv, gm1);
#pragma unroll
    for (int rr = 0; rr < n; rr++)
#pragma unroll
      for (int c = 0; c < S; c++) arg[rr][c] = u[c];
  }
#pragma unroll
  for (int c = 0; c < S; c++) {
    Fsum[c] = f0[c];
    Fprev[c] = f0[c];
  }
#pragma unroll
  for (int k = 2; k <= n; k++) {
    R U[S];
#pragma unroll
    for (int c = 0; c < S; c++) U[c] = R(0);
#pragma unroll
    for (int r = 0; r < n; r++)
#pragma unroll
      for (int c = 0; c < S; c++) U[c] = fma(g1r[r], __shfl_sync(mask, Fprev[c], base + r), U[c]);
    R acc[S];
#pragma unroll
    for (int c = 0; c < S; c++) acc[c] = TB::gk(p, k - 1, p - 1) * f0[c];
#pragma unroll
    for (int rr = 0; rr < n; rr++) {
      if (rr == p - 1) continue;  // r = 0: f(u_j) itself
      const R cr = TB::taylor(p, rr, k - 1);
      R fr[S];
#pragma unroll
      for (int c = 0; c < S; c++) arg[rr][c] = fma(cr, U[c], arg[rr][c]);
      Phys<FLUX>::flux(arg[rr], fr, adv, gm1);
#pragma unroll
      for (int c = 0; c < S; c++) acc[c] = fma(TB::gk(p, k - 1, rr), fr[c], acc[c]);
    }
#pragma unroll
    for (int c = 0; c < S; c++) {
      Fprev[c] = acc[c];
      Fsum[c] = fma(TB::invfact(k), acc[c], Fsum[c]);
    }
  }
  const R w = TB::gh(p, l);
#pragma unroll
  for (int c = 0; c < S; c++) {
    const R v = w * Fsum[c];
    R t = __shfl_sync(mask, v, base);
#pragma unroll
    for (int r = 1; r < n; r++) t += __shfl_sync(mask, v, base + r);
    Fout[c] = t;
  }
}

// FL-CAT2 flux (Eq. 3.4), FP64: the CAT2 flux (p = 1 recursion, Eqs.
// 2.16-2.17) blended with Rusanov by the limiter psi^1. Worked by the L lanes
// of the interface group (all of them call it): lanes of even and odd rank
// evaluate the two nodes' fluxes and wave speeds, exchanged by shuffles, and
// the limiter's ratios are spread over the group. Every lane returns F.
template <int FLUX, int L>
__device__ __forceinline__ void flcat2_flux(const double *q, int cs, int l, unsigned gmask, double lam,
                                            double adv, double gamma, int limiter_form, int lo_flux,
                                            double *F) {
  constexpr int S = Phys<FLUX>::S;
  const double gm1 = gamma - 1.0;
  const int me = l & 1;  // node i + me
  double u[S], f[S], a[S], t[S], u0[S], u1[S], f0[S], f1[S], t0[S], t1[S];
#pragma unroll
  for (int c = 0; c < S; c++) u[c] = q[c * cs + me];
  Phys<FLUX>::flux(u, f, adv, gm1);
#pragma unroll
  for (int c = 0; c < S; c++) {
    const double o = __shfl_xor_sync(gmask, f[c], 1);
    f0[c] = me ? o : f[c];
    f1[c] = me ? f[c] : o;
    u0[c] = q[c * cs];
    u1[c] = q[c * cs + 1];
    const double U = -lam * (f1[c] - f0[c]);  // gamma^{1,j}_1 = (-1, 1), both nodes
    a[c] = u[c] + U;
  }
  Phys<FLUX>::flux(a, t, adv, gm1);
  bool ok;
  const double s = Phys<FLUX>::speed(u, adv, gamma, ok);
  const double so = __shfl_xor_sync(gmask, s, 1);
  const double s0 = me ? so : s, s1 = me ? s : so;
#pragma unroll
  for (int c = 0; c < S; c++) {
    const double o = __shfl_xor_sync(gmask, t[c], 1);
    t0[c] = me ? o : t[c];
    t1[c] = me ? t[c] : o;
  }
  double n0 = 0.0, x0 = 0.0, n1 = 0.0, x1 = 0.0;
  if (lo_flux == ACAT_LO_HLL) {
    double n, x;
    Phys<FLUX>::eig(u, adv, gamma, n, x);
    const double no = __shfl_xor_sync(gmask, n, 1), xo = __shfl_xor_sync(gmask, x, 1);
    n0 = me ? no : n;
    x0 = me ? xo : x;
    n1 = me ? n : no;
    x1 = me ? x : xo;
  }
  double Flo[S];
  flux_lo<S, double>(lo_flux, u0, u1, f0, f1, s0, s1, n0, x0, n1, x1, lam, Flo);
  const double w = psi1_group<S, L>([=](int c, int k) { return q[c * cs + k]; },
                                    FLUX == ACAT_FLUX_LINEAR ? 0 : 1, limiter_form, adv, l, gmask);
#pragma unroll
  for (int c = 0; c < S; c++) {
    const double F1 = 0.5 * (f0[c] + f1[c]) + 0.25 * ((t0[c] - f0[c]) + (t1[c] - f1[c]));
    F[c] = w * F1 + (1.0 - w) * Flo[c];
  }
}

// ---------------------------------------------------------------------------
// FP32 delta formulation. The flux at x_{i+1/2} is written F = f(u_i) + G and
// every term of G is built from flux increments df(u; d) = f(u + d) - f(u)
// evaluated in a cancellation-free algebraic form, so that float rounding is
// relative to the (small) increments and not to |f|:
//   - the time-derivative sums sum_r gamma^{k,0}_r f(arg_r), k >= 1, equal
//     sum_{r != 0} gamma^{k,0}_r df(u_j; arg_r - u_j) since the weights of a
//     derivative sum to zero;
//   - the spatial derivative of f~^(0) equals that of df(u_i; u_j - u_i);
//   - the k = 1 flux term sum_j gamma^{0,1/2}_j f(u_j) equals
//     f(u_i) + sum_j gamma^{0,1/2}_j df(u_i; u_j - u_i) (weights sum to one).
// The update u_i += lambda (F_{i-1/2} - F_{i+1/2}) then needs only
// f(u_{i-1}) - f(u_i) = df(u_i; u_{i-1} - u_i) and the G's, all small. The
// identities are used symbolically; nothing relies on rounded weights summing
// to zero.
// ---------------------------------------------------------------------------
template <int FLUX>
struct DPhys;

template <>
struct DPhys<ACAT_FLUX_LINEAR> {
  static constexpr int S = 1;
  struct Base {
    float a;
  };
  __device__ static __forceinline__ Base base(const float *, float a, float) { return Base{a}; }
  __device__ static __forceinline__ Base base2(const float *, const float *, float a, float) { return Base{a}; }
  __device__ static __forceinline__ void dflux(const Base &b, const float *d, float *df) {
    df[0] = b.a * d[0];
  }
  __device__ static __forceinline__ void dflux_pair(const Base &b, const float *dh, const float *dl, float *df) {
    df[0] = b.a * (dh[0] + dl[0]);
  }
  // two increments at once, packed in the lanes of float2 values
  __device__ static __forceinline__ void dflux_x2(const Base &b, const float2 *d, float2 *df) {
    df[0] = f2mul(f2dup(b.a), d[0]);
  }
  __device__ static __forceinline__ float speed(const float *, float a, float) { return fabsf(a); }
  __device__ static __forceinline__ bool physical(const float *u, float) { return isfinite(u[0]); }
};

template <>
struct DPhys<ACAT_FLUX_BURGERS> {
  static constexpr int S = 1;
  struct Base {
    float u;
  };
  __device__ static __forceinline__ Base base(const float *u, float, float) { return Base{u[0]}; }
  __device__ static __forceinline__ Base base2(const float *h, const float *, float, float) { return Base{h[0]}; }
  // (u + d)^2/2 - u^2/2 = d (u + d/2)
  __device__ static __forceinline__ void dflux(const Base &b, const float *d, float *df) {
    df[0] = d[0] * fmaf(0.5f, d[0], b.u);
  }
  __device__ static __forceinline__ void dflux_pair(const Base &b, const float *dh, const float *dl, float *df) {
    const float d[1] = {dh[0] + dl[0]};
    dflux(b, d, df);
  }
  __device__ static __forceinline__ void dflux_x2(const Base &b, const float2 *d, float2 *df) {
    df[0] = f2mul(d[0], f2fma(f2dup(0.5f), d[0], f2dup(b.u)));
  }
  __device__ static __forceinline__ float speed(const float *u, float, float) { return fabsf(u[0]); }
  __device__ static __forceinline__ bool physical(const float *u, float) { return isfinite(u[0]); }
};

template <>
struct DPhys<ACAT_FLUX_EULER1D> {
  static constexpr int S = 3;
  struct Base {
    float rho, m, v, vl, H, gm1;  // v + vl: the velocity as a float-float pair
  };
  __device__ static __forceinline__ Base base(const float *u, float, float gm1) {
    Base b;
    b.rho = u[0];
    b.m = u[1];
    b.v = __fmul_rn(u[1], recip(u[0]));
    b.vl = 0.0f;
    const float p = __fmul_rn(gm1, fmaf(__fmul_rn(-0.5f, u[1]), b.v, u[2]));
    b.H = __fadd_rn(u[2], p);
    b.gm1 = gm1;
    return b;
  }
  // The base of a compensated state hi + lo, with the velocity m / rho carried
  // to float-float accuracy: v = fl(m_hi / rho_hi), and vl from the residual
  // m - v rho (its leading part m_hi - v rho_hi exact in one FMA). Increments
  // at constant velocity (an entropy wave) have b = v a exactly, and the
  // numerator b - v a of dv cancels: with v rounded to float it would leave
  // eps32 |v a| of noise in every energy and momentum increment, which the
  // (2p-1)-th difference of tau_p amplifies over a run.
  __device__ static __forceinline__ Base base2(const float *h, const float *l, float, float gm1) {
    Base b;
    b.rho = h[0];
    b.m = h[1];
    const float r = recip(h[0]);
    b.v = __fmul_rn(h[1], r);
    b.vl = __fmul_rn(__fadd_rn(fmaf(-b.v, h[0], h[1]), fmaf(-b.v, l[0], l[1])), r);
    const float p = __fmul_rn(gm1, fmaf(__fmul_rn(-0.5f, h[1]), b.v, h[2]));
    b.H = __fadd_rn(h[2], p);
    b.gm1 = gm1;
    return b;
  }
  // With u = (rho, m, E), d = (a, b, c), v = m/rho, H = E + p:
  //   dv = (b - v a) / (rho + a)          [v' - v]
  //   d(mv) = m dv + b (v + dv)
  //   dp = (gamma - 1)(c - d(mv)/2)
  //   df = (b, d(mv) + dp, dv H + (v + dv)(c + dp))
  // Every operation is rounded as written (no contraction left to the
  // compiler), so that every kernel instantiating it gives the same bits.
  __device__ static __forceinline__ void dflux(const Base &B, const float *d, float *df) {
    const float dv = __fmul_rn(fmaf(-B.vl, d[0], fmaf(-B.v, d[0], d[1])), recip(__fadd_rn(B.rho, d[0])));
    rest(B, d, dv, df);
  }
  __device__ static __forceinline__ void rest(const Base &B, const float *d, float dv, float *df) {
    const float vn = __fadd_rn(B.v, dv);
    const float dmv = fmaf(B.m, dv, __fmul_rn(d[1], vn));
    const float dp = __fmul_rn(B.gm1, fmaf(-0.5f, dmv, d[2]));
    df[0] = d[1];
    df[1] = __fadd_rn(dmv, dp);
    df[2] = fmaf(dv, B.H, __fmul_rn(vn, __fadd_rn(d[2], dp)));
  }
  // the increment d = dh + dl given as an unevaluated pair (dh: difference of
  // the hi parts, exact for nearby values; dl: of the lo parts): the
  // cancelling numerator of dv is formed from both parts
  __device__ static __forceinline__ void dflux_pair(const Base &B, const float *dh, const float *dl, float *df) {
    const float d[3] = {__fadd_rn(dh[0], dl[0]), __fadd_rn(dh[1], dl[1]), __fadd_rn(dh[2], dl[2])};
    const float num = fmaf(-B.vl, dh[0], __fadd_rn(fmaf(-B.v, dh[0], dh[1]), fmaf(-B.v, dl[0], dl[1])));
    rest(B, d, __fmul_rn(num, recip(__fadd_rn(B.rho, d[0]))), df);
  }
  // the same for two increments packed in float2 lanes
  __device__ static __forceinline__ void dflux_x2(const Base &B, const float2 *d, float2 *df) {
    const float2 t = f2fma(f2dup(-B.vl), d[0], f2fma(f2dup(-B.v), d[0], d[1]));
    const float2 den = f2add(f2dup(B.rho), d[0]);
    const float2 dv = f2mul(t, make_float2(recip(den.x), recip(den.y)));
    const float2 vn = f2add(f2dup(B.v), dv);
    const float2 dmv = f2fma(f2dup(B.m), dv, f2mul(d[1], vn));
    const float2 dp = f2mul(f2dup(B.gm1), f2fma(f2dup(-0.5f), dmv, d[2]));
    df[0] = d[1];
    df[1] = f2add(dmv, dp);
    df[2] = f2fma(dv, f2dup(B.H), f2mul(vn, f2add(d[2], dp)));
  }
  __device__ static __forceinline__ float speed(const float *u, float, float gamma) {
    const float v = __fdiv_rn(u[1], u[0]);
    const float p = __fmul_rn(__fsub_rn(gamma, 1.0f), __fsub_rn(u[2], __fmul_rn(__fmul_rn(0.5f, u[1]), v)));
    return __fadd_rn(fabsf(v), __fsqrt_rn(fmaxf(__fdiv_rn(__fmul_rn(gamma, p), u[0]), 0.0f)));
  }
  __device__ static __forceinline__ bool physical(const float *u, float gamma) {
    const float v = __fdiv_rn(u[1], u[0]);
    const float p = __fmul_rn(__fsub_rn(gamma, 1.0f), __fsub_rn(u[2], __fmul_rn(__fmul_rn(0.5f, u[1]), v)));
    return u[0] > 0.0f && p > 0.0f && isfinite(u[0]) && isfinite(u[1]) && isfinite(u[2]);
  }
};

// CAT2p increment G of one interface by a group of 2p lanes (lane l <-> node
// j = l - p + 1). hi/lo point at cell i of component 0 of the compensated
// tile, components `cs` apart. xg: the group's exchange slots in shared
// memory (node r at xg[r], two sets XSET apart used alternately by k),
// through which the lanes of the group read the F^(k-2) of all nodes of a
// system: one 16-byte store and 2p 16-byte broadcast loads per lane and order
// instead of 2p s shuffles (scalar laws shuffle). Every lane returns G.
template <int p, int FLUX>
__device__ __forceinline__ void cat_delta(const float *hi, const float *lo, int cs, int l, int base,
                                          float lam, float adv, float gm1, float4 *xg, float *Gout) {
  using TB = Tab<float>;
  using DP = DPhys<FLUX>;
  constexpr int S = DP::S;
  constexpr int n = 2 * p;
  const unsigned mask = ((1u << n) - 1u) << base;
  const int j = l - p + 1;
  // the node's derivative weights scaled by -lambda once (no multiply per
  // component and order)
  float g1r[n];
#pragma unroll
  for (int r = 0; r < n; r++) g1r[r] = __fmul_rn(TB::g1(p, l, r), -lam);
  float ui[S], uil[S], uj[S], ujl[S], dh[S], dl[S];
#pragma unroll
  for (int c = 0; c < S; c++) {
    ui[c] = hi[c * cs];
    uil[c] = lo[c * cs];
    uj[c] = hi[c * cs + j];
    ujl[c] = lo[c * cs + j];
    dh[c] = uj[c] - ui[c];
    dl[c] = ujl[c] - uil[c];
  }
  // the 2p - 1 time levels r != 0 (level q <-> table row q < p - 1 ? q : q + 1)
  // are worked in pairs packed in float2 lanes (p <= 3; at p = 4 the pairs
  // would cost the registers of a fourth resident CTA), the last one alone
  constexpr int NL = n - 1, NP = p <= 3 ? NL / 2 : 0;
  float D[S], Fsum[S], Fprev[S], dels[NL - 2 * NP][S];
  float2 del2[NP > 0 ? NP : 1][S];
  DP::dflux_pair(DP::base2(ui, uil, adv, gm1), dh, dl, D);  // f(u_j) - f(u_i)
  const typename DP::Base bj = DP::base2(uj, ujl, adv, gm1);
#pragma unroll
  for (int c = 0; c < S; c++) {
    Fsum[c] = D[c];
    Fprev[c] = D[c];
  }
#pragma unroll
  for (int q = 0; q < NL - 2 * NP; q++)
#pragma unroll
    for (int c = 0; c < S; c++) dels[q][c] = 0.0f;
#pragma unroll
  for (int q = 0; q < NP; q++)
#pragma unroll
    for (int c = 0; c < S; c++) del2[q][c] = make_float2(0.0f, 0.0f);
#pragma unroll
  for (int k = 2; k <= n; k++) {
    float U[S];
#pragma unroll
    for (int c = 0; c < S; c++) U[c] = 0.0f;
    if constexpr (S == 3 && p >= 3) {
      // the slot set of order k was last read at order k - 2, before every
      // lane of the group passed the barrier of order k - 1. At p >= 3
      // components 0 and 1 of the sum run packed in float2 lanes (each
      // rounded as the scalar FMA); at p = 2 the scalar form is faster.
      float4 *xb = xg + (k & 1) * XSET;
      xb[l] = make_float4(Fprev[0], Fprev[1], Fprev[S > 2 ? 2 : 0], 0.0f);
      __syncwarp(mask);
      float2 u01 = make_float2(0.0f, 0.0f);
#pragma unroll
      for (int r = 0; r < n; r++) {
        const float4 f = xb[r];
        u01 = f2fma(f2dup(g1r[r]), make_float2(f.x, f.y), u01);
        U[S > 2 ? 2 : 0] = fmaf(g1r[r], f.z, U[S > 2 ? 2 : 0]);
      }
      U[0] = u01.x;
      U[1] = u01.y;
    } else if constexpr (S > 1) {
      float4 *xb = xg + (k & 1) * XSET;
      xb[l] = make_float4(Fprev[0], Fprev[1], Fprev[S > 2 ? 2 : 0], 0.0f);
      __syncwarp(mask);
#pragma unroll
      for (int r = 0; r < n; r++) {
        const float4 f = xb[r];
        const float fr[3] = {f.x, f.y, f.z};
#pragma unroll
        for (int c = 0; c < S; c++) U[c] = fmaf(g1r[r], fr[c], U[c]);
      }
    } else {  // a scalar law: one shuffle per node
#pragma unroll
      for (int r = 0; r < n; r++) U[0] = fmaf(g1r[r], __shfl_sync(mask, Fprev[0], base + r), U[0]);
    }
    float acc[S];
    float2 acc2[S];
#pragma unroll
    for (int c = 0; c < S; c++) {
      acc[c] = 0.0f;
      acc2[c] = make_float2(0.0f, 0.0f);
    }
#pragma unroll
    for (int q = 0; q < NP; q++) {
      const int ra = 2 * q < p - 1 ? 2 * q : 2 * q + 1, rb = 2 * q + 1 < p - 1 ? 2 * q + 1 : 2 * q + 2;
      const float2 cr = make_float2(TB::taylor(p, ra, k - 1), TB::taylor(p, rb, k - 1));
      const float2 wk = make_float2(TB::gk(p, k - 1, ra), TB::gk(p, k - 1, rb));
      float2 E2[S];
#pragma unroll
      for (int c = 0; c < S; c++) del2[q][c] = f2fma(cr, f2dup(U[c]), del2[q][c]);
      DP::dflux_x2(bj, del2[q], E2);
#pragma unroll
      for (int c = 0; c < S; c++) acc2[c] = f2fma(wk, E2[c], acc2[c]);
    }
#pragma unroll
    for (int q = 2 * NP; q < NL; q++) {  // levels not paired
      const int rs = q < p - 1 ? q : q + 1;
      const float cr = TB::taylor(p, rs, k - 1), wk = TB::gk(p, k - 1, rs);
      float *dq = dels[q - 2 * NP];
      float E[S];
      if constexpr (S == 3 && p >= 3) {
        const float2 d01 = f2fma(f2dup(cr), make_float2(U[0], U[1]), make_float2(dq[0], dq[1]));
        dq[0] = d01.x;
        dq[1] = d01.y;
        dq[S > 2 ? 2 : 0] = fmaf(cr, U[S > 2 ? 2 : 0], dq[S > 2 ? 2 : 0]);
        DP::dflux(bj, dq, E);
        const float2 a01 = f2fma(f2dup(wk), make_float2(E[0], E[1]), make_float2(acc[0], acc[1]));
        acc[0] = a01.x;
        acc[1] = a01.y;
        acc[S > 2 ? 2 : 0] = fmaf(wk, E[S > 2 ? 2 : 0], acc[S > 2 ? 2 : 0]);
      } else {
#pragma unroll
        for (int c = 0; c < S; c++) dq[c] = fmaf(cr, U[c], dq[c]);
        DP::dflux(bj, dq, E);
#pragma unroll
        for (int c = 0; c < S; c++) acc[c] = fmaf(wk, E[c], acc[c]);
      }
    }
    if constexpr (S == 3 && p >= 3) {
      // a + (x + y) and the order's Taylor sum, components 0 and 1 packed
      const float ifk = TB::invfact(k);
      const float2 s01 = f2add(make_float2(acc[0], acc[1]),
                               f2add(make_float2(acc2[0].x, acc2[1].x), make_float2(acc2[0].y, acc2[1].y)));
      const float2 f01 = f2fma(f2dup(ifk), s01, make_float2(Fsum[0], Fsum[1]));
      Fprev[0] = s01.x;
      Fprev[1] = s01.y;
      Fsum[0] = f01.x;
      Fsum[1] = f01.y;
      constexpr int c2 = S > 2 ? 2 : 0;
      acc[c2] += acc2[c2].x + acc2[c2].y;
      Fprev[c2] = acc[c2];
      Fsum[c2] = fmaf(ifk, acc[c2], Fsum[c2]);
    } else {
#pragma unroll
      for (int c = 0; c < S; c++) {
        acc[c] += acc2[c].x + acc2[c].y;
        Fprev[c] = acc[c];
        Fsum[c] = fmaf(TB::invfact(k), acc[c], Fsum[c]);
      }
    }
  }
  const float w = TB::gh(p, l);
#pragma unroll
  for (int c = 0; c < S; c++) {
    const float v = w * Fsum[c];
    float t = 0.0f;
#pragma unroll
    for (int r = 0; r < n; r++) t += __shfl_sync(mask, v, base + r);
    Gout[c] = t;
  }
}

// cat_delta by a group of 4p lanes, two per node: lane l <-> node
// m = l >> 1 (j = m - p + 1), half h = l & 1. The two lanes of a node split
// the recursion's work and add their partial sums with one shuffle:
//   - U^(k-1)_j: half h sums the nodes r = h p .. h p + p - 1;
//   - the 2p - 1 time levels r != 0: half h takes the levels h p .. h p + p - 1
//     that exist, in float2 pairs; the empty places of a pair carry zero
//     weights.
// Both lanes of a node then hold the same F^(k-1)_j. The sums are grouped
// differently from cat_delta (two partial sums instead of one running sum),
// so the two forms agree to float rounding, not bit for bit. Every lane
// returns G.
template <int p, int FLUX>
__device__ __forceinline__ void cat_delta2(const float *hi, const float *lo, int cs, int l, int base,
                                           float lam, float adv, float gm1, float *Gout) {
  using TB = Tab<float>;
  using DP = DPhys<FLUX>;
  constexpr int S = DP::S;
  constexpr int n = 2 * p;
  constexpr int NL = n - 1;  // time levels r != 0 (level q <-> table row q < p - 1 ? q : q + 1)
  constexpr int K = p;       // levels per half: ceil(NL / 2)
  constexpr int KP = (K + 1) / 2;
  const unsigned mask = ((1u << (2 * n)) - 1u) << base;
  const int m = l >> 1, h = l & 1;
  const int j = m - p + 1;
  float g1h[p];
#pragma unroll
  for (int i = 0; i < p; i++) g1h[i] = TB::g1(p, m, h * p + i);
  float ui[S], uil[S], uj[S], ujl[S], dh[S], dl[S];
#pragma unroll
  for (int c = 0; c < S; c++) {
    ui[c] = hi[c * cs];
    uil[c] = lo[c * cs];
    uj[c] = hi[c * cs + j];
    ujl[c] = lo[c * cs + j];
    dh[c] = uj[c] - ui[c];
    dl[c] = ujl[c] - uil[c];
  }
  float D[S], Fsum[S], Fprev[S];
  float2 del2[KP][S];
  DP::dflux_pair(DP::base2(ui, uil, adv, gm1), dh, dl, D);  // f(u_j) - f(u_i)
  const typename DP::Base bj = DP::base2(uj, ujl, adv, gm1);
#pragma unroll
  for (int c = 0; c < S; c++) {
    Fsum[c] = D[c];
    Fprev[c] = D[c];
  }
#pragma unroll
  for (int q = 0; q < KP; q++)
#pragma unroll
    for (int c = 0; c < S; c++) del2[q][c] = make_float2(0.0f, 0.0f);
#pragma unroll
  for (int k = 2; k <= n; k++) {
    float U[S];
#pragma unroll
    for (int c = 0; c < S; c++) U[c] = 0.0f;
#pragma unroll
    for (int i = 0; i < p; i++)
#pragma unroll
      for (int c = 0; c < S; c++) U[c] = fmaf(g1h[i], __shfl_sync(mask, Fprev[c], base + 2 * (h * p + i)), U[c]);
#pragma unroll
    for (int c = 0; c < S; c++) U[c] = -lam * (U[c] + __shfl_xor_sync(mask, U[c], 1));
    float2 acc2[S];
#pragma unroll
    for (int c = 0; c < S; c++) acc2[c] = make_float2(0.0f, 0.0f);
#pragma unroll
    for (int q = 0; q < KP; q++) {
      // the slot's two levels in either half (a level >= NL is empty)
      float cr0[2], cr1[2], wk0[2], wk1[2];
#pragma unroll
      for (int e = 0; e < 2; e++) {
        const int q0 = 2 * q + e, q1 = K + 2 * q + e;
        const int r0 = q0 < p - 1 ? q0 : q0 + 1, r1 = q1 < p - 1 ? q1 : q1 + 1;
        const bool v0 = q0 < K, v1 = q1 < NL;
        cr0[e] = v0 ? TB::taylor(p, r0, k - 1) : 0.0f;
        wk0[e] = v0 ? TB::gk(p, k - 1, r0) : 0.0f;
        cr1[e] = v1 ? TB::taylor(p, r1, k - 1) : 0.0f;
        wk1[e] = v1 ? TB::gk(p, k - 1, r1) : 0.0f;
      }
      const float2 cr = h ? make_float2(cr1[0], cr1[1]) : make_float2(cr0[0], cr0[1]);
      const float2 wk = h ? make_float2(wk1[0], wk1[1]) : make_float2(wk0[0], wk0[1]);
      float2 E2[S];
#pragma unroll
      for (int c = 0; c < S; c++) del2[q][c] = f2fma(cr, f2dup(U[c]), del2[q][c]);
      DP::dflux_x2(bj, del2[q], E2);
#pragma unroll
      for (int c = 0; c < S; c++) acc2[c] = f2fma(wk, E2[c], acc2[c]);
    }
#pragma unroll
    for (int c = 0; c < S; c++) {
      float a = acc2[c].x + acc2[c].y;
      a += __shfl_xor_sync(mask, a, 1);
      Fprev[c] = a;
      Fsum[c] = fmaf(TB::invfact(k), a, Fsum[c]);
    }
  }
  const float w = TB::gh(p, m);
#pragma unroll
  for (int c = 0; c < S; c++) {
    const float v = w * Fsum[c];
    float t = 0.0f;
#pragma unroll
    for (int r = 0; r < n; r++) t += __shfl_sync(mask, v, base + 2 * r);
    Gout[c] = t;
  }
}

// FL-CAT2 increment G (F* = f(u_i) + G), worked by the L lanes of the
// interface group (all of them call it; the limiter's ratios are spread over
// the lanes, every lane returns G). With D1 = f(u_{i+1}) -
// f(u_i), U = -lambda D1, T0 = df(u_i; U), T1 = df(u_i; u_{i+1} - u_i + U):
//   CAT2:    F1 - f(u_i) = (T0 + T1 + D1) / 4
//   Rusanov, global LF: Flo - f(u_i) = D1 / 2 - alpha (u_{i+1} - u_i) / 2
//   HLL: 0 (s_l >= 0), D1 (s_r <= 0), s_l (s_r (u_{i+1} - u_i) - D1) / (s_r - s_l)
template <int FLUX, int L>
__device__ __forceinline__ void flcat2_delta(const float *hi, const float *lo, int cs, int l, unsigned gmask,
                                             float lam, float adv, float gamma, double advd,
                                             int limiter_form, int lo_flux, float *G) {
  using DP = DPhys<FLUX>;
  constexpr int S = DP::S;
  const float gm1 = gamma - 1.0f;
  float u0[S], u0l[S], u1[S], dh[S], dl[S], du[S], D1[S], U[S], d1[S], T0[S], T1[S];
#pragma unroll
  for (int c = 0; c < S; c++) {
    u0[c] = hi[c * cs];
    u0l[c] = lo[c * cs];
    u1[c] = hi[c * cs + 1];
    dh[c] = u1[c] - u0[c];
    dl[c] = lo[c * cs + 1] - u0l[c];
    du[c] = dh[c] + dl[c];
  }
  const typename DP::Base b0 = DP::base2(u0, u0l, adv, gm1);
  DP::dflux_pair(b0, dh, dl, D1);
#pragma unroll
  for (int c = 0; c < S; c++) {
    U[c] = __fmul_rn(-lam, D1[c]);
    d1[c] = __fadd_rn(du[c], U[c]);
  }
  DP::dflux(b0, U, T0);
  DP::dflux(b0, d1, T1);
  const float s0 = DP::speed(u0, adv, gamma), s1 = DP::speed(u1, adv, gamma);
  const float alpha = lo_flux == ACAT_LO_GLOBAL_LF ? __fdiv_rn(1.0f, lam) : (s1 > s0 ? s1 : s0);
  float sl = 0.0f, sr = 0.0f;
  if (lo_flux == ACAT_LO_HLL) {
    float n0, x0, n1, x1;
    Phys<FLUX>::eig(u0, adv, gamma, n0, x0);
    Phys<FLUX>::eig(u1, adv, gamma, n1, x1);
    sl = n1 < n0 ? n1 : n0;
    sr = x1 > x0 ? x1 : x0;
  }
  // scalar laws with the Roe-speed side: the side decision in FP64 on hi + lo;
  // systems (and the min form): float-float ratios
  const float w =
      (S == 1 && limiter_form == 0)
          ? (float)psi1_g<S>([=](int c, int k) { return (double)hi[c * cs + k] + (double)lo[c * cs + k]; },
                             FLUX == ACAT_FLUX_LINEAR ? 0 : 1, limiter_form, advd)
          : psi1_group_ff<S, L>(hi, lo, cs, 1, l, gmask);
#pragma unroll
  for (int c = 0; c < S; c++) {
    const float G1 = __fmul_rn(0.25f, __fadd_rn(__fadd_rn(T0[c], T1[c]), D1[c]));
    float Glo;
    if (lo_flux == ACAT_LO_HLL)
      Glo = sl >= 0.0f ? 0.0f
                       : (sr <= 0.0f ? D1[c]
                                     : __fdiv_rn(__fmul_rn(sl, __fsub_rn(__fmul_rn(sr, du[c]), D1[c])),
                                                 __fsub_rn(sr, sl)));
    else
      Glo = __fsub_rn(__fmul_rn(0.5f, D1[c]), __fmul_rn(__fmul_rn(0.5f, alpha), du[c]));
    G[c] = fmaf(w, __fsub_rn(G1, Glo), Glo);
  }
}

// Resident CTAs per SM the step kernels are compiled for (register cap
// 65536 / (256 x value)): enough warps to hide the recursion's latency
// without spilling.
template <int P, bool F32>
struct MinCtas {
  static constexpr int value = F32 ? 4 : 2;
};

// dt of this step from the reduced wave speed (1D CFL rule), clipped at
// t_end; no side effects. *t receives the time at the start of the step.
__device__ double step_dt_value(const Step1DArgs &a, double *t, bool *bad) {
  double dt;
  *bad = false;
  if (a.dt_in) {
    dt = *a.dt_in;
  } else if (a.dt_fixed > 0.0) {
    dt = a.dt_fixed;
  } else {
    const double smax = __longlong_as_double((long long)a.smax[a.slot]);
    if (!(smax > 0.0) || !isfinite(smax)) {
      *bad = true;
      dt = 0.0;
    } else {
      dt = a.cfl * a.dx / smax;
    }
  }
  *t = 0.0;
  if (a.tslot) {
    *t = a.tslot[a.slot];
    if (a.t_end > 0.0) {
      if (*t >= a.t_end) dt = 0.0;
      else if (dt > a.t_end - *t) dt = a.t_end - *t;
    }
  }
  return dt;
}

// step_dt_value, and block 0 advances the simulated time, records dt,
// flags a bad wave speed and recycles the slot two steps ahead.
__device__ double step_dt(const Step1DArgs &a) {
  double t;
  bool bad;
  const double dt = step_dt_value(a, &t, &bad);
  if (blockIdx.x == 0) {
    if (bad) atomicOr(a.status, (unsigned)ACAT_STATUS_BAD_DT);
    if (a.tslot) a.tslot[(a.slot + 1) % 3] = t + dt;
    if (a.dt_out) *a.dt_out = dt;
    a.smax[(a.slot + 2) % 3] = 0ull;
  }
  return dt;
}

// Shared-memory workspace of one 1D tile of NW warps.
template <int P, int S, int NW = NT / 32>
struct Smem64 {
  double tile[S][Tiling<P, NW>::TW];
  double Fs[Tiling<P, NW>::NI][S];
  double red[NW];
};
template <int P, int S, int NW = NT / 32, int LPN = 1, int R = 1>
struct Smem32 {
  float thi[S][Tiling<P, NW, LPN, R>::TW], tlo[S][Tiling<P, NW, LPN, R>::TW];
  float Gs[Tiling<P, NW, LPN, R>::NI][S];
  unsigned char rej[S][Tiling<P, NW, LPN, R>::NI];  // rejected orders per (component, interface)
  float redf[NW];
};

// Block-wide maximum of `v` over NW warps (thread 0 returns it).
template <int NW = NT / 32>
__device__ __forceinline__ double block_max(double v, double *red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double r = red[0];
  if (threadIdx.x == 0)
    for (int w = 1; w < NW; w++) r = fmax(r, red[w]);
  return r;
}

// One FP64 tile: cells [i0, i0 + T) of an instance of N cells whose state
// starts at cell `off` of arrays with component stride M; orders (nullable)
// points at the instance's interface 0; the tile's maximal wave speed goes to
// *smax_out. The CTA has NW warps.
template <int P, int FLUX, int NW = NT / 32>
__device__ __forceinline__ void tile_f64(const Step1DArgs &a, Smem64<P, Phys<FLUX>::S, NW> &sm,
                                         const double *__restrict__ uin, double *__restrict__ uout,
                                         long off, long M, long N, long i0, double lam,
                                         int8_t *orders, unsigned long long *smax_out) {
  using TL = Tiling<P, NW>;
  constexpr int NTB = NW * 32;
  constexpr int S = Phys<FLUX>::S;
  for (int q = threadIdx.x; q < S * TL::TW; q += NTB) {
    const int c = q / TL::TW, k = q - c * TL::TW;
    const long g = bc_index(i0 - TL::GH + k, N, a.bc);
    if (acat_in_bounds(g >= 0 && g < N && off + N <= M, a.status)) sm.tile[c][k] = uin[c * M + off + g];
  }
  __syncthreads();
  const double gm1 = a.gamma - 1.0;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int grp = lane / TL::L, l = lane - grp * TL::L;
  const bool valid = grp < TL::GPW;
  const int il = warp * TL::GPW + grp;  // local interface
  const long m = i0 + il;               // interface between cells m-1 and m
  const bool active = valid && m <= N;
  const int ic = il - 1 + TL::GH;       // tile index of cell m-1

  const FiltConst FC = filt_const(a.epsf, a.rf, a.factf);
  const int ps = select_order<P, S, false>(&sm.tile[0][valid ? ic : 0], nullptr, nullptr, TL::TW, l,
                                           grp, active, valid, FC, a.eps, a.thr, a.fact_tau, a.psi2_mod);

  double F[S];
  const int base = grp * TL::L;
  const double *q0 = &sm.tile[0][ic];
  if (active && acat_in_bounds(ic - P + 1 >= 0 && ic + P < TL::TW && il < TL::NI && m <= N, a.status)) {
    if (ps == 4) {
      if constexpr (P >= 4) cat_flux<4, FLUX, double>(q0, TL::TW, l, base, lam, a.adv, gm1, F);
    } else if (ps == 3) {
      if constexpr (P >= 3) if (l < 6) cat_flux<3, FLUX, double>(q0, TL::TW, l, base, lam, a.adv, gm1, F);
    } else if (ps == 2) {
      if constexpr (P >= 2) if (l < 4) cat_flux<2, FLUX, double>(q0, TL::TW, l, base, lam, a.adv, gm1, F);
    } else {
      flcat2_flux<FLUX, TL::L>(q0, TL::TW, l, ((1u << TL::L) - 1u) << base, lam, a.adv, a.gamma,
                               a.limiter_form, a.lo_flux, F);
    }
    if (l == 0) {
#pragma unroll
      for (int c = 0; c < S; c++) sm.Fs[il][c] = F[c];
      if (orders && (il < TL::T || m == N)) orders[m] = (int8_t)ps;
    }
  }
  __syncthreads();

  double smax = 0.0;
  bool bad = false;
  for (int t = threadIdx.x; t < TL::T; t += NTB) {
    const long i = i0 + t;
    if (i >= N) break;
    if (!acat_in_bounds(t + 1 < TL::NI && t + TL::GH < TL::TW && off + i < M, a.status)) continue;
    double un[S];
#pragma unroll
    for (int c = 0; c < S; c++) {
      un[c] = sm.tile[c][t + TL::GH] + lam * (sm.Fs[t][c] - sm.Fs[t + 1][c]);
      uout[c * M + off + i] = un[c];
    }
    bool ok;
    const double sp = Phys<FLUX>::speed(un, a.adv, a.gamma, ok);
    bad |= !ok;
    smax = fmax(smax, sp);
  }
  if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(a.status, (unsigned)ACAT_STATUS_NONPHYSICAL);
  const double v = block_max<NW>(smax, sm.red);
  if (threadIdx.x == 0) atomic_max_pos(smax_out, v);
  __syncthreads();
}

// Order selection and flux increment G of interface il of an FP32 tile, by
// the L lanes of group grp (all 32 lanes of the warp call it; lane l of the
// group). thi, tlo: component 0 of the staged tile (components tw apart),
// cell k of the tile at index k; interface il lies between tile cells
// il - 1 + GH and il + GH. xw: the warp's exchange slots. Every lane of an
// active group returns the code p_s and G (lanes beyond the selected order's
// 2p return G unset).
// rej (nullable): the tile's rejected orders per (component, interface), from
// reject_pass_f32; the group then ORs its interface's bits instead of
// deciding in select_order.
template <int P, int FLUX, int LPN>
__device__ __forceinline__ int iface_f32(const Step1DArgs &a, const float *thi, const float *tlo, int tw,
                                         int il, int grp, int l, bool valid, bool active, float lam,
                                         const FiltConst &FC, float4 *xw, float *G,
                                         const unsigned char *rej = nullptr, int ni = 0) {
  using TL = Tiling<P, NT / 32, LPN>;
  using DP = DPhys<FLUX>;
  constexpr int S = DP::S;
  const float adv = a.advf, gam = a.gammaf, gm1 = a.gm1f;
  const int ic = il - 1 + TL::GH;
  const int icv = valid ? ic : 0;
  int ps = 1;
  if (rej) {
    if constexpr (P >= 2) {
      unsigned r = 0;
      if (active) {
#pragma unroll
        for (int c = 0; c < S; c++) r |= rej[c * ni + il];
      }
      const unsigned accept = ~r & ((1u << (P - 1)) - 1u);
      ps = accept ? (32 - __clz(accept)) + 1 : 1;
    }
  } else {
    ps = select_order<P, S, true, LPN>(nullptr, thi + icv, tlo + icv, tw, l, grp, active, valid, FC, a.eps,
                                       a.thr, a.fact_tau, a.psi2_mod);
  }
  const int base = grp * TL::L;
  float4 *const xg = xw + (P >= 3 ? xslot(base) : base);
  if (active && acat_in_bounds(ic - P + 1 >= 0 && ic + P < tw, a.status)) {
    const float *h0 = thi + ic, *l0 = tlo + ic;
    if (ps == 4) {
      if constexpr (P >= 4) {
        if constexpr (LPN == 2) cat_delta2<4, FLUX>(h0, l0, tw, l, base, lam, adv, gm1, G);
        else cat_delta<4, FLUX>(h0, l0, tw, l, base, lam, adv, gm1, xg, G);
      }
    } else if (ps == 3) {
      if constexpr (P >= 3) {
        if constexpr (LPN == 2) {
          if (l < 12) cat_delta2<3, FLUX>(h0, l0, tw, l, base, lam, adv, gm1, G);
        } else if (l < 6) {
          cat_delta<3, FLUX>(h0, l0, tw, l, base, lam, adv, gm1, xg, G);
        }
      }
    } else if (ps == 2) {
      if constexpr (P >= 2) {
        if constexpr (LPN == 2) {
          if (l < 8) cat_delta2<2, FLUX>(h0, l0, tw, l, base, lam, adv, gm1, G);
        } else if (l < 4) {
          cat_delta<2, FLUX>(h0, l0, tw, l, base, lam, adv, gm1, xg, G);
        }
      }
    } else {
      flcat2_delta<FLUX, TL::L>(h0, l0, tw, l, ((1u << TL::L) - 1u) << base, lam, adv, gam, a.adv,
                                a.limiter_form, a.lo_flux, G);
    }
  }
  return ps;
}

// The order decisions of a staged FP32 tile, spread over all nthreads
// threads: for every (component c, interface il < ni) with i0 + il <= N, the
// rejected orders of component c (reject_set32: the filtered decision with its
// literal FP64 fallback on hi + lo, as select_order takes it), written to
// rej[c ni + il]. Component-major, so that the threads of a warp read
// consecutive cells. Interfaces beyond the instance get 0 (never used).
template <int P, int S, int GH>
__device__ __forceinline__ void reject_pass_f32(const Step1DArgs &a, const float *thi, const float *tlo, int tw,
                                                int ni, long i0, long N, const FiltConst &FC, unsigned char *rej,
                                                int nthreads) {
  if constexpr (P >= 2) {
    for (int q = threadIdx.x; q < S * ni; q += nthreads) {
      const int c = q / ni, il = q - c * ni;
      unsigned r = 0;
      if (i0 + il <= N && acat_in_bounds(il - 1 + GH - P + 1 >= 0 && il - 1 + GH + P < tw, a.status)) {
        const int ic = il - 1 + GH;
        r = reject_set32<P>(thi + c * tw + ic, tlo + c * tw + ic, 1, c == 0, FC, a.eps, a.thr, a.fact_tau,
                            a.psi2_mod);
      }
      rej[q] = (unsigned char)r;
    }
  }
}

// Conservative update (Eq. 2.12) of the cell at tile index k of an FP32 tile
// (component 0 rows thi, tlo, components tw apart) with the flux increments
// Gl = G_{i-1/2}, Gr = G_{i+1/2}: u += lam (f(u_{i-1}) - f(u_i) + Gl - Gr)
// added to the pair (hi, lo) by TwoSum then Fast2Sum, written to cell i of
// the output (component stride M from offset off). Folds the new state's
// float wave speed into *smax and its physicality into *bad.
template <int FLUX>
__device__ __forceinline__ void update_cell_f32(const Step1DArgs &a, const float *thi, const float *tlo, int tw,
                                                int k, float lam, const float *Gl, const float *Gr,
                                                float *__restrict__ uout, long M, long off, long i, float *smax,
                                                bool *bad) {
  using DP = DPhys<FLUX>;
  constexpr int S = DP::S;
  if (!acat_in_bounds(k >= 1 && k < tw && i >= 0 && off + i < M, a.status)) return;
  const float adv = a.advf, gam = a.gammaf, gm1 = a.gm1f;
  float ui[S], uil[S], dh[S], dl[S], B[S];
#pragma unroll
  for (int c = 0; c < S; c++) {
    ui[c] = thi[c * tw + k];
    uil[c] = tlo[c * tw + k];
    dh[c] = thi[c * tw + k - 1] - ui[c];
    dl[c] = tlo[c * tw + k - 1] - uil[c];
  }
  DP::dflux_pair(DP::base2(ui, uil, adv, gm1), dh, dl, B);  // f(u_{i-1}) - f(u_i)
  float un[S], lo_[S];
#pragma unroll
  for (int c = 0; c < S; c++) {
    const float d = __fmul_rn(lam, __fadd_rn(B[c], __fsub_rn(Gl[c], Gr[c])));
    const float h = ui[c], w = uil[c];
    // TwoSum(h, d): s + e = h + d exactly
    const float s = __fadd_rn(h, d);
    const float bp = __fsub_rn(s, h);
    const float e = __fadd_rn(__fsub_rn(h, __fsub_rn(s, bp)), __fsub_rn(d, bp));
    const float w2 = __fadd_rn(w, e);
    // Fast2Sum(s, w2), |s| >= |w2|: renormalised pair
    const float hn = __fadd_rn(s, w2);
    const float ln = __fsub_rn(w2, __fsub_rn(hn, s));
    uout[c * M + off + i] = hn;
    uout[(S + c) * M + off + i] = ln;
    un[c] = hn;
    lo_[c] = ln;
  }
  // wave speed in float (the FP32 path's dt is exact to float rounding);
  // a state that looks non-physical in float is re-checked in FP64
  const float sf = DP::speed(un, adv, gam);
  if (!DP::physical(un, gam)) {
    double ud[S];
#pragma unroll
    for (int c = 0; c < S; c++) ud[c] = (double)un[c] + (double)lo_[c];
    bool ok;
    Phys<FLUX>::speed(ud, a.adv, a.gamma, ok);
    *bad |= !ok;
  }
  *smax = fmaxf(*smax, sf);
}

// One FP32 tile on the compensated state [hi(s x M); lo(s x M)].
// Three CTA barriers per tile: after staging (which also publishes *lam_sm,
// written by the caller before the call), after the order decisions, and
// between the flux and update phases. There is none at the end: a caller that loops over tiles
// alternates between two workspaces (and two lam slots), so the next tile's
// staging cannot overwrite what a slower warp still reads. The wave speed
// maximum goes out per warp (atomic max of the warps that updated cells).
template <int P, int FLUX, int NW = NT / 32, int LPN = 1, int R = 1>
__device__ __forceinline__ void tile_f32(const Step1DArgs &a, Smem32<P, DPhys<FLUX>::S, NW, LPN, R> &sm,
                                         const float *__restrict__ uin, float *__restrict__ uout,
                                         long off, long M, long N, long i0, const float *lam_sm,
                                         int8_t *orders, unsigned long long *smax_out) {
  using TL = Tiling<P, NW, LPN, R>;
  constexpr int NTB = NW * 32;
  using DP = DPhys<FLUX>;
  constexpr int S = DP::S;
  for (int q = threadIdx.x; q < S * TL::TW; q += NTB) {
    const int c = q / TL::TW, k = q - c * TL::TW;
    const long g = bc_index(i0 - TL::GH + k, N, a.bc);
    if (!acat_in_bounds(g >= 0 && g < N && off + N <= M, a.status)) continue;
    sm.thi[c][k] = uin[c * M + off + g];
    sm.tlo[c][k] = uin[(S + c) * M + off + g];
  }
  __syncthreads();
  const float lam = *lam_sm;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int grp = lane / TL::L, l = lane - grp * TL::L;
  const bool valid = grp < TL::GPW;

  // the warps' shuffle-free exchange slots of the one-lane-per-node recursion
  __shared__ float4 xs[(LPN == 1 && P >= 2 && S > 1) ? NW * 2 * XSET : 1];
  const FiltConst FC = filt_const(a.epsf, a.rf, a.factf);
  // every order decision of the tile first, over all threads (a group's
  // lanes beyond its S components would otherwise wait through them)
  reject_pass_f32<P, S, TL::GH>(a, &sm.thi[0][0], &sm.tlo[0][0], TL::TW, TL::NI, i0, N, FC, &sm.rej[0][0], NTB);
  if (P >= 2) __syncthreads();
  // R rounds: round rnd takes the interfaces (rnd NW + warp) GPW + grp, so
  // each round covers NW GPW consecutive interfaces; the tile's barriers
  // serve all R rounds
#pragma unroll 1
  for (int rnd = 0; rnd < R; rnd++) {
    if (rnd > 0) __syncwarp();  // the exchange slots of the last round are read
    const int il = (rnd * NW + warp) * TL::GPW + grp;
    const long m = i0 + il;
    const bool active = valid && m <= N;
    float G[S];
    const int ps = iface_f32<P, FLUX, LPN>(a, &sm.thi[0][0], &sm.tlo[0][0], TL::TW, il, grp, l, valid, active,
                                           lam, FC, &xs[warp * 2 * XSET], G, &sm.rej[0][0], TL::NI);
    if (active && l == 0 && acat_in_bounds(il < TL::NI && m <= N, a.status)) {
#pragma unroll
      for (int c = 0; c < S; c++) sm.Gs[il][c] = G[c];
      if (orders && (il < TL::T || m == N)) orders[m] = (int8_t)ps;
    }
  }  // rounds
  __syncthreads();

  float smax = 0.0f;
  bool bad = false;
  for (int t = threadIdx.x; t < TL::T; t += NTB) {
    const long i = i0 + t;
    if (i >= N) break;
    if (!acat_in_bounds(t + 1 < TL::NI, a.status)) continue;
    update_cell_f32<FLUX>(a, &sm.thi[0][0], &sm.tlo[0][0], TL::TW, t + TL::GH, lam, sm.Gs[t], sm.Gs[t + 1], uout,
                          M, off, i, &smax, &bad);
  }
  if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(a.status, (unsigned)ACAT_STATUS_NONPHYSICAL);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) smax = fmaxf(smax, __shfl_xor_sync(0xffffffffu, smax, o));
  if (lane == 0 && warp * 32 < TL::T) atomic_max_pos(smax_out, (double)smax);
}
}  // namespace
