// step1d.cu -- the 1D ACAT step on sm_103a CUDA cores (FP64, and FP32 on a
// compensated state).
//
// One CTA owns T consecutive cells and computes the T+1 interface fluxes
// around them (the last one is recomputed by the next CTA). The cells
// [i0 - GH, i0 + T + GH) are staged once in shared memory with the boundary
// condition applied while loading. Each interface is worked by a group of 2P
// lanes of one warp, one lane per stencil node j = -p+1..p:
//   - the (p, component) pairs of the indicators psi^p (Eqs. 3.8-3.12, the
//     minimum over components of Sec. 3.4) are spread over the group's lanes.
//     Each pair is decided by a float test with a certified error margin
//     (psi_filter); only when the margin cannot settle it is psi^p evaluated
//     literally with explicitly rounded FP64 operations in the order of its
//     definition. Either way the decision is the one a literal FP64
//     evaluation of the same state takes. An OR-reduction over the group
//     gives p_s = max A (Eqs. 3.2-3.3);
//   - for p_s >= 2 every lane runs the local Taylor recursion of Sec. 2.2 for
//     its node in registers, in the dt-scaled form
//         U^(k-1)_j = -lambda sum_r gamma^{1,j}_r F^(k-2)_r     (shuffles)
//         F^(k-1)_j = sum_r gamma^{k-1,0}_r f(u_j + sum_l r^l/l! U^(l)_j)
//     (U^(l) = dt^l u~^(l), F^(k) = dt^k f~^(k)), keeping the Taylor sums at
//     the 2p-1 time levels r != 0 as running values (one FMA per level and
//     order instead of a Horner pass); the flux is sum_k 1/k! sum_j
//     gamma^{0,1/2}_j F^(k-1)_j (Eq. 2.14) reduced across the group;
//   - for p_s = 1 lane 0 evaluates FL-CAT2 (Eqs. 3.4-3.7).
// The conservative update (Eq. 2.12) follows from shared memory, and its
// epilogue reduces the wave speed of the new state for the next step's CFL
// dt into a triple-buffered slot (atomic max on ordered double bits).
//
// FP32 variant: the state is a compensated float pair (hi, lo). The order
// decisions are those of FP64 on the exact value hi + lo (the filtered test
// falls back to FP64 on hi + lo), and so is the limiter psi^1 of FL-CAT2
// interfaces; the wave speed for the next step's dt is reduced in float. The
// recursion runs in float in a delta formulation (see cat_delta):
// every flux is carried as f(u_i) + G, G built from flux increments computed
// in a cancellation-free form, so float rounding is relative to increments of
// size O(dx) rather than to |f|. The update adds lambda (f(u_{i-1}) - f(u_i) +
// G_{i-1/2} - G_{i+1/2}) to the pair with an error-free transformation
// (Knuth's TwoSum, then Dekker's Fast2Sum).
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
  R g1r[n];
#pragma unroll
  for (int r = 0; r < n; r++) g1r[r] = TB::g1(p, l, r);
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
    for (int c = 0; c < S; c++) {
      U[c] *= -lam;
      acc[c] = TB::gk(p, k - 1, p - 1) * f0[c];
    }
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
    R t = R(0);
#pragma unroll
    for (int r = 0; r < n; r++) t += __shfl_sync(mask, v, base + r);
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
  __device__ static __forceinline__ void dflux(const Base &b, const float *d, float *df) {
    df[0] = b.a * d[0];
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
  // (u + d)^2/2 - u^2/2 = d (u + d/2)
  __device__ static __forceinline__ void dflux(const Base &b, const float *d, float *df) {
    df[0] = d[0] * fmaf(0.5f, d[0], b.u);
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
    float rho, m, v, H, gm1;
  };
  __device__ static __forceinline__ Base base(const float *u, float, float gm1) {
    Base b;
    b.rho = u[0];
    b.m = u[1];
    b.v = u[1] * __frcp_rn(u[0]);
    const float p = gm1 * fmaf(-0.5f * u[1], b.v, u[2]);
    b.H = u[2] + p;
    b.gm1 = gm1;
    return b;
  }
  // With u = (rho, m, E), d = (a, b, c), v = m/rho, H = E + p:
  //   dv = (b - v a) / (rho + a)          [v' - v]
  //   d(mv) = m dv + b (v + dv)
  //   dp = (gamma - 1)(c - d(mv)/2)
  //   df = (b, d(mv) + dp, dv H + (v + dv)(c + dp))
  __device__ static __forceinline__ void dflux(const Base &B, const float *d, float *df) {
    const float dv = fmaf(-B.v, d[0], d[1]) * __frcp_rn(B.rho + d[0]);
    const float vn = B.v + dv;
    const float dmv = fmaf(B.m, dv, d[1] * vn);
    const float dp = B.gm1 * fmaf(-0.5f, dmv, d[2]);
    df[0] = d[1];
    df[1] = dmv + dp;
    df[2] = fmaf(dv, B.H, vn * (d[2] + dp));
  }
  // the same for two increments packed in float2 lanes
  __device__ static __forceinline__ void dflux_x2(const Base &B, const float2 *d, float2 *df) {
    const float2 t = f2fma(f2dup(-B.v), d[0], d[1]);
    const float2 den = f2add(f2dup(B.rho), d[0]);
    const float2 dv = f2mul(t, make_float2(__frcp_rn(den.x), __frcp_rn(den.y)));
    const float2 vn = f2add(f2dup(B.v), dv);
    const float2 dmv = f2fma(f2dup(B.m), dv, f2mul(d[1], vn));
    const float2 dp = f2mul(f2dup(B.gm1), f2fma(f2dup(-0.5f), dmv, d[2]));
    df[0] = d[1];
    df[1] = f2add(dmv, dp);
    df[2] = f2fma(dv, f2dup(B.H), f2mul(vn, f2add(d[2], dp)));
  }
  __device__ static __forceinline__ float speed(const float *u, float, float gamma) {
    const float v = u[1] / u[0];
    const float p = (gamma - 1.0f) * (u[2] - 0.5f * u[1] * v);
    return fabsf(v) + sqrtf(fmaxf(gamma * p / u[0], 0.0f));
  }
  __device__ static __forceinline__ bool physical(const float *u, float gamma) {
    const float p = (gamma - 1.0f) * (u[2] - 0.5f * u[1] * (u[1] / u[0]));
    return u[0] > 0.0f && p > 0.0f && isfinite(u[0]) && isfinite(u[1]) && isfinite(u[2]);
  }
};

// CAT2p increment G of one interface by a group of 2p lanes (lane l <-> node
// j = l - p + 1). hi/lo point at cell i of component 0 of the compensated
// tile, components `cs` apart. Every lane returns G.
template <int p, int FLUX>
__device__ __forceinline__ void cat_delta(const float *hi, const float *lo, int cs, int l, int base,
                                          float lam, float adv, float gm1, float *Gout) {
  using TB = Tab<float>;
  using DP = DPhys<FLUX>;
  constexpr int S = DP::S;
  constexpr int n = 2 * p;
  const unsigned mask = ((1u << n) - 1u) << base;
  const int j = l - p + 1;
  float g1r[n];
#pragma unroll
  for (int r = 0; r < n; r++) g1r[r] = TB::g1(p, l, r);
  float ui[S], uj[S], d0[S];
#pragma unroll
  for (int c = 0; c < S; c++) {
    ui[c] = hi[c * cs];
    uj[c] = hi[c * cs + j];
    d0[c] = (hi[c * cs + j] - hi[c * cs]) + (lo[c * cs + j] - lo[c * cs]);
  }
  // the 2p - 1 time levels r != 0 (level q <-> table row q < p - 1 ? q : q + 1)
  // are worked in pairs packed in float2 lanes (p <= 3; at p = 4 the pairs
  // would cost the registers of a fourth resident CTA), the last one alone
  constexpr int NL = n - 1, NP = p <= 3 ? NL / 2 : 0;
  float D[S], Fsum[S], Fprev[S], dels[NL - 2 * NP][S];
  float2 del2[NP > 0 ? NP : 1][S];
  DP::dflux(DP::base(ui, adv, gm1), d0, D);  // f(u_j) - f(u_i)
  const typename DP::Base bj = DP::base(uj, adv, gm1);
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
#pragma unroll
    for (int r = 0; r < n; r++)
#pragma unroll
      for (int c = 0; c < S; c++) U[c] = fmaf(g1r[r], __shfl_sync(mask, Fprev[c], base + r), U[c]);
    float acc[S];
    float2 acc2[S];
#pragma unroll
    for (int c = 0; c < S; c++) {
      U[c] *= -lam;
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
      float E[S];
#pragma unroll
      for (int c = 0; c < S; c++) dels[q - 2 * NP][c] = fmaf(TB::taylor(p, rs, k - 1), U[c], dels[q - 2 * NP][c]);
      DP::dflux(bj, dels[q - 2 * NP], E);
#pragma unroll
      for (int c = 0; c < S; c++) acc[c] = fmaf(TB::gk(p, k - 1, rs), E[c], acc[c]);
    }
#pragma unroll
    for (int c = 0; c < S; c++) {
      acc[c] += acc2[c].x + acc2[c].y;
      Fprev[c] = acc[c];
      Fsum[c] = fmaf(TB::invfact(k), acc[c], Fsum[c]);
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
  float u0[S], u1[S], du[S], D1[S], U[S], d1[S], T0[S], T1[S];
#pragma unroll
  for (int c = 0; c < S; c++) {
    u0[c] = hi[c * cs];
    u1[c] = hi[c * cs + 1];
    du[c] = (hi[c * cs + 1] - hi[c * cs]) + (lo[c * cs + 1] - lo[c * cs]);
  }
  const typename DP::Base b0 = DP::base(u0, adv, gm1);
  DP::dflux(b0, du, D1);
#pragma unroll
  for (int c = 0; c < S; c++) {
    U[c] = -lam * D1[c];
    d1[c] = du[c] + U[c];
  }
  DP::dflux(b0, U, T0);
  DP::dflux(b0, d1, T1);
  const float s0 = DP::speed(u0, adv, gamma), s1 = DP::speed(u1, adv, gamma);
  const float alpha = lo_flux == ACAT_LO_GLOBAL_LF ? 1.0f / lam : (s1 > s0 ? s1 : s0);
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
    const float G1 = 0.25f * (T0[c] + T1[c] + D1[c]);
    float Glo;
    if (lo_flux == ACAT_LO_HLL)
      Glo = sl >= 0.0f ? 0.0f : (sr <= 0.0f ? D1[c] : sl * (sr * du[c] - D1[c]) / (sr - sl));
    else
      Glo = 0.5f * D1[c] - 0.5f * alpha * du[c];
    G[c] = fmaf(w, G1 - Glo, Glo);
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

// Shared-memory workspace of one 1D tile.
template <int P, int S>
struct Smem64 {
  double tile[S][Tiling<P>::TW];
  double Fs[Tiling<P>::NI][S];
  double red[NT / 32];
};
template <int P, int S>
struct Smem32 {
  float thi[S][Tiling<P>::TW], tlo[S][Tiling<P>::TW];
  float Gs[Tiling<P>::NI][S];
  float redf[NT / 32];
};

// Block-wide maximum of a non-negative float `v` (thread 0 returns it).
__device__ __forceinline__ float block_max_f(float v, float *red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < NT / 32; w++) v = fmaxf(v, red[w]);
  }
  return v;
}

// Block-wide maximum of `v` (thread 0 returns it).
__device__ __forceinline__ double block_max(double v, double *red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double r = red[0];
  if (threadIdx.x == 0)
    for (int w = 1; w < NT / 32; w++) r = fmax(r, red[w]);
  return r;
}

// One FP64 tile: cells [i0, i0 + T) of an instance of N cells whose state
// starts at cell `off` of arrays with component stride M; orders (nullable)
// points at the instance's interface 0; the tile's maximal wave speed goes to
// *smax_out.
template <int P, int FLUX>
__device__ __forceinline__ void tile_f64(const Step1DArgs &a, Smem64<P, Phys<FLUX>::S> &sm,
                                         const double *__restrict__ uin, double *__restrict__ uout,
                                         long off, long M, long N, long i0, double lam,
                                         int8_t *orders, unsigned long long *smax_out) {
  using TL = Tiling<P>;
  constexpr int S = Phys<FLUX>::S;
  for (int q = threadIdx.x; q < S * TL::TW; q += NT) {
    const int c = q / TL::TW, k = q - c * TL::TW;
    sm.tile[c][k] = uin[c * M + off + bc_index(i0 - TL::GH + k, N, a.bc)];
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
  if (active) {
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
  for (int t = threadIdx.x; t < TL::T; t += NT) {
    const long i = i0 + t;
    if (i >= N) break;
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
  const double v = block_max(smax, sm.red);
  if (threadIdx.x == 0) atomic_max_pos(smax_out, v);
  __syncthreads();
}

// One FP32 tile on the compensated state [hi(s x M); lo(s x M)].
// Two CTA barriers per tile: after staging (which also publishes *lam_sm,
// written by the caller before the call) and between the flux and update
// phases. There is none at the end: a caller that loops over tiles
// alternates between two workspaces (and two lam slots), so the next tile's
// staging cannot overwrite what a slower warp still reads. The wave speed
// maximum goes out per warp (atomic max of the warps that updated cells).
template <int P, int FLUX>
__device__ __forceinline__ void tile_f32(const Step1DArgs &a, Smem32<P, DPhys<FLUX>::S> &sm,
                                         const float *__restrict__ uin, float *__restrict__ uout,
                                         long off, long M, long N, long i0, const float *lam_sm,
                                         int8_t *orders, unsigned long long *smax_out) {
  using TL = Tiling<P>;
  using DP = DPhys<FLUX>;
  constexpr int S = DP::S;
  for (int q = threadIdx.x; q < S * TL::TW; q += NT) {
    const int c = q / TL::TW, k = q - c * TL::TW;
    const long g = off + bc_index(i0 - TL::GH + k, N, a.bc);
    sm.thi[c][k] = uin[c * M + g];
    sm.tlo[c][k] = uin[(S + c) * M + g];
  }
  __syncthreads();
  const float lam = *lam_sm;
  const float adv = a.advf, gam = a.gammaf, gm1 = a.gm1f;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int grp = lane / TL::L, l = lane - grp * TL::L;
  const bool valid = grp < TL::GPW;
  const int il = warp * TL::GPW + grp;
  const long m = i0 + il;
  const bool active = valid && m <= N;
  const int ic = il - 1 + TL::GH;

  const FiltConst FC = filt_const(a.epsf, a.rf, a.factf);
  const int icv = valid ? ic : 0;
  const int ps = select_order<P, S, true>(nullptr, &sm.thi[0][icv], &sm.tlo[0][icv], TL::TW, l, grp,
                                          active, valid, FC, a.eps, a.thr, a.fact_tau, a.psi2_mod);

  float G[S];
  const int base = grp * TL::L;
  if (active) {
    const float *h0 = &sm.thi[0][ic], *l0 = &sm.tlo[0][ic];
    if (ps == 4) {
      if constexpr (P >= 4) cat_delta<4, FLUX>(h0, l0, TL::TW, l, base, lam, adv, gm1, G);
    } else if (ps == 3) {
      if constexpr (P >= 3) if (l < 6) cat_delta<3, FLUX>(h0, l0, TL::TW, l, base, lam, adv, gm1, G);
    } else if (ps == 2) {
      if constexpr (P >= 2) if (l < 4) cat_delta<2, FLUX>(h0, l0, TL::TW, l, base, lam, adv, gm1, G);
    } else {
      flcat2_delta<FLUX, TL::L>(h0, l0, TL::TW, l, ((1u << TL::L) - 1u) << base, lam, adv, gam, a.adv,
                                a.limiter_form, a.lo_flux, G);
    }
    if (l == 0) {
#pragma unroll
      for (int c = 0; c < S; c++) sm.Gs[il][c] = G[c];
      if (orders && (il < TL::T || m == N)) orders[m] = (int8_t)ps;
    }
  }
  __syncthreads();

  float smax = 0.0f;
  bool bad = false;
  for (int t = threadIdx.x; t < TL::T; t += NT) {
    const long i = i0 + t;
    if (i >= N) break;
    const int k = t + TL::GH;
    float ui[S], dl[S], B[S];
#pragma unroll
    for (int c = 0; c < S; c++) {
      ui[c] = sm.thi[c][k];
      dl[c] = (sm.thi[c][k - 1] - sm.thi[c][k]) + (sm.tlo[c][k - 1] - sm.tlo[c][k]);
    }
    DP::dflux(DP::base(ui, adv, gm1), dl, B);  // f(u_{i-1}) - f(u_i)
    float un[S], lo_[S];
#pragma unroll
    for (int c = 0; c < S; c++) {
      const float d = __fmul_rn(lam, __fadd_rn(B[c], __fsub_rn(sm.Gs[t][c], sm.Gs[t + 1][c])));
      const float h = sm.thi[c][k], w = sm.tlo[c][k];
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
      bad |= !ok;
    }
    smax = fmaxf(smax, sf);
  }
  if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(a.status, (unsigned)ACAT_STATUS_NONPHYSICAL);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) smax = fmaxf(smax, __shfl_xor_sync(0xffffffffu, smax, o));
  if (lane == 0 && warp * 32 < TL::T) atomic_max_pos(smax_out, (double)smax);
}

template <int P, int FLUX>
__global__ void __launch_bounds__(NT, MinCtas<P, false>::value) k_step1d_f64(const Step1DArgs a) {
  __shared__ Smem64<P, Phys<FLUX>::S> sm;
  __shared__ double s_lam;
  if (threadIdx.x == 0) s_lam = step_dt(a) / a.dx;
  __syncthreads();
  tile_f64<P, FLUX>(a, sm, static_cast<const double *>(a.u_in), static_cast<double *>(a.u_out), 0,
                    a.N, a.N, (long)blockIdx.x * Tiling<P>::T, s_lam, a.orders,
                    &a.smax[(a.slot + 1) % 3]);
}

template <int P, int FLUX>
__global__ void __launch_bounds__(NT, MinCtas<P, true>::value) k_step1d_f32(const Step1DArgs a) {
  __shared__ Smem32<P, DPhys<FLUX>::S> sm;
  __shared__ float s_lam;
  if (threadIdx.x == 0) s_lam = (float)(step_dt(a) / a.dx);
  tile_f32<P, FLUX>(a, sm, static_cast<const float *>(a.u_in), static_cast<float *>(a.u_out), 0,
                    a.N, a.N, (long)blockIdx.x * Tiling<P>::T, &s_lam, a.orders,
                    &a.smax[(a.slot + 1) % 3]);
}

// FP64 step in small CTAs (NWF warps): CTA b computes the NI interfaces
// [b NI, b NI + NI) and updates the cells between them; the cell between
// two CTAs is updated by whichever of the two finishes second. Each CTA
// publishes its edge fluxes, fences, and counts itself in at the boundary
// counters of its left and right neighbours (atomicAdd; no CTA ever waits):
// the one that reads 1 owns the boundary cell, reads the other edge flux from
// L2 and resets the counter for the next step. Small CTAs spread a step's
// interfaces evenly over the SMs, and no interface is computed twice.
template <int P, int FLUX>
__global__ void __launch_bounds__(NWF * 32, 16 / NWF) k_step1d_fine(const Step1DArgs a) {
  using TL = Tiling<P, NWF>;
  constexpr int S = Phys<FLUX>::S;
  constexpr int NTF = NWF * 32;
  __shared__ double tile[S][TL::TW];
  __shared__ double Fs[TL::NI][S];
  __shared__ double red[NWF];
  __shared__ double s_lam;
  __shared__ int s_own[2];
  const long N = a.N, i0 = (long)blockIdx.x * TL::NI;
  const double *__restrict__ uin = static_cast<const double *>(a.u_in);
  double *__restrict__ uout = static_cast<double *>(a.u_out);
  if (threadIdx.x == 0) s_lam = step_dt(a) / a.dx;
  for (int q = threadIdx.x; q < S * TL::TW; q += NTF) {
    const int c = q / TL::TW, k = q - c * TL::TW;
    tile[c][k] = uin[c * N + bc_index(i0 - TL::GH + k, N, a.bc)];
  }
  __syncthreads();
  const double lam = s_lam, gm1 = a.gamma - 1.0;
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
  if (active) {
    double F[S];
    const int base = grp * TL::L;
    const double *q0 = &tile[0][ic];
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
      for (int c = 0; c < S; c++) Fs[il][c] = F[c];
      if (a.orders) a.orders[m] = (int8_t)ps;
    }
  }
  __syncthreads();
  const long nI = (N + 1 - i0) < TL::NI ? (N + 1 - i0) : TL::NI;  // interfaces of this CTA
  const bool has_left = blockIdx.x > 0, has_right = i0 + TL::NI <= N;
  if (threadIdx.x == 0) {
    // publish the edge fluxes, then count in at both boundaries
#pragma unroll
    for (int c = 0; c < S; c++) {
      if (has_left) a.flux_buf[c * (N + 1) + i0] = Fs[0][c];
      if (has_right) a.flux_buf[c * (N + 1) + i0 + TL::NI - 1] = Fs[TL::NI - 1][c];
    }
    __threadfence();
    int own0 = 0, own1 = 0;
    if (has_left && atomicAdd(&a.cnt[blockIdx.x - 1], 1) == 1) {
      own0 = 1;
      a.cnt[blockIdx.x - 1] = 0;
    }
    if (has_right && atomicAdd(&a.cnt[blockIdx.x], 1) == 1) {
      own1 = 1;
      a.cnt[blockIdx.x] = 0;
    }
    s_own[0] = own0;
    s_own[1] = own1;
  }
  __syncthreads();
  double smax = 0.0;
  bool bad = false;
  // cells t = 0 .. nI - 2 lie between two interfaces of this CTA; task nI - 1
  // is the left boundary cell i0 - 1, task nI the right one i0 + NI - 1
  for (int t = threadIdx.x; t <= nI; t += NTF) {
    long i;
    int k;
    double Fl[S], Fr[S];
    if (t < nI - 1) {
      i = i0 + t;
      k = t + TL::GH;
#pragma unroll
      for (int c = 0; c < S; c++) {
        Fl[c] = Fs[t][c];
        Fr[c] = Fs[t + 1][c];
      }
    } else if (t == nI - 1) {
      if (!s_own[0]) continue;
      i = i0 - 1;
      k = TL::GH - 1;
#pragma unroll
      for (int c = 0; c < S; c++) {
        Fl[c] = __ldcg(&a.flux_buf[c * (N + 1) + i0 - 1]);
        Fr[c] = Fs[0][c];
      }
    } else {
      if (!s_own[1]) continue;
      i = i0 + TL::NI - 1;
      k = TL::NI - 1 + TL::GH;
#pragma unroll
      for (int c = 0; c < S; c++) {
        Fl[c] = Fs[TL::NI - 1][c];
        Fr[c] = __ldcg(&a.flux_buf[c * (N + 1) + i0 + TL::NI]);
      }
    }
    double un[S];
#pragma unroll
    for (int c = 0; c < S; c++) {
      un[c] = tile[c][k] + lam * (Fl[c] - Fr[c]);
      uout[c * N + i] = un[c];
    }
    bool ok;
    smax = fmax(smax, Phys<FLUX>::speed(un, a.adv, a.gamma, ok));
    bad |= !ok;
  }
  if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(a.status, (unsigned)ACAT_STATUS_NONPHYSICAL);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) smax = fmax(smax, __shfl_xor_sync(0xffffffffu, smax, o));
  if (lane == 0) red[warp] = smax;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = red[0];
#pragma unroll
    for (int w = 1; w < NWF; w++) v = fmax(v, red[w]);
    atomic_max_pos(&a.smax[(a.slot + 1) % 3], v);
  }
}

// dt of instance b of a batch (1D CFL rule on the instance's own wave speed
// and grid); the instance's first tile advances its time and recycles its
// slot two steps ahead.
__device__ double batch_dt(const Step1DArgs &a, const BatchArgs &bt, int b, bool leader, double dx) {
  const long B = bt.B;
  double dt;
  if (a.dt_fixed > 0.0) {
    dt = a.dt_fixed;
  } else {
    const double smax = __longlong_as_double((long long)bt.smax[a.slot * B + b]);
    if (!(smax > 0.0) || !isfinite(smax)) {
      if (leader) atomicOr(a.status, (unsigned)ACAT_STATUS_BAD_DT);
      dt = 0.0;
    } else {
      dt = a.cfl * dx / smax;
    }
  }
  const double t = bt.t[a.slot * B + b];
  if (a.t_end > 0.0) {
    if (t >= a.t_end) dt = 0.0;
    else if (dt > a.t_end - t) dt = a.t_end - t;
  }
  if (leader) {
    bt.t[((a.slot + 1) % 3) * B + b] = t + dt;
    bt.smax[((a.slot + 2) % 3) * B + b] = 0ull;
    if (bt.dt_out) bt.dt_out[b] = dt;
  }
  return dt;
}

// Persistent batched step: the CTAs stride over the (instance, first cell)
// work list; every instance is advanced with its own dt.
template <int P, int FLUX, bool F32>
__global__ void __launch_bounds__(NT, MinCtas<P, F32>::value) k_batch1d(const Step1DArgs a, const BatchArgs bt) {
  using SM = typename std::conditional<F32, Smem32<P, Phys<FLUX>::S>, Smem64<P, Phys<FLUX>::S>>::type;
  // FP32: two workspaces used alternately (tile_f32 ends without a barrier)
  __shared__ SM sm[F32 ? 2 : 1];
  __shared__ double s_lam;
  __shared__ float s_lamf[2];
  int par = 0;
  for (long w = blockIdx.x; w < bt.ntiles; w += gridDim.x) {
    const int b = bt.tiles[w].b;
    const long i0 = (long)bt.tiles[w].tile * Tiling<P>::T;
    const long off = bt.offs[b], N = bt.offs[b + 1] - off;
    if (threadIdx.x == 0) {
      const double dx = bt.xlen / (double)N;
      const double l = batch_dt(a, bt, b, i0 == 0, dx) / dx;
      if constexpr (F32) s_lamf[par] = (float)l;
      else s_lam = l;
    }
    int8_t *ord = bt.orders ? bt.orders + off + b : nullptr;
    unsigned long long *so = &bt.smax[((a.slot + 1) % 3) * (long)bt.B + b];
    if constexpr (F32) {
      tile_f32<P, FLUX>(a, sm[par], static_cast<const float *>(a.u_in), static_cast<float *>(a.u_out), off,
                        bt.M, N, i0, &s_lamf[par], ord, so);
      par ^= 1;
    } else {
      __syncthreads();
      tile_f64<P, FLUX>(a, sm[0], static_cast<const double *>(a.u_in), static_cast<double *>(a.u_out),
                        off, bt.M, N, i0, s_lam, ord, so);
    }
  }
}

// Wave speed of every instance of a batch into its slot (one CTA per
// instance); also sets the instances' time to 0.
template <int FLUX, bool F32>
__global__ void __launch_bounds__(NT) k_smax_batch(const Step1DArgs a, const BatchArgs bt) {
  constexpr int S = Phys<FLUX>::S;
  __shared__ double red[NT / 32];
  for (long b = blockIdx.x; b < bt.B; b += gridDim.x) {
    const long off = bt.offs[b], N = bt.offs[b + 1] - off;
    double smax = 0.0;
    bool bad = false;
    for (long i = threadIdx.x; i < N; i += NT) {
      double u[S];
#pragma unroll
      for (int c = 0; c < S; c++) {
        if constexpr (F32) {
          const float *p = static_cast<const float *>(a.u_in);
          u[c] = (double)p[c * bt.M + off + i] + (double)p[(S + c) * bt.M + off + i];
        } else {
          u[c] = static_cast<const double *>(a.u_in)[c * bt.M + off + i];
        }
      }
      bool ok;
      smax = fmax(smax, Phys<FLUX>::speed(u, a.adv, a.gamma, ok));
      bad |= !ok;
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0)
      atomicOr(a.status, (unsigned)ACAT_STATUS_NONPHYSICAL);
    const double v = block_max(smax, red);
    if (threadIdx.x == 0) {
      atomic_max_pos(&bt.smax[a.slot * bt.B + b], v);
      bt.t[a.slot * bt.B + b] = 0.0;
    }
    __syncthreads();
  }
}

// Wave speed of a state into smax[slot]; block 0 also sets tslot[slot] = 0.
template <int FLUX, bool F32>
__global__ void __launch_bounds__(NT) k_smax1d(const Step1DArgs a) {
  constexpr int S = Phys<FLUX>::S;
  __shared__ double s_red[NT / 32];
  double smax = 0.0;
  bool bad = false;
  for (long i = (long)blockIdx.x * NT + threadIdx.x; i < a.N; i += (long)gridDim.x * NT) {
    double u[S];
#pragma unroll
    for (int c = 0; c < S; c++) {
      if constexpr (F32) {
        const float *uin = static_cast<const float *>(a.u_in);
        u[c] = (double)uin[c * (long)a.N + i] + (double)uin[(S + c) * (long)a.N + i];
      } else {
        u[c] = static_cast<const double *>(a.u_in)[c * (long)a.N + i];
      }
    }
    bool ok;
    smax = fmax(smax, Phys<FLUX>::speed(u, a.adv, a.gamma, ok));
    bad |= !ok;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(a.status, (unsigned)ACAT_STATUS_NONPHYSICAL);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) smax = fmax(smax, __shfl_xor_sync(0xffffffffu, smax, o));
  if (lane == 0) s_red[warp] = smax;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = s_red[0];
    for (int w = 1; w < NT / 32; w++) v = fmax(v, s_red[w]);
    atomic_max_pos(&a.smax[a.slot], v);
    if (blockIdx.x == 0 && a.tslot) a.tslot[a.slot] = 0.0;
  }
}

template <int P, int FLUX, bool F32>
int launch_p(const Step1DArgs &a, cudaStream_t st) {
  using TL = Tiling<P>;
  if constexpr (!F32) {
    if (a.flux_buf && a.cnt) {  // small-CTA step with boundary hand-off
      const unsigned g = (unsigned)acat_fine_ctas_1d(P, a.N);
      k_step1d_fine<P, FLUX><<<g, NWF * 32, 0, st>>>(a);
      return (int)cudaGetLastError();
    }
  }
  const unsigned grid = (unsigned)((a.N + TL::T - 1) / TL::T);
  if constexpr (F32) k_step1d_f32<P, FLUX><<<grid, NT, 0, st>>>(a);
  else k_step1d_f64<P, FLUX><<<grid, NT, 0, st>>>(a);
  return (int)cudaGetLastError();
}

template <int FLUX, bool F32>
int launch_f(int P, const Step1DArgs &a, cudaStream_t st) {
  switch (P) {
  case 1: return launch_p<1, FLUX, F32>(a, st);
  case 2: return launch_p<2, FLUX, F32>(a, st);
  case 3: return launch_p<3, FLUX, F32>(a, st);
  case 4: return launch_p<4, FLUX, F32>(a, st);
  }
  return (int)cudaErrorInvalidValue;
}

template <bool F32>
int launch_prec(int P, int flux, const Step1DArgs &a, cudaStream_t st) {
  switch (flux) {
  case ACAT_FLUX_LINEAR: return launch_f<ACAT_FLUX_LINEAR, F32>(P, a, st);
  case ACAT_FLUX_BURGERS: return launch_f<ACAT_FLUX_BURGERS, F32>(P, a, st);
  case ACAT_FLUX_EULER1D: return launch_f<ACAT_FLUX_EULER1D, F32>(P, a, st);
  }
  return (int)cudaErrorInvalidValue;
}

template <bool F32>
int launch_smax(int flux, const Step1DArgs &a, cudaStream_t st) {
  const long blocks = (a.N + NT - 1) / NT;
  const unsigned grid = (unsigned)(blocks < 1024 ? blocks : 1024);
  switch (flux) {
  case ACAT_FLUX_LINEAR: k_smax1d<ACAT_FLUX_LINEAR, F32><<<grid, NT, 0, st>>>(a); break;
  case ACAT_FLUX_BURGERS: k_smax1d<ACAT_FLUX_BURGERS, F32><<<grid, NT, 0, st>>>(a); break;
  case ACAT_FLUX_EULER1D: k_smax1d<ACAT_FLUX_EULER1D, F32><<<grid, NT, 0, st>>>(a); break;
  default: return (int)cudaErrorInvalidValue;
  }
  return (int)cudaGetLastError();
}

template <int FLUX, bool F32>
int launch_batch_f(int P, const Step1DArgs &a, const BatchArgs &bt, cudaStream_t st) {
  int dev = 0, sms = 0, occ = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  switch (P) {
#define ACAT_BATCH_CASE(PP)                                                                      \
  case PP:                                                                                       \
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_batch1d<PP, FLUX, F32>, NT, 0);        \
    k_batch1d<PP, FLUX, F32><<<(unsigned)(sms * (occ > 0 ? occ : 1)), NT, 0, st>>>(a, bt);      \
    break;
    ACAT_BATCH_CASE(1)
    ACAT_BATCH_CASE(2)
    ACAT_BATCH_CASE(3)
    ACAT_BATCH_CASE(4)
#undef ACAT_BATCH_CASE
  default: return (int)cudaErrorInvalidValue;
  }
  return (int)cudaGetLastError();
}

template <bool F32>
int launch_batch(int P, int flux, const Step1DArgs &a, const BatchArgs &bt, cudaStream_t st) {
  switch (flux) {
  case ACAT_FLUX_LINEAR: return launch_batch_f<ACAT_FLUX_LINEAR, F32>(P, a, bt, st);
  case ACAT_FLUX_BURGERS: return launch_batch_f<ACAT_FLUX_BURGERS, F32>(P, a, bt, st);
  case ACAT_FLUX_EULER1D: return launch_batch_f<ACAT_FLUX_EULER1D, F32>(P, a, bt, st);
  }
  return (int)cudaErrorInvalidValue;
}

template <bool F32>
int launch_smax_batch(int flux, const Step1DArgs &a, const BatchArgs &bt, cudaStream_t st) {
  const unsigned grid = (unsigned)(bt.B < 4096 ? bt.B : 4096);
  switch (flux) {
  case ACAT_FLUX_LINEAR: k_smax_batch<ACAT_FLUX_LINEAR, F32><<<grid, NT, 0, st>>>(a, bt); break;
  case ACAT_FLUX_BURGERS: k_smax_batch<ACAT_FLUX_BURGERS, F32><<<grid, NT, 0, st>>>(a, bt); break;
  case ACAT_FLUX_EULER1D: k_smax_batch<ACAT_FLUX_EULER1D, F32><<<grid, NT, 0, st>>>(a, bt); break;
  default: return (int)cudaErrorInvalidValue;
  }
  return (int)cudaGetLastError();
}

}  // namespace

int acat_launch_batch1d(int P, int flux, int prec, const Step1DArgs &a, const BatchArgs &bt,
                        void *stream) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  return prec == ACAT_PREC_F32 ? launch_batch<true>(P, flux, a, bt, st)
                               : launch_batch<false>(P, flux, a, bt, st);
}

int acat_launch_smax_batch(int flux, int prec, const Step1DArgs &a, const BatchArgs &bt, void *stream) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  return prec == ACAT_PREC_F32 ? launch_smax_batch<true>(flux, a, bt, st)
                               : launch_smax_batch<false>(flux, a, bt, st);
}

int acat_cells_per_cta_1d(int P, int /*prec*/) {
  switch (P) {
  case 1: return Tiling<1>::T;
  case 2: return Tiling<2>::T;
  case 3: return Tiling<3>::T;
  case 4: return Tiling<4>::T;
  }
  return 0;
}

int acat_fine_ctas_1d(int P, long N) {
  int ni = 0;
  switch (P) {
  case 1: ni = Tiling<1, NWF>::NI; break;
  case 2: ni = Tiling<2, NWF>::NI; break;
  case 3: ni = Tiling<3, NWF>::NI; break;
  case 4: ni = Tiling<4, NWF>::NI; break;
  default: return -1;
  }
  return (int)((N + 1 + ni - 1) / ni);
}

int acat_launch_step1d(int P, int flux, int prec, const Step1DArgs &a, void *stream) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (prec == ACAT_PREC_F64) return launch_prec<false>(P, flux, a, st);
  if (prec == ACAT_PREC_F32) return launch_prec<true>(P, flux, a, st);
  return (int)cudaErrorInvalidValue;
}

int acat_launch_smax1d(int flux, int prec, const Step1DArgs &a, void *stream) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (prec == ACAT_PREC_F64) return launch_smax<false>(flux, a, st);
  if (prec == ACAT_PREC_F32) return launch_smax<true>(flux, a, st);
  return (int)cudaErrorInvalidValue;
}

int acat_upload_tables_1d(const AcatTables *T) { return (int)cudaMemcpyToSymbol(c_tab, T, sizeof *T); }

int acat_upload_tables_current_device() {
  AcatTables T;
  acat_build_tables(&T);
  int e = acat_upload_tables_1d(&T);
  if (e == 0) e = acat_upload_tables_2d(&T);
  if (e == 0) e = acat_upload_tables_adj(&T);
  return e;
}
