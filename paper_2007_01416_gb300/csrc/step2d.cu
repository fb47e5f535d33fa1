// step2d.cu -- the 2D ACAT step (Sec. 4) on sm_103a CUDA cores, for the 2D
// Euler equations and 2D linear transport, P <= 2.
//
// A CTA owns a 15 x 15 tile of cells and the 16 x 16 corner anchors
// (x, y), x0-1 <= x < x0+15, y0-1 <= y < y0+15, that carry the x-flux F at
// (x+1/2, y) and the y-flux G at (x, y+1/2) around its cells (Eq. 4.9). The
// cells the anchors' stencils reach (a halo of max(P, 2)) are staged once in
// shared memory with the boundary condition applied. Each anchor is worked by
// a group of 16 lanes, one lane per node of the 4 x 4 block S_2:
//   - the indicators are taken dimension by dimension (p_1 from the row
//     through the anchor, p_2 from its column; Sec. 4, admissible sets A_1,
//     A_2), one (direction, component) pair per lane, in explicitly rounded
//     FP64 as in 1D;
//   - when a direction selects p = 2, the group runs the block recursion of
//     Sec. 4 (Eqs. 4.5-4.6): u~^(k-1) at every node from the x-derivative of
//     f~ along its row and the y-derivative of g~ along its column (lane
//     shuffles), f and g at the 2p - 1 other time levels, and F from row 0,
//     G from column 0. One block serves both directions when both select it;
//   - a direction that selects nothing uses FL-CAT2 (Eqs. 4.3-4.4 blended as
//     Eqs. 4.7-4.8) on one lane.
// The update and the dt epilogue (both directions' maximal speeds, Sec. 5.5
// CFL rule) follow as in 1D. The FP32 variant uses the delta formulation of
// the 1D kernel: F = f(u_a) + G_F, G = g(u_a) + G_G about the anchor state.
#include <type_traits>

#include "device_common.cuh"

namespace {

constexpr int TXY = 15;       // cells per CTA side
constexpr int NA = TXY + 1;   // anchors per CTA side
constexpr int GH2 = 2;        // ghost width (P <= 2)
constexpr int TW2 = TXY + 2 * GH2;

template <int FLUX>
struct Phys2;

template <>
struct Phys2<ACAT_FLUX_LINEAR> {
  static constexpr int S = 1;
  template <typename R>
  __device__ static __forceinline__ void flux2(const R *u, R *f, R *g, R ax, R ay, R) {
    f[0] = ax * u[0];
    g[0] = ay * u[0];
  }
  __device__ static __forceinline__ void speed2(const double *u, double ax, double ay, double,
                                                double &sx, double &sy, bool &ok) {
    sx = fabs(ax);
    sy = fabs(ay);
    ok = isfinite(u[0]);
  }
  template <typename R>
  __device__ static __forceinline__ void eig2(const R *, R ax, R ay, R, int dir, R &lmin, R &lmax) {
    lmin = lmax = dir == 0 ? ax : ay;
  }
  struct Base {
    float ax, ay;
  };
  __device__ static __forceinline__ Base base(const float *, float ax, float ay, float) {
    return Base{ax, ay};
  }
  __device__ static __forceinline__ Base base2(const float *, const float *, float ax, float ay, float) {
    return Base{ax, ay};
  }
  __device__ static __forceinline__ void dflux2(const Base &B, const float *d, float *df, float *dg) {
    df[0] = B.ax * d[0];
    dg[0] = B.ay * d[0];
  }
  __device__ static __forceinline__ void dflux2_pair(const Base &B, const float *dh, const float *dl, float *df,
                                                     float *dg) {
    const float d[1] = {dh[0] + dl[0]};
    dflux2(B, d, df, dg);
  }
  __device__ static __forceinline__ void dflux2_x2(const Base &B, const float2 *d, float2 *df, float2 *dg) {
    df[0] = f2mul(f2dup(B.ax), d[0]);
    dg[0] = f2mul(f2dup(B.ay), d[0]);
  }
  __device__ static __forceinline__ float fspeed(const float *, float ax, float ay, float, int dir) {
    return dir == 0 ? fabsf(ax) : fabsf(ay);
  }
  __device__ static __forceinline__ bool fphysical(const float *u, float) { return isfinite(u[0]); }
};

template <>
struct Phys2<ACAT_FLUX_EULER2D> {
  static constexpr int S = 4;
  template <typename R>
  __device__ static __forceinline__ void flux2(const R *u, R *f, R *g, R, R, R gm1) {
    const R ri = recip(u[0]);
    const R v = u[1] * ri, w = u[2] * ri;
    const R p = gm1 * (u[3] - R(0.5) * (u[1] * v + u[2] * w));
    const R H = u[3] + p;
    f[0] = u[1];
    f[1] = u[1] * v + p;
    f[2] = u[1] * w;
    f[3] = v * H;
    g[0] = u[2];
    g[1] = u[2] * v;
    g[2] = u[2] * w + p;
    g[3] = w * H;
  }
  // |v| + c and |w| + c, every operation rounded as written (bit-exact dt)
  __device__ static __forceinline__ void speed2(const double *u, double, double, double gamma,
                                                double &sx, double &sy, bool &ok) {
    const double v = __ddiv_rn(u[1], u[0]), w = __ddiv_rn(u[2], u[0]);
    const double ke = __dmul_rn(__dmul_rn(0.5, u[0]), __dadd_rn(__dmul_rn(v, v), __dmul_rn(w, w)));
    const double p = __dmul_rn(__dsub_rn(gamma, 1.0), __dsub_rn(u[3], ke));
    const double c = __dsqrt_rn(__ddiv_rn(__dmul_rn(gamma, p), u[0]));
    sx = __dadd_rn(fabs(v), c);
    sy = __dadd_rn(fabs(w), c);
    ok = (u[0] > 0.0) && (p > 0.0) && isfinite(u[0]) && isfinite(u[1]) && isfinite(u[2]) &&
         isfinite(u[3]);
  }
  // smallest and largest eigenvalue v_n -/+ c in direction dir (HLL bounds)
  template <typename R>
  __device__ static __forceinline__ void eig2(const R *u, R, R, R gamma, int dir, R &lmin, R &lmax) {
    const R v = u[1] / u[0], w = u[2] / u[0];
    const R p = (gamma - R(1)) * (u[3] - R(0.5) * (u[1] * v + u[2] * w));
    const R c = sqrt(gamma * p / u[0]);
    const R vn = dir == 0 ? v : w;
    lmin = vn - c;
    lmax = vn + c;
  }
  struct Base {
    float mx, my, v, w, vl, wl, H, rho, gm1;  // v + vl, w + wl: float-float velocities
  };
  __device__ static __forceinline__ Base base(const float *u, float, float, float gm1) {
    Base b;
    b.rho = u[0];
    b.mx = u[1];
    b.my = u[2];
    const float ri = recip(u[0]);
    b.v = u[1] * ri;
    b.w = u[2] * ri;
    b.vl = b.wl = 0.0f;
    const float p = gm1 * (u[3] - 0.5f * fmaf(u[1], b.v, u[2] * b.w));
    b.H = u[3] + p;
    b.gm1 = gm1;
    return b;
  }
  // The base of a compensated state hi + lo with both velocities to
  // float-float accuracy (the 1D base2: at constant velocity the numerators
  // b - v a of the velocity increments cancel, and a velocity rounded to float
  // would leave eps32 |v a| of noise in the increments).
  __device__ static __forceinline__ Base base2(const float *h, const float *l, float, float, float gm1) {
    Base b;
    b.rho = h[0];
    b.mx = h[1];
    b.my = h[2];
    const float ri = recip(h[0]);
    b.v = h[1] * ri;
    b.w = h[2] * ri;
    b.vl = (fmaf(-b.v, h[0], h[1]) + fmaf(-b.v, l[0], l[1])) * ri;
    b.wl = (fmaf(-b.w, h[0], h[2]) + fmaf(-b.w, l[0], l[2])) * ri;
    const float p = gm1 * (h[3] - 0.5f * fmaf(h[1], b.v, h[2] * b.w));
    b.H = h[3] + p;
    b.gm1 = gm1;
    return b;
  }
  // Increments of f and g for u -> u + d, d = (a, bx, by, c):
  //   dv = (bx - v a)/(rho + a), dw = (by - w a)/(rho + a)
  //   d(mx v) = mx dv + bx (v + dv), d(my w) = my dw + by (w + dw),
  //   d(mx w) = mx dw + bx (w + dw), dp = (gamma - 1)(c - (d(mx v) + d(my w))/2)
  __device__ static __forceinline__ void dflux2(const Base &B, const float *d, float *df, float *dg) {
    const float ri = recip(B.rho + d[0]);
    const float dv = fmaf(-B.vl, d[0], fmaf(-B.v, d[0], d[1])) * ri;
    const float dw = fmaf(-B.wl, d[0], fmaf(-B.w, d[0], d[2])) * ri;
    dflux2_rest(B, d, dv, dw, df, dg);
  }
  // the increment d = dh + dl as an unevaluated pair (differences of the hi
  // and of the lo parts): the cancelling numerators take both parts
  __device__ static __forceinline__ void dflux2_pair(const Base &B, const float *dh, const float *dl, float *df,
                                                     float *dg) {
    const float d[4] = {dh[0] + dl[0], dh[1] + dl[1], dh[2] + dl[2], dh[3] + dl[3]};
    const float ri = recip(B.rho + d[0]);
    const float dv = fmaf(-B.vl, dh[0], fmaf(-B.v, dh[0], dh[1]) + fmaf(-B.v, dl[0], dl[1])) * ri;
    const float dw = fmaf(-B.wl, dh[0], fmaf(-B.w, dh[0], dh[2]) + fmaf(-B.w, dl[0], dl[2])) * ri;
    dflux2_rest(B, d, dv, dw, df, dg);
  }
  __device__ static __forceinline__ void dflux2_rest(const Base &B, const float *d, float dv, float dw, float *df,
                                                     float *dg) {
    const float vn = B.v + dv, wn = B.w + dw;
    const float dmv = fmaf(B.mx, dv, d[1] * vn), dmw = fmaf(B.my, dw, d[2] * wn);
    const float dxy = fmaf(B.mx, dw, d[1] * wn);
    const float dp = B.gm1 * fmaf(-0.5f, dmv + dmw, d[3]);
    const float dH = d[3] + dp;
    df[0] = d[1];
    df[1] = dmv + dp;
    df[2] = dxy;
    df[3] = fmaf(dv, B.H, vn * dH);
    dg[0] = d[2];
    dg[1] = dxy;
    dg[2] = dmw + dp;
    dg[3] = fmaf(dw, B.H, wn * dH);
  }
  // the same for two increments packed in float2 lanes
  __device__ static __forceinline__ void dflux2_x2(const Base &B, const float2 *d, float2 *df, float2 *dg) {
    const float2 den = f2add(f2dup(B.rho), d[0]);
    const float2 ri = make_float2(recip(den.x), recip(den.y));
    const float2 dv = f2mul(f2fma(f2dup(-B.vl), d[0], f2fma(f2dup(-B.v), d[0], d[1])), ri);
    const float2 dw = f2mul(f2fma(f2dup(-B.wl), d[0], f2fma(f2dup(-B.w), d[0], d[2])), ri);
    const float2 vn = f2add(f2dup(B.v), dv), wn = f2add(f2dup(B.w), dw);
    const float2 dmv = f2fma(f2dup(B.mx), dv, f2mul(d[1], vn)), dmw = f2fma(f2dup(B.my), dw, f2mul(d[2], wn));
    const float2 dxy = f2fma(f2dup(B.mx), dw, f2mul(d[1], wn));
    const float2 dp = f2mul(f2dup(B.gm1), f2fma(f2dup(-0.5f), f2add(dmv, dmw), d[3]));
    const float2 dH = f2add(d[3], dp);
    df[0] = d[1];
    df[1] = f2add(dmv, dp);
    df[2] = dxy;
    df[3] = f2fma(dv, f2dup(B.H), f2mul(vn, dH));
    dg[0] = d[2];
    dg[1] = dxy;
    dg[2] = f2add(dmw, dp);
    dg[3] = f2fma(dw, f2dup(B.H), f2mul(wn, dH));
  }
  __device__ static __forceinline__ float fspeed(const float *u, float, float, float gamma, int dir) {
    const float v = u[1] / u[0], w = u[2] / u[0];
    const float p = (gamma - 1.0f) * (u[3] - 0.5f * (u[1] * v + u[2] * w));
    return fabsf(dir == 0 ? v : w) + sqrtf(fmaxf(gamma * p / u[0], 0.0f));
  }
  __device__ static __forceinline__ bool fphysical(const float *u, float gamma) {
    const float ri = 1.0f / u[0];
    const float p = (gamma - 1.0f) * (u[3] - 0.5f * (u[1] * u[1] + u[2] * u[2]) * ri);
    return u[0] > 0.0f && p > 0.0f && isfinite(u[0]) && isfinite(u[1]) && isfinite(u[2]) &&
           isfinite(u[3]);
  }
};

// ---------------------------------------------------------------------------
// FP64 block recursion (Eqs. 4.5-4.6) by 16 lanes; lane l <-> node
// (a1, b1) = (l % n, l / n). q points at the anchor for component 0; `cs`
// between components, `rs` between rows. Every lane returns F and G.
// ---------------------------------------------------------------------------
template <int p, int FLUX>
__device__ __forceinline__ void cat2d_f64(const double *q, int cs, int rs, int l, int base,
                                          double lx, double ly, double ax, double ay, double gm1,
                                          double *Fo, double *Go) {
  using TB = Tab<double>;
  constexpr int S = Phys2<FLUX>::S;
  constexpr int n = 2 * p;
  const unsigned mask = ((1u << (n * n)) - 1u) << base;
  const int a1 = l % n, b1 = l / n;
  // the node's row and column weights scaled by -lambda_x and -lambda_y once:
  // each order's U = -lambda_x sum_r gx_r F_r - lambda_y sum_r gy_r G_r is then
  // one accumulation over both directions
  double gx[n], gy[n];
#pragma unroll
  for (int r = 0; r < n; r++) {
    gx[r] = TB::g1(p, a1, r) * -lx;
    gy[r] = TB::g1(p, b1, r) * -ly;
  }
  double f0[S], g0[S], Ff[S], Fg[S], Pf[S], Pg[S], arg[n][S];
  {
    double u[S];
#pragma unroll
    for (int c = 0; c < S; c++) u[c] = q[c * cs + (b1 - p + 1) * rs + (a1 - p + 1)];
    Phys2<FLUX>::flux2(u, f0, g0, ax, ay, gm1);
#pragma unroll
    for (int rr = 0; rr < n; rr++)
#pragma unroll
      for (int c = 0; c < S; c++) arg[rr][c] = u[c];
  }
#pragma unroll
  for (int c = 0; c < S; c++) {
    Ff[c] = Pf[c] = f0[c];
    Fg[c] = Pg[c] = g0[c];
  }
#pragma unroll
  for (int k = 2; k <= n; k++) {
    double U[S], af[S], ag[S];
#pragma unroll
    for (int c = 0; c < S; c++) U[c] = 0.0;
#pragma unroll
    for (int r = 0; r < n; r++)
#pragma unroll
      for (int c = 0; c < S; c++) U[c] = fma(gx[r], __shfl_sync(mask, Pf[c], base + b1 * n + r), U[c]);
#pragma unroll
    for (int r = 0; r < n; r++)
#pragma unroll
      for (int c = 0; c < S; c++) U[c] = fma(gy[r], __shfl_sync(mask, Pg[c], base + r * n + a1), U[c]);
#pragma unroll
    for (int c = 0; c < S; c++) {
      af[c] = TB::gk(p, k - 1, p - 1) * f0[c];
      ag[c] = TB::gk(p, k - 1, p - 1) * g0[c];
    }
#pragma unroll
    for (int rr = 0; rr < n; rr++) {
      if (rr == p - 1) continue;
      const double cr = TB::taylor(p, rr, k - 1), wk = TB::gk(p, k - 1, rr);
      double fr[S], gr[S];
#pragma unroll
      for (int c = 0; c < S; c++) arg[rr][c] = fma(cr, U[c], arg[rr][c]);
      Phys2<FLUX>::flux2(arg[rr], fr, gr, ax, ay, gm1);
#pragma unroll
      for (int c = 0; c < S; c++) {
        af[c] = fma(wk, fr[c], af[c]);
        ag[c] = fma(wk, gr[c], ag[c]);
      }
    }
#pragma unroll
    for (int c = 0; c < S; c++) {
      Pf[c] = af[c];
      Pg[c] = ag[c];
      Ff[c] = fma(TB::invfact(k), af[c], Ff[c]);
      Fg[c] = fma(TB::invfact(k), ag[c], Fg[c]);
    }
  }
#pragma unroll
  for (int c = 0; c < S; c++) {
    const double vF = TB::gh(p, a1) * Ff[c], vG = TB::gh(p, b1) * Fg[c];
    double tF = 0.0, tG = 0.0;
#pragma unroll
    for (int r = 0; r < n; r++) {
      tF += __shfl_sync(mask, vF, base + (p - 1) * n + r);
      tG += __shfl_sync(mask, vG, base + r * n + (p - 1));
    }
    Fo[c] = tF;
    Go[c] = tG;
  }
}

// FP32 block recursion in the delta formulation about the anchor state u_a:
// returns G_F = F - f(u_a) and G_G = G - g(u_a). xw: the warp's 128 exchange
// slots in shared memory (two sets of 2 x 32 used alternately by k), through
// which a system's nodes read the F^(k-2) of their row and the G^(k-2) of
// their column: two 16-byte stores and 2 x 2p 16-byte loads per lane and
// order instead of 2 x 2p s shuffles (scalar laws shuffle).
template <int p, int FLUX>
__device__ __forceinline__ void cat2d_f32(const float *hi, const float *lo, int cs, int rs, int l,
                                          int base, float lx, float ly, float ax, float ay, float gm1,
                                          float4 *xw, float *GFo, float *GGo) {
  using TB = Tab<float>;
  using PH = Phys2<FLUX>;
  constexpr int S = PH::S;
  constexpr int n = 2 * p;
  const unsigned mask = ((1u << (n * n)) - 1u) << base;
  const int a1 = l % n, b1 = l / n;
  const int off = (b1 - p + 1) * rs + (a1 - p + 1);
  float gx[n], gy[n];
#pragma unroll
  for (int r = 0; r < n; r++) {
    gx[r] = TB::g1(p, a1, r);
    gy[r] = TB::g1(p, b1, r);
  }
  float ua[S], ual[S], uj[S], ujl[S], dh[S], dl[S];
#pragma unroll
  for (int c = 0; c < S; c++) {
    ua[c] = hi[c * cs];
    ual[c] = lo[c * cs];
    uj[c] = hi[c * cs + off];
    ujl[c] = lo[c * cs + off];
    dh[c] = uj[c] - ua[c];
    dl[c] = ujl[c] - ual[c];
  }
  float Df[S], Dg[S];
  PH::dflux2_pair(PH::base2(ua, ual, ax, ay, gm1), dh, dl, Df, Dg);  // f(u_j) - f(u_a), g(u_j) - g(u_a)
  const typename PH::Base bj = PH::base2(uj, ujl, ax, ay, gm1);
  // the 2p - 1 levels r != 0 in pairs packed in float2 lanes, the last alone
  constexpr int NL = n - 1, NP = NL / 2;
  float Ff[S], Fg[S], Pf[S], Pg[S], dels[S];
  float2 del2[NP][S];
#pragma unroll
  for (int c = 0; c < S; c++) {
    Ff[c] = Pf[c] = Df[c];
    Fg[c] = Pg[c] = Dg[c];
    dels[c] = 0.0f;
  }
#pragma unroll
  for (int q = 0; q < NP; q++)
#pragma unroll
    for (int c = 0; c < S; c++) del2[q][c] = make_float2(0.0f, 0.0f);
#pragma unroll
  for (int k = 2; k <= n; k++) {
    float Ux[S], Uy[S];
#pragma unroll
    for (int c = 0; c < S; c++) Ux[c] = Uy[c] = 0.0f;
    if constexpr (S > 1) {
      // the slot set of order k was last read at order k - 2, before every
      // lane of the block passed the barrier of order k - 1
      float4 *xb = xw + (k & 1) * 64;
      xb[base + l] = make_float4(Pf[0], Pf[1], S > 2 ? Pf[S > 2 ? 2 : 0] : 0.0f, S > 3 ? Pf[S > 3 ? 3 : 0] : 0.0f);
      xb[32 + base + l] =
          make_float4(Pg[0], Pg[1], S > 2 ? Pg[S > 2 ? 2 : 0] : 0.0f, S > 3 ? Pg[S > 3 ? 3 : 0] : 0.0f);
      __syncwarp(mask);
#pragma unroll
      for (int r = 0; r < n; r++) {
        const float4 f = xb[base + b1 * n + r], g = xb[32 + base + r * n + a1];
        const float fr[4] = {f.x, f.y, f.z, f.w}, gr[4] = {g.x, g.y, g.z, g.w};
#pragma unroll
        for (int c = 0; c < S; c++) {
          Ux[c] = fmaf(gx[r], fr[c], Ux[c]);
          Uy[c] = fmaf(gy[r], gr[c], Uy[c]);
        }
      }
    } else {
#pragma unroll
      for (int r = 0; r < n; r++) {
        Ux[0] = fmaf(gx[r], __shfl_sync(mask, Pf[0], base + b1 * n + r), Ux[0]);
        Uy[0] = fmaf(gy[r], __shfl_sync(mask, Pg[0], base + r * n + a1), Uy[0]);
      }
    }
    float U[S], af[S], ag[S];
#pragma unroll
    for (int c = 0; c < S; c++) {
      U[c] = -(lx * Ux[c]) - ly * Uy[c];
      af[c] = ag[c] = 0.0f;
    }
    float2 af2[S], ag2[S];
#pragma unroll
    for (int c = 0; c < S; c++) af2[c] = ag2[c] = make_float2(0.0f, 0.0f);
#pragma unroll
    for (int q = 0; q < NP; q++) {
      const int ra = 2 * q < p - 1 ? 2 * q : 2 * q + 1, rb = 2 * q + 1 < p - 1 ? 2 * q + 1 : 2 * q + 2;
      const float2 cr = make_float2(TB::taylor(p, ra, k - 1), TB::taylor(p, rb, k - 1));
      const float2 wk = make_float2(TB::gk(p, k - 1, ra), TB::gk(p, k - 1, rb));
      float2 ef[S], eg[S];
#pragma unroll
      for (int c = 0; c < S; c++) del2[q][c] = f2fma(cr, f2dup(U[c]), del2[q][c]);
      PH::dflux2_x2(bj, del2[q], ef, eg);
#pragma unroll
      for (int c = 0; c < S; c++) {
        af2[c] = f2fma(wk, ef[c], af2[c]);
        ag2[c] = f2fma(wk, eg[c], ag2[c]);
      }
    }
    {
      constexpr int rs = NL - 1 < p - 1 ? NL - 1 : NL;  // the last level
      const float cr = TB::taylor(p, rs, k - 1), wk = TB::gk(p, k - 1, rs);
      float ef[S], eg[S];
#pragma unroll
      for (int c = 0; c < S; c++) dels[c] = fmaf(cr, U[c], dels[c]);
      PH::dflux2(bj, dels, ef, eg);
#pragma unroll
      for (int c = 0; c < S; c++) {
        af[c] = fmaf(wk, ef[c], af[c]);
        ag[c] = fmaf(wk, eg[c], ag[c]);
      }
    }
#pragma unroll
    for (int c = 0; c < S; c++) {
      af[c] += af2[c].x + af2[c].y;
      ag[c] += ag2[c].x + ag2[c].y;
      Pf[c] = af[c];
      Pg[c] = ag[c];
      Ff[c] = fmaf(TB::invfact(k), af[c], Ff[c]);
      Fg[c] = fmaf(TB::invfact(k), ag[c], Fg[c]);
    }
  }
#pragma unroll
  for (int c = 0; c < S; c++) {
    const float vF = TB::gh(p, a1) * Ff[c], vG = TB::gh(p, b1) * Fg[c];
    float tF = 0.0f, tG = 0.0f;
#pragma unroll
    for (int r = 0; r < n; r++) {
      tF += __shfl_sync(mask, vF, base + (p - 1) * n + r);
      tG += __shfl_sync(mask, vG, base + r * n + (p - 1));
    }
    GFo[c] = tF;
    GGo[c] = tG;
  }
}

// F^lo of Eq. 3.4 along one direction (ACAT_LO_*), as in 1D: Rusanov with the
// larger spectral radius, global LF with alpha = 1 / lambda_dir, HLL with the
// states' eigenvalue bounds.
template <int S, typename R>
__device__ __forceinline__ void flux_lo2(int lo_flux, const R *u0, const R *u1, const R *f0, const R *f1, R s0,
                                         R s1, R n0, R x0, R n1, R x1, R lam, R *Flo) {
  if (lo_flux == ACAT_LO_HLL) {
    const R sl = n1 < n0 ? n1 : n0, sr = x1 > x0 ? x1 : x0;
#pragma unroll
    for (int c = 0; c < S; c++) {
      if (sl >= R(0)) Flo[c] = f0[c];
      else if (sr <= R(0)) Flo[c] = f1[c];
      else Flo[c] = (sr * f0[c] - sl * f1[c] + sl * sr * (u1[c] - u0[c])) / (sr - sl);
    }
    return;
  }
  const R alpha = lo_flux == ACAT_LO_GLOBAL_LF ? R(1) / lam : (s1 > s0 ? s1 : s0);
#pragma unroll
  for (int c = 0; c < S; c++) Flo[c] = R(0.5) * (f0[c] + f1[c]) - R(0.5) * alpha * (u1[c] - u0[c]);
}

// FP64 FL-CAT2 in 2D (one lane): the 2D CAT2 fluxes of Eqs. 4.3-4.4 on the
// 2 x 2 block at the anchor, blended with Rusanov by psi^1 of the row (F) or
// the column (G) as in Eqs. 4.7-4.8.
template <int FLUX>
__device__ __forceinline__ void flcat2_2d_f64(const double *q, int cs, int rs, bool wantF, bool wantG,
                                              double lx, double ly, double ax, double ay,
                                              double gamma, int limiter_form, int lo_flux, double *F,
                                              double *G) {
  using PH = Phys2<FLUX>;
  constexpr int S = PH::S;
  const double gm1 = gamma - 1.0;
  double u00[S], u10[S], u01[S], u11[S];
#pragma unroll
  for (int c = 0; c < S; c++) {
    u00[c] = q[c * cs];
    u10[c] = q[c * cs + 1];
    u01[c] = q[c * cs + rs];
    u11[c] = q[c * cs + rs + 1];
  }
  double f00[S], g00[S], f10[S], g10[S], f01[S], g01[S], f11[S], g11[S];
  PH::flux2(u00, f00, g00, ax, ay, gm1);
  PH::flux2(u10, f10, g10, ax, ay, gm1);
  PH::flux2(u01, f01, g01, ax, ay, gm1);
  PH::flux2(u11, f11, g11, ax, ay, gm1);
  const int kind = 0;  // 2D scalar law here is linear transport
  if (wantF) {
    double a0[S], a1[S], t0[S], t1[S], tg[S];
#pragma unroll
    for (int c = 0; c < S; c++) {
      a0[c] = u00[c] + (-lx * (f10[c] - f00[c]) - ly * (g01[c] - g00[c]));
      a1[c] = u10[c] + (-lx * (f10[c] - f00[c]) - ly * (g11[c] - g10[c]));
    }
    PH::flux2(a0, t0, tg, ax, ay, gm1);
    PH::flux2(a1, t1, tg, ax, ay, gm1);
    double sx0, sy0, sx1, sy1;
    bool ok;
    PH::speed2(u00, ax, ay, gamma, sx0, sy0, ok);
    PH::speed2(u10, ax, ay, gamma, sx1, sy1, ok);
    double n0 = 0.0, x0 = 0.0, n1 = 0.0, x1 = 0.0;
    if (lo_flux == ACAT_LO_HLL) {
      PH::eig2(u00, ax, ay, gamma, 0, n0, x0);
      PH::eig2(u10, ax, ay, gamma, 0, n1, x1);
    }
    double Flo[S];
    flux_lo2<S, double>(lo_flux, u00, u10, f00, f10, sx0, sx1, n0, x0, n1, x1, lx, Flo);
    const double w = psi1_line<S>(q, cs, 1, kind, limiter_form, ax);
#pragma unroll
    for (int c = 0; c < S; c++) {
      const double F1 = 0.25 * (t0[c] + t1[c] + f00[c] + f10[c]);
      F[c] = w * F1 + (1.0 - w) * Flo[c];
    }
  }
  if (wantG) {
    double a0[S], a1[S], t0[S], t1[S], tf[S];
#pragma unroll
    for (int c = 0; c < S; c++) {
      a0[c] = u00[c] + (-lx * (f10[c] - f00[c]) - ly * (g01[c] - g00[c]));
      a1[c] = u01[c] + (-lx * (f11[c] - f01[c]) - ly * (g01[c] - g00[c]));
    }
    PH::flux2(a0, tf, t0, ax, ay, gm1);
    PH::flux2(a1, tf, t1, ax, ay, gm1);
    double sx0, sy0, sx1, sy1;
    bool ok;
    PH::speed2(u00, ax, ay, gamma, sx0, sy0, ok);
    PH::speed2(u01, ax, ay, gamma, sx1, sy1, ok);
    double n0 = 0.0, x0 = 0.0, n1 = 0.0, x1 = 0.0;
    if (lo_flux == ACAT_LO_HLL) {
      PH::eig2(u00, ax, ay, gamma, 1, n0, x0);
      PH::eig2(u01, ax, ay, gamma, 1, n1, x1);
    }
    double Glo[S];
    flux_lo2<S, double>(lo_flux, u00, u01, g00, g01, sy0, sy1, n0, x0, n1, x1, ly, Glo);
    const double w = psi1_line<S>(q, cs, rs, kind, limiter_form, ay);
#pragma unroll
    for (int c = 0; c < S; c++) {
      const double G1 = 0.25 * (t0[c] + t1[c] + g00[c] + g01[c]);
      G[c] = w * G1 + (1.0 - w) * Glo[c];
    }
  }
}

// FP32 FL-CAT2 in 2D, delta form about the anchor state a (one lane).
template <int FLUX>
__device__ __forceinline__ void flcat2_2d_f32(const float *hi, const float *lo, int cs, int rs,
                                              bool wantF, bool wantG, float lx,
                                              float ly, float ax, float ay, float gamma, float gm1,
                                              int limiter_form, int lo_flux, float *GF, float *GG) {
  using PH = Phys2<FLUX>;
  constexpr int S = PH::S;
  const bool roe_linear = FLUX == ACAT_FLUX_LINEAR && limiter_form == 0;
  float ua[S], ual[S], d10[S], d01[S], d11[S], u10[S], u01[S];
  float h10[S], l10[S], h01[S], l01[S], h11[S], l11[S];
#pragma unroll
  for (int c = 0; c < S; c++) {
    const int o = c * cs;
    ua[c] = hi[o];
    ual[c] = lo[o];
    u10[c] = hi[o + 1];
    u01[c] = hi[o + rs];
    h10[c] = hi[o + 1] - hi[o];
    l10[c] = lo[o + 1] - lo[o];
    h01[c] = hi[o + rs] - hi[o];
    l01[c] = lo[o + rs] - lo[o];
    h11[c] = hi[o + rs + 1] - hi[o];
    l11[c] = lo[o + rs + 1] - lo[o];
    d10[c] = h10[c] + l10[c];
    d01[c] = h01[c] + l01[c];
    d11[c] = h11[c] + l11[c];
  }
  const typename PH::Base B = PH::base2(ua, ual, ax, ay, gm1);
  float Df10[S], Dg10[S], Df01[S], Dg01[S], Df11[S], Dg11[S];
  PH::dflux2_pair(B, h10, l10, Df10, Dg10);
  PH::dflux2_pair(B, h01, l01, Df01, Dg01);
  PH::dflux2_pair(B, h11, l11, Df11, Dg11);
  float U00[S];
#pragma unroll
  for (int c = 0; c < S; c++) U00[c] = -lx * Df10[c] - ly * Dg01[c];
  float e00f[S], e00g[S];
  PH::dflux2(B, U00, e00f, e00g);
  if (wantF) {
    float x1[S], ef[S], eg[S];
#pragma unroll
    for (int c = 0; c < S; c++) x1[c] = d10[c] + (-lx * Df10[c] - ly * (Dg11[c] - Dg10[c]));
    PH::dflux2(B, x1, ef, eg);  // f(u10 + U10) - f(u_a)
    const float s0 = PH::fspeed(ua, ax, ay, gamma, 0), s1 = PH::fspeed(u10, ax, ay, gamma, 0);
    const float alpha = lo_flux == ACAT_LO_GLOBAL_LF ? 1.0f / lx : (s1 > s0 ? s1 : s0);
    float sl = 0.0f, sr = 0.0f;
    if (lo_flux == ACAT_LO_HLL) {
      float n0, x0, n1, x1;
      PH::eig2(ua, ax, ay, gamma, 0, n0, x0);
      PH::eig2(u10, ax, ay, gamma, 0, n1, x1);
      sl = n1 < n0 ? n1 : n0;
      sr = x1 > x0 ? x1 : x0;
    }
    const float w = psi1_line_ff<S>(hi, lo, cs, 1, roe_linear, ax);
#pragma unroll
    for (int c = 0; c < S; c++) {
      // F1 - f(a) = Df10/2 + (e00 + (ef - Df10))/4 ; Flo - f(a) = Df10/2 - alpha d10/2 (LF
      // forms), HLL: 0, Df10 or sl (sr d10 - Df10) / (sr - sl)
      const float G1 = 0.5f * Df10[c] + 0.25f * (e00f[c] + ef[c] - Df10[c]);
      float Glo;
      if (lo_flux == ACAT_LO_HLL)
        Glo = sl >= 0.0f ? 0.0f : (sr <= 0.0f ? Df10[c] : sl * (sr * d10[c] - Df10[c]) / (sr - sl));
      else
        Glo = 0.5f * Df10[c] - 0.5f * alpha * d10[c];
      GF[c] = fmaf(w, G1 - Glo, Glo);
    }
  }
  if (wantG) {
    float x1[S], ef[S], eg[S];
#pragma unroll
    for (int c = 0; c < S; c++) x1[c] = d01[c] + (-lx * (Df11[c] - Df01[c]) - ly * Dg01[c]);
    PH::dflux2(B, x1, ef, eg);  // g(u01 + U01) - g(u_a)
    const float s0 = PH::fspeed(ua, ax, ay, gamma, 1), s1 = PH::fspeed(u01, ax, ay, gamma, 1);
    const float alpha = lo_flux == ACAT_LO_GLOBAL_LF ? 1.0f / ly : (s1 > s0 ? s1 : s0);
    float sl = 0.0f, sr = 0.0f;
    if (lo_flux == ACAT_LO_HLL) {
      float n0, x0, n1, x1;
      PH::eig2(ua, ax, ay, gamma, 1, n0, x0);
      PH::eig2(u01, ax, ay, gamma, 1, n1, x1);
      sl = n1 < n0 ? n1 : n0;
      sr = x1 > x0 ? x1 : x0;
    }
    const float w = psi1_line_ff<S>(hi, lo, cs, rs, roe_linear, ay);
#pragma unroll
    for (int c = 0; c < S; c++) {
      const float G1 = 0.5f * Dg01[c] + 0.25f * (e00g[c] + eg[c] - Dg01[c]);
      float Glo;
      if (lo_flux == ACAT_LO_HLL)
        Glo = sl >= 0.0f ? 0.0f : (sr <= 0.0f ? Dg01[c] : sl * (sr * d01[c] - Dg01[c]) / (sr - sl));
      else
        Glo = 0.5f * Dg01[c] - 0.5f * alpha * d01[c];
      GG[c] = fmaf(w, G1 - Glo, Glo);
    }
  }
}

// dt of a 2D step: CFL/2 min(dx / s^max_x, dy / s^max_y) (Sec. 5.5).
__device__ double step_dt2(const Step2DArgs &a) {
  double dt;
  if (a.dt_fixed > 0.0) {
    dt = a.dt_fixed;
  } else {
    const double sx = __longlong_as_double((long long)a.smax[a.slot * 2 + 0]);
    const double sy = __longlong_as_double((long long)a.smax[a.slot * 2 + 1]);
    const double inf = __longlong_as_double(0x7ff0000000000000LL);
    if (!isfinite(sx) || !isfinite(sy) || !(sx > 0.0 || sy > 0.0)) {
      if (blockIdx.x == 0 && blockIdx.y == 0) atomicOr(a.status, (unsigned)ACAT_STATUS_BAD_DT);
      dt = 0.0;
    } else {
      const double tx = sx > 0.0 ? __ddiv_rn(a.dx, sx) : inf;
      const double ty = sy > 0.0 ? __ddiv_rn(a.dy, sy) : inf;
      dt = __dmul_rn(a.cfl / 2.0, tx < ty ? tx : ty);
    }
  }
  double t = 0.0;
  if (a.tslot) {
    t = a.tslot[a.slot];
    if (a.t_end > 0.0) {
      if (t >= a.t_end) dt = 0.0;
      else if (dt > a.t_end - t) dt = a.t_end - t;
    }
  }
  if (blockIdx.x == 0 && blockIdx.y == 0) {
    if (a.tslot) a.tslot[(a.slot + 1) % 3] = t + dt;
    if (a.dt_out) *a.dt_out = dt;
    const int z = (a.slot + 2) % 3;
    a.smax[z * 2 + 0] = 0ull;
    a.smax[z * 2 + 1] = 0ull;
  }
  return dt;
}

__device__ __forceinline__ long bc2(long g, long n, int bc) { return bc_index(g, n, bc); }

template <int P, int FLUX, bool F32>
__global__ void __launch_bounds__(NT, F32 ? 3 : (FLUX == ACAT_FLUX_LINEAR ? 3 : 2)) k_step2d(const Step2DArgs a) {
  using PH = Phys2<FLUX>;
  constexpr int S = PH::S;
  using R = typename std::conditional<F32, float, double>::type;
  __shared__ double tile[F32 ? 1 : S][F32 ? 1 : TW2][F32 ? 1 : TW2];
  __shared__ float thi[F32 ? S : 1][F32 ? TW2 : 1][F32 ? TW2 : 1];
  __shared__ float tlo[F32 ? S : 1][F32 ? TW2 : 1][F32 ? TW2 : 1];
  __shared__ R Fx[TXY][TXY + 1][S];
  __shared__ R Gy[TXY + 1][TXY][S];
  __shared__ double s_dt;
  __shared__ double s_red[2][NT / 32];
  const long NXl = a.NX, NYl = a.NY;
  const long x0 = (long)blockIdx.x * TXY, y0 = (long)blockIdx.y * TXY;

  __shared__ double s_lx, s_ly;
  __shared__ float s_lxf, s_lyf;
  if (threadIdx.x == 0) {
    s_dt = step_dt2(a);
    s_lx = s_dt / a.dx;
    s_ly = s_dt / a.dy;
    s_lxf = (float)s_lx;
    s_lyf = (float)s_ly;
  }
  constexpr int CELLS = TW2 * TW2;
  for (int q = threadIdx.x; q < S * CELLS; q += NT) {
    const int c = q / CELLS, rem = q - c * CELLS, yy = rem / TW2, xx = rem - yy * TW2;
    const long gx = bc2(x0 - GH2 + xx, NXl, a.bc), gy = bc2(y0 - GH2 + yy, NYl, a.bc);
    const long gi = ((long)c * NYl + gy) * NXl + gx;
    if (!acat_in_bounds(gx >= 0 && gx < NXl && gy >= 0 && gy < NYl, a.status)) continue;
    if constexpr (F32) {
      const float *u = static_cast<const float *>(a.u_in);
      thi[c][yy][xx] = u[gi];
      tlo[c][yy][xx] = u[(long)S * NYl * NXl + gi];
    } else {
      tile[c][yy][xx] = static_cast<const double *>(a.u_in)[gi];
    }
  }
  __syncthreads();
  const double lxd = s_lx, lyd = s_ly;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int grp = lane >> 4, l = lane & 15, base = grp * 16;
  // the warps' exchange slots of the FP32 block recursion of systems
  __shared__ float4 xs2[(F32 && S > 1 && P >= 2) ? (NT / 32) * 128 : 1];
  constexpr int CS = TW2 * TW2, RS = TW2;
  const FiltConst FC = filt_const(a.epsf, a.rf, a.factf);
  // --- dimension-by-dimension order decisions of every anchor first, one
  // (direction, component, anchor) per thread and pass: rejected orders
  // (Eqs. 3.2-3.3 on the row through the anchor for x, its column for y)
  __shared__ unsigned char rej2[P >= 2 ? 2 * S * NA * NA : 1];
  if constexpr (P >= 2) {
    for (int q = threadIdx.x; q < 2 * S * NA * NA; q += NT) {
      const int dc = q / (NA * NA), an = q - dc * NA * NA, dir = dc / S, c = dc - dir * S;
      const int ax = an % NA - 1, ay = an / NA - 1;
      const bool inside = x0 + ax < NXl && y0 + ay < NYl;
      unsigned r = 0;
      if (inside && (dir == 0 ? ay >= 0 : ax >= 0)) {
        const int tx = ax + GH2, ty = ay + GH2;
        if constexpr (F32)
          r = reject_set32<P>(&thi[c][ty][tx], &tlo[c][ty][tx], dir == 0 ? 1 : RS, c == 0, FC, a.eps, a.thr,
                              a.fact_tau, a.psi2_mod);
        else
          r = reject_set64<P>(&tile[c][ty][tx], dir == 0 ? 1 : RS, c == 0, FC, a.eps, a.thr, a.fact_tau,
                              a.psi2_mod);
      }
      rej2[q] = (unsigned char)r;
    }
    __syncthreads();
  }

  for (int round = 0; round < NA * NA / 16; round++) {
    const int an = round * 16 + warp * 2 + grp;
    const int ax = an % NA - 1, ay = an / NA - 1;  // anchor relative to (x0, y0)
    const long gxa = x0 + ax, gya = y0 + ay;
    const bool inside = gxa < NXl && gya < NYl;
    const bool needF = inside && ay >= 0;
    const bool needG = inside && ax >= 0;
    const int tx = ax + GH2, ty = ay + GH2;
    const double *q64 = F32 ? nullptr : &tile[0][F32 ? 0 : ty][F32 ? 0 : tx];
    unsigned rej = 0;
    if constexpr (P >= 2) {
#pragma unroll
      for (int c = 0; c < S; c++) {
        rej |= rej2[c * NA * NA + an];
        rej |= (unsigned)rej2[(S + c) * NA * NA + an] << (P - 1);
      }
    }
    int px = 1, py = 1;
    if (P >= 2) {
      const unsigned all = (1u << (P - 1)) - 1u;
      const unsigned accx = ~rej & all, accy = ~(rej >> (P - 1)) & all;
      px = accx ? (32 - __clz(accx)) + 1 : 1;
      py = accy ? (32 - __clz(accy)) + 1 : 1;
    }
    const bool blkF = needF && px >= 2, blkG = needG && py >= 2;
    R F[S], G[S];
    if (P >= 2 && (blkF || blkG)) {
      if constexpr (P >= 2) {
        if constexpr (F32) {
          cat2d_f32<2, FLUX>(&thi[0][ty][tx], &tlo[0][ty][tx], CS, RS, l, base, s_lxf, s_lyf, a.advf[0],
                             a.advf[1], a.gm1f, &xs2[warp * 128], F, G);
        } else {
          cat2d_f64<2, FLUX>(q64, CS, RS, l, base, lxd, lyd, a.adv[0], a.adv[1], a.gamma - 1.0, F, G);
        }
      }
    }
    const bool flF = needF && !blkF, flG = needG && !blkG;
    if (l == 0 && (flF || flG)) {
      R F1[S], G1[S];
      if constexpr (F32) {
        flcat2_2d_f32<FLUX>(&thi[0][ty][tx], &tlo[0][ty][tx], CS, RS, flF, flG, s_lxf, s_lyf, a.advf[0],
                            a.advf[1], a.gammaf, a.gm1f, a.limiter_form, a.lo_flux, F1, G1);
      } else {
        flcat2_2d_f64<FLUX>(q64, CS, RS, flF, flG, lxd, lyd, a.adv[0], a.adv[1], a.gamma,
                            a.limiter_form, a.lo_flux, F1, G1);
      }
#pragma unroll
      for (int c = 0; c < S; c++) {
        if (flF) F[c] = F1[c];
        if (flG) G[c] = G1[c];
      }
    }
    if (l == 0) {
      if (needF) {
#pragma unroll
        for (int c = 0; c < S; c++) Fx[ay][ax + 1][c] = F[c];
        if (a.ord_x && (ax >= 0 || gxa == -1)) a.ord_x[gya * (NXl + 1) + (gxa + 1)] = (int8_t)px;
      }
      if (needG) {
#pragma unroll
        for (int c = 0; c < S; c++) Gy[ay + 1][ax][c] = G[c];
        if (a.ord_y && (ay >= 0 || gya == -1)) a.ord_y[(gya + 1) * NXl + gxa] = (int8_t)py;
      }
    }
  }
  __syncthreads();

  // --- update and wave-speed epilogue ------------------------------------------
  R mx = 0, my = 0;
  bool bad = false;
  for (int t = threadIdx.x; t < TXY * TXY; t += NT) {
    const int cy = t / TXY, cx = t - cy * TXY;
    const long gx = x0 + cx, gy = y0 + cy;
    if (gx >= NXl || gy >= NYl) continue;
    const int tx = cx + GH2, ty = cy + GH2;
    double un[S];
    if constexpr (F32) {
      float uc[S], ucl[S], hx[S], lx_[S], hy[S], ly_[S], Bx[S], By[S], junk[S], hf[S], lf[S];
#pragma unroll
      for (int c = 0; c < S; c++) {
        uc[c] = thi[c][ty][tx];
        ucl[c] = tlo[c][ty][tx];
        hx[c] = thi[c][ty][tx - 1] - uc[c];
        lx_[c] = tlo[c][ty][tx - 1] - ucl[c];
        hy[c] = thi[c][ty - 1][tx] - uc[c];
        ly_[c] = tlo[c][ty - 1][tx] - ucl[c];
      }
      const typename PH::Base B = PH::base2(uc, ucl, a.advf[0], a.advf[1], a.gm1f);
      PH::dflux2_pair(B, hx, lx_, Bx, junk);  // f(u_{x-1,y}) - f(u)
      PH::dflux2_pair(B, hy, ly_, junk, By);  // g(u_{x,y-1}) - g(u)
      float *uo = static_cast<float *>(a.u_out);
      const float lx = s_lxf, ly = s_lyf;
#pragma unroll
      for (int c = 0; c < S; c++) {
        const float dx_ = __fmul_rn(lx, __fadd_rn(Bx[c], __fsub_rn(Fx[cy][cx][c], Fx[cy][cx + 1][c])));
        const float dy_ = __fmul_rn(ly, __fadd_rn(By[c], __fsub_rn(Gy[cy][cx][c], Gy[cy + 1][cx][c])));
        const float d = __fadd_rn(dx_, dy_);
        const float h = thi[c][ty][tx], w = tlo[c][ty][tx];
        const float s = __fadd_rn(h, d);
        const float bp = __fsub_rn(s, h);
        const float e = __fadd_rn(__fsub_rn(h, __fsub_rn(s, bp)), __fsub_rn(d, bp));
        const float w2 = __fadd_rn(w, e);
        const float hn = __fadd_rn(s, w2);
        const float ln = __fsub_rn(w2, __fsub_rn(hn, s));
        const long gi = ((long)c * NYl + gy) * NXl + gx;
        uo[gi] = hn;
        uo[(long)S * NYl * NXl + gi] = ln;
        hf[c] = hn;
        lf[c] = ln;
      }
      // wave speeds in float; a state that looks non-physical is re-checked in FP64
      const float g = a.gammaf;
      const float sxf = PH::fspeed(hf, a.advf[0], a.advf[1], g, 0);
      const float syf = PH::fspeed(hf, a.advf[0], a.advf[1], g, 1);
      if (!PH::fphysical(hf, g)) {
#pragma unroll
        for (int c = 0; c < S; c++) un[c] = (double)hf[c] + (double)lf[c];
        double sx, sy;
        bool ok;
        PH::speed2(un, a.adv[0], a.adv[1], a.gamma, sx, sy, ok);
        bad |= !ok;
      }
      mx = fmaxf(mx, sxf);
      my = fmaxf(my, syf);
      continue;
    } else {
      double *uo = static_cast<double *>(a.u_out);
#pragma unroll
      for (int c = 0; c < S; c++) {
        un[c] = tile[c][ty][tx] + lxd * (Fx[cy][cx][c] - Fx[cy][cx + 1][c]) +
                lyd * (Gy[cy][cx][c] - Gy[cy + 1][cx][c]);
        uo[((long)c * NYl + gy) * NXl + gx] = un[c];
      }
    }
    double sx, sy;
    bool ok;
    PH::speed2(un, a.adv[0], a.adv[1], a.gamma, sx, sy, ok);
    bad |= !ok;
    if constexpr (!F32) {
      mx = fmax(mx, sx);
      my = fmax(my, sy);
    }
  }
  if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(a.status, (unsigned)ACAT_STATUS_NONPHYSICAL);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const R ox = __shfl_xor_sync(0xffffffffu, mx, o), oy = __shfl_xor_sync(0xffffffffu, my, o);
    mx = ox > mx ? ox : mx;
    my = oy > my ? oy : my;
  }
  if (lane == 0) {
    s_red[0][warp] = (double)mx;
    s_red[1][warp] = (double)my;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double vx = s_red[0][0], vy = s_red[1][0];
    for (int w = 1; w < NT / 32; w++) {
      vx = fmax(vx, s_red[0][w]);
      vy = fmax(vy, s_red[1][w]);
    }
    const int z = (a.slot + 1) % 3;
    atomic_max_pos(&a.smax[z * 2 + 0], vx);
    atomic_max_pos(&a.smax[z * 2 + 1], vy);
  }
}

template <int FLUX, bool F32>
__global__ void __launch_bounds__(NT) k_smax2d(const Step2DArgs a) {
  constexpr int S = Phys2<FLUX>::S;
  __shared__ double s_red[2][NT / 32];
  const long NC = (long)a.NX * a.NY;
  double mx = 0.0, my = 0.0;
  bool bad = false;
  for (long i = (long)blockIdx.x * NT + threadIdx.x; i < NC; i += (long)gridDim.x * NT) {
    double u[S];
#pragma unroll
    for (int c = 0; c < S; c++) {
      if constexpr (F32) {
        const float *p = static_cast<const float *>(a.u_in);
        u[c] = (double)p[c * NC + i] + (double)p[(S + c) * NC + i];
      } else {
        u[c] = static_cast<const double *>(a.u_in)[c * NC + i];
      }
    }
    double sx, sy;
    bool ok;
    Phys2<FLUX>::speed2(u, a.adv[0], a.adv[1], a.gamma, sx, sy, ok);
    mx = fmax(mx, sx);
    my = fmax(my, sy);
    bad |= !ok;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(a.status, (unsigned)ACAT_STATUS_NONPHYSICAL);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    my = fmax(my, __shfl_xor_sync(0xffffffffu, my, o));
  }
  if (lane == 0) {
    s_red[0][warp] = mx;
    s_red[1][warp] = my;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double vx = s_red[0][0], vy = s_red[1][0];
    for (int w = 1; w < NT / 32; w++) {
      vx = fmax(vx, s_red[0][w]);
      vy = fmax(vy, s_red[1][w]);
    }
    atomic_max_pos(&a.smax[a.slot * 2 + 0], vx);
    atomic_max_pos(&a.smax[a.slot * 2 + 1], vy);
    if (blockIdx.x == 0 && a.tslot) a.tslot[a.slot] = 0.0;
  }
}

// ---------------------------------------------------------------------------
// 2D step for P = 3, 4 (FP64). Blocks of 2p x 2p nodes exceed a warp for
// p >= 3, so the block recursion (Eqs. 4.5-4.6) runs with one thread per node
// and the F^(k), G^(k) of the nodes exchanged through shared memory. A CTA
// owns TXH x TXH cells and their (TXH+1)^2 anchors:
//   1. dt, staging of the cells with a halo of P;
//   2. the order decisions of every (anchor, direction, p, component),
//      spread over all threads (filtered / literal as in 1D);
//   3. per anchor: the orders p_1 (row) and p_2 (column); a block task for
//      p_1 = p_2 (serving F and G), else one task per direction with p >= 2
//      (square blocks S_{p_1}, S_{p_2}); FL-CAT2 directions done in place;
//   4. for p = 2..P, the tasks of that p in rounds that pack NT / (2p)^2
//      blocks densely onto the threads, every round in lockstep;
//   5. the conservative update (Eq. 4.9) and the wave speeds for the next dt.
// ---------------------------------------------------------------------------
constexpr int TXH = 12;        // cells per CTA side
constexpr int NAH = TXH + 1;   // anchors per CTA side
constexpr unsigned WANT_F = 1u << 8, WANT_G = 1u << 9;

template <int P, int FLUX>
struct Smem2H {
  static constexpr int S = Phys2<FLUX>::S;
  static constexpr int TW = TXH + 2 * P;
  double tile[S][TW][TW];
  double Fx[TXH][TXH + 1][S];
  double Gy[TXH + 1][TXH][S];
  double X[NT][S], Y[NT][S];  // F^(k), G^(k) of the nodes of a round
  unsigned rej[NAH * NAH];    // rejected orders: bit dir * (P - 1) + (p - 2)
  unsigned short task[P + 1][2 * NAH * NAH];
  int ntask[P + 1];
  unsigned rtask[2 * NAH * NAH];  // rectangular blocks: anchor | wants | p1 << 10 | p2 << 13
  int nrtask;
  double lx, ly;
};

// The block tasks of order p, NT / (2p)^2 per round (node (ia, ib) of task ti
// on thread ti (2p)^2 + ib 2p + ia).
template <int p, int P, int FLUX>
__device__ __forceinline__ void block_tasks(Smem2H<P, FLUX> &sm, const Step2DArgs &a, double lx, double ly) {
  using TB = Tab<double>;
  using PH = Phys2<FLUX>;
  constexpr int S = PH::S;
  constexpr int n = 2 * p, nn = n * n, per = NT / nn, z = p - 1;
  const double gm1 = a.gamma - 1.0, axv = a.adv[0], ayv = a.adv[1];
  const int nt = sm.ntask[p];
  const int tid = threadIdx.x, ti = tid / nn, node = tid - ti * nn;
  const int ia = node % n, ib = node / n;
  // row and column weights scaled by -lambda_x, -lambda_y once (one
  // accumulation of U over both directions per order)
  double gx[n], gy[n];
#pragma unroll
  for (int r = 0; r < n; r++) {
    gx[r] = TB::g1(p, ia, r) * -lx;
    gy[r] = TB::g1(p, ib, r) * -ly;
  }
  for (int base = 0; base < nt; base += per) {
    const bool act = ti < per && base + ti < nt;
    const unsigned tk = act ? sm.task[p][base + ti] : 0u;
    const int an = (int)(tk & 0xffu);
    const int ax = an % NAH - 1, ay = an / NAH - 1;
    double u[S], f0[S], g0[S], Fs[S], Gs[S], arg[n][S];
    if (act) {
      const int tx = acat_tile_index(ax + P - p + 1 + ia, Smem2H<P, FLUX>::TW, a.status);
      const int ty = acat_tile_index(ay + P - p + 1 + ib, Smem2H<P, FLUX>::TW, a.status);
#pragma unroll
      for (int c = 0; c < S; c++) u[c] = sm.tile[c][ty][tx];
      PH::flux2(u, f0, g0, axv, ayv, gm1);
    } else {
#pragma unroll
      for (int c = 0; c < S; c++) u[c] = f0[c] = g0[c] = 0.0;
    }
#pragma unroll
    for (int c = 0; c < S; c++) {
      Fs[c] = f0[c];
      Gs[c] = g0[c];
      sm.X[tid][c] = f0[c];
      sm.Y[tid][c] = g0[c];
    }
#pragma unroll
    for (int rr = 0; rr < n; rr++)
#pragma unroll
      for (int c = 0; c < S; c++) arg[rr][c] = u[c];
#pragma unroll 1
    for (int k = 2; k <= n; k++) {
      __syncthreads();
      double U[S];
      if (act) {
#pragma unroll
        for (int c = 0; c < S; c++) U[c] = 0.0;
#pragma unroll
        for (int r = 0; r < n; r++)
#pragma unroll
          for (int c = 0; c < S; c++) U[c] = fma(gx[r], sm.X[ti * nn + ib * n + r][c], U[c]);
#pragma unroll
        for (int r = 0; r < n; r++)
#pragma unroll
          for (int c = 0; c < S; c++) U[c] = fma(gy[r], sm.Y[ti * nn + r * n + ia][c], U[c]);
      }
      __syncthreads();
      if (act) {
        double af[S], ag[S];
#pragma unroll
        for (int c = 0; c < S; c++) {
          af[c] = TB::gk(p, k - 1, z) * f0[c];
          ag[c] = TB::gk(p, k - 1, z) * g0[c];
        }
#pragma unroll
        for (int rr = 0; rr < n; rr++) {
          if (rr == z) continue;
          const double cr = TB::taylor(p, rr, k - 1), wk = TB::gk(p, k - 1, rr);
          double fr[S], gr[S];
#pragma unroll
          for (int c = 0; c < S; c++) arg[rr][c] = fma(cr, U[c], arg[rr][c]);
          PH::flux2(arg[rr], fr, gr, axv, ayv, gm1);
#pragma unroll
          for (int c = 0; c < S; c++) {
            af[c] = fma(wk, fr[c], af[c]);
            ag[c] = fma(wk, gr[c], ag[c]);
          }
        }
#pragma unroll
        for (int c = 0; c < S; c++) {
          sm.X[tid][c] = af[c];
          sm.Y[tid][c] = ag[c];
          Fs[c] = fma(TB::invfact(k), af[c], Fs[c]);
          Gs[c] = fma(TB::invfact(k), ag[c], Gs[c]);
        }
      }
    }
    __syncthreads();
    if (act) {
#pragma unroll
      for (int c = 0; c < S; c++) {
        if (ib == z) sm.X[tid][c] = TB::gh(p, ia) * Fs[c];
        if (ia == z) sm.Y[tid][c] = TB::gh(p, ib) * Gs[c];
      }
    }
    __syncthreads();
    if (act && node == 0) {
      if (tk & WANT_F)
#pragma unroll
        for (int c = 0; c < S; c++) {
          double t = 0.0;
#pragma unroll
          for (int r = 0; r < n; r++) t += sm.X[ti * nn + z * n + r][c];
          sm.Fx[ay][ax + 1][c] = t;
        }
      if (tk & WANT_G)
#pragma unroll
        for (int c = 0; c < S; c++) {
          double t = 0.0;
#pragma unroll
          for (int r = 0; r < n; r++) t += sm.Y[ti * nn + r * n + z][c];
          sm.Gy[ay + 1][ax][c] = t;
        }
    }
    __syncthreads();
  }
}

// The rectangular block tasks (rect_2d): one block S_{p1,p2} of 2 p1 x 2 p2
// nodes per task, p1 != p2 (a direction on FL-CAT2 counts as p = 1). The
// recursion of block_tasks with runtime extents: x-derivatives over the
// 2 p1 nodes of a row, y-derivatives over the 2 p2 nodes of a column, the
// 2 pm time levels of pm = max(p1, p2), the recursion to k = 2 pm; F sums to
// k = 2 p1 along the row j2 = 0, G to k = 2 p2 along the column j1 = 0.
// (2P)^2 threads per task, node (ia, ib) on thread ti (2P)^2 + ib 2P + ia.
template <int P, int FLUX>
__device__ __forceinline__ void rect_tasks(Smem2H<P, FLUX> &sm, const Step2DArgs &a, double lx, double ly) {
  using TB = Tab<double>;
  using PH = Phys2<FLUX>;
  constexpr int S = PH::S;
  constexpr int NM = 2 * P, NN = NM * NM, per = NT / NN;
  const double gm1 = a.gamma - 1.0, axv = a.adv[0], ayv = a.adv[1];
  const int nt = sm.nrtask;
  const int tid = threadIdx.x, ti = tid / NN, node = tid - ti * NN;
  const int ia = node % NM, ib = node / NM;
  for (int base = 0; base < nt; base += per) {
    const bool slot_ok = ti < per && base + ti < nt;
    const unsigned tk = slot_ok ? sm.rtask[base + ti] : 0u;
    const int an = (int)(tk & 0xffu);
    const int p1 = slot_ok ? (int)((tk >> 10) & 7u) : 1, p2 = slot_ok ? (int)((tk >> 13) & 7u) : 1;
    const int n1 = 2 * p1, n2 = 2 * p2, pm = p1 > p2 ? p1 : p2, n = 2 * pm, zt = pm - 1;
    const bool act = slot_ok && ia < n1 && ib < n2;
    const int ax = an % NAH - 1, ay = an / NAH - 1;
    double u[S], f0[S], g0[S], Fs[S], Gs[S], arg[NM][S];
    if (act) {
      const int tx = acat_tile_index(ax + P - p1 + 1 + ia, Smem2H<P, FLUX>::TW, a.status);
      const int ty = acat_tile_index(ay + P - p2 + 1 + ib, Smem2H<P, FLUX>::TW, a.status);
#pragma unroll
      for (int c = 0; c < S; c++) u[c] = sm.tile[c][ty][tx];
      PH::flux2(u, f0, g0, axv, ayv, gm1);
    } else {
#pragma unroll
      for (int c = 0; c < S; c++) u[c] = f0[c] = g0[c] = 0.0;
    }
#pragma unroll
    for (int c = 0; c < S; c++) {
      Fs[c] = f0[c];
      Gs[c] = g0[c];
      sm.X[tid][c] = f0[c];
      sm.Y[tid][c] = g0[c];
    }
#pragma unroll
    for (int rr = 0; rr < NM; rr++)
#pragma unroll
      for (int c = 0; c < S; c++) arg[rr][c] = u[c];
#pragma unroll 1
    for (int k = 2; k <= NM; k++) {
      __syncthreads();
      const bool go = act && k <= n;
      double U[S];
      if (go) {
        double Ux[S], Uy[S];
#pragma unroll
        for (int c = 0; c < S; c++) Ux[c] = Uy[c] = 0.0;
#pragma unroll
        for (int r = 0; r < NM; r++) {
          if (r < n1) {
            const double w = TB::g1(p1, ia, r);
#pragma unroll
            for (int c = 0; c < S; c++) Ux[c] = fma(w, sm.X[ti * NN + ib * NM + r][c], Ux[c]);
          }
          if (r < n2) {
            const double w = TB::g1(p2, ib, r);
#pragma unroll
            for (int c = 0; c < S; c++) Uy[c] = fma(w, sm.Y[ti * NN + r * NM + ia][c], Uy[c]);
          }
        }
#pragma unroll
        for (int c = 0; c < S; c++) U[c] = -(lx * Ux[c]) - ly * Uy[c];
      }
      __syncthreads();
      if (go) {
        double af[S], ag[S];
#pragma unroll
        for (int c = 0; c < S; c++) {
          af[c] = TB::gk(pm, k - 1, zt) * f0[c];
          ag[c] = TB::gk(pm, k - 1, zt) * g0[c];
        }
#pragma unroll
        for (int rr = 0; rr < NM; rr++) {
          if (rr >= n || rr == zt) continue;
          const double cr = TB::taylor(pm, rr, k - 1), wk = TB::gk(pm, k - 1, rr);
          double fr[S], gr[S];
#pragma unroll
          for (int c = 0; c < S; c++) arg[rr][c] = fma(cr, U[c], arg[rr][c]);
          PH::flux2(arg[rr], fr, gr, axv, ayv, gm1);
#pragma unroll
          for (int c = 0; c < S; c++) {
            af[c] = fma(wk, fr[c], af[c]);
            ag[c] = fma(wk, gr[c], ag[c]);
          }
        }
#pragma unroll
        for (int c = 0; c < S; c++) {
          sm.X[tid][c] = af[c];
          sm.Y[tid][c] = ag[c];
          if (k <= n1) Fs[c] = fma(TB::invfact(k), af[c], Fs[c]);
          if (k <= n2) Gs[c] = fma(TB::invfact(k), ag[c], Gs[c]);
        }
      }
    }
    __syncthreads();
    if (act) {
#pragma unroll
      for (int c = 0; c < S; c++) {
        if (ib == p2 - 1) sm.X[tid][c] = TB::gh(p1, ia) * Fs[c];
        if (ia == p1 - 1) sm.Y[tid][c] = TB::gh(p2, ib) * Gs[c];
      }
    }
    __syncthreads();
    if (slot_ok && node == 0) {
      if (tk & WANT_F)
#pragma unroll
        for (int c = 0; c < S; c++) {
          double t = 0.0;
          for (int r = 0; r < n1; r++) t += sm.X[ti * NN + (p2 - 1) * NM + r][c];
          sm.Fx[ay][ax + 1][c] = t;
        }
      if (tk & WANT_G)
#pragma unroll
        for (int c = 0; c < S; c++) {
          double t = 0.0;
          for (int r = 0; r < n2; r++) t += sm.Y[ti * NN + r * NM + (p1 - 1)][c];
          sm.Gy[ay + 1][ax][c] = t;
        }
    }
    __syncthreads();
  }
}

template <int P, int FLUX>
__global__ void __launch_bounds__(NT, 1) k_step2d_hi(const Step2DArgs a) {
  using PH = Phys2<FLUX>;
  constexpr int S = PH::S;
  constexpr int TW = Smem2H<P, FLUX>::TW;
  constexpr int CELLS = TW * TW;
  __shared__ Smem2H<P, FLUX> sm;
  const int tid = threadIdx.x;
  const long NXl = a.NX, NYl = a.NY;
  const long x0 = (long)blockIdx.x * TXH, y0 = (long)blockIdx.y * TXH;
  if (tid == 0) {
    const double dt = step_dt2(a);
    sm.lx = dt / a.dx;
    sm.ly = dt / a.dy;
  }
  if (tid <= P) sm.ntask[tid] = 0;
  if (tid == 0) sm.nrtask = 0;
  for (int q = tid; q < NAH * NAH; q += NT) sm.rej[q] = 0u;
  const double *uin = static_cast<const double *>(a.u_in);
  for (int q = tid; q < S * CELLS; q += NT) {
    const int c = q / CELLS, rem = q - c * CELLS, yy = rem / TW, xx = rem - yy * TW;
    const long gx = bc2(x0 - P + xx, NXl, a.bc), gy = bc2(y0 - P + yy, NYl, a.bc);
    if (!acat_in_bounds(gx >= 0 && gx < NXl && gy >= 0 && gy < NYl, a.status)) continue;
    sm.tile[c][yy][xx] = uin[((long)c * NYl + gy) * NXl + gx];
  }
  __syncthreads();
  const double lx = sm.lx, ly = sm.ly;
  // --- order decisions of every (anchor, direction, p, component) ----------
  constexpr int NPAIR = 2 * S;  // (direction, component): every order p = 2..P at once
  const FiltConst FC = filt_const(a.epsf, a.rf, a.factf);
  for (int q = tid; q < NAH * NAH * NPAIR; q += NT) {
    const int an = q / NPAIR, pr = q - an * NPAIR;
    const int dir = pr / S, c = pr - dir * S;
    const int ax = an % NAH - 1, ay = an / NAH - 1;
    const bool inside = x0 + ax < NXl && y0 + ay < NYl;
    // rectangular blocks take both orders of every anchor that has a flux
    const bool skip = a.rect_2d ? (ax < 0 && ay < 0) : (dir == 0 ? ay < 0 : ax < 0);
    if (!inside || skip) continue;
    const unsigned r = reject_set64<P>(&sm.tile[c][ay + P][ax + P], dir == 0 ? 1 : TW, c == 0, FC, a.eps, a.thr,
                                       a.fact_tau, a.psi2_mod);
    if (r) atomicOr(&sm.rej[an], r << (dir * (P - 1)));
  }
  __syncthreads();
  // --- orders, block tasks, FL-CAT2 directions -----------------------------
  for (int an = tid; an < NAH * NAH; an += NT) {
    const int ax = an % NAH - 1, ay = an / NAH - 1;
    const long gxa = x0 + ax, gya = y0 + ay;
    const bool inside = gxa < NXl && gya < NYl;
    const bool needF = inside && ay >= 0, needG = inside && ax >= 0;
    const unsigned rej = sm.rej[an], all = (1u << (P - 1)) - 1u;
    const unsigned accx = ~rej & all, accy = ~(rej >> (P - 1)) & all;
    const int px = accx ? (32 - __clz(accx)) + 1 : 1, py = accy ? (32 - __clz(accy)) + 1 : 1;
    if (needF && a.ord_x && (ax >= 0 || gxa == -1)) a.ord_x[gya * (NXl + 1) + (gxa + 1)] = (int8_t)px;
    if (needG && a.ord_y && (ay >= 0 || gya == -1)) a.ord_y[(gya + 1) * NXl + gxa] = (int8_t)py;
    const bool bF = needF && px >= 2, bG = needG && py >= 2;
    if (a.rect_2d) {
      // one block S_{px,py} serves both directions of the anchor
      const unsigned want = (bF ? WANT_F : 0u) | (bG ? WANT_G : 0u);
      if (want && px == py) sm.task[px][atomicAdd(&sm.ntask[px], 1)] = (unsigned short)(an | want);
      else if (want) sm.rtask[atomicAdd(&sm.nrtask, 1)] = (unsigned)an | want | ((unsigned)px << 10) | ((unsigned)py << 13);
    } else if (bF && bG && px == py) {
      sm.task[px][atomicAdd(&sm.ntask[px], 1)] = (unsigned short)(an | WANT_F | WANT_G);
    } else {
      if (bF) sm.task[px][atomicAdd(&sm.ntask[px], 1)] = (unsigned short)(an | WANT_F);
      if (bG) sm.task[py][atomicAdd(&sm.ntask[py], 1)] = (unsigned short)(an | WANT_G);
    }
    const bool flF = needF && px < 2, flG = needG && py < 2;
    if (flF || flG) {
      double F1[S], G1[S];
      flcat2_2d_f64<FLUX>(&sm.tile[0][ay + P][ax + P], CELLS, TW, flF, flG, lx, ly, a.adv[0], a.adv[1],
                          a.gamma, a.limiter_form, a.lo_flux, F1, G1);
#pragma unroll
      for (int c = 0; c < S; c++) {
        if (flF) sm.Fx[ay][ax + 1][c] = F1[c];
        if (flG) sm.Gy[ay + 1][ax][c] = G1[c];
      }
    }
  }
  __syncthreads();
  // --- block recursions, one order at a time ------------------------------
  block_tasks<2, P, FLUX>(sm, a, lx, ly);
  if constexpr (P >= 3) block_tasks<3, P, FLUX>(sm, a, lx, ly);
  if constexpr (P >= 4) block_tasks<4, P, FLUX>(sm, a, lx, ly);
  if (a.rect_2d) rect_tasks<P, FLUX>(sm, a, lx, ly);
  // --- update and wave-speed epilogue (Eq. 4.9) ---------------------------
  double mx = 0.0, my = 0.0;
  bool bad = false;
  double *uo = static_cast<double *>(a.u_out);
  for (int t = tid; t < TXH * TXH; t += NT) {
    const int cy = t / TXH, cx = t - cy * TXH;
    const long gx = x0 + cx, gy = y0 + cy;
    if (gx >= NXl || gy >= NYl) continue;
    double un[S];
#pragma unroll
    for (int c = 0; c < S; c++) {
      un[c] = sm.tile[c][cy + P][cx + P] + lx * (sm.Fx[cy][cx][c] - sm.Fx[cy][cx + 1][c]) +
              ly * (sm.Gy[cy][cx][c] - sm.Gy[cy + 1][cx][c]);
      uo[((long)c * NYl + gy) * NXl + gx] = un[c];
    }
    double sx, sy;
    bool ok;
    PH::speed2(un, a.adv[0], a.adv[1], a.gamma, sx, sy, ok);
    bad |= !ok;
    mx = fmax(mx, sx);
    my = fmax(my, sy);
  }
  const int lane = tid & 31;
  if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(a.status, (unsigned)ACAT_STATUS_NONPHYSICAL);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    my = fmax(my, __shfl_xor_sync(0xffffffffu, my, o));
  }
  if (lane == 0) {
    const int zs = (a.slot + 1) % 3;
    atomic_max_pos(&a.smax[zs * 2 + 0], mx);
    atomic_max_pos(&a.smax[zs * 2 + 1], my);
  }
}

template <int P, int FLUX, bool F32>
int launch2(const Step2DArgs &a, cudaStream_t st) {
  dim3 grid((unsigned)((a.NX + TXY - 1) / TXY), (unsigned)((a.NY + TXY - 1) / TXY));
  k_step2d<P, FLUX, F32><<<grid, NT, 0, st>>>(a);
  return (int)cudaGetLastError();
}

// ---------------------------------------------------------------------------
// 2D step for P = 3, 4 in FP32, and the rectangular stencils in FP32 at
// P = 2..4: the structure of k_step2d_hi on the compensated state. Every
// block task (square or rectangular) runs one thread per node on a
// (2P)^2-thread slot with runtime extents 2 p1 x 2 p2, in the delta
// formulation of the P <= 2 FP32 kernel: node j carries increments about the
// anchor state u_a, f(u_j) - f(u_a) from a cancellation-free difference, and
// every time level's flux increment f(u_j + del) - f(u_j) likewise; the
// fluxes leave as F - f(u_a), G - g(u_a), and the update adds
// f(u_{i-1}) - f(u_i) itself (TwoSum / Fast2Sum into the pair).
// ---------------------------------------------------------------------------
// The float weight tables in shared memory: the FP32 block tasks index them
// with per-task orders and a per-thread node, which constant memory serves
// one address at a time.
struct TabSF {
  float g1[ACAT_MAXP + 1][ACAT_MAXN][ACAT_MAXN];
  float gk[ACAT_MAXP + 1][ACAT_MAXN][ACAT_MAXN];
  float taylor[ACAT_MAXP + 1][ACAT_MAXN][ACAT_MAXN];
  float gh[ACAT_MAXP + 1][ACAT_MAXN];
  float invfact[ACAT_MAXN + 1];
};

// Tiles of the FP32 high-order step: TXF x TXF cells and their (TXF+1)^2
// anchors. Below P = 4 they are larger than the FP64 kernel's (its double
// tiles fill the shared memory at TXH): fewer of the anchors on a tile's left
// column and bottom row, whose block recursions the neighbouring CTA repeats.
// At P = 4 the larger tile measured slower (fewer CTAs per SM) and TXH is kept.
// Task words: anchor in bits 0-9, the wanted fluxes in bits 10-11, p1 and p2
// from bits 12 and 15.
template <int P>
constexpr int TXF = P >= 4 ? TXH : 16;
template <int P>
constexpr int NAF = TXF<P> + 1;
constexpr unsigned WF32 = 1u << 10, WG32 = 1u << 11;
template <int P, int FLUX>
struct Smem2HF {
  static constexpr int S = Phys2<FLUX>::S;
  static constexpr int TW = TXF<P> + 2 * P;
  float thi[S][TW][TW], tlo[S][TW][TW];
  float Fx[TXF<P>][TXF<P> + 1][S];
  float Gy[TXF<P> + 1][TXF<P>][S];
  // F^(k), G^(k) increments of the nodes of a round, a task's 2P x 2P nodes
  // by rows (X) and by columns (Y). At P = 2, 4 each row (column) is padded to
  // 2P + 1 slots, so that the loads of node r of a warp's rows (columns) fall
  // in distinct 16-byte bank quads instead of 4 to a quad (5 % faster). At
  // P = 3 the packed rows meet at most 2 to a quad, and X and Y stay packed
  // in thread order (the padded form measured 2 % slower there). RW: slots
  // between rows of X; YC, YS: between columns and between the nodes of a
  // column of Y; TS: per task. Room for the idle threads past the last task.
  static constexpr bool PAD = P != 3;
  static constexpr int RW = PAD ? 2 * P + 1 : 2 * P, TS = 2 * P * RW;
  static constexpr int YC = PAD ? RW : 1, YS = PAD ? 1 : 2 * P;
  static constexpr int XS = (NT / (4 * P * P) + 1) * TS;
  float X[XS][S], Y[XS][S];
  unsigned rej[NAF<P> * NAF<P>];    // rejected orders: bit dir * (P - 1) + (p - 2)
  unsigned task[2 * NAF<P> * NAF<P>];  // anchor | wants | p1 << 12 | p2 << 15
  int ntask;
  float lx, ly;
  TabSF tab;
};

template <int P, int FLUX>
__device__ __forceinline__ void block_tasks_f32(Smem2HF<P, FLUX> &sm, const Step2DArgs &a, float lx, float ly) {
  const TabSF &TB = sm.tab;
  using PH = Phys2<FLUX>;
  constexpr int S = PH::S;
  constexpr int NM = 2 * P, NN = NM * NM, per = NT / NN;
  const float gm1 = a.gm1f, axv = a.advf[0], ayv = a.advf[1];
  const int nt = sm.ntask;
  const int tid = threadIdx.x, ti = tid / NN, node = tid - ti * NN;
  const int ia = node % NM, ib = node / NM;
  using SM = Smem2HF<P, FLUX>;
  const int xrow = ti * SM::TS + ib * SM::RW, ycol = ti * SM::TS + ia * SM::YC;  // row / column
  const int xw = xrow + ia, yw = ycol + ib * SM::YS;                             // own slots
  for (int base = 0; base < nt; base += per) {
    const bool slot_ok = ti < per && base + ti < nt;
    const unsigned tk = slot_ok ? sm.task[base + ti] : 0u;
    const int an = (int)(tk & 0x3ffu);
    const int p1 = slot_ok ? (int)((tk >> 12) & 7u) : 1, p2 = slot_ok ? (int)((tk >> 15) & 7u) : 1;
    const int n1 = 2 * p1, n2 = 2 * p2, pm = p1 > p2 ? p1 : p2, n = 2 * pm, zt = pm - 1;
    const bool act = slot_ok && ia < n1 && ib < n2;
    const int ax = an % NAF<P> - 1, ay = an / NAF<P> - 1;
    float Ff[S], Fg[S], dels[NM][S];
    typename PH::Base bj;
    if (act) {
      const int tx = acat_tile_index(ax + P - p1 + 1 + ia, Smem2HF<P, FLUX>::TW, a.status);
      const int ty = acat_tile_index(ay + P - p2 + 1 + ib, Smem2HF<P, FLUX>::TW, a.status);
      float ua[S], ual[S], uj[S], ujl[S], dh[S], dl[S];
#pragma unroll
      for (int c = 0; c < S; c++) {
        ua[c] = sm.thi[c][ay + P][ax + P];
        ual[c] = sm.tlo[c][ay + P][ax + P];
        uj[c] = sm.thi[c][ty][tx];
        ujl[c] = sm.tlo[c][ty][tx];
        dh[c] = uj[c] - ua[c];
        dl[c] = ujl[c] - ual[c];
      }
      PH::dflux2_pair(PH::base2(ua, ual, axv, ayv, gm1), dh, dl, Ff, Fg);  // f(u_j) - f(u_a), g(u_j) - g(u_a)
      bj = PH::base2(uj, ujl, axv, ayv, gm1);
    } else {
      float z[S];
#pragma unroll
      for (int c = 0; c < S; c++) z[c] = Ff[c] = Fg[c] = 0.0f;
      bj = PH::base(z, axv, ayv, gm1);
    }
#pragma unroll
    for (int c = 0; c < S; c++) {
      sm.X[xw][c] = Ff[c];
      sm.Y[yw][c] = Fg[c];
    }
#pragma unroll
    for (int rr = 0; rr < NM; rr++)
#pragma unroll
      for (int c = 0; c < S; c++) dels[rr][c] = 0.0f;
    // the derivative weights of the node's row and column, read once per task
    // at P <= 3 (at P = 4 they would cost the registers of the second CTA per
    // SM, and the loop reads them from the shared table)
    constexpr bool HW = P <= 3;
    float wx[HW ? NM : 1], wy[HW ? NM : 1];
    if constexpr (HW) {
#pragma unroll
      for (int r = 0; r < NM; r++) {  // scaled by -lambda_x, -lambda_y once
        wx[r] = act && r < n1 ? __fmul_rn(TB.g1[p1][ia][r], -lx) : 0.0f;
        wy[r] = act && r < n2 ? __fmul_rn(TB.g1[p2][ib][r], -ly) : 0.0f;
      }
    }
#pragma unroll 1
    for (int k = 2; k <= NM; k++) {
      __syncthreads();
      const bool go = act && k <= n;
      float U[S];
      if (go) {
        if constexpr (HW) {  // the scaled weights: one accumulation over row and column
#pragma unroll
          for (int c = 0; c < S; c++) U[c] = 0.0f;
#pragma unroll
          for (int r = 0; r < NM; r++) {
            if (r < n1) {
#pragma unroll
              for (int c = 0; c < S; c++) U[c] = fmaf(wx[r], sm.X[xrow + r][c], U[c]);
            }
            if (r < n2) {
#pragma unroll
              for (int c = 0; c < S; c++) U[c] = fmaf(wy[r], sm.Y[ycol + r * SM::YS][c], U[c]);
            }
          }
        } else {
          float Ux[S], Uy[S];
#pragma unroll
          for (int c = 0; c < S; c++) Ux[c] = Uy[c] = 0.0f;
#pragma unroll
          for (int r = 0; r < NM; r++) {
            if (r < n1) {
              const float w = TB.g1[p1][ia][r];
#pragma unroll
              for (int c = 0; c < S; c++) Ux[c] = fmaf(w, sm.X[xrow + r][c], Ux[c]);
            }
            if (r < n2) {
              const float w = TB.g1[p2][ib][r];
#pragma unroll
              for (int c = 0; c < S; c++) Uy[c] = fmaf(w, sm.Y[ycol + r * SM::YS][c], Uy[c]);
            }
          }
#pragma unroll
          for (int c = 0; c < S; c++) U[c] = -(lx * Ux[c]) - ly * Uy[c];
        }
      }
      __syncthreads();
      if (go) {
        float af[S], ag[S];
#pragma unroll
        for (int c = 0; c < S; c++) af[c] = ag[c] = 0.0f;
#pragma unroll
        for (int rr = 0; rr < NM; rr++) {
          if (rr >= n || rr == zt) continue;
          const float cr = TB.taylor[pm][rr][k - 1], wk = TB.gk[pm][k - 1][rr];
          float ef[S], eg[S];
#pragma unroll
          for (int c = 0; c < S; c++) dels[rr][c] = fmaf(cr, U[c], dels[rr][c]);
          PH::dflux2(bj, dels[rr], ef, eg);  // f(u_j + del) - f(u_j): the level's weights sum to 0
#pragma unroll
          for (int c = 0; c < S; c++) {
            af[c] = fmaf(wk, ef[c], af[c]);
            ag[c] = fmaf(wk, eg[c], ag[c]);
          }
        }
#pragma unroll
        for (int c = 0; c < S; c++) {
          sm.X[xw][c] = af[c];
          sm.Y[yw][c] = ag[c];
          if (k <= n1) Ff[c] = fmaf(TB.invfact[k], af[c], Ff[c]);
          if (k <= n2) Fg[c] = fmaf(TB.invfact[k], ag[c], Fg[c]);
        }
      }
    }
    __syncthreads();
    if (act) {
#pragma unroll
      for (int c = 0; c < S; c++) {
        if (ib == p2 - 1) sm.X[xw][c] = TB.gh[p1][ia] * Ff[c];
        if (ia == p1 - 1) sm.Y[yw][c] = TB.gh[p2][ib] * Fg[c];
      }
    }
    __syncthreads();
    if (slot_ok && node == 0) {
      if (tk & WF32)
#pragma unroll
        for (int c = 0; c < S; c++) {
          float t = 0.0f;
          for (int r = 0; r < n1; r++) t += sm.X[ti * SM::TS + (p2 - 1) * SM::RW + r][c];
          sm.Fx[ay][ax + 1][c] = t;
        }
      if (tk & WG32)
#pragma unroll
        for (int c = 0; c < S; c++) {
          float t = 0.0f;
          for (int r = 0; r < n2; r++) t += sm.Y[ti * SM::TS + (p1 - 1) * SM::YC + r * SM::YS][c];
          sm.Gy[ay + 1][ax][c] = t;
        }
    }
    __syncthreads();
  }
}

template <int P, int FLUX>
__global__ void __launch_bounds__(NT, 2) k_step2d_hi_f32(const Step2DArgs a) {
  using PH = Phys2<FLUX>;
  constexpr int S = PH::S;
  constexpr int TW = Smem2HF<P, FLUX>::TW;
  constexpr int CELLS = TW * TW;
  __shared__ Smem2HF<P, FLUX> sm;
  __shared__ double s_red[2][NT / 32];
  const int tid = threadIdx.x;
  const long NXl = a.NX, NYl = a.NY;
  const long x0 = (long)blockIdx.x * TXF<P>, y0 = (long)blockIdx.y * TXF<P>;
  if (tid == 0) {
    const double dt = step_dt2(a);
    sm.lx = (float)(dt / a.dx);
    sm.ly = (float)(dt / a.dy);
    sm.ntask = 0;
  }
  for (int q = tid; q < NAF<P> * NAF<P>; q += NT) sm.rej[q] = 0u;
  {
    constexpr int NW3 = (ACAT_MAXP + 1) * ACAT_MAXN * ACAT_MAXN;
    for (int q = tid; q < NW3; q += NT) {
      (&sm.tab.g1[0][0][0])[q] = (&c_tab.g1f[0][0][0])[q];
      (&sm.tab.gk[0][0][0])[q] = (&c_tab.gkf[0][0][0])[q];
      (&sm.tab.taylor[0][0][0])[q] = (&c_tab.taylorf[0][0][0])[q];
    }
    for (int q = tid; q < (ACAT_MAXP + 1) * ACAT_MAXN; q += NT) (&sm.tab.gh[0][0])[q] = (&c_tab.ghf[0][0])[q];
    for (int q = tid; q <= ACAT_MAXN; q += NT) sm.tab.invfact[q] = c_tab.invfactf[q];
  }
  const float *uin = static_cast<const float *>(a.u_in);
  for (int q = tid; q < S * CELLS; q += NT) {
    const int c = q / CELLS, rem = q - c * CELLS, yy = rem / TW, xx = rem - yy * TW;
    const long gx = bc2(x0 - P + xx, NXl, a.bc), gy = bc2(y0 - P + yy, NYl, a.bc);
    const long gi = ((long)c * NYl + gy) * NXl + gx;
    if (!acat_in_bounds(gx >= 0 && gx < NXl && gy >= 0 && gy < NYl, a.status)) continue;
    sm.thi[c][yy][xx] = uin[gi];
    sm.tlo[c][yy][xx] = uin[(long)S * NYl * NXl + gi];
  }
  __syncthreads();
  const float lx = sm.lx, ly = sm.ly;
  // --- order decisions: every (anchor, direction, component), all orders at once
  constexpr int NPAIR = 2 * S;
  const FiltConst FC = filt_const(a.epsf, a.rf, a.factf);
  for (int q = tid; q < NAF<P> * NAF<P> * NPAIR; q += NT) {
    const int an = q / NPAIR, pr = q - an * NPAIR;
    const int dir = pr / S, c = pr - dir * S;
    const int ax = an % NAF<P> - 1, ay = an / NAF<P> - 1;
    const bool inside = x0 + ax < NXl && y0 + ay < NYl;
    const bool skip = a.rect_2d ? (ax < 0 && ay < 0) : (dir == 0 ? ay < 0 : ax < 0);
    if (!inside || skip) continue;
    const unsigned r = reject_set32<P>(&sm.thi[c][ay + P][ax + P], &sm.tlo[c][ay + P][ax + P], dir == 0 ? 1 : TW,
                                       c == 0, FC, a.eps, a.thr, a.fact_tau, a.psi2_mod);
    if (r) atomicOr(&sm.rej[an], r << (dir * (P - 1)));
  }
  __syncthreads();
  // --- orders, block tasks, FL-CAT2 directions
  for (int an = tid; an < NAF<P> * NAF<P>; an += NT) {
    const int ax = an % NAF<P> - 1, ay = an / NAF<P> - 1;
    const long gxa = x0 + ax, gya = y0 + ay;
    const bool inside = gxa < NXl && gya < NYl;
    const bool needF = inside && ay >= 0, needG = inside && ax >= 0;
    const unsigned rej = sm.rej[an], all = (1u << (P - 1)) - 1u;
    const unsigned accx = ~rej & all, accy = ~(rej >> (P - 1)) & all;
    const int px = accx ? (32 - __clz(accx)) + 1 : 1, py = accy ? (32 - __clz(accy)) + 1 : 1;
    if (needF && a.ord_x && (ax >= 0 || gxa == -1)) a.ord_x[gya * (NXl + 1) + (gxa + 1)] = (int8_t)px;
    if (needG && a.ord_y && (ay >= 0 || gya == -1)) a.ord_y[(gya + 1) * NXl + gxa] = (int8_t)py;
    const bool bF = needF && px >= 2, bG = needG && py >= 2;
    const unsigned ua = (unsigned)an;
    if (a.rect_2d) {
      const unsigned want = (bF ? WF32 : 0u) | (bG ? WG32 : 0u);
      if (want) sm.task[atomicAdd(&sm.ntask, 1)] = ua | want | ((unsigned)px << 12) | ((unsigned)py << 15);
    } else if (bF && bG && px == py) {
      sm.task[atomicAdd(&sm.ntask, 1)] = ua | WF32 | WG32 | ((unsigned)px << 12) | ((unsigned)px << 15);
    } else {
      if (bF) sm.task[atomicAdd(&sm.ntask, 1)] = ua | WF32 | ((unsigned)px << 12) | ((unsigned)px << 15);
      if (bG) sm.task[atomicAdd(&sm.ntask, 1)] = ua | WG32 | ((unsigned)py << 12) | ((unsigned)py << 15);
    }
    const bool flF = needF && px < 2, flG = needG && py < 2;
    if (flF || flG) {
      float F1[S], G1[S];
      flcat2_2d_f32<FLUX>(&sm.thi[0][ay + P][ax + P], &sm.tlo[0][ay + P][ax + P], CELLS, TW, flF, flG, lx, ly,
                          a.advf[0], a.advf[1], a.gammaf, a.gm1f, a.limiter_form, a.lo_flux, F1, G1);
#pragma unroll
      for (int c = 0; c < S; c++) {
        if (flF) sm.Fx[ay][ax + 1][c] = F1[c];
        if (flG) sm.Gy[ay + 1][ax][c] = G1[c];
      }
    }
  }
  __syncthreads();
  block_tasks_f32<P, FLUX>(sm, a, lx, ly);
  // --- update on the compensated pair and the wave-speed epilogue (Eq. 4.9)
  float mx = 0.0f, my = 0.0f;
  bool bad = false;
  float *uo = static_cast<float *>(a.u_out);
  for (int t = tid; t < TXF<P> * TXF<P>; t += NT) {
    const int cy = t / TXF<P>, cx = t - cy * TXF<P>;
    const long gx = x0 + cx, gy = y0 + cy;
    if (gx >= NXl || gy >= NYl) continue;
    const int tx = cx + P, ty = cy + P;
    float uc[S], ucl[S], hx[S], lx_[S], hy[S], ly_[S], Bx[S], By[S], junk[S], hf[S], lf[S];
#pragma unroll
    for (int c = 0; c < S; c++) {
      uc[c] = sm.thi[c][ty][tx];
      ucl[c] = sm.tlo[c][ty][tx];
      hx[c] = sm.thi[c][ty][tx - 1] - uc[c];
      lx_[c] = sm.tlo[c][ty][tx - 1] - ucl[c];
      hy[c] = sm.thi[c][ty - 1][tx] - uc[c];
      ly_[c] = sm.tlo[c][ty - 1][tx] - ucl[c];
    }
    const typename PH::Base B = PH::base2(uc, ucl, a.advf[0], a.advf[1], a.gm1f);
    PH::dflux2_pair(B, hx, lx_, Bx, junk);  // f(u_{x-1,y}) - f(u)
    PH::dflux2_pair(B, hy, ly_, junk, By);  // g(u_{x,y-1}) - g(u)
#pragma unroll
    for (int c = 0; c < S; c++) {
      const float dx_ = __fmul_rn(lx, __fadd_rn(Bx[c], __fsub_rn(sm.Fx[cy][cx][c], sm.Fx[cy][cx + 1][c])));
      const float dy_ = __fmul_rn(ly, __fadd_rn(By[c], __fsub_rn(sm.Gy[cy][cx][c], sm.Gy[cy + 1][cx][c])));
      const float d = __fadd_rn(dx_, dy_);
      const float h = sm.thi[c][ty][tx], w = sm.tlo[c][ty][tx];
      // TwoSum(h, d), then Fast2Sum with the low part
      const float s = __fadd_rn(h, d);
      const float bp = __fsub_rn(s, h);
      const float e = __fadd_rn(__fsub_rn(h, __fsub_rn(s, bp)), __fsub_rn(d, bp));
      const float w2 = __fadd_rn(w, e);
      const float hn = __fadd_rn(s, w2);
      const float ln = __fsub_rn(w2, __fsub_rn(hn, s));
      const long gi = ((long)c * NYl + gy) * NXl + gx;
      uo[gi] = hn;
      uo[(long)S * NYl * NXl + gi] = ln;
      hf[c] = hn;
      lf[c] = ln;
    }
    const float g = a.gammaf;
    const float sxf = PH::fspeed(hf, a.advf[0], a.advf[1], g, 0);
    const float syf = PH::fspeed(hf, a.advf[0], a.advf[1], g, 1);
    if (!PH::fphysical(hf, g)) {
      double un[S], sx, sy;
#pragma unroll
      for (int c = 0; c < S; c++) un[c] = (double)hf[c] + (double)lf[c];
      bool ok;
      PH::speed2(un, a.adv[0], a.adv[1], a.gamma, sx, sy, ok);
      bad |= !ok;
    }
    mx = fmaxf(mx, sxf);
    my = fmaxf(my, syf);
  }
  const int lane = tid & 31, warp = tid >> 5;
  if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(a.status, (unsigned)ACAT_STATUS_NONPHYSICAL);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    my = fmaxf(my, __shfl_xor_sync(0xffffffffu, my, o));
  }
  if (lane == 0) {
    s_red[0][warp] = (double)mx;
    s_red[1][warp] = (double)my;
  }
  __syncthreads();
  if (tid == 0) {
    double vx = s_red[0][0], vy = s_red[1][0];
    for (int w = 1; w < NT / 32; w++) {
      vx = fmax(vx, s_red[0][w]);
      vy = fmax(vy, s_red[1][w]);
    }
    const int zs = (a.slot + 1) % 3;
    atomic_max_pos(&a.smax[zs * 2 + 0], vx);
    atomic_max_pos(&a.smax[zs * 2 + 1], vy);
  }
}

template <int P, int FLUX>
int launch2_hi_f32(const Step2DArgs &a, cudaStream_t st) {
  dim3 grid((unsigned)((a.NX + TXF<P> - 1) / TXF<P>), (unsigned)((a.NY + TXF<P> - 1) / TXF<P>));
  k_step2d_hi_f32<P, FLUX><<<grid, NT, 0, st>>>(a);
  return (int)cudaGetLastError();
}

template <int P, int FLUX>
int launch2_hi(const Step2DArgs &a, cudaStream_t st) {
  dim3 grid((unsigned)((a.NX + TXH - 1) / TXH), (unsigned)((a.NY + TXH - 1) / TXH));
  k_step2d_hi<P, FLUX><<<grid, NT, 0, st>>>(a);
  return (int)cudaGetLastError();
}

template <int FLUX, bool F32>
int launch2_p(int P, const Step2DArgs &a, cudaStream_t st) {
  if (P == 1) return launch2<1, FLUX, F32>(a, st);
  if constexpr (F32) {
    if (P == 2 && a.rect_2d) return launch2_hi_f32<2, FLUX>(a, st);  // blocks S_{2,1}, S_{1,2}
    if (P == 2) return launch2<2, FLUX, F32>(a, st);
    if (P == 3) return launch2_hi_f32<3, FLUX>(a, st);
    if (P == 4) return launch2_hi_f32<4, FLUX>(a, st);
  } else {
    if (P == 2 && a.rect_2d) return launch2_hi<2, FLUX>(a, st);  // blocks S_{2,1}, S_{1,2}
    if (P == 2) return launch2<2, FLUX, F32>(a, st);
    if (P == 3) return launch2_hi<3, FLUX>(a, st);
    if (P == 4) return launch2_hi<4, FLUX>(a, st);
  }
  return (int)cudaErrorInvalidValue;
}

}  // namespace

int acat_launch_step2d(int P, int flux, int prec, const Step2DArgs &a, void *stream) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const bool f32 = prec == ACAT_PREC_F32;
  if (flux == ACAT_FLUX_EULER2D)
    return f32 ? launch2_p<ACAT_FLUX_EULER2D, true>(P, a, st) : launch2_p<ACAT_FLUX_EULER2D, false>(P, a, st);
  if (flux == ACAT_FLUX_LINEAR)
    return f32 ? launch2_p<ACAT_FLUX_LINEAR, true>(P, a, st) : launch2_p<ACAT_FLUX_LINEAR, false>(P, a, st);
  return (int)cudaErrorInvalidValue;
}

int acat_launch_smax2d(int flux, int prec, const Step2DArgs &a, void *stream) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const long NC = (long)a.NX * a.NY;
  const long blocks = (NC + NT - 1) / NT;
  const unsigned grid = (unsigned)(blocks < 2048 ? blocks : 2048);
  const bool f32 = prec == ACAT_PREC_F32;
  if (flux == ACAT_FLUX_EULER2D) {
    if (f32) k_smax2d<ACAT_FLUX_EULER2D, true><<<grid, NT, 0, st>>>(a);
    else k_smax2d<ACAT_FLUX_EULER2D, false><<<grid, NT, 0, st>>>(a);
  } else if (flux == ACAT_FLUX_LINEAR) {
    if (f32) k_smax2d<ACAT_FLUX_LINEAR, true><<<grid, NT, 0, st>>>(a);
    else k_smax2d<ACAT_FLUX_LINEAR, false><<<grid, NT, 0, st>>>(a);
  } else {
    return (int)cudaErrorInvalidValue;
  }
  return (int)cudaGetLastError();
}

int acat_upload_tables_2d(const AcatTables *T) { return (int)cudaMemcpyToSymbol(c_tab, T, sizeof *T); }
