// device_common.cuh -- device helpers shared by the 1D and 2D ACAT kernels.
// Each translation unit that includes it gets its own copy of the weight
// tables in constant memory; acat_upload_tables_current_device fills all.
#pragma once
#include <utility>

#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/acat.h"
#include "acat_internal.h"

static __constant__ AcatTables c_tab;

namespace {

constexpr int NT = 256;  // threads per CTA

// ---------------------------------------------------------------------------
// Arithmetic helpers
// ---------------------------------------------------------------------------
// 1/x for normal x: the hardware approximation y0 = rcp.approx.ftz.f64(x)
// refined by the truncated geometric series of 1/x = y0 / (1 - e),
// e = 1 - x y0:  1/x ~ y0 (1 + e + e^2), three FMAs. Measured on sm_103a
// over 2^24 inputs spanning 2^-200..2^200: |e| <= 2^-19.9, so the neglected
// e^3 term is below 2^-59 and the result is within one ulp of the correctly
// rounded reciprocal (equal to it for 99.97 % of the inputs).
__device__ __forceinline__ double recip(double x) {
  double y;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  const double e = fma(-x, y, 1.0);
  return fma(y, fma(e, e, e), y);
}
// float 1/x: the hardware approximation rcp.approx.ftz.f32 (within about an
// ulp; inputs are densities, far from the subnormal range it flushes). The
// FP32 path applies it to O(1) quantities whose rounding enters the flux
// increments only relatively.
__device__ __forceinline__ float recip(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Packed pairs of floats (sm_100+ f32x2 instructions: one issue slot for two
// lanes' worth of add, multiply or fused multiply-add, each rounded to
// nearest exactly as the scalar instruction).
__device__ __forceinline__ unsigned long long f2bits(float2 a) {
  return (unsigned long long)__float_as_uint(a.x) | ((unsigned long long)__float_as_uint(a.y) << 32);
}
__device__ __forceinline__ float2 f2from(unsigned long long b) {
  return make_float2(__uint_as_float((unsigned)b), __uint_as_float((unsigned)(b >> 32)));
}
__device__ __forceinline__ float2 f2add(float2 a, float2 b) {
  unsigned long long d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(f2bits(a)), "l"(f2bits(b)));
  return f2from(d);
}
__device__ __forceinline__ float2 f2mul(float2 a, float2 b) {
  unsigned long long d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(f2bits(a)), "l"(f2bits(b)));
  return f2from(d);
}
__device__ __forceinline__ float2 f2fma(float2 a, float2 b, float2 c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(f2bits(a)), "l"(f2bits(b)), "l"(f2bits(c)));
  return f2from(d);
}
__device__ __forceinline__ float2 f2dup(float a) { return make_float2(a, a); }

// operations rounded as written, in the arithmetic type of their arguments
// (no contraction into FMAs: the same bits in every kernel that inlines them)
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float div_rn(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ double div_rn(double a, double b) { return __ddiv_rn(a, b); }
__device__ __forceinline__ float sqrt_rn(float a) { return __fsqrt_rn(a); }
__device__ __forceinline__ double sqrt_rn(double a) { return __dsqrt_rn(a); }

// fused multiply-add in the arithmetic type of its arguments
__device__ __forceinline__ double fmar(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fmar(float a, float b, float c) { return fmaf(a, b, c); }

template <typename R>
struct Tab;
template <>
struct Tab<double> {
  __device__ static double g1(int p, int j, int r) { return c_tab.g1[p][j][r]; }
  __device__ static double gk(int p, int k, int r) { return c_tab.gk[p][k][r]; }
  __device__ static double gh(int p, int j) { return c_tab.gh[p][j]; }
  __device__ static double taylor(int p, int r, int l) { return c_tab.taylor[p][r][l]; }
  __device__ static double invfact(int k) { return c_tab.invfact[k]; }
};
template <>
struct Tab<float> {
  __device__ static float g1(int p, int j, int r) { return c_tab.g1f[p][j][r]; }
  __device__ static float gk(int p, int k, int r) { return c_tab.gkf[p][k][r]; }
  __device__ static float gh(int p, int j) { return c_tab.ghf[p][j]; }
  __device__ static float taylor(int p, int r, int l) { return c_tab.taylorf[p][r][l]; }
  __device__ static float invfact(int k) { return c_tab.invfactf[k]; }
};

// Index checks of the bounds-checked build (compiled with ACAT_BOUNDS_CHECK):
// acat_in_bounds(cond, status) records a failed check in the status word
// (ACAT_STATUS_BOUNDS) and returns false, and the caller skips the access.
// Without the flag it returns true and the check compiles away.
__device__ __forceinline__ bool acat_in_bounds(bool cond, unsigned *status) {
#ifdef ACAT_BOUNDS_CHECK
  if (!cond && status) atomicOr(status, (unsigned)ACAT_STATUS_BOUNDS);
  return cond;
#else
  (void)cond;
  (void)status;
  return true;
#endif
}

// A tile index checked by the bounds-checked build: i itself when
// 0 <= i < n, else (recorded in the status word) 0, a safe index.
__device__ __forceinline__ int acat_tile_index(int i, int n, unsigned *status) {
  return acat_in_bounds(i >= 0 && i < n, status) ? i : 0;
}

// Programmatic dependent launch of the 1D step kernels. They are launched
// with programmatic stream serialization, so that the next step's launch
// overlaps the end of the current step. acat_pdl_wait() is the first
// statement of such a kernel: it waits until the previous kernel of the
// stream has completed and its memory is visible (no memory access of the
// step comes before). acat_pdl_release() is its last: the next launch begins
// once every CTA of this grid has passed it, when nearly every SM is free, so
// the next grid's CTAs spread over the SMs as a plain launch spreads them.
// (Released at the start of the kernel, the next grid's CTAs took the first
// SMs to free up, and steps of one uneven wave lost their balance.) In a
// kernel launched without the attribute both instructions return at once.
__device__ __forceinline__ void acat_pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void acat_pdl_release() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Host side: launch a kernel of that form with programmatic stream
// serialization (returns 0 or a cudaError_t value).
template <typename... Params, typename... Args>
int acat_launch_dep(void (*kernel)(Params...), unsigned grid, unsigned block, cudaStream_t st, Args &&...args) {
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return (int)cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// Node-exchange slots of the FP32 1D recursion. A lane stores its F^(k-2) in
// a 16-byte slot that the other lanes of its group read back by broadcast. In
// tiles of P >= 3 the slots of the group whose first lane is b start at
// xslot(b) = b + (b >> 3): the groups of a warp, 6 or 8 lanes apart, then
// start in distinct 16-byte bank quads, and each broadcast load is one
// shared-memory wavefront instead of two (P = 3) or four (P = 4). At P = 2
// (4 lanes apart) the same padding also removes four-way conflicts but
// measured slower, and the slots start at b. A warp holds two sets of XSET.
constexpr int XSET = 36;
__device__ __forceinline__ int xslot(int b) { return b + (b >> 3); }

__device__ __forceinline__ long bc_index(long g, long N, int bc) {
  if (bc == ACAT_BC_PERIODIC) {
    if (g >= 0 && g < N) return g;
    long r = g % N;
    return r < 0 ? r + N : r;
  }
  return g < 0 ? 0 : (g >= N ? N - 1 : g);
}

// ---------------------------------------------------------------------------
// Indicators and limiter: explicit round-to-nearest FP64 operations, no FMA
// contraction, in the order of Eqs. 3.6-3.12.
// ---------------------------------------------------------------------------
// q(j) returns the FP64 value of cell i + j.
template <class Get>
__device__ __forceinline__ double psi_p_comp_g(Get q, int p, double eps, double fact) {
  double IL = 0.0, IR = 0.0;
  for (int j = -p + 1; j <= -1; j++) {
    const double d = __dsub_rn(q(1 + j), q(j));
    IL = __dadd_rn(IL, __dmul_rn(d, d));
  }
  IL = __dadd_rn(IL, eps);
  for (int j = 1; j <= p - 1; j++) {
    const double d = __dsub_rn(q(1 + j), q(j));
    IR = __dadd_rn(IR, __dmul_rn(d, d));
  }
  IR = __dadd_rn(IR, eps);
  const double I = __ddiv_rn(__dmul_rn(IL, IR), __dadd_rn(IL, IR));
  double S = 0.0;
  for (int j = -p + 1; j <= p; j++) S = __dadd_rn(S, __dmul_rn(c_tab.gd[p][j + p - 1], q(j)));
  const double D = __dmul_rn(fact, S);
  const double tau = __dmul_rn(D, D);
  return __ddiv_rn(I, __dadd_rn(I, tau));
}

// Modified indicator psi~^2 (Sec. 3.2): the two splits of the three
// differences of S_2 into lateral weights that keep the central one,
// I^1 = (d_-^2 + eps, d_0^2 + d_+^2 + eps), I^2 = (d_-^2 + d_0^2 + eps, d_+^2 + eps),
// and the larger of I^j / (I^j + tau_2), in the order of the definition.
template <class Get>
__device__ __forceinline__ double psi2m_comp_g(Get q, double eps, double fact) {
  const double dm = __dsub_rn(q(0), q(-1)), d0 = __dsub_rn(q(1), q(0)), dp = __dsub_rn(q(2), q(1));
  const double sm = __dmul_rn(dm, dm), s0 = __dmul_rn(d0, d0), sp = __dmul_rn(dp, dp);
  const double I1L = __dadd_rn(sm, eps), I1R = __dadd_rn(__dadd_rn(s0, sp), eps);
  const double I2L = __dadd_rn(__dadd_rn(sm, s0), eps), I2R = __dadd_rn(sp, eps);
  const double I1 = __ddiv_rn(__dmul_rn(I1L, I1R), __dadd_rn(I1L, I1R));
  const double I2 = __ddiv_rn(__dmul_rn(I2L, I2R), __dadd_rn(I2L, I2R));
  double S = 0.0;
  for (int j = -1; j <= 2; j++) S = __dadd_rn(S, __dmul_rn(c_tab.gd[2][j + 1], q(j)));
  const double D = __dmul_rn(fact, S);
  const double tau = __dmul_rn(D, D);
  const double a = __ddiv_rn(I1, __dadd_rn(I1, tau)), b = __ddiv_rn(I2, __dadd_rn(I2, tau));
  return a > b ? a : b;
}

__device__ __forceinline__ double lim_ratio(double upw, double loc) {
  if (loc == 0.0) {
    if (upw == 0.0) return 1.0;
    return upw > 0.0 ? __longlong_as_double(0x7ff0000000000000LL)
                     : __longlong_as_double((long long)0xfff0000000000000ULL);
  }
  return __ddiv_rn(upw, loc);
}

__device__ __forceinline__ double superbee(double r) {
  const double r2 = __dmul_rn(2.0, r);
  const double a = r2 < 1.0 ? r2 : 1.0;
  const double b = r < 2.0 ? r : 2.0;
  const double m = a > b ? a : b;
  return m > 0.0 ? m : 0.0;
}

// ---------------------------------------------------------------------------
// Filtered order decision. psi^p >= thr (thr < 1) holds exactly when
// I (1 - thr) >= thr tau, i.e. I >= r tau with r = thr / (1 - thr). The test is
// first evaluated in float from the first differences d_k = u_{k+1} - u_k,
// k = -p+1..p-1, each with an absolute error bound e_k:
//   I_L, I_R, I from the d_k (relative error below 4e-6 while the errors
//   the d_k carry into I_L and I_R stay below 8e-7 of them; undecided
//   otherwise),
//   Delta^{2p-1} u = Delta^{2p-2} d by repeated differencing, its bound
//   propagated as e' = e_{k+1} + e_k + 2^-24 |t'|,
// and the decision is taken only when the bounds leave no doubt (with a
// further relative margin of 1e-5, far above the rounding of a literal FP64
// evaluation). Otherwise it is undecided and the caller evaluates psi^p
// literally in FP64. The same decision as the literal FP64 evaluation
// results in every case.
// ---------------------------------------------------------------------------
// The filtered decision for psi~^2 (differences d_0..d_2 of S_2 with bounds
// e): accept when either split's I certainly reaches r tau, reject when
// neither can, else undecided; the bounds are those of psi_filter_all.
__device__ __forceinline__ int psi2m_filter(const float *d, const float *e, float eps, float r, float fact) {
  const float sm = d[0] * d[0], s0 = d[1] * d[1], sp = d[2] * d[2];
  const float I1L = sm + eps, I1R = (s0 + sp) + eps, I2L = (sm + s0) + eps, I2R = sp + eps;
  const float mn = fminf(fminf(I1L, I1R), fminf(I2L, I2R)), mx = fmaxf(fmaxf(I1L, I1R), fmaxf(I2L, I2R));
  if (!(mn > 1e-30f) || !(mx < 1e30f)) return -1;
  const float I1 = I1L * I1R / (I1L + I1R), I2 = I2L * I2R / (I2L + I2R);
  float t[3], b[3];
#pragma unroll
  for (int k = 0; k < 3; k++) {
    t[k] = d[k];
    b[k] = e[k];
  }
#pragma unroll
  for (int lev = 1; lev < 3; lev++)
#pragma unroll
    for (int k = 0; k < 3 - lev; k++) {
      t[k] = t[k + 1] - t[k];
      b[k] = (b[k + 1] + b[k]) + 5.97e-8f * fabsf(t[k]) + 1e-44f;
    }
  const float S = fabsf(t[0]), eS = 1.01f * b[0];
  const float Dhi = (S + eS) * fact * 1.0000005f;
  const float Dlo = fmaxf(S - eS, 0.0f) * fact * 0.9999995f;
  const float thi = r * (Dhi * Dhi) * 1.00001f, tlo = r * (Dlo * Dlo) * 0.99999f;
  if (I1 * (1.0f - 4e-6f) > thi || I2 * (1.0f - 4e-6f) > thi) return 1;
  if (I1 * (1.0f + 4e-6f) < tlo && I2 * (1.0f + 4e-6f) < tlo) return 0;
  return -1;
}

// Float constants of the filter.
struct FiltConst {
  float eps, r;
  float fact[ACAT_MAXP + 1];
};
// From the float constants computed once on the host (no FP64 work per thread).
__device__ __forceinline__ FiltConst filt_const(float eps, float r, const float *fact) {
  FiltConst f;
  f.eps = eps;
  f.r = r;
#pragma unroll
  for (int q = 0; q <= ACAT_MAXP; q++) f.fact[q] = fact[q];
  return f;
}

// The filtered decision for every order p = 2..PM of one component at once.
// The stencils S_2 c S_3 c ... c S_PM are nested around the same interface,
// so their first differences are windows of those of S_PM:
//   d_k = u_{k-PM+2} - u_{k-PM+1}, k = 0..2PM-2 (bounds e_k),
// S_p taking d_{PM-p} .. d_{PM+p-2}. One differencing triangle over all d
// holds Delta^{2p-2} d of the window of S_p at level 2p-2, entry PM-p: each
// entry depends on its own window only, so it is the value (and bound) that
// differencing that window alone would give. I_L and I_R grow outwards by
// one square per order. Bit p-2 of *acc: accepted, of *und: undecided.
template <int PM>
__device__ __forceinline__ void psi_filter_all(const float *d, const float *e, float eps, float r,
                                               const float *fact, unsigned *acc, unsigned *und) {
  constexpr int n = 2 * PM - 1;
  float t[n], b[n], S[PM + 1], eS[PM + 1];
#pragma unroll
  for (int k = 0; k < n; k++) {
    t[k] = d[k];
    b[k] = e[k];
  }
#pragma unroll
  for (int lev = 1; lev < n; lev++) {
#pragma unroll
    for (int k = 0; k < n - lev; k++) {
      t[k] = t[k + 1] - t[k];
      b[k] = (b[k + 1] + b[k]) + 5.97e-8f * fabsf(t[k]) + 1e-44f;
    }
    if (lev % 2 == 0) {
      const int p = lev / 2 + 1;
      S[p] = fabsf(t[PM - p]);
      eS[p] = 1.01f * b[PM - p];
    }
  }
  unsigned a = 0, u = 0;
  float il = 0.0f, ir = 0.0f, el = 0.0f, er = 0.0f;
#pragma unroll
  for (int p = 2; p <= PM; p++) {
    const unsigned bit = 1u << (p - 2);
    const float dl = d[PM - p], dr = d[PM + p - 2], bl = e[PM - p], br = e[PM + p - 2];
    il = fmaf(dl, dl, il);
    ir = fmaf(dr, dr, ir);
    // bounds of the error that the differences' errors carry into the sums
    el = fmaf(bl, 2.0f * fabsf(dl) + bl, el);
    er = fmaf(br, 2.0f * fabsf(dr) + br, er);
    const float IL = il + eps, IR = ir + eps;
    if (!(IL > 1e-30f && IR > 1e-30f) || !(IL < 1e30f && IR < 1e30f)) {
      u |= bit;
      continue;
    }
    // the relative error of I stays below 4e-6 only while these carried
    // errors are below 8e-7 of I_L and I_R (differences much smaller than
    // the rounding of the state, with a small eps): otherwise undecided
    if (!(el <= 8e-7f * IL && er <= 8e-7f * IR)) {
      u |= bit;
      continue;
    }
    const float I = IL * IR / (IL + IR);
    const float Dhi = (S[p] + eS[p]) * fact[p] * 1.0000005f;
    const float Dlo = fmaxf(S[p] - eS[p], 0.0f) * fact[p] * 0.9999995f;
    if (I * (1.0f - 4e-6f) > r * (Dhi * Dhi) * 1.00001f) a |= bit;
    else if (!(I * (1.0f + 4e-6f) < r * (Dlo * Dlo) * 0.99999f)) u |= bit;
  }
  *acc = a;
  *und = u;
}

// The rejected orders p = 2..PM (bit p - 2) of one component, from the
// filtered decisions of psi_filter_all (psi2m_filter for p = 2 when
// psi2_mod) and, where a decision is undecided, the literal FP64 evaluation
// of psi^p on q(j) (the FP64 value of cell i + j). `first`: the first
// component (a NaN there rejects, a NaN in a later component is ignored, as
// in a minimum taken from the first component). d, e: the differences of
// S_PM and their bounds, as for psi_filter_all.
template <int PM, class Get>
__device__ __forceinline__ unsigned reject_set(const float *d, const float *e, Get q, bool first,
                                               const FiltConst &F, double eps, double thr, const double *fact,
                                               int psi2_mod) {
  unsigned acc, und;
  psi_filter_all<PM>(d, e, F.eps, F.r, F.fact, &acc, &und);
  unsigned rej = 0;
#pragma unroll
  for (int p = 2; p <= PM; p++) {
    const unsigned bit = 1u << (p - 2);
    const bool mod = p == 2 && psi2_mod;
    const int dec = mod ? psi2m_filter(d + PM - 2, e + PM - 2, F.eps, F.r, F.fact[2])
                        : ((und & bit) ? -1 : ((acc & bit) ? 1 : 0));
    bool ok;
    if (dec >= 0) {
      ok = dec == 1;
    } else {
      const double v = mod ? psi2m_comp_g(q, eps, fact[2]) : psi_p_comp_g(q, p, eps, fact[p]);
      ok = first ? (v >= thr) : !(v < thr);
    }
    if (!ok) rej |= bit;
  }
  return rej;
}

// reject_set of one component of an FP64 state, values at q[j*st],
// j = -PM+1..PM.
template <int PM>
__device__ __forceinline__ unsigned reject_set64(const double *q, int st, bool first, const FiltConst &F,
                                                 double eps, double thr, const double *fact, int psi2_mod) {
  float d[2 * PM - 1], e[2 * PM - 1];
#pragma unroll
  for (int k = 0; k < 2 * PM - 1; k++) {
    const int j = k - PM + 1;
    d[k] = (float)__dsub_rn(q[(j + 1) * st], q[j * st]);
    e[k] = 6.0e-8f * fabsf(d[k]) + 1e-44f;
  }
  return reject_set<PM>(d, e, [=](int j) { return q[j * st]; }, first, F, eps, thr, fact, psi2_mod);
}

// The same for a compensated float state hi + lo (the literal fallback reads
// the exact value hi + lo).
template <int PM>
__device__ __forceinline__ unsigned reject_set32(const float *hi, const float *lo, int st, bool first,
                                                 const FiltConst &F, double eps, double thr, const double *fact,
                                                 int psi2_mod) {
  float d[2 * PM - 1], e[2 * PM - 1];
#pragma unroll
  for (int k = 0; k < 2 * PM - 1; k++) {
    const int j = k - PM + 1;
    const float h1 = hi[(j + 1) * st], h0 = hi[j * st];
    d[k] = (h1 - h0) + (lo[(j + 1) * st] - lo[j * st]);
    e[k] = 1.2e-7f * fabsf(d[k]) + 1.5e-14f * (fabsf(h1) + fabsf(h0)) + 1e-44f;
  }
  return reject_set<PM>(d, e, [=](int j) { return (double)hi[j * st] + (double)lo[j * st]; }, first, F, eps, thr,
                        fact, psi2_mod);
}

// psi^1 (Eqs. 3.5-3.7, superbee) at the interface between q[0] (cell i) and
// q[st]: components `cs` apart, cells `st` apart. Scalar laws (S == 1; kind
// 0: linear transport with speed `adv`, kind 1: Burgers) use the Roe-speed
// side unless limiter_form is 1; systems use min(psi(r+), psi(r-)) per
// component and the minimum over components.
template <int S, class Get>
__device__ __forceinline__ double psi1_g(Get q, int kind, int limiter_form, double adv) {
  if (S == 1 && limiter_form == 0) {
    const double um = q(0, -1), u0 = q(0, 0), u1 = q(0, 1), u2 = q(0, 2);
    double a;
    if (u0 != u1) {
      double f0, f1;
      if (kind == 0) {
        f0 = __dmul_rn(adv, u0);
        f1 = __dmul_rn(adv, u1);
      } else {
        f0 = __dmul_rn(__dmul_rn(0.5, u0), u0);
        f1 = __dmul_rn(__dmul_rn(0.5, u1), u1);
      }
      a = __ddiv_rn(__dsub_rn(f1, f0), __dsub_rn(u1, u0));
    } else {
      a = (kind == 0) ? adv : u0;
    }
    const double upw = a > 0.0 ? __dsub_rn(u0, um) : __dsub_rn(u2, u1);
    return superbee(lim_ratio(upw, __dsub_rn(u1, u0)));
  }
  double best = 2.0;
#pragma unroll
  for (int c = 0; c < S; c++) {
    const double v0 = q(c, 0), v1 = q(c, 1);
    const double loc = __dsub_rn(v1, v0);
    const double pm = superbee(lim_ratio(__dsub_rn(v0, q(c, -1)), loc));
    const double pp = superbee(lim_ratio(__dsub_rn(q(c, 2), v1), loc));
    const double v = pp < pm ? pp : pm;
    if (v < best) best = v;
  }
  return best;
}

template <int S>
__device__ __forceinline__ double psi1_line(const double *q, int cs, int st, int kind,
                                            int limiter_form, double adv) {
  return psi1_g<S>([=](int c, int k) { return q[c * cs + k * st]; }, kind, limiter_form, adv);
}

// psi1_g evaluated by the L lanes of an interface group (lane l of the
// group, gmask its lanes; all of them must call it): for systems the
// (component, side) ratios are spread over the lanes and the minimum is
// reduced across the group, which gives the serial minimum's value for
// finite data (the candidates lie in [0, 2] and ties are equal values).
// Every lane returns the limiter.
template <int S, int L, class Get>
__device__ __forceinline__ double psi1_group(Get q, int kind, int limiter_form, double adv, int l,
                                             unsigned gmask) {
  if (S == 1 && limiter_form == 0) return psi1_g<S>(q, kind, limiter_form, adv);
  double best = 2.0;
  for (int k = l; k < 2 * S; k += L) {
    const int c = k >> 1;
    const double v0 = q(c, 0), v1 = q(c, 1);
    const double loc = __dsub_rn(v1, v0);
    const double upw = (k & 1) ? __dsub_rn(q(c, 2), v1) : __dsub_rn(v0, q(c, -1));
    const double v = superbee(lim_ratio(upw, loc));
    if (v < best) best = v;
  }
  // group minimum over the lanes that hold candidates (L need not be a power of two)
  const int base = __ffs(gmask) - 1;
  double m = best;
#pragma unroll
  for (int r = 0; r < (L < 2 * S ? L : 2 * S); r++) {
    const double w = __shfl_sync(gmask, best, base + r);
    if (w < m) m = w;
  }
  return m;
}

// ---------------------------------------------------------------------------
// psi^1 of systems on a compensated float state, in float-float arithmetic
// (an unevaluated sum hi + lo of two floats: Knuth's TwoSum and Dekker's
// Fast2Sum renormalisation, division by one correction of the quotient). The
// jumps of hi + lo are formed to about 2^-44 relative, the ratio r is rounded
// to float once, so psi^1 = superbee(r) carries only the rounding of a float
// result (the FP32 path rounds the limiter to float in any case).
// ---------------------------------------------------------------------------
struct FF {
  float h, l;
};

// (h1 + l1) - (h0 + l0)
__device__ __forceinline__ FF ff_jump(float h0, float l0, float h1, float l1) {
  const float s = __fsub_rn(h1, h0);
  const float bb = __fsub_rn(s, h1);
  const float e = __fadd_rn(__fsub_rn(h1, __fsub_rn(s, bb)), __fsub_rn(-h0, bb));
  const float t = __fadd_rn(e, __fsub_rn(l1, l0));
  const float hi = __fadd_rn(s, t);
  return FF{hi, __fsub_rn(t, __fsub_rn(hi, s))};
}

// the limiter ratio u / d rounded to float, with the conventions of lim_ratio
// for d == 0
__device__ __forceinline__ float ff_ratio(FF u, FF d) {
  if (d.h == 0.0f) {
    if (u.h == 0.0f) return 1.0f;
    return u.h > 0.0f ? __int_as_float(0x7f800000) : __int_as_float((int)0xff800000u);
  }
  const float q = __fdiv_rn(u.h, d.h);
  const float r = fmaf(-q, d.h, u.h);             // u.h - q d.h, exact
  const float rem = fmaf(-q, d.l, __fadd_rn(r, u.l));
  return __fadd_rn(q, __fdiv_rn(rem, d.h));
}

__device__ __forceinline__ float superbee_f(float r) {
  const float r2 = 2.0f * r;
  const float a = r2 < 1.0f ? r2 : 1.0f;
  const float b = r < 2.0f ? r : 2.0f;
  const float m = a > b ? a : b;
  return m > 0.0f ? m : 0.0f;
}

// psi^1 of a system interface on the compensated state (min form, Eq. 3.7),
// the (component, side) ratios spread over the L lanes of the group (gmask;
// all lanes call it); every lane returns it.
template <int S, int L>
__device__ __forceinline__ float psi1_group_ff(const float *hi, const float *lo, int cs, int st, int l,
                                               unsigned gmask) {
  float best = 2.0f;
  for (int k = l; k < 2 * S; k += L) {
    const int c = k >> 1;
    const float *h = hi + c * cs, *w = lo + c * cs;
    const FF loc = ff_jump(h[0], w[0], h[st], w[st]);
    const FF upw = (k & 1) ? ff_jump(h[st], w[st], h[2 * st], w[2 * st]) : ff_jump(h[-st], w[-st], h[0], w[0]);
    const float v = superbee_f(ff_ratio(upw, loc));
    if (v < best) best = v;
  }
  const int base = __ffs(gmask) - 1;
  float m = best;
#pragma unroll
  for (int r = 0; r < (L < 2 * S ? L : 2 * S); r++) {
    const float w = __shfl_sync(gmask, best, base + r);
    if (w < m) m = w;
  }
  return m;
}

// psi^1 along a line of the compensated state by one lane, float-float
// ratios: systems (and the min form) take the minimum over (component, side);
// linear transport with the Roe-speed form takes the upwind side of the
// constant speed adv (r- for adv > 0, else r+).
template <int S>
__device__ __forceinline__ float psi1_line_ff(const float *hi, const float *lo, int cs, int st, bool roe_linear,
                                              float adv) {
  float best = 2.0f;
#pragma unroll
  for (int k = 0; k < 2 * S; k++) {
    const int c = k >> 1;
    if (roe_linear && ((k & 1) == (adv > 0.0f ? 1 : 0))) continue;
    const float *h = hi + c * cs, *w = lo + c * cs;
    const FF loc = ff_jump(h[0], w[0], h[st], w[st]);
    const FF upw = (k & 1) ? ff_jump(h[st], w[st], h[2 * st], w[2 * st]) : ff_jump(h[-st], w[-st], h[0], w[0]);
    const float v = superbee_f(ff_ratio(upw, loc));
    if (roe_linear) return v;
    if (v < best) best = v;
  }
  return best;
}

template <int S>
__device__ __forceinline__ double psi1_pair(const float *hi, const float *lo, int cs, int st, int kind,
                                            int limiter_form, double adv) {
  return psi1_g<S>(
      [=](int c, int k) { return (double)hi[c * cs + k * st] + (double)lo[c * cs + k * st]; }, kind,
      limiter_form, adv);
}

__device__ __forceinline__ void atomic_max_pos(unsigned long long *addr, double v) {
  // non-negative doubles (and +inf) order like their bit patterns
  atomicMax(addr, (unsigned long long)__double_as_longlong(v));
}

}  // namespace
