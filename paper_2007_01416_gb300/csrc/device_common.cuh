// device_common.cuh -- device helpers shared by the 1D and 2D ACAT kernels.
// Each translation unit that includes it gets its own copy of the weight
// tables in constant memory; acat_upload_tables_current_device fills all.
#pragma once

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
// 1/x for x > 0: the hardware approximation rcp.approx.ftz.f64 (about 23
// correct bits) refined by two Newton-Raphson steps y <- y + y (1 - x y), each
// doubling the number of correct bits (error within an ulp of 1/x).
__device__ __forceinline__ double recip(double x) {
  double y;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  double e = fma(-x, y, 1.0);
  y = fma(y, e, y);
  e = fma(-x, y, 1.0);
  return fma(y, e, y);
}
__device__ __forceinline__ float recip(float x) { return __frcp_rn(x); }

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

__device__ __forceinline__ long bc_index(long g, long N, int bc) {
  if (bc == ACAT_BC_PERIODIC) {
    long r = g % N;
    return r < 0 ? r + N : r;
  }
  return g < 0 ? 0 : (g >= N ? N - 1 : g);
}

// ---------------------------------------------------------------------------
// Indicators and limiter: explicit round-to-nearest FP64 operations, no FMA
// contraction, in the order of Eqs. 3.6-3.12.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double psi_p_comp(const double *q, int st, int p, double eps, double fact) {
  double IL = 0.0, IR = 0.0;
  for (int j = -p + 1; j <= -1; j++) {
    const double d = __dsub_rn(q[(1 + j) * st], q[j * st]);
    IL = __dadd_rn(IL, __dmul_rn(d, d));
  }
  IL = __dadd_rn(IL, eps);
  for (int j = 1; j <= p - 1; j++) {
    const double d = __dsub_rn(q[(1 + j) * st], q[j * st]);
    IR = __dadd_rn(IR, __dmul_rn(d, d));
  }
  IR = __dadd_rn(IR, eps);
  const double I = __ddiv_rn(__dmul_rn(IL, IR), __dadd_rn(IL, IR));
  double S = 0.0;
  for (int j = -p + 1; j <= p; j++) S = __dadd_rn(S, __dmul_rn(c_tab.gd[p][j + p - 1], q[j * st]));
  const double D = __dmul_rn(fact, S);
  const double tau = __dmul_rn(D, D);
  return __ddiv_rn(I, __dadd_rn(I, tau));
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

// psi^1 (Eqs. 3.5-3.7, superbee) at the interface between q[0] (cell i) and
// q[st]: components `cs` apart, cells `st` apart. Scalar laws (S == 1; kind
// 0: linear transport with speed `adv`, kind 1: Burgers) use the Roe-speed
// side unless limiter_form is 1; systems use min(psi(r+), psi(r-)) per
// component and the minimum over components.
template <int S>
__device__ __forceinline__ double psi1_line(const double *q, int cs, int st, int kind,
                                            int limiter_form, double adv) {
  if (S == 1 && limiter_form == 0) {
    const double um = q[-st], u0 = q[0], u1 = q[st], u2 = q[2 * st];
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
    const double *p = q + c * cs;
    const double loc = __dsub_rn(p[st], p[0]);
    const double pm = superbee(lim_ratio(__dsub_rn(p[0], p[-st]), loc));
    const double pp = superbee(lim_ratio(__dsub_rn(p[2 * st], p[st]), loc));
    const double v = pp < pm ? pp : pm;
    if (v < best) best = v;
  }
  return best;
}

__device__ __forceinline__ void atomic_max_pos(unsigned long long *addr, double v) {
  // non-negative doubles (and +inf) order like their bit patterns
  atomicMax(addr, (unsigned long long)__double_as_longlong(v));
}

}  // namespace
