// phys1d.cuh -- 1D physics, tiling and order selection shared by the 1D step
// and adjoint kernels.
#pragma once

#include "device_common.cuh"

namespace {

// ---------------------------------------------------------------------------
// Physics
// ---------------------------------------------------------------------------
template <int FLUX>
struct Phys;

template <>
struct Phys<ACAT_FLUX_LINEAR> {
  static constexpr int S = 1;
  template <typename R>
  __device__ static __forceinline__ void flux(const R *u, R *f, R a, R /*gm1*/) { f[0] = a * u[0]; }
  __device__ static __forceinline__ double speed(const double *u, double a, double, bool &ok) {
    ok = isfinite(u[0]);
    return fabs(a);
  }
  template <typename R>
  __device__ static __forceinline__ void eig(const R *, R a, R, R &lmin, R &lmax) { lmin = lmax = a; }
};

template <>
struct Phys<ACAT_FLUX_BURGERS> {
  static constexpr int S = 1;
  template <typename R>
  __device__ static __forceinline__ void flux(const R *u, R *f, R, R) { f[0] = R(0.5) * u[0] * u[0]; }
  __device__ static __forceinline__ double speed(const double *u, double, double, bool &ok) {
    ok = isfinite(u[0]);
    return fabs(u[0]);
  }
  template <typename R>
  __device__ static __forceinline__ void eig(const R *u, R, R, R &lmin, R &lmax) { lmin = lmax = u[0]; }
};

template <>
struct Phys<ACAT_FLUX_EULER1D> {
  static constexpr int S = 3;
  template <typename R>
  __device__ static __forceinline__ void flux(const R *u, R *f, R, R gm1) {
    const R ri = recip(u[0]);
    const R v = u[1] * ri;
    const R p = gm1 * (u[2] - R(0.5) * u[1] * v);
    f[0] = u[1];
    f[1] = u[1] * v + p;
    f[2] = v * (u[2] + p);
  }
  // |v| + c with c = sqrt(gamma p / rho), every operation rounded as written
  // (no contraction), so that the CFL dt is reproducible bit for bit
  __device__ static __forceinline__ double speed(const double *u, double, double gamma, bool &ok) {
    const double v = __ddiv_rn(u[1], u[0]);
    const double ke = __dmul_rn(__dmul_rn(__dmul_rn(0.5, u[0]), v), v);
    const double p = __dmul_rn(__dsub_rn(gamma, 1.0), __dsub_rn(u[2], ke));
    ok = (u[0] > 0.0) && (p > 0.0) && isfinite(u[0]) && isfinite(u[1]) && isfinite(u[2]);
    return __dadd_rn(fabs(v), __dsqrt_rn(__ddiv_rn(__dmul_rn(gamma, p), u[0])));
  }
  // smallest and largest eigenvalue v -/+ c (HLL wave-speed bounds)
  template <typename R>
  __device__ static __forceinline__ void eig(const R *u, R, R gamma, R &lmin, R &lmax) {
    const R v = div_rn(u[1], u[0]);
    const R p = mul_rn(sub_rn(gamma, R(1)), sub_rn(u[2], mul_rn(mul_rn(R(0.5), u[1]), v)));
    const R c = sqrt_rn(div_rn(mul_rn(gamma, p), u[0]));
    lmin = sub_rn(v, c);
    lmax = add_rn(v, c);
  }
};

// F^lo of Eq. 3.4 between the states u0 | u1 with fluxes f0, f1 (ACAT_LO_*):
// Rusanov with the larger of the spectral radii s0, s1; global LF with
// alpha = 1 / lambda (= dx / dt); HLL with the bounds min(n0, n1), max(x0, x1)
// of the states' eigenvalues.
template <int S, typename R>
__device__ __forceinline__ void flux_lo(int lo_flux, const R *u0, const R *u1, const R *f0, const R *f1, R s0,
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

// psi^1 of a 1D interface (cells consecutive in the tile).
template <int FLUX>
__device__ __forceinline__ double psi1(const double *q, int cs, int limiter_form, double adv) {
  return psi1_line<Phys<FLUX>::S>(q, cs, 1, FLUX == ACAT_FLUX_LINEAR ? 0 : 1, limiter_form, adv);
}

// Interface tiling of a CTA of NW warps: groups of L = 2P x LPN lanes (LPN
// lanes per stencil node), one interface per group and round (R rounds); a
// fused step tile updates T = NI - 1 cells, a flux-only tile computes NI
// interfaces. TW cells are staged (GH ghosts each side).
template <int P, int NW = NT / 32, int LPN = 1, int R = 1>
struct Tiling {
  static constexpr int L = 2 * P * LPN;       // lanes per interface
  static constexpr int GPW = 32 / L;          // interface groups per warp
  static constexpr int NI = NW * GPW * R;     // interfaces per CTA (R rounds per group)
  static constexpr int T = NI - 1;            // cells per CTA
  static constexpr int GH = P > 2 ? P : 2;    // ghost cells each side
  static constexpr int TW = T + 2 * GH;       // staged cells
};

// Warps per CTA of the flux-only and adjoint kernels: small CTAs spread a
// step's interfaces evenly over the SMs (no CTA-sized tail).
constexpr int NWF = 2;

// Order selection of the interface of lane group `grp`: lane c < S of the
// group decides every order p = 2..P of component c (reject_set: the
// filtered indicator decisions of all nested stencils at once); a group
// OR-reduction of the rejected orders gives p_s = max A (1 when A is empty).
// A component's psi is admissible when psi >= thr; as in a literal minimum
// over components taken from the first component, a NaN in the first
// component rejects p and a NaN elsewhere is ignored. Groups have LPN lanes
// per node. Must be called by all 32 lanes.
template <int P, int S, bool F32, int LPN = 1>
__device__ __forceinline__ int select_order(const double *t0, const float *h0, const float *l0, int cs,
                                            int l, int grp, bool active, bool valid,
                                            const FiltConst &FC, double eps, double thr,
                                            const double *fact, int psi2_mod) {
  using TL = Tiling<P, NT / 32, LPN>;
  if (P < 2) return 1;
  static_assert(S <= 2 * P || P < 2, "one lane per component");
  unsigned rej = 0;
  if (active && l < S) {
    if constexpr (P >= 2) {
      if constexpr (F32)
        rej = reject_set32<P>(h0 + l * cs, l0 + l * cs, 1, l == 0, FC, eps, thr, fact, psi2_mod);
      else
        rej = reject_set64<P>(t0 + l * cs, 1, l == 0, FC, eps, thr, fact, psi2_mod);
    }
  }
  constexpr unsigned spare = (TL::GPW * TL::L >= 32) ? 0u : (0xffffffffu << (TL::GPW * TL::L));
  const unsigned gmask = valid ? (((1u << TL::L) - 1u) << (grp * TL::L)) : spare;
  rej = __reduce_or_sync(gmask, rej);
  const unsigned accept = ~rej & ((1u << (P - 1)) - 1u);
  return accept ? (32 - __clz(accept)) + 1 : 1;
}

}  // namespace
