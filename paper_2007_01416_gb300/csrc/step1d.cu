// step1d.cu -- the 1D ACAT step on sm_103a CUDA cores (FP64, and FP32 on a
// compensated state).
//
// One CTA owns T consecutive cells and computes the T+1 interface fluxes
// around them (the last one is recomputed by the next CTA). The cells
// [i0 - GH, i0 + T + GH) are staged once in shared memory with the boundary
// condition applied while loading. Each interface is worked by a group of 2P
// lanes of one warp, one lane per stencil node j = -p+1..p:
//   - the indicators psi^p (Eqs. 3.8-3.12, the minimum over components of
//     Sec. 3.4): lane c of the group decides every order p = 2..P of
//     component c from the differences of the largest stencil (the smaller
//     ones are nested in it). Each decision is a float test with a certified
//     error margin (psi_filter_all); only when the margin cannot settle it
//     is psi^p evaluated literally with explicitly rounded FP64 operations
//     in the order of its definition. Either way the decision is the one a
//     literal FP64 evaluation of the same state takes. An OR-reduction over
//     the group gives p_s = max A (Eqs. 3.2-3.3);
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
#include "step1d_core.cuh"

namespace {

template <int P, int FLUX>
__global__ void __launch_bounds__(NT, MinCtas<P, false>::value) k_step1d_f64(const Step1DArgs a) {
  acat_pdl_wait();
  __shared__ Smem64<P, Phys<FLUX>::S> sm;
  __shared__ double s_lam;
  if (threadIdx.x == 0) s_lam = step_dt(a) / a.dx;
  __syncthreads();
  tile_f64<P, FLUX>(a, sm, static_cast<const double *>(a.u_in), static_cast<double *>(a.u_out), 0,
                    a.N, a.N, (long)blockIdx.x * Tiling<P>::T, s_lam, a.orders,
                    &a.smax[(a.slot + 1) % 3]);
  acat_pdl_release();
}

// The fused FP32 step in CTAs of NW warps: 8, or 7, whose tiles of 7 GPW - 1
// cells let a step of a few waves fill every SM with the same number of CTAs
// (N = 16384 at P = 4: 607 CTAs, 4 on every SM, against 529 of 8 warps, 4 on
// some SMs and 3 on the others); the same register cap per thread.
template <int P, int FLUX, int LPN, int NW = NT / 32>
__global__ void __launch_bounds__(NW * 32, MinCtas<P, true>::value) k_step1d_f32(const Step1DArgs a) {
  acat_pdl_wait();
  __shared__ Smem32<P, DPhys<FLUX>::S, NW, LPN> sm;
  __shared__ float s_lam;
  if (threadIdx.x == 0) s_lam = (float)(step_dt(a) / a.dx);
  tile_f32<P, FLUX, NW, LPN>(a, sm, static_cast<const float *>(a.u_in), static_cast<float *>(a.u_out), 0, a.N,
                             a.N, (long)blockIdx.x * Tiling<P, NW, LPN>::T, &s_lam, a.orders,
                             &a.smax[(a.slot + 1) % 3]);
  acat_pdl_release();
}

// FP64 step in small CTAs (NWF warps): CTA b computes the NI interfaces
// [b NI, b NI + NI) and updates the cells between them; the cell between
// two CTAs is updated by whichever of the two finishes second. Each CTA
// publishes its edge fluxes, fences (release), and counts itself in at the
// boundary counters of its left and right neighbours (atomicAdd; no CTA ever
// waits): the one that reads 1 fences again (acquire), owns the boundary
// cell, reads the other edge flux from L2 and resets the counter for the next
// step. Small CTAs spread a step's interfaces evenly over the SMs, and no
// interface is computed twice.
template <int P, int FLUX>
__global__ void __launch_bounds__(NWF * 32, 16 / NWF) k_step1d_fine(const Step1DArgs a) {
  acat_pdl_wait();
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
  if (active && acat_in_bounds(ic - P + 1 >= 0 && ic + P < TL::TW && il < TL::NI, a.status)) {
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
  // the hand-off indices: this CTA's edge slots and counters
  const bool ho_ok = acat_in_bounds(i0 + TL::NI - 1 <= N || !has_right, a.status) &&
                     acat_in_bounds(blockIdx.x < gridDim.x && (long)gridDim.x * TL::NI >= N + 1, a.status);
  if (threadIdx.x == 0 && ho_ok) {
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
    // acquire: the neighbour's edge flux, published before its fence and
    // atomic, is read (by any thread, after the barrier below) only after
    // this fence, which follows the atomic that observed it
    if (own0 | own1) __threadfence();
    s_own[0] = own0;
    s_own[1] = own1;
  }
  if (threadIdx.x == 0 && !ho_ok) s_own[0] = s_own[1] = 0;
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
    if (!acat_in_bounds(k >= 0 && k < TL::TW && i >= 0 && i < N, a.status)) continue;
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
  acat_pdl_release();
}

// FP32 step in small CTAs (NWF warps), the boundary hand-off of
// k_step1d_fine on the compensated state: CTA b computes the flux increments
// G of the NI interfaces [b NI, b NI + NI) (iface_f32, as the fused FP32 tile)
// and updates the cells between them (update_cell_f32); it publishes its two
// edge increments (float, s x (N+1) in flux_buf), fences, and counts in at
// both boundary counters; the CTA that reads 1 fences again and updates the
// boundary cell. Small CTAs spread the interfaces evenly over the SMs where
// whole 8-warp CTAs leave some SMs with one CTA more than others; measured at
// N = 16384 the fused step is still faster (the two device-scope fences and
// the serial update phase of every small CTA weigh more at FP32 step times),
// so this is a selectable launch shape (nw = 2), not the default.
template <int P, int FLUX>
__global__ void __launch_bounds__(NWF * 32, 16) k_step1d_fine_f32(const Step1DArgs a) {
  acat_pdl_wait();
  using TL = Tiling<P, NWF>;
  using DP = DPhys<FLUX>;
  constexpr int S = DP::S;
  constexpr int NTF = NWF * 32;
  __shared__ float thi[S][TL::TW], tlo[S][TL::TW];
  __shared__ float Gs[TL::NI][S];
  __shared__ unsigned char rej[S][TL::NI];
  __shared__ float4 xs[(P >= 2 && S > 1) ? NWF * 2 * XSET : 1];
  __shared__ float s_lam;
  __shared__ int s_own[2];
  const long N = a.N, i0 = (long)blockIdx.x * TL::NI;
  const float *__restrict__ uin = static_cast<const float *>(a.u_in);
  float *__restrict__ uout = static_cast<float *>(a.u_out);
  float *__restrict__ gbuf = reinterpret_cast<float *>(a.flux_buf);
  if (threadIdx.x == 0) s_lam = (float)(step_dt(a) / a.dx);
  for (int q = threadIdx.x; q < S * TL::TW; q += NTF) {
    const int c = q / TL::TW, k = q - c * TL::TW;
    const long g = bc_index(i0 - TL::GH + k, N, a.bc);
    thi[c][k] = uin[c * N + g];
    tlo[c][k] = uin[(S + c) * N + g];
  }
  __syncthreads();
  const float lam = s_lam;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int grp = lane / TL::L, l = lane - grp * TL::L;
  const bool valid = grp < TL::GPW;
  const int il = warp * TL::GPW + grp;
  const long m = i0 + il;
  const bool active = valid && m <= N;
  const FiltConst FC = filt_const(a.epsf, a.rf, a.factf);
  reject_pass_f32<P, S, TL::GH>(a, &thi[0][0], &tlo[0][0], TL::TW, TL::NI, i0, N, FC, &rej[0][0], NTF);
  if (P >= 2) __syncthreads();
  float G[S];
  const int ps = iface_f32<P, FLUX, 1>(a, &thi[0][0], &tlo[0][0], TL::TW, il, grp, l, valid, active, lam, FC,
                                       &xs[warp * 2 * XSET], G, &rej[0][0], TL::NI);
  if (active && l == 0) {
#pragma unroll
    for (int c = 0; c < S; c++) Gs[il][c] = G[c];
    if (a.orders) a.orders[m] = (int8_t)ps;
  }
  __syncthreads();
  const long nI = (N + 1 - i0) < TL::NI ? (N + 1 - i0) : TL::NI;  // interfaces of this CTA
  const bool has_left = blockIdx.x > 0, has_right = i0 + TL::NI <= N;
  const bool ho_ok = acat_in_bounds(i0 + TL::NI - 1 <= N || !has_right, a.status) &&
                     acat_in_bounds((long)gridDim.x * TL::NI >= N + 1, a.status);
  if (threadIdx.x == 0 && ho_ok) {
#pragma unroll
    for (int c = 0; c < S; c++) {
      if (has_left) gbuf[c * (N + 1) + i0] = Gs[0][c];
      if (has_right) gbuf[c * (N + 1) + i0 + TL::NI - 1] = Gs[TL::NI - 1][c];
    }
    __threadfence();  // release: the edge increments before the counts
    int own0 = 0, own1 = 0;
    if (has_left && atomicAdd(&a.cnt[blockIdx.x - 1], 1) == 1) {
      own0 = 1;
      a.cnt[blockIdx.x - 1] = 0;
    }
    if (has_right && atomicAdd(&a.cnt[blockIdx.x], 1) == 1) {
      own1 = 1;
      a.cnt[blockIdx.x] = 0;
    }
    if (own0 | own1) __threadfence();  // acquire: the neighbour's increments after its count
    s_own[0] = own0;
    s_own[1] = own1;
  }
  if (threadIdx.x == 0 && !ho_ok) s_own[0] = s_own[1] = 0;
  __syncthreads();
  float smax = 0.0f;
  bool bad = false;
  // cells t = 0 .. nI - 2 lie between two interfaces of this CTA; task nI - 1
  // is the left boundary cell i0 - 1, task nI the right one i0 + NI - 1
  for (int t = threadIdx.x; t <= nI; t += NTF) {
    float Gl[S], Gr[S];
    long i;
    int k;
    if (t < nI - 1) {
      i = i0 + t;
      k = t + TL::GH;
#pragma unroll
      for (int c = 0; c < S; c++) {
        Gl[c] = Gs[t][c];
        Gr[c] = Gs[t + 1][c];
      }
    } else if (t == nI - 1) {
      if (!s_own[0]) continue;
      i = i0 - 1;
      k = TL::GH - 1;
#pragma unroll
      for (int c = 0; c < S; c++) {
        Gl[c] = __ldcg(&gbuf[c * (N + 1) + i0 - 1]);
        Gr[c] = Gs[0][c];
      }
    } else {
      if (!s_own[1]) continue;
      i = i0 + TL::NI - 1;
      k = TL::NI - 1 + TL::GH;
#pragma unroll
      for (int c = 0; c < S; c++) {
        Gl[c] = Gs[TL::NI - 1][c];
        Gr[c] = __ldcg(&gbuf[c * (N + 1) + i0 + TL::NI]);
      }
    }
    update_cell_f32<FLUX>(a, &thi[0][0], &tlo[0][0], TL::TW, k, lam, Gl, Gr, uout, N, 0, i, &smax, &bad);
  }
  if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(a.status, (unsigned)ACAT_STATUS_NONPHYSICAL);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) smax = fmaxf(smax, __shfl_xor_sync(0xffffffffu, smax, o));
  if (lane == 0) atomic_max_pos(&a.smax[(a.slot + 1) % 3], (double)smax);
  acat_pdl_release();
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
    if (a.flux_buf && a.cnt)  // small-CTA step with boundary hand-off
      return acat_launch_dep(k_step1d_fine<P, FLUX>, (unsigned)acat_fine_ctas_1d(P, a.N), NWF * 32, st, a);
  }
  if constexpr (F32) {
    if (a.flux_buf && a.cnt && a.lpn == 1)  // small-CTA step with boundary hand-off
      return acat_launch_dep(k_step1d_fine_f32<P, FLUX>, (unsigned)acat_fine_ctas_1d(P, a.N), NWF * 32, st, a);
    if constexpr (P == 2 || P == 4) {
      if (a.lpn == 2) {
        using T2 = Tiling<P, NT / 32, 2>;
        return acat_launch_dep(k_step1d_f32<P, FLUX, 2>, (unsigned)((a.N + T2::T - 1) / T2::T), NT, st, a);
      }
    }
    if (a.lpn != 1) return (int)cudaErrorInvalidValue;
    if (a.nw == 7) {
      using T7 = Tiling<P, 7>;
      return acat_launch_dep(k_step1d_f32<P, FLUX, 1, 7>, (unsigned)((a.N + T7::T - 1) / T7::T), 7 * 32, st, a);
    }
    if (a.nw != 0 && a.nw != NT / 32) return (int)cudaErrorInvalidValue;
  }
  const unsigned grid = (unsigned)((a.N + TL::T - 1) / TL::T);
  if constexpr (F32) return acat_launch_dep(k_step1d_f32<P, FLUX, 1>, grid, NT, st, a);
  else return acat_launch_dep(k_step1d_f64<P, FLUX>, grid, NT, st, a);
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

}  // namespace

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
  if (e == 0) e = acat_upload_tables_batch(&T);
  return e;
}
