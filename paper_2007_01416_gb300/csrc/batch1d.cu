// batch1d.cu -- the batched 1D step: independent instances of ragged sizes,
// concatenated along the cell index, advanced in one persistent launch per
// step. CTAs take the tiles of an (instance, tile) work list from a queue;
// each tile is the tile of the single-instance step (step1d_core.cuh) with
// the instance's own dt, and per-instance wave speeds are reduced into
// per-instance slots for the next step's dt.
#include "step1d_core.cuh"

namespace {

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

// dt and lambda = dt / dx of every instance for this step, one thread per
// instance (batch_dt: the instance's time advanced, its wave-speed slot two
// steps ahead recycled). The step kernel's tiles then read lambda: the FP64
// divisions are done once per instance, not once per tile (in the tile they
// held the whole CTA at its staging barrier behind one thread).
__global__ void __launch_bounds__(NT) k_batch_dt(const Step1DArgs a, const BatchArgs bt) {
  if (blockIdx.x == 0 && threadIdx.x == 0) *bt.next = 0;  // the step kernel's tile queue
  for (long b = (long)blockIdx.x * NT + threadIdx.x; b < bt.B; b += (long)gridDim.x * NT) {
    const long N = bt.offs[b + 1] - bt.offs[b];
    const double dx = bt.xlen / (double)N;
    const double l = batch_dt(a, bt, (int)b, true, dx) / dx;
    bt.lam[b] = l;
    bt.lamf[b] = (float)l;
  }
}

// Interface rounds per lane group in a tile of the FP32 batched step: eight
// rounds (two at 16 warps, within 48 KB of static shared memory) make tiles
// of R NW GPW interfaces, so the tile's CTA barriers, order-decision pass and
// update phase are shared by R times the flux work.
template <int NW>
struct RoundsB32 {
  static constexpr int value = NW >= 16 ? 2 : 8;
};

// Persistent batched step: CTAs of NW warps take the tiles of the (instance,
// first cell) work list, Tiling<P, NW, LPN, R>::T cells wide (R =
// RoundsB32<NW> in FP32, 1 in FP64), from a queue: CTA c starts with tile c,
// and each further tile is claimed with one atomic on the queue counter
// (set to 0 by k_batch_dt), issued before the current tile so that its
// latency hides behind the tile's work. Tiles cost unevenly (FL-CAT2
// interfaces, the order decisions left to the FP64 fallback, partial last
// tiles), and the queue keeps the CTAs busy to the end. Results do not
// depend on which CTA takes a tile. Every instance is advanced with its own
// dt (lambda from k_batch_dt). The register cap per thread is that of the
// 8-warp kernels (MinCtas x 8 / NW resident CTAs).
template <int P, int FLUX, bool F32, int NW, int LPN>
__global__ void __launch_bounds__(NW * 32, MinCtas<P, F32>::value * 8 / NW)
    k_batch1d(const Step1DArgs a, const BatchArgs bt) {
  constexpr int R = F32 ? RoundsB32<NW>::value : 1;
  using SM =
      typename std::conditional<F32, Smem32<P, Phys<FLUX>::S, NW, LPN, R>, Smem64<P, Phys<FLUX>::S, NW>>::type;
  // FP32: two workspaces used alternately (tile_f32 ends without a barrier)
  __shared__ SM sm[F32 ? 2 : 1];
  // the next tile of this CTA, claimed by thread 0 before the current one and
  // read after it: the tile's staging barrier publishes it, and the two slots
  // alternate, so a claim never overwrites a slot another thread still reads
  __shared__ long long s_next[2];
  int par = 0;
  for (long w = blockIdx.x; w < bt.ntiles; par ^= 1) {
    if (threadIdx.x == 0) s_next[par] = (long long)gridDim.x + atomicAdd(bt.next, 1);
    const int b = bt.tiles[w].b;
    const long i0 = (long)bt.tiles[w].tile * Tiling<P, NW, LPN, R>::T;
    const long off = bt.offs[b], N = bt.offs[b + 1] - off;
    int8_t *ord = bt.orders ? bt.orders + off + b : nullptr;
    unsigned long long *so = &bt.smax[((a.slot + 1) % 3) * (long)bt.B + b];
    if constexpr (F32) {
      tile_f32<P, FLUX, NW, LPN, R>(a, sm[par], static_cast<const float *>(a.u_in),
                                    static_cast<float *>(a.u_out), off, bt.M, N, i0, &bt.lamf[b], ord, so);
    } else {
      tile_f64<P, FLUX, NW>(a, sm[0], static_cast<const double *>(a.u_in), static_cast<double *>(a.u_out),
                            off, bt.M, N, i0, bt.lam[b], ord, so);
    }
    w = (long)s_next[par];
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

// Resident CTAs per SM of the batched kernel with NW warps and LPN lanes per
// node, and its launch on sms x cps CTAs (cps <= 0 or above the occupancy:
// the occupancy). With occ_out set, only the occupancy is returned.
template <int P, int FLUX, bool F32, int NW, int LPN>
int launch_batch_nw(const Step1DArgs &a, const BatchArgs &bt, cudaStream_t st, int *occ_out) {
  int dev = 0, sms = 0, occ = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_batch1d<P, FLUX, F32, NW, LPN>, NW * 32, 0);
  if (occ < 1) occ = 1;
  if (occ_out) {
    *occ_out = occ;
    return 0;
  }
  const int cps = (bt.cps > 0 && bt.cps < occ) ? bt.cps : occ;
  const unsigned gdt = (unsigned)((bt.B + NT - 1) / NT);
  k_batch_dt<<<gdt < 1024u ? gdt : 1024u, NT, 0, st>>>(a, bt);
  const int e = (int)cudaGetLastError();
  if (e) return e;
  k_batch1d<P, FLUX, F32, NW, LPN><<<(unsigned)(sms * cps), NW * 32, 0, st>>>(a, bt);
  return (int)cudaGetLastError();
}

template <int P, int FLUX, bool F32, int LPN>
int launch_batch_lpn(const Step1DArgs &a, const BatchArgs &bt, cudaStream_t st, int *occ_out) {
  switch (bt.nw) {
  case 4: return launch_batch_nw<P, FLUX, F32, 4, LPN>(a, bt, st, occ_out);
  case 8: return launch_batch_nw<P, FLUX, F32, 8, LPN>(a, bt, st, occ_out);
  case 16: return launch_batch_nw<P, FLUX, F32, 16, LPN>(a, bt, st, occ_out);
  }
  return (int)cudaErrorInvalidValue;
}

template <int P, int FLUX, bool F32>
int launch_batch_p(const Step1DArgs &a, const BatchArgs &bt, cudaStream_t st, int *occ_out) {
  if constexpr (F32 && (P == 2 || P == 4)) {
    if (bt.lpn == 2) return launch_batch_lpn<P, FLUX, F32, 2>(a, bt, st, occ_out);
  }
  if (bt.lpn != 1) return (int)cudaErrorInvalidValue;
  return launch_batch_lpn<P, FLUX, F32, 1>(a, bt, st, occ_out);
}

template <int FLUX, bool F32>
int launch_batch_f(int P, const Step1DArgs &a, const BatchArgs &bt, cudaStream_t st, int *occ_out) {
  switch (P) {
  case 1: return launch_batch_p<1, FLUX, F32>(a, bt, st, occ_out);
  case 2: return launch_batch_p<2, FLUX, F32>(a, bt, st, occ_out);
  case 3: return launch_batch_p<3, FLUX, F32>(a, bt, st, occ_out);
  case 4: return launch_batch_p<4, FLUX, F32>(a, bt, st, occ_out);
  }
  return (int)cudaErrorInvalidValue;
}

template <bool F32>
int launch_batch(int P, int flux, const Step1DArgs &a, const BatchArgs &bt, cudaStream_t st, int *occ_out) {
  switch (flux) {
  case ACAT_FLUX_LINEAR: return launch_batch_f<ACAT_FLUX_LINEAR, F32>(P, a, bt, st, occ_out);
  case ACAT_FLUX_BURGERS: return launch_batch_f<ACAT_FLUX_BURGERS, F32>(P, a, bt, st, occ_out);
  case ACAT_FLUX_EULER1D: return launch_batch_f<ACAT_FLUX_EULER1D, F32>(P, a, bt, st, occ_out);
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
  return prec == ACAT_PREC_F32 ? launch_batch<true>(P, flux, a, bt, st, nullptr)
                               : launch_batch<false>(P, flux, a, bt, st, nullptr);
}

int acat_batch_occupancy(int P, int flux, int prec, int nw, int lpn) {
  BatchArgs bt;
  std::memset(&bt, 0, sizeof bt);
  bt.nw = nw;
  bt.lpn = lpn;
  Step1DArgs a;
  std::memset(&a, 0, sizeof a);
  int occ = 0;
  const int e = prec == ACAT_PREC_F32 ? launch_batch<true>(P, flux, a, bt, nullptr, &occ)
                                      : launch_batch<false>(P, flux, a, bt, nullptr, &occ);
  return e ? -1 : occ;
}

namespace {
template <int NW, int LPN, bool F32>
int cells_per_tile(int P) {
  constexpr int R = F32 ? RoundsB32<NW>::value : 1;
  switch (P) {
  case 1: return Tiling<1, NW, LPN, R>::T;
  case 2: return Tiling<2, NW, LPN, R>::T;
  case 3: return Tiling<3, NW, LPN, R>::T;
  case 4: return Tiling<4, NW, LPN, R>::T;
  }
  return 0;
}
template <int LPN, bool F32>
int cells_per_tile_nw(int P, int nw) {
  switch (nw) {
  case 4: return cells_per_tile<4, LPN, F32>(P);
  case 8: return cells_per_tile<8, LPN, F32>(P);
  case 16: return cells_per_tile<16, LPN, F32>(P);
  }
  return 0;
}
}  // namespace

int acat_cells_per_tile_1d(int P, int prec, int nw, int lpn) {
  if (prec != ACAT_PREC_F32) return lpn == 1 ? cells_per_tile_nw<1, false>(P, nw) : 0;
  if (lpn == 1) return cells_per_tile_nw<1, true>(P, nw);
  if (lpn == 2 && (P == 2 || P == 4)) return cells_per_tile_nw<2, true>(P, nw);
  return 0;
}

int acat_launch_smax_batch(int flux, int prec, const Step1DArgs &a, const BatchArgs &bt, void *stream) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  return prec == ACAT_PREC_F32 ? launch_smax_batch<true>(flux, a, bt, st)
                               : launch_smax_batch<false>(flux, a, bt, st);
}

int acat_upload_tables_batch(const AcatTables *T) { return (int)cudaMemcpyToSymbol(c_tab, T, sizeof *T); }
