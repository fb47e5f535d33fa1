// api.cu -- the C ABI of libacat (declared in include/acat.h): context
// lifetime, argument checks, the step and run entry points (CUDA-graph replay of
// the time loop with the dt reduction kept on the device), status words.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include "../../include/acat.h"
#include "acat_internal.h"

struct acat_ctx {
  acat_params p;
  int s = 1;
  int dim = 1;
  int device = 0;
  long cells = 0;
  unsigned long long *d_smax = nullptr;  // 3 slots
  double *d_t = nullptr;                 // 3 slots
  unsigned *d_status = nullptr;
  void *d_work = nullptr;                // second state buffer (run ping-pong)
  void *d_host_stage = nullptr;          // device buffer for acat_run_host
  cudaStream_t cap_stream = nullptr;     // stream used for graph capture
  cudaGraphExec_t chain = nullptr;       // GRAPH_STEPS steps, starting at step % 6 == 0
  void *chain_u = nullptr;
  double chain_t_end = 0.0;
  double fact_tau[ACAT_MAXP + 1] = {0};  // (2p-1)! or 1 (tau_factorial)
  int64_t launches = 0;
  // batch of independent 1D instances (acat_create_batched)
  int batched = 0;
  int B = 0;
  long long *d_offs = nullptr;
  TileRef *d_tiles = nullptr;
  long long ntiles = 0;
  std::vector<int32_t> sizes;             // cells of each instance
  int bnw = 8;                            // warps per CTA of the batched kernel
  int bcps = 0;                           // its CTAs per SM (0: occupancy)
  int lpn = 1;                            // 1D FP32: lanes per stencil node
  unsigned long long *d_smaxb = nullptr;  // 3 x B
  double *d_tb = nullptr;                 // 3 x B
  double *d_lamb = nullptr;               // B: dt / dx of each instance for the current step
  float *d_lambf = nullptr;               // B: the same in float
  int *d_next = nullptr;                  // batched: the step kernel's tile queue counter
  double *d_contrib = nullptr;            // adjoint: per-interface node cotangents
  void *d_seg = nullptr;                  // adjoint run: recomputed states of a segment
  size_t seg_bytes = 0;
  void *d_bar = nullptr;                  // adjoint run: second cotangent buffer
  double *d_flux = nullptr;               // 1D: CTA-edge fluxes (FP32: increments) of the small-CTA step
  int *d_cnt = nullptr;                   // 1D: its boundary hand-off counters
  int snw = 8;                            // 1D FP32 single instance: warps per CTA (8 or 7 fused, 2 small-CTA)
};

namespace {

constexpr int GRAPH_STEPS = 48;  // multiple of 2 (ping-pong) and 3 (dt slots)
constexpr int NWF_API = 2;       // warps per CTA of the small-CTA 1D steps

std::mutex g_tab_mu;
bool g_tab_done[64] = {false};

int nvars(int flux) {
  switch (flux) {
  case ACAT_FLUX_EULER1D: return 3;
  case ACAT_FLUX_EULER2D: return 4;
  default: return 1;
  }
}

int cuda_err(cudaError_t e) { return e == cudaSuccess ? ACAT_OK : ACAT_ERR_CUDA; }

// Whether lpn lanes per stencil node exist for (P, precision): two lanes per
// node only for the FP32 recursion at P = 2, 4.
bool acat_lpn_ok(int P, int prec, int lpn) {
  return lpn == 1 || (lpn == 2 && prec == ACAT_PREC_F32 && (P == 2 || P == 4));
}

int check_params(const acat_params *p) {
  if (!p) return ACAT_ERR_INVALID_ARG;
  if (p->P < 1 || p->P > ACAT_MAXP) return ACAT_ERR_INVALID_ARG;
  if (p->flux < ACAT_FLUX_LINEAR || p->flux > ACAT_FLUX_EULER2D) return ACAT_ERR_INVALID_ARG;
  if (p->bc != ACAT_BC_PERIODIC && p->bc != ACAT_BC_TRANSMISSIVE) return ACAT_ERR_INVALID_ARG;
  if (p->precision != ACAT_PREC_F64 && p->precision != ACAT_PREC_F32) return ACAT_ERR_INVALID_ARG;
  if (p->ny < 1 || p->nx < 2 * (p->P > 2 ? p->P : 2)) return ACAT_ERR_INVALID_ARG;
  if (!(p->cfl > 0.0) || !std::isfinite(p->cfl)) return ACAT_ERR_INVALID_ARG;
  if (!(p->x1 > p->x0) || !(p->y1 > p->y0)) return ACAT_ERR_INVALID_ARG;
  if (!(p->psi_tol >= 0.0 && p->psi_tol < 1.0)) return ACAT_ERR_INVALID_ARG;
  if (!(p->eps >= 0.0) || !std::isfinite(p->eps)) return ACAT_ERR_INVALID_ARG;
  if (p->psi2_mod != 0 && p->psi2_mod != 1) return ACAT_ERR_INVALID_ARG;
  if (p->lo_flux < ACAT_LO_RUSANOV || p->lo_flux > ACAT_LO_HLL) return ACAT_ERR_INVALID_ARG;
  if (p->rect_2d != 0 && p->rect_2d != 1) return ACAT_ERR_INVALID_ARG;
  if ((p->flux == ACAT_FLUX_EULER1D || p->flux == ACAT_FLUX_EULER2D) && !(p->gamma > 1.0))
    return ACAT_ERR_INVALID_ARG;
  const bool is2d = p->ny > 1 || p->flux == ACAT_FLUX_EULER2D;
  if (is2d) {
    if (p->ny < 2 * (p->P > 2 ? p->P : 2)) return ACAT_ERR_INVALID_ARG;
    if (p->flux != ACAT_FLUX_EULER2D && p->flux != ACAT_FLUX_LINEAR) return ACAT_ERR_UNSUPPORTED;

    if ((long)p->nx * (long)p->ny > (1l << 31)) return ACAT_ERR_TOO_LARGE;
    return ACAT_OK;
  }
  if ((long)p->nx > (1l << 30)) return ACAT_ERR_TOO_LARGE;
  return ACAT_OK;
}

Step1DArgs base_args(acat_ctx *c) {
  Step1DArgs a;
  std::memset(&a, 0, sizeof a);
  const acat_params &p = c->p;
  a.N = p.nx;
  a.bc = p.bc;
  a.limiter_form = p.limiter_form;
  a.psi2_mod = p.psi2_mod;
  a.lo_flux = p.lo_flux;
  a.dx = (p.x1 - p.x0) / (double)p.nx;
  a.cfl = p.cfl;
  a.dt_fixed = -1.0;
  a.t_end = -1.0;
  a.gamma = p.gamma;
  a.adv = p.adv[0];
  a.eps = p.eps;
  a.thr = 1.0 - p.psi_tol;
  for (int q = 0; q <= ACAT_MAXP; q++) {
    a.fact_tau[q] = c->fact_tau[q];
    a.factf[q] = (float)c->fact_tau[q];
  }
  a.epsf = (float)p.eps;
  a.rf = (float)(a.thr / (1.0 - a.thr));
  a.advf = (float)p.adv[0];
  a.gammaf = (float)p.gamma;
  a.gm1f = (float)(p.gamma - 1.0);
  a.smax = c->d_smax;
  a.status = c->d_status;
  // the small-CTA step: FP64 whenever its buffers exist, FP32 when chosen
  const bool fine = c->d_flux && (p.precision != ACAT_PREC_F32 || c->snw == NWF_API);
  a.flux_buf = fine ? c->d_flux : nullptr;
  a.cnt = fine ? c->d_cnt : nullptr;
  a.lpn = c->lpn;
  a.nw = p.precision == ACAT_PREC_F32 && c->snw == 7 ? 7 : 0;
  return a;
}

Step2DArgs base_args2(acat_ctx *c) {
  Step2DArgs a;
  std::memset(&a, 0, sizeof a);
  const acat_params &p = c->p;
  a.NX = p.nx;
  a.NY = p.ny;
  a.bc = p.bc;
  a.limiter_form = p.limiter_form;
  a.psi2_mod = p.psi2_mod;
  a.lo_flux = p.lo_flux;
  a.rect_2d = p.rect_2d;
  a.dx = (p.x1 - p.x0) / (double)p.nx;
  a.dy = (p.y1 - p.y0) / (double)p.ny;
  a.cfl = p.cfl;
  a.dt_fixed = -1.0;
  a.t_end = -1.0;
  a.gamma = p.gamma;
  a.adv[0] = p.adv[0];
  a.adv[1] = p.adv[1];
  a.eps = p.eps;
  a.thr = 1.0 - p.psi_tol;
  for (int q = 0; q <= ACAT_MAXP; q++) {
    a.fact_tau[q] = c->fact_tau[q];
    a.factf[q] = (float)c->fact_tau[q];
  }
  a.epsf = (float)p.eps;
  a.rf = (float)(a.thr / (1.0 - a.thr));
  a.advf[0] = (float)p.adv[0];
  a.advf[1] = (float)p.adv[1];
  a.gammaf = (float)p.gamma;
  a.gm1f = (float)(p.gamma - 1.0);
  a.smax = c->d_smax;
  a.status = c->d_status;
  return a;
}

int launch_step(acat_ctx *c, const Step1DArgs &a, cudaStream_t st) {
  int e = acat_launch_step1d(c->p.P, c->p.flux, c->p.precision, a, st);
  c->launches++;
  return e ? ACAT_ERR_CUDA : ACAT_OK;
}

BatchArgs batch_args(acat_ctx *c) {
  BatchArgs bt;
  std::memset(&bt, 0, sizeof bt);
  bt.offs = c->d_offs;
  bt.tiles = c->d_tiles;
  bt.ntiles = c->ntiles;
  bt.B = c->B;
  bt.M = c->cells;
  bt.xlen = c->p.x1 - c->p.x0;
  bt.smax = c->d_smaxb;
  bt.t = c->d_tb;
  bt.lam = c->d_lamb;
  bt.lamf = c->d_lambf;
  bt.next = c->d_next;
  bt.nw = c->bnw;
  bt.cps = c->bcps;
  bt.lpn = c->lpn;
  return bt;
}

// (Re)builds the batch's work list for tiles of the kernel with nw warps and
// lpn lanes per node: one (instance, tile) entry per tile, instances in order.
int build_tiles(acat_ctx *c, int nw, int lpn) {
  const int T = acat_cells_per_tile_1d(c->p.P, c->p.precision, nw, lpn);
  if (T <= 0) return ACAT_ERR_INVALID_ARG;
  long long ntiles = 0;
  for (int32_t n : c->sizes) ntiles += (n + T - 1) / T;
  if (ntiles > (1ll << 31)) return ACAT_ERR_TOO_LARGE;
  std::vector<TileRef> tiles;
  tiles.reserve((size_t)ntiles);
  for (int b = 0; b < (int)c->sizes.size(); b++)
    for (int k = 0; k < (c->sizes[b] + T - 1) / T; k++) tiles.push_back(TileRef{b, k});
  TileRef *d = nullptr;
  cudaError_t e = cudaMalloc(&d, sizeof(TileRef) * (size_t)ntiles);
  if (e == cudaSuccess) e = cudaMemcpy(d, tiles.data(), sizeof(TileRef) * (size_t)ntiles, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(d);
    return e == cudaErrorMemoryAllocation ? ACAT_ERR_NOMEM : ACAT_ERR_CUDA;
  }
  // the old list may still be read by queued work and by the captured chain
  if (cudaDeviceSynchronize() != cudaSuccess) {
    cudaFree(d);
    return ACAT_ERR_CUDA;
  }
  if (c->chain) {
    cudaGraphExecDestroy(c->chain);
    c->chain = nullptr;
  }
  cudaFree(c->d_tiles);
  c->d_tiles = d;
  c->ntiles = ntiles;
  c->bnw = nw;
  c->lpn = lpn;
  return ACAT_OK;
}

// Steps n..n+count-1 of a run on (u, work), dt slots n % 3.
int issue_steps(acat_ctx *c, void *u, long n, int count, double t_end, cudaStream_t st) {
  if (c->batched) {
    Step1DArgs a = base_args(c);
    a.t_end = t_end;
    BatchArgs bt = batch_args(c);
    for (int k = 0; k < count; k++, n++) {
      a.u_in = (n % 2 == 0) ? u : c->d_work;
      a.u_out = (n % 2 == 0) ? c->d_work : u;
      a.slot = (int)(n % 3);
      int e = acat_launch_batch1d(c->p.P, c->p.flux, c->p.precision, a, bt, st);
      c->launches += ACAT_BATCH_LAUNCHES_PER_STEP;
      if (e) return ACAT_ERR_CUDA;
    }
    return ACAT_OK;
  }
  if (c->dim == 2) {
    Step2DArgs a = base_args2(c);
    a.t_end = t_end;
    a.tslot = c->d_t;
    for (int k = 0; k < count; k++, n++) {
      a.u_in = (n % 2 == 0) ? u : c->d_work;
      a.u_out = (n % 2 == 0) ? c->d_work : u;
      a.slot = (int)(n % 3);
      int e = acat_launch_step2d(c->p.P, c->p.flux, c->p.precision, a, st);
      c->launches++;
      if (e) return ACAT_ERR_CUDA;
    }
    return ACAT_OK;
  }
  Step1DArgs a = base_args(c);
  a.t_end = t_end;
  a.tslot = c->d_t;
  for (int k = 0; k < count; k++, n++) {
    a.u_in = (n % 2 == 0) ? u : c->d_work;
    a.u_out = (n % 2 == 0) ? c->d_work : u;
    a.slot = (int)(n % 3);
    int rc = launch_step(c, a, st);
    if (rc) return rc;
  }
  return ACAT_OK;
}

int ensure_chain(acat_ctx *c, void *u, double t_end) {
  if (c->chain && c->chain_u == u && c->chain_t_end == t_end) return ACAT_OK;
  if (c->chain) {
    cudaGraphExecDestroy(c->chain);
    c->chain = nullptr;
  }
  cudaGraph_t g = nullptr;
  if (cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
    return ACAT_ERR_CUDA;
  const int64_t before = c->launches;
  int rc = issue_steps(c, u, 0, GRAPH_STEPS, t_end, c->cap_stream);
  c->launches = before;  // captured, not launched
  cudaError_t e = cudaStreamEndCapture(c->cap_stream, &g);
  if (rc || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return ACAT_ERR_CUDA;
  }
  e = cudaGraphInstantiate(&c->chain, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    c->chain = nullptr;
    return ACAT_ERR_CUDA;
  }
  c->chain_u = u;
  c->chain_t_end = t_end;
  return ACAT_OK;
}

}  // namespace

// The weight tables of every kernel file, uploaded once per device with that
// device current (shared by acat_create and acat_run_noalloc).
int acat_ensure_tables(int dev) {
  std::lock_guard<std::mutex> lk(g_tab_mu);
  if (dev < 0 || dev >= 64) return ACAT_ERR_UNSUPPORTED;
  if (!g_tab_done[dev]) {
    if (acat_upload_tables_current_device() != 0) return ACAT_ERR_CUDA;
    g_tab_done[dev] = true;
  }
  return ACAT_OK;
}

extern "C" {

void acat_default_params(acat_params *p) {
  if (!p) return;
  std::memset(p, 0, sizeof *p);
  p->flux = ACAT_FLUX_BURGERS;
  p->P = 2;
  p->nx = 64;
  p->ny = 1;
  p->bc = ACAT_BC_PERIODIC;
  p->precision = ACAT_PREC_F64;
  p->tau_factorial = 1;
  p->limiter_form = 0;
  p->gamma = 1.4;
  p->adv[0] = 1.0;
  p->adv[1] = 1.0;
  p->cfl = 0.5;
  p->x0 = 0.0;
  p->x1 = 1.0;
  p->y0 = 0.0;
  p->y1 = 1.0;
  p->psi_tol = 0.1;
  p->eps = 1e-12;
}

int acat_create(const acat_params *p, acat_ctx **out) {
  if (!out) return ACAT_ERR_INVALID_ARG;
  *out = nullptr;
  int rc = check_params(p);
  if (rc) return rc;
  acat_ctx *c = new (std::nothrow) acat_ctx();
  if (!c) return ACAT_ERR_NOMEM;
  c->p = *p;
  c->s = nvars(p->flux);
  c->cells = (long)p->nx * p->ny;
  c->dim = (p->ny > 1 || p->flux == ACAT_FLUX_EULER2D) ? 2 : 1;
  {
    AcatTables T;
    acat_build_tables(&T);
    for (int q = 0; q <= ACAT_MAXP; q++) c->fact_tau[q] = p->tau_factorial ? T.fact[q] : 1.0;
  }
  if (cudaGetDevice(&c->device) != cudaSuccess) {
    delete c;
    return ACAT_ERR_CUDA;
  }
  {
    const int rt = acat_ensure_tables(c->device);
    if (rt != ACAT_OK) {
      delete c;
      return rt;
    }
  }
  const size_t sb = (size_t)acat_state_bytes(c);
  cudaError_t e = cudaMalloc(&c->d_smax, 6 * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMalloc(&c->d_t, 3 * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&c->d_status, sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMalloc(&c->d_work, sb);
  // 1D FP64: the small-CTA step when the 8-warp fused step would not fit its
  // CTAs in ~3/4 of one wave at 2 CTAs per SM (it then leaves SMs idle)
  int sms = 0;
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
  const long fused_ctas = (p->nx + acat_cells_per_cta_1d(p->P, ACAT_PREC_F64) - 1) /
                          acat_cells_per_cta_1d(p->P, ACAT_PREC_F64);
  // 1D FP32: the small-CTA step is available to every context through
  // acat_set_launch_shape and the autotuner; the fused step (8 or 7 warps, set
  // below) stays the default (at FP32 step times the hand-off's fences and the
  // small CTAs' serial update phases cost more than their even load saves)
  const bool f64_fine = p->precision == ACAT_PREC_F64 && 4 * fused_ctas > 3 * 2 * (long)sms;
  const bool f32_fine = p->precision == ACAT_PREC_F32;
  if (e == cudaSuccess && c->dim == 1 && (f64_fine || f32_fine)) {
    const size_t nc = (size_t)acat_fine_ctas_1d(p->P, p->nx);
    e = cudaMalloc(&c->d_flux, (size_t)c->s * (size_t)(p->nx + 1) * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&c->d_cnt, nc * sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(c->d_cnt, 0, nc * sizeof(int));
  }
  // 1D FP32, fused step: 8 or 7 warps per CTA, whichever leaves the busiest
  // SM the fewer warps of work: ceil(CTAs / SMs) x warps per CTA, with
  // CTAs = ceil(N / T) and T = warps x floor(32 / 2P) - 1 cells per tile
  // (N = 16384: 7 at P = 2 and 4, 8 at P = 3; ties keep 8)
  if (e == cudaSuccess && c->dim == 1 && p->precision == ACAT_PREC_F32 && sms > 0) {
    long load[2] = {0, 0};
    const int nws[2] = {8, 7};
    for (int q = 0; q < 2; q++) {
      const long T = (long)nws[q] * (32 / (2 * p->P)) - 1;
      const long ctas = (p->nx + T - 1) / T;
      load[q] = (ctas + sms - 1) / sms * nws[q];
    }
    c->snw = load[1] < load[0] ? 7 : 8;
  }
  if (e == cudaSuccess) e = cudaMemset(c->d_smax, 0, 6 * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMemset(c->d_t, 0, 3 * sizeof(double));
  if (e == cudaSuccess) e = cudaMemset(c->d_status, 0, sizeof(unsigned));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    acat_destroy(c);
    return e == cudaErrorMemoryAllocation ? ACAT_ERR_NOMEM : ACAT_ERR_CUDA;
  }
  *out = c;
  return ACAT_OK;
}

int acat_create_batched(const acat_params *p, int n_inst, const int32_t *n_per_inst, acat_ctx **out) {
  if (!out || !p || n_inst < 1 || !n_per_inst) return ACAT_ERR_INVALID_ARG;
  *out = nullptr;
  if (p->ny != 1 || p->flux == ACAT_FLUX_EULER2D) return ACAT_ERR_INVALID_ARG;
  const int gh = p->P > 2 ? p->P : 2;
  long long M = 0;
  for (int b = 0; b < n_inst; b++) {
    if (n_per_inst[b] < 2 * gh) return ACAT_ERR_INVALID_ARG;
    M += n_per_inst[b];
  }
  if (M > (1ll << 31)) return ACAT_ERR_TOO_LARGE;
  acat_params q = *p;
  q.nx = n_per_inst[0];
  acat_ctx *c = nullptr;
  int rc = acat_create(&q, &c);
  if (rc) return rc;
  // replace the single-instance workspace by the batch's
  cudaFree(c->d_work);
  c->d_work = nullptr;
  cudaFree(c->d_flux);
  c->d_flux = nullptr;
  cudaFree(c->d_cnt);
  c->d_cnt = nullptr;
  c->batched = 1;
  c->B = n_inst;
  c->cells = M;
  c->sizes.assign(n_per_inst, n_per_inst + n_inst);
  std::vector<long long> offs((size_t)n_inst + 1, 0);
  for (int b = 0; b < n_inst; b++) offs[b + 1] = offs[b] + n_per_inst[b];
  rc = build_tiles(c, 8, 1);
  if (rc) {
    acat_destroy(c);
    return rc;
  }
  cudaError_t e = cudaMalloc(&c->d_work, (size_t)acat_state_bytes(c));
  if (e == cudaSuccess) e = cudaMalloc(&c->d_offs, sizeof(long long) * (size_t)(n_inst + 1));
  if (e == cudaSuccess) e = cudaMalloc(&c->d_smaxb, 3 * sizeof(unsigned long long) * (size_t)n_inst);
  if (e == cudaSuccess) e = cudaMalloc(&c->d_tb, 3 * sizeof(double) * (size_t)n_inst);
  if (e == cudaSuccess) e = cudaMalloc(&c->d_lamb, sizeof(double) * (size_t)n_inst);
  if (e == cudaSuccess) e = cudaMalloc(&c->d_lambf, sizeof(float) * (size_t)n_inst);
  if (e == cudaSuccess) e = cudaMalloc(&c->d_next, sizeof(int));
  if (e == cudaSuccess)
    e = cudaMemcpy(c->d_offs, offs.data(), sizeof(long long) * (size_t)(n_inst + 1), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(c->d_smaxb, 0, 3 * sizeof(unsigned long long) * (size_t)n_inst);
  if (e == cudaSuccess) e = cudaMemset(c->d_tb, 0, 3 * sizeof(double) * (size_t)n_inst);
  if (e != cudaSuccess) {
    acat_destroy(c);
    return e == cudaErrorMemoryAllocation ? ACAT_ERR_NOMEM : ACAT_ERR_CUDA;
  }
  *out = c;
  return ACAT_OK;
}

int acat_launch_shape(const acat_ctx *c, int *nw, int *lpn, int *cps) {
  if (!c) return ACAT_ERR_INVALID_ARG;
  if (c->dim != 1) return ACAT_ERR_UNSUPPORTED;
  int w = 8, k = 0;
  if (c->batched) {
    w = c->bnw;
    k = c->bcps > 0 ? c->bcps : acat_batch_occupancy(c->p.P, c->p.flux, c->p.precision, c->bnw, c->lpn);
  } else if (c->p.precision == ACAT_PREC_F32) {
    w = c->snw;
  } else if (c->d_flux) {
    w = NWF_API;  // the small-CTA FP64 step
  }
  if (nw) *nw = w;
  if (lpn) *lpn = c->lpn;
  if (cps) *cps = k;
  return ACAT_OK;
}

int acat_set_launch_shape(acat_ctx *c, int nw, int lpn, int cps) {
  if (!c || cps < 0) return ACAT_ERR_INVALID_ARG;
  if (c->dim != 1) return ACAT_ERR_UNSUPPORTED;
  if (!c->batched) {
    int w0 = 0, l0 = 0, k0 = 0;
    acat_launch_shape(c, &w0, &l0, &k0);
    if (cps != 0) return ACAT_ERR_UNSUPPORTED;
    if (c->p.precision != ACAT_PREC_F32) {  // fixed for a single FP64 instance
      if (nw != w0) return ACAT_ERR_UNSUPPORTED;
      return lpn == c->lpn ? ACAT_OK : ACAT_ERR_UNSUPPORTED;
    }
    // FP32: the fused step of 8 warps (one or two lanes per node) or 7 warps (one
    // lane per node), or the small-CTA step
    if (nw != 8 && nw != 7 && !(nw == NWF_API && c->d_flux)) return ACAT_ERR_UNSUPPORTED;
    if (!acat_lpn_ok(c->p.P, c->p.precision, lpn) || ((nw == NWF_API || nw == 7) && lpn != 1))
      return ACAT_ERR_INVALID_ARG;
    if (lpn == c->lpn && nw == c->snw) return ACAT_OK;
    if (c->chain) {
      if (cudaDeviceSynchronize() != cudaSuccess) return ACAT_ERR_CUDA;
      cudaGraphExecDestroy(c->chain);
      c->chain = nullptr;
    }
    c->lpn = lpn;
    c->snw = nw;
    return ACAT_OK;
  }
  if (!acat_lpn_ok(c->p.P, c->p.precision, lpn) || acat_cells_per_tile_1d(c->p.P, c->p.precision, nw, lpn) <= 0)
    return ACAT_ERR_INVALID_ARG;
  const int occ = acat_batch_occupancy(c->p.P, c->p.flux, c->p.precision, nw, lpn);
  if (occ < 1) return ACAT_ERR_CUDA;
  if (cps > occ) return ACAT_ERR_INVALID_ARG;
  if (nw != c->bnw || lpn != c->lpn) {
    int rc = build_tiles(c, nw, lpn);
    if (rc) return rc;
  }
  if (cps != c->bcps && c->chain) {
    if (cudaDeviceSynchronize() != cudaSuccess) return ACAT_ERR_CUDA;
    cudaGraphExecDestroy(c->chain);
    c->chain = nullptr;
  }
  c->bcps = cps;
  return ACAT_OK;
}

int acat_autotune(acat_ctx *c, const void *u_dev, int steps, void *stream, int *nw_out, int *lpn_out,
                  int *cps_out) {
  if (!c || !u_dev || steps < 1) return ACAT_ERR_INVALID_ARG;
  if (c->dim != 1 || !(c->batched || c->p.precision == ACAT_PREC_F32)) return ACAT_ERR_UNSUPPORTED;
  // candidate shapes: (warps per CTA, lanes per node, CTAs per SM; 0 = occupancy)
  struct Shape {
    int nw, lpn, cps;
  };
  std::vector<Shape> cands;
  const int lpns[2] = {1, 2};
  for (int lpn : lpns) {
    if (!acat_lpn_ok(c->p.P, c->p.precision, lpn)) continue;
    if (!c->batched) {
      cands.push_back(Shape{8, lpn, 0});
      if (lpn == 1) cands.push_back(Shape{7, 1, 0});
      if (lpn == 1 && c->d_flux) cands.push_back(Shape{NWF_API, 1, 0});
      continue;
    }
    const int nws[3] = {8, 4, 16};
    for (int nw : nws) {
      const int occ = acat_batch_occupancy(c->p.P, c->p.flux, c->p.precision, nw, lpn);
      if (occ < 1) continue;
      cands.push_back(Shape{nw, lpn, 0});
      if (occ / 2 >= 1) cands.push_back(Shape{nw, lpn, occ / 2});
    }
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t sb = (size_t)acat_state_bytes(c);
  void *trial = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaMalloc(&trial, sb);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  int rc = e == cudaSuccess ? ACAT_OK : (e == cudaErrorMemoryAllocation ? ACAT_ERR_NOMEM : ACAT_ERR_CUDA);
  Shape old{0, 0, 0};
  if (rc == ACAT_OK) acat_launch_shape(c, &old.nw, &old.lpn, &old.cps);
  old.cps = c->bcps;
  Shape best = old;
  float best_ms = 0.0f;
  for (size_t i = 0; i < cands.size() && rc == ACAT_OK; i++) {
    rc = acat_set_launch_shape(c, cands[i].nw, cands[i].lpn, cands[i].cps);
    float ms = 0.0f;
    // untimed pass (first launch of this shape), then the timed one
    for (int pass = 0; pass < 2 && rc == ACAT_OK; pass++) {
      if (cudaMemcpyAsync(trial, u_dev, sb, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
          cudaEventRecord(e0, st) != cudaSuccess) {
        rc = ACAT_ERR_CUDA;
        break;
      }
      rc = acat_run(c, trial, steps, -1.0, stream, nullptr);
      if (rc == ACAT_OK && (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                            cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
        rc = ACAT_ERR_CUDA;
    }
    if (rc == ACAT_OK && (best_ms == 0.0f || ms < best_ms)) {
      best_ms = ms;
      best = cands[i];
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (cudaStreamSynchronize(st) != cudaSuccess && rc == ACAT_OK) rc = ACAT_ERR_CUDA;
  if (c->chain) {  // captured on the trial buffer
    cudaGraphExecDestroy(c->chain);
    c->chain = nullptr;
  }
  cudaFree(trial);
  if (rc != ACAT_OK) {
    if (old.nw) acat_set_launch_shape(c, old.nw, old.lpn, old.cps);
    return rc;
  }
  rc = acat_set_launch_shape(c, best.nw, best.lpn, best.cps);
  if (rc) return rc;
  return acat_launch_shape(c, nw_out, lpn_out, cps_out);
}

int acat_destroy(acat_ctx *c) {
  if (!c) return ACAT_ERR_INVALID_ARG;
  cudaDeviceSynchronize();
  if (c->chain) cudaGraphExecDestroy(c->chain);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  cudaFree(c->d_smax);
  cudaFree(c->d_t);
  cudaFree(c->d_status);
  cudaFree(c->d_work);
  cudaFree(c->d_host_stage);
  cudaFree(c->d_offs);
  cudaFree(c->d_tiles);
  cudaFree(c->d_smaxb);
  cudaFree(c->d_tb);
  cudaFree(c->d_lamb);
  cudaFree(c->d_lambf);
  cudaFree(c->d_next);
  cudaFree(c->d_contrib);
  cudaFree(c->d_seg);
  cudaFree(c->d_bar);
  cudaFree(c->d_flux);
  cudaFree(c->d_cnt);
  delete c;
  return ACAT_OK;
}

int64_t acat_state_bytes(const acat_ctx *c) {
  if (!c) return ACAT_ERR_INVALID_ARG;
  const int64_t n = (int64_t)c->s * c->cells;
  return c->p.precision == ACAT_PREC_F64 ? n * 8 : n * 8;  // FP32: hi + lo floats
}

int acat_step(acat_ctx *c, const void *u_in, void *u_out, double dt, void *stream, double *dt_dev,
              int8_t *orders_dev) {
  if (!c || !u_in || !u_out || u_in == u_out) return ACAT_ERR_INVALID_ARG;
  if (!(dt > 0.0) && dt != dt) return ACAT_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (c->batched) {
    Step1DArgs a = base_args(c);
    a.u_in = u_in;
    a.u_out = u_out;
    a.slot = 0;
    BatchArgs bt = batch_args(c);
    bt.dt_out = dt_dev;
    bt.orders = orders_dev;
    if (cudaMemsetAsync(c->d_smaxb, 0, 3 * (size_t)c->B * sizeof(unsigned long long), st) != cudaSuccess)
      return ACAT_ERR_CUDA;
    if (dt > 0.0) {
      a.dt_fixed = dt;
      if (cudaMemsetAsync(c->d_tb, 0, 3 * (size_t)c->B * sizeof(double), st) != cudaSuccess)
        return ACAT_ERR_CUDA;
    } else {
      if (acat_launch_smax_batch(c->p.flux, c->p.precision, a, bt, st)) return ACAT_ERR_CUDA;
      c->launches++;
    }
    int e3 = acat_launch_batch1d(c->p.P, c->p.flux, c->p.precision, a, bt, st);
    c->launches += ACAT_BATCH_LAUNCHES_PER_STEP;
    return e3 ? ACAT_ERR_CUDA : ACAT_OK;
  }
  if (c->dim == 2) {
    Step2DArgs a = base_args2(c);
    a.u_in = u_in;
    a.u_out = u_out;
    a.slot = 0;
    a.dt_out = dt_dev;
    if (orders_dev) {
      a.ord_x = orders_dev;
      a.ord_y = orders_dev + (long)c->p.ny * (c->p.nx + 1);
    }
    if (cudaMemsetAsync(c->d_smax, 0, 6 * sizeof(unsigned long long), st) != cudaSuccess)
      return ACAT_ERR_CUDA;
    if (dt > 0.0) {
      a.dt_fixed = dt;
    } else {
      if (acat_launch_smax2d(c->p.flux, c->p.precision, a, st)) return ACAT_ERR_CUDA;
      c->launches++;
    }
    int e2 = acat_launch_step2d(c->p.P, c->p.flux, c->p.precision, a, st);
    c->launches++;
    return e2 ? ACAT_ERR_CUDA : ACAT_OK;
  }
  Step1DArgs a = base_args(c);
  a.u_in = u_in;
  a.u_out = u_out;
  a.slot = 0;
  a.orders = orders_dev;
  a.dt_out = dt_dev;
  cudaError_t e = cudaMemsetAsync(c->d_smax, 0, 6 * sizeof(unsigned long long), st);
  if (e != cudaSuccess) return ACAT_ERR_CUDA;
  if (dt > 0.0) {
    a.dt_fixed = dt;
  } else {
    if (acat_launch_smax1d(c->p.flux, c->p.precision, a, st)) return ACAT_ERR_CUDA;
    c->launches++;
  }
  return launch_step(c, a, st);
}

int acat_run(acat_ctx *c, void *u, int nsteps, double t_end, void *stream, double *t_dev) {
  if (!c || !u || nsteps < 0) return ACAT_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (t_end != t_end) return ACAT_ERR_INVALID_ARG;
  if (cudaMemsetAsync(c->d_smax, 0, 6 * sizeof(unsigned long long), st) != cudaSuccess)
    return ACAT_ERR_CUDA;
  if (c->batched) {
    Step1DArgs a = base_args(c);
    a.u_in = u;
    a.slot = 0;
    BatchArgs bt = batch_args(c);
    if (cudaMemsetAsync(c->d_smaxb, 0, 3 * (size_t)c->B * sizeof(unsigned long long), st) != cudaSuccess)
      return ACAT_ERR_CUDA;
    if (acat_launch_smax_batch(c->p.flux, c->p.precision, a, bt, st)) return ACAT_ERR_CUDA;
  } else if (c->dim == 2) {
    Step2DArgs a = base_args2(c);
    a.u_in = u;
    a.slot = 0;
    a.tslot = c->d_t;
    if (acat_launch_smax2d(c->p.flux, c->p.precision, a, st)) return ACAT_ERR_CUDA;
  } else {
    Step1DArgs a = base_args(c);
    a.u_in = u;
    a.slot = 0;
    a.tslot = c->d_t;
    if (acat_launch_smax1d(c->p.flux, c->p.precision, a, st)) return ACAT_ERR_CUDA;
  }
  c->launches++;
  long n = 0;
  const int chunks = nsteps / GRAPH_STEPS;
  if (chunks > 0) {
    int rc = ensure_chain(c, u, t_end);
    if (rc) return rc;
    for (int k = 0; k < chunks; k++) {
      if (cudaGraphLaunch(c->chain, st) != cudaSuccess) return ACAT_ERR_CUDA;
      c->launches += GRAPH_STEPS;
    }
    n = (long)chunks * GRAPH_STEPS;
  }
  int rc = issue_steps(c, u, n, nsteps - (int)n, t_end, st);
  if (rc) return rc;
  if (nsteps % 2 == 1) {
    if (cudaMemcpyAsync(u, c->d_work, (size_t)acat_state_bytes(c), cudaMemcpyDeviceToDevice, st) !=
        cudaSuccess)
      return ACAT_ERR_CUDA;
  }
  if (t_dev) {
    const double *src = c->batched ? c->d_tb + (size_t)(nsteps % 3) * c->B : c->d_t + (nsteps % 3);
    const size_t nb = (c->batched ? (size_t)c->B : 1) * sizeof(double);
    if (cudaMemcpyAsync(t_dev, src, nb, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
      return ACAT_ERR_CUDA;
  }
  return ACAT_OK;
}

int acat_run_host(acat_ctx *c, const void *u_host_in, void *u_host_out, int nsteps, double t_end,
                  void *stream, double *t_host) {
  if (!c || !u_host_in || !u_host_out) return ACAT_ERR_INVALID_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t sb = (size_t)acat_state_bytes(c);
  const size_t nt = c->batched ? (size_t)c->B : 1;  // time values returned
  if (!c->d_host_stage) {
    cudaError_t e = cudaMalloc(&c->d_host_stage, sb + nt * sizeof(double));
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? ACAT_ERR_NOMEM : ACAT_ERR_CUDA;
  }
  double *d_tfin = reinterpret_cast<double *>(static_cast<char *>(c->d_host_stage) + sb);
  if (cudaMemcpyAsync(c->d_host_stage, u_host_in, sb, cudaMemcpyHostToDevice, st) != cudaSuccess)
    return ACAT_ERR_CUDA;
  int rc = acat_run(c, c->d_host_stage, nsteps, t_end, stream, d_tfin);
  if (rc) return rc;
  if (cudaMemcpyAsync(u_host_out, c->d_host_stage, sb, cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return ACAT_ERR_CUDA;
  if (t_host && cudaMemcpyAsync(t_host, d_tfin, nt * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return ACAT_ERR_CUDA;
  return cuda_err(cudaStreamSynchronize(st));
}

namespace {

int ensure_contrib(acat_ctx *c) {
  if (c->d_contrib) return ACAT_OK;
  const size_t n = (size_t)(c->p.nx + 1) * (size_t)acat_adjoint_slots(c->p.P) * (size_t)c->s;
  cudaError_t e = cudaMalloc(&c->d_contrib, n * sizeof(double));
  if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? ACAT_ERR_NOMEM : ACAT_ERR_CUDA;
  return ACAT_OK;
}

int adjoint_launch(acat_ctx *c, const void *u_n, double dt, const double *dt_dev, const void *ubar1,
                   void *ubar0, cudaStream_t st) {
  Step1DArgs a = base_args(c);
  a.u_in = u_n;
  a.dt_fixed = dt;
  a.dt_in = dt_dev;
  int e = acat_launch_adjoint1d(c->p.P, c->p.flux, c->p.precision, a, ubar1, c->d_contrib, ubar0, st);
  c->launches += 2;
  return e ? ACAT_ERR_CUDA : ACAT_OK;
}

bool adjoint_ctx(const acat_ctx *c) { return c->dim == 1 && !c->batched; }

}  // namespace

int acat_adjoint_step(acat_ctx *c, const void *u_n, double dt, const void *ubar_np1, void *ubar_n,
                      void *stream) {
  if (!c || !u_n || !ubar_np1 || !ubar_n || ubar_np1 == ubar_n) return ACAT_ERR_INVALID_ARG;
  if (!(dt > 0.0) || !std::isfinite(dt)) return ACAT_ERR_INVALID_ARG;
  if (!adjoint_ctx(c)) return ACAT_ERR_UNSUPPORTED;
  int rc = ensure_contrib(c);
  if (rc) return rc;
  return adjoint_launch(c, u_n, dt, nullptr, ubar_np1, ubar_n, static_cast<cudaStream_t>(stream));
}

int acat_run_record(acat_ctx *c, const void *u0, void *u_out, int nsteps, int every, void *ckpt,
                    double *dts, void *stream) {
  if (!c || !u0 || !u_out || u0 == u_out || nsteps < 0 || every < 1) return ACAT_ERR_INVALID_ARG;
  if (nsteps > 0 && (!ckpt || !dts)) return ACAT_ERR_INVALID_ARG;
  if (!adjoint_ctx(c)) return ACAT_ERR_UNSUPPORTED;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t sb = (size_t)acat_state_bytes(c);
  if (cudaMemsetAsync(c->d_smax, 0, 6 * sizeof(unsigned long long), st) != cudaSuccess) return ACAT_ERR_CUDA;
  Step1DArgs a = base_args(c);
  a.tslot = c->d_t;
  a.u_in = u0;
  a.slot = 0;
  if (acat_launch_smax1d(c->p.flux, c->p.precision, a, st)) return ACAT_ERR_CUDA;
  c->launches++;
  const void *cur = u0;
  for (long n = 0; n < nsteps; n++) {
    if (n % every == 0 &&
        cudaMemcpyAsync(static_cast<char *>(ckpt) + (size_t)(n / every) * sb, cur, sb, cudaMemcpyDeviceToDevice,
                        st) != cudaSuccess)
      return ACAT_ERR_CUDA;
    void *nxt = (cur == u_out) ? c->d_work : u_out;
    a.u_in = cur;
    a.u_out = nxt;
    a.slot = (int)(n % 3);
    a.dt_out = dts + n;
    int rc = launch_step(c, a, st);
    if (rc) return rc;
    cur = nxt;
  }
  if (cur != u_out && cudaMemcpyAsync(u_out, cur, sb, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return ACAT_ERR_CUDA;
  return ACAT_OK;
}

int acat_adjoint_run(acat_ctx *c, const void *ckpt, const double *dts, int nsteps, int every, const void *ubar_n,
                     void *ubar_0, void *stream) {
  if (!c || !ubar_n || !ubar_0 || nsteps < 0 || every < 1) return ACAT_ERR_INVALID_ARG;
  if (nsteps > 0 && (!ckpt || !dts)) return ACAT_ERR_INVALID_ARG;
  if (!adjoint_ctx(c)) return ACAT_ERR_UNSUPPORTED;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t sb = (size_t)acat_state_bytes(c);
  int rc = ensure_contrib(c);
  if (rc) return rc;
  const size_t need = (size_t)(every - 1) * sb;
  if (need > c->seg_bytes) {
    if (c->d_seg && cudaStreamSynchronize(st) != cudaSuccess) return ACAT_ERR_CUDA;
    cudaFree(c->d_seg);
    c->d_seg = nullptr;
    c->seg_bytes = 0;
    cudaError_t e = cudaMalloc(&c->d_seg, need);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? ACAT_ERR_NOMEM : ACAT_ERR_CUDA;
    c->seg_bytes = need;
  }
  if (!c->d_bar) {
    cudaError_t e = cudaMalloc(&c->d_bar, sb);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? ACAT_ERR_NOMEM : ACAT_ERR_CUDA;
  }
  if (ubar_n != ubar_0 && cudaMemcpyAsync(ubar_0, ubar_n, sb, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return ACAT_ERR_CUDA;
  // the cotangent lives in ubar_0 between steps, d_bar takes the odd copies
  void *cur = ubar_0;
  Step1DArgs a = base_args(c);
  const int nseg = (nsteps + every - 1) / every;
  for (int seg = nseg - 1; seg >= 0; seg--) {
    const long start = (long)seg * every;
    const long end = std::min((long)nsteps, start + every);
    const char *base = static_cast<const char *>(ckpt) + (size_t)seg * sb;
    auto state = [&](long n) -> const void * {
      return n == start ? static_cast<const void *>(base)
                        : static_cast<const void *>(static_cast<char *>(c->d_seg) + (size_t)(n - start - 1) * sb);
    };
    for (long n = start; n < end - 1; n++) {
      a.u_in = state(n);
      a.u_out = const_cast<void *>(state(n + 1));
      a.slot = 0;
      a.dt_in = dts + n;
      rc = launch_step(c, a, st);
      if (rc) return rc;
    }
    for (long n = end - 1; n >= start; n--) {
      void *nxt = (cur == ubar_0) ? c->d_bar : ubar_0;
      rc = adjoint_launch(c, state(n), -1.0, dts + n, cur, nxt, st);
      if (rc) return rc;
      cur = nxt;
    }
  }
  if (cur != ubar_0 && cudaMemcpyAsync(ubar_0, cur, sb, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return ACAT_ERR_CUDA;
  return ACAT_OK;
}

int acat_status(acat_ctx *c, unsigned *flags) {
  if (!c) return ACAT_ERR_INVALID_ARG;
  unsigned f = 0;
  if (cudaDeviceSynchronize() != cudaSuccess) return ACAT_ERR_CUDA;
  if (cudaMemcpy(&f, c->d_status, sizeof f, cudaMemcpyDeviceToHost) != cudaSuccess) return ACAT_ERR_CUDA;
  if (flags) *flags = f;
  return f ? ACAT_ERR_NONPHYSICAL : ACAT_OK;
}

int acat_clear_status(acat_ctx *c) {
  if (!c) return ACAT_ERR_INVALID_ARG;
  return cuda_err(cudaMemset(c->d_status, 0, sizeof(unsigned)));
}

const char *acat_strerror(int code) {
  switch (code) {
  case ACAT_OK: return "ok";
  case ACAT_ERR_INVALID_ARG: return "invalid argument";
  case ACAT_ERR_CUDA: return "CUDA runtime error";
  case ACAT_ERR_NOMEM: return "out of device memory";
  case ACAT_ERR_NONPHYSICAL: return "non-physical state or bad time step detected on the device";
  case ACAT_ERR_UNSUPPORTED: return "configuration not supported";
  case ACAT_ERR_TOO_LARGE: return "size exceeds the supported maximum";
  }
  return "unknown error";
}

int64_t acat_launch_count(const acat_ctx *c) { return c ? c->launches : -1; }

double acat_measure_fma_peak(int precision, void *stream) {
  if (precision != 0 && precision != 1) return -1.0;
  return acat_fma_peak_run(precision, stream);
}

}  // extern "C"
