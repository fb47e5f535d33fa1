// noalloc.cu -- acat_run_noalloc: the 1D run for callers that must not
// allocate device memory.
//
// Some callers cannot call cudaMalloc: a host application that owns all
// device memory through its own pool and forbids other allocations, a plugin
// loaded into such an application, or code whose latency budget cannot absorb
// an allocation (which may synchronise the device). acat_create allocates a
// context (work buffer, dt slots, status word); this entry point instead takes
// the problem description directly and keeps all of its scratch in one
// file-scope device array of fixed size, so it never allocates.
//
// The scratch array: 256 bytes of slots (three wave-speed slots, three time
// slots, the status word) followed by a work buffer of ACAT_NOALLOC_MAX_STATE
// bytes for the ping-pong of the time loop. Every GPU that loads the library
// holds it until the process exits. All calls on a device share it and it keeps
// the last call's contents; the slots are cleared at the start of every call.
// Calls that overlap on the GPU (different streams, or several host threads)
// race on it: issue them on one stream.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>

#include "../../include/acat.h"
#include "acat_internal.h"

namespace {

constexpr size_t kSlotBytes = 256;
constexpr size_t kMaxState = (size_t)ACAT_NOALLOC_MAX_STATE;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kSlotBytes + kMaxState];

int nvars1d(int flux) { return flux == ACAT_FLUX_EULER1D ? 3 : 1; }

int validate(const acat_params *p) {
  if (!p) return ACAT_ERR_INVALID_ARG;
  if (p->P < 1 || p->P > ACAT_MAXP) return ACAT_ERR_INVALID_ARG;
  if (p->flux < ACAT_FLUX_LINEAR || p->flux > ACAT_FLUX_EULER2D) return ACAT_ERR_INVALID_ARG;
  if (p->bc != ACAT_BC_PERIODIC && p->bc != ACAT_BC_TRANSMISSIVE) return ACAT_ERR_INVALID_ARG;
  if (p->ny < 1 || p->nx < 2 * (p->P > 2 ? p->P : 2)) return ACAT_ERR_INVALID_ARG;
  if (!(p->cfl > 0.0) || !std::isfinite(p->cfl)) return ACAT_ERR_INVALID_ARG;
  if (!(p->x1 > p->x0)) return ACAT_ERR_INVALID_ARG;
  if (!(p->psi_tol >= 0.0 && p->psi_tol < 1.0)) return ACAT_ERR_INVALID_ARG;
  if (!(p->eps >= 0.0) || !std::isfinite(p->eps)) return ACAT_ERR_INVALID_ARG;
  if (p->psi2_mod != 0 && p->psi2_mod != 1) return ACAT_ERR_INVALID_ARG;
  if (p->lo_flux < ACAT_LO_RUSANOV || p->lo_flux > ACAT_LO_HLL) return ACAT_ERR_INVALID_ARG;
  if (p->rect_2d != 0 && p->rect_2d != 1) return ACAT_ERR_INVALID_ARG;
  if (p->flux == ACAT_FLUX_EULER1D && !(p->gamma > 1.0)) return ACAT_ERR_INVALID_ARG;
  if (p->ny != 1 || p->flux == ACAT_FLUX_EULER2D || p->precision != ACAT_PREC_F64)
    return ACAT_ERR_UNSUPPORTED;
  return ACAT_OK;
}

// With the device current: the weight tables in constant memory (uploaded
// once per device, shared with acat_create), then the device address of the
// scratch array, asked on every call so that no address outlives the context
// it was taken in.
int setup(int dev, unsigned char **ptr) {
  const int rc = acat_ensure_tables(dev);
  if (rc != ACAT_OK) return rc;
  void *addr = nullptr;
  if (cudaGetSymbolAddress(&addr, g_noalloc_scratch) != cudaSuccess || !addr) return ACAT_ERR_CUDA;
  *ptr = static_cast<unsigned char *>(addr);
  return ACAT_OK;
}

}  // namespace

extern "C" int acat_run_noalloc(const acat_params *p, void *u_dev, int nsteps, double t_end,
                                void *stream, double *t_dev, unsigned *status_dev) {
  int rc = validate(p);
  if (rc) return rc;
  if (!u_dev || nsteps < 0 || t_end != t_end) return ACAT_ERR_INVALID_ARG;
  const size_t bytes = (size_t)nvars1d(p->flux) * (size_t)p->nx * sizeof(double);
  if (bytes > kMaxState) return ACAT_ERR_TOO_LARGE;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return ACAT_ERR_CUDA;
  unsigned char *base = nullptr;
  rc = setup(dev, &base);
  if (rc) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  unsigned long long *smax = reinterpret_cast<unsigned long long *>(base);
  double *tslot = reinterpret_cast<double *>(base + 32);
  unsigned *status = reinterpret_cast<unsigned *>(base + 64);
  void *work = base + kSlotBytes;
  if (cudaMemsetAsync(base, 0, kSlotBytes, st) != cudaSuccess) return ACAT_ERR_CUDA;

  AcatTables T;
  acat_build_tables(&T);
  Step1DArgs a;
  std::memset(&a, 0, sizeof a);
  a.N = p->nx;
  a.lpn = 1;
  a.bc = p->bc;
  a.limiter_form = p->limiter_form;
  a.psi2_mod = p->psi2_mod;
  a.lo_flux = p->lo_flux;
  a.dx = (p->x1 - p->x0) / (double)p->nx;
  a.cfl = p->cfl;
  a.dt_fixed = -1.0;
  a.t_end = t_end;
  a.gamma = p->gamma;
  a.adv = p->adv[0];
  a.eps = p->eps;
  a.thr = 1.0 - p->psi_tol;
  for (int q = 0; q <= ACAT_MAXP; q++) {
    a.fact_tau[q] = p->tau_factorial ? T.fact[q] : 1.0;
    a.factf[q] = (float)a.fact_tau[q];
  }
  a.epsf = (float)p->eps;
  a.rf = (float)(a.thr / (1.0 - a.thr));
  a.advf = (float)p->adv[0];
  a.gammaf = (float)p->gamma;
  a.gm1f = (float)(p->gamma - 1.0);
  a.smax = smax;
  a.tslot = tslot;
  a.status = status;

  a.u_in = u_dev;
  a.slot = 0;
  if (acat_launch_smax1d(p->flux, p->precision, a, st)) return ACAT_ERR_CUDA;
  for (long n = 0; n < nsteps; n++) {
    a.u_in = (n % 2 == 0) ? u_dev : work;
    a.u_out = (n % 2 == 0) ? work : u_dev;
    a.slot = (int)(n % 3);
    if (acat_launch_step1d(p->P, p->flux, p->precision, a, st)) return ACAT_ERR_CUDA;
  }
  if (nsteps % 2 == 1 && cudaMemcpyAsync(u_dev, work, bytes, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return ACAT_ERR_CUDA;
  if (t_dev && cudaMemcpyAsync(t_dev, tslot + (nsteps % 3), sizeof(double), cudaMemcpyDeviceToDevice,
                               st) != cudaSuccess)
    return ACAT_ERR_CUDA;
  if (status_dev &&
      cudaMemcpyAsync(status_dev, status, sizeof(unsigned), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return ACAT_ERR_CUDA;
  return ACAT_OK;
}
