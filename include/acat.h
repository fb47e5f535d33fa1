/*
 * acat.h -- C ABI of libacat, the GB300 (sm_103a) implementation of the
 * explicit time step of the Adaptive Compact Approximate Taylor (ACAT) method
 * of Carrillo, Macca, Pares, Russo and Zorio, "An order-adaptive compact
 * approximation Taylor method for systems of conservation laws"
 * (arXiv 2007.01416).
 *
 * One step (Sec. 3.3, Eq. 3.19; 2D: Sec. 4, Eq. 4.9) does, at every
 * interface x_{i+1/2}:
 *   - the smoothness indicators psi^p, p = 2..P, on the centred stencils S_p
 *     (Eqs. 3.8-3.12; systems: minimum over components, Sec. 3.4);
 *   - the order selection p_s = max A (Eqs. 3.2-3.3);
 *   - the CAT2p_s flux by the local Taylor recursion (Sec. 2.2, Eq. 2.14),
 *     or, when A is empty, the FL-CAT2 flux psi^1 F^CAT2 + (1-psi^1) F^lo with
 *     the superbee limiter (Eqs. 3.4-3.7) and a Rusanov F^lo;
 *   - the conservative update u_i += dt/dx (F_{i-1/2} - F_{i+1/2}) (Eq. 2.12);
 * with dt = CFL dx / s^max (1D) or CFL/2 min(dx/s^max_x, dy/s^max_y) (2D,
 * Sec. 5.5), s^max reduced on the device.
 *
 * Conventions
 *   - Every pointer named *_dev is a device pointer on the current device; the
 *     caller owns it. *_host pointers are host memory.
 *   - State layout, FP64: SoA doubles, 1D u[c][i] (c < s, i < nx),
 *     2D u[c][y][x]; s = 1 (linear, Burgers), 3 (Euler 1D), 4 (Euler 2D).
 *   - State layout, FP32 (ACAT_PREC_F32): a compensated pair of float SoA
 *     arrays, hi[s][...] followed by lo[s][...]; the represented value is
 *     hi + lo.
 *   - Interfaces, 1D: m = 0..nx, interface m between cells m-1 and m. 2D:
 *     x-interfaces [y][m] (m = 0..nx), y-interfaces [m][x] (m = 0..ny).
 *   - Order codes (int8): p_s in 2..P, or 1 when the FL-CAT2 flux was used.
 *   - `stream` is a cudaStream_t (NULL: the legacy default stream). All calls
 *     except acat_create, acat_destroy and acat_status are asynchronous on it.
 *   - The weight tables are uploaded to each device's constant memory once,
 *     by the first acat_create (or acat_run_noalloc) on that device. Do not use
 *     the library across a reset of the device (cudaDeviceReset): the tables
 *     would not be uploaded again.
 *   - Return values: ACAT_OK (0) or a negative ACAT_ERR_* code; no call
 *     throws. Errors the device detects (non-physical states, a bad dt) are
 *     recorded as sticky ACAT_STATUS_* bits, read by acat_status.
 */
#ifndef ACAT_H
#define ACAT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct acat_ctx acat_ctx; /* opaque, owned by the library */

enum { ACAT_FLUX_LINEAR = 0, ACAT_FLUX_BURGERS = 1, ACAT_FLUX_EULER1D = 2, ACAT_FLUX_EULER2D = 3 };
enum { ACAT_BC_PERIODIC = 0, ACAT_BC_TRANSMISSIVE = 1 };
enum { ACAT_PREC_F64 = 0, ACAT_PREC_F32 = 1 };
/* robust first-order flux F^lo of FL-CAT2 (Eq. 3.4 leaves it open) */
enum { ACAT_LO_RUSANOV = 0, ACAT_LO_GLOBAL_LF = 1, ACAT_LO_HLL = 2 };

enum {
  ACAT_OK = 0,
  ACAT_ERR_INVALID_ARG = -1,
  ACAT_ERR_CUDA = -2,
  ACAT_ERR_NOMEM = -3,
  ACAT_ERR_NONPHYSICAL = -4,
  ACAT_ERR_UNSUPPORTED = -5,
  ACAT_ERR_TOO_LARGE = -6
};

/* sticky device status bits */
enum {
  ACAT_STATUS_NONPHYSICAL = 1u, /* rho <= 0, p <= 0 or a non-finite state  */
  ACAT_STATUS_BAD_DT = 2u,      /* s^max not positive and finite           */
  ACAT_STATUS_BOUNDS = 4u       /* only in a library built with
                                   ACAT_BOUNDS_CHECK: a kernel computed a
                                   tile, shared-memory or global index
                                   outside its buffer and skipped the access */
};

/* Problem description in the terms of the paper.
 *   flux          ACAT_FLUX_*; Euler uses gamma (Sec. 5.3, 5.5), linear
 *                 transport uses adv[0] (x) and adv[1] (y) (Eqs. 5.1, 5.13).
 *   P             maximal half-width 1..4 (order up to 2P); P = 1 is FL-CAT2.
 *   nx, ny        cells; ny = 1 for 1D.
 *   x0..y1        domain; cell centres x_i = x0 + (i + 1/2) dx.
 *   bc            ACAT_BC_PERIODIC or ACAT_BC_TRANSMISSIVE (zero-gradient
 *                 ghost cells, the "outflow"/"free" conditions of Sec. 5).
 *   precision     ACAT_PREC_F64, or ACAT_PREC_F32 (float arithmetic on a
 *                 compensated float-pair state; the order decisions are
 *                 those of FP64 on the state value hi + lo).
 *   cfl           CFL number of the dt rule above.
 *   psi_tol       p is admissible when psi^p >= 1 - psi_tol (the paper's
 *                 "psi^p ~ 1", Eq. 3.2, has no threshold; default 0.1).
 *   eps           epsilon of the lateral weights (Eq. 3.8), default 1e-12.
 *   tau_factorial 1 (default): tau_p = ((2p-1)! Delta^{2p-1})^2 as printed
 *                 in Eq. 3.12; 0 drops the factorial.
 *   limiter_form  0 (default): Roe-speed side for scalar laws (Eq. 3.6),
 *                 min form for systems (Eq. 3.7); 1: min form everywhere.
 *   psi2_mod      1: the modified indicator psi~^2 of Sec. 3.2 (the larger of
 *                 the two lateral-weight splits that keep the central
 *                 difference) in place of psi^2; 0 (default): Eq. 3.12.
 *   lo_flux       F^lo of FL-CAT2: ACAT_LO_RUSANOV (default, local LF with
 *                 the larger spectral radius), ACAT_LO_GLOBAL_LF (alpha =
 *                 dx / dt), ACAT_LO_HLL (wave-speed bounds: the smaller of the
 *                 two states' smallest eigenvalues, the larger of their
 *                 largest).
 *   rect_2d       2D stencils (Sec. 4, end). 0 (default): the x-flux of order
 *                 2 p1 from the square block S_{p1}, the y-flux of order 2 p2
 *                 from S_{p2}. 1: both from one rectangular block S_{p1,p2} of
 *                 2 p1 x 2 p2 nodes per anchor (a direction on FL-CAT2 counts
 *                 as p = 1), x-derivatives over its rows, y-derivatives over
 *                 its columns, time derivatives on 2 max(p1, p2) time levels.
 *                 No effect in 1D. */
typedef struct {
  int flux;
  int P;
  int nx, ny;
  int bc;
  int precision;
  int tau_factorial;
  int limiter_form;
  int psi2_mod;
  int lo_flux;
  int rect_2d;
  double gamma;
  double adv[2];
  double cfl;
  double x0, x1, y0, y1;
  double psi_tol;
  double eps;
} acat_params;

/* Fills *p with the defaults above (gamma 1.4, CFL 0.5, psi_tol 0.1,
 * eps 1e-12, [0,1]^2, periodic, FP64, P = 2, Burgers, nx = 64, ny = 1). */
void acat_default_params(acat_params *p);

/* Validates *p, uploads the differentiation-weight tables (Eq. 2.10; the flux
 * weights of Eq. 2.14 are those that satisfy Eq. 2.11 at k = 1) to the
 * current device and allocates the context's device workspace (dt/time
 * slots, status word). Errors: INVALID_ARG (bad field, nx or ny < 2 max(P, 2),
 * P outside 1..4), UNSUPPORTED (2D with a flux other than Euler or linear
 * transport), TOO_LARGE, NOMEM, CUDA. */
int acat_create(const acat_params *p, acat_ctx **out);

/* A batch of n_inst independent 1D problems of ragged sizes n_per_inst[b]
 * (host array; each >= 2 max(P, 2)), all with the parameters *p (p->nx is
 * ignored) and each on the whole domain [x0, x1] with its own dx. The state
 * is the concatenation along the cell index, u[c][M] with M = sum n_b and
 * instance b at cells off_b = n_0 + ... + n_{b-1} (FP32: hi[c][M] then
 * lo[c][M]). Every step advances all instances in one persistent launch,
 * each with its own CFL dt reduced on the device (Eq. 2.12 per instance).
 * With a batched ctx: acat_step's dt_dev receives n_inst values and
 * orders_dev M + n_inst codes (instance b at off_b + b); acat_run's t_dev and
 * acat_run_host's t_host receive n_inst times. Errors as acat_create, plus
 * INVALID_ARG for a 2D problem or a too small instance. */
int acat_create_batched(const acat_params *p, int n_inst, const int32_t *n_per_inst, acat_ctx **out);

/* Launch shape of a 1D context's step kernel: warps per CTA (nw), lanes per
 * stencil node (lpn) and CTAs per SM (cps).
 *   - An interface is worked by a group of 2P x lpn lanes (Sec. 2.2: one
 *     lane per node of its stencil S_P, or two that split the node's sums of
 *     the recursion and its time levels). lpn = 2 exists for FP32 contexts
 *     with P = 2 or 4. The two forms group the recursion's sums differently,
 *     so they agree to float rounding (both within the FP32 parity bar), not
 *     bit for bit.
 *   - Batched contexts: the batch is cut into tiles of
 *     T = R nw floor(32 / (2P lpn)) - 1 consecutive cells of one instance,
 *     R = 8 interface rounds per lane group in FP32 (2 at nw = 16), 1 in
 *     FP64 (P = 3, nw = 8, lpn = 1: 319 in FP32, 39 in FP64); one CTA of nw
 *     warps per tile at a time,
 *     on a grid of (SM count) x cps CTAs that take the tiles from a queue
 *     (cps = 0: the kernel's occupancy). nw in {4, 8, 16}. At a fixed lpn,
 *     nw and cps only move work between CTAs: every interface flux, wave
 *     speed and update is computed from the same values, so the states are
 *     bit-identical.
 *   - Single-instance contexts: cps is 0. FP64: nw is fixed (8; 2 for the
 *     small-CTA step of large grids). FP32: nw = 8 (the fused step, lpn 1
 *     or 2), nw = 7 (the fused step in tiles of 7 floor(32 / 2P) - 1
 *     cells, lpn = 1: a grid of a few waves then fills every SM with the
 *     same number of CTAs) or nw = 2 (the small-CTA step with the boundary
 *     hand-off, lpn = 1); all compute every interface and cell from the
 *     same values, so at lpn = 1 they are bit-identical.
 * Defaults: nw = 8, lpn = 1, cps = 0; a single 1D FP32 instance starts with
 * nw = 7 where that leaves the busiest SM fewer warps of work
 * (ceil(ceil(N / T) / SMs) x nw against the same at nw = 8).
 * acat_launch_shape returns the current shape (cps resolved to a number for
 * a batch). acat_set_launch_shape sets one; for a batch, changing nw or lpn
 * rebuilds the tile list (a device allocation and a device synchronisation);
 * any change drops the captured step graph.
 * Errors: INVALID_ARG (a shape that does not exist, cps above the
 * occupancy), UNSUPPORTED (2D contexts; a single-instance nw or cps other
 * than its own, lpn on an FP64 single instance), NOMEM, CUDA. */
int acat_launch_shape(const acat_ctx *ctx, int *nw_out, int *lpn_out, int *cps_out);
int acat_set_launch_shape(acat_ctx *ctx, int nw, int lpn, int cps);

/* Autotuner of the launch shape (batched contexts, and single-instance 1D
 * FP32 contexts). Times `steps` steps (acat_run) from u_dev for every
 * candidate shape: batched: nw in {8, 4, 16} x lpn in {1, 2 where it exists}
 * x cps in {occupancy, occupancy / 2}; single FP32: (nw, lpn) in {(8, 1),
 * (8, 2) where it exists, (7, 1), (2, 1)}. Each candidate runs on a context-allocated copy of u_dev (u_dev is
 * only read), once untimed and once timed with CUDA events on `stream`. The
 * fastest shape is kept (acat_set_launch_shape) and returned in *nw_out,
 * *lpn_out, *cps_out (each nullable). Synchronises `stream` and the device;
 * must not be called during stream capture. Its launches count in
 * acat_launch_count.
 * Errors: INVALID_ARG, UNSUPPORTED (2D, or a single-instance FP64 context),
 * NOMEM, CUDA, with the previous shape restored. */
int acat_autotune(acat_ctx *ctx, const void *u_dev, int steps, void *stream, int *nw_out, int *lpn_out,
                  int *cps_out);

/* Frees every device and host resource of ctx (synchronises first). */
int acat_destroy(acat_ctx *ctx);

/* Size in bytes of one state buffer of ctx (s * cells * 8, or 2 * s *
 * cells * 4 in FP32). */
int64_t acat_state_bytes(const acat_ctx *ctx);

/* One ACAT step u_in -> u_out (device buffers, must not alias).
 *   dt > 0 imposes that time step; dt <= 0 computes the CFL time step of
 *   u_in on the device.
 *   dt_dev (nullable): receives the dt used (one double).
 *   orders_dev (nullable): receives the order codes, nx + 1 int8 (1D) or
 *   ny*(nx+1) + (ny+1)*nx (2D: x-interfaces then y-interfaces). */
int acat_step(acat_ctx *ctx, const void *u_in_dev, void *u_out_dev, double dt, void *stream,
              double *dt_dev, int8_t *orders_dev);

/* nsteps ACAT steps in place on u_dev, each with the CFL dt of its own
 * state, reduced on the device (dt never returns to the host). With
 * t_end > 0 the last step is clipped so that t stops at t_end and further
 * steps do nothing. The step sequence is replayed from CUDA graphs.
 * t_dev (nullable): receives the final time (one double). */
int acat_run(acat_ctx *ctx, void *u_dev, int nsteps, double t_end, void *stream, double *t_dev);

/* acat_run on host memory: copies u_host_in to the device, runs, copies the
 * result to u_host_out (may equal u_host_in), all on `stream`, and
 * synchronises it. Pinned host memory makes the copies asynchronous. */
int acat_run_host(acat_ctx *ctx, const void *u_host_in, void *u_host_out, int nsteps, double t_end,
                  void *stream, double *t_host);

/* Adjoint (transposed Jacobian) of one 1D step:
 *   ubar_n = (d u^{n+1} / d u^n)^T ubar_np1,
 * with u^{n+1} = step(u^n) taken with the time step dt (treated as a
 * constant: the dt the forward step used) and every discrete choice frozen as
 * the forward step takes it at u_n: the selected orders (Eqs. 3.2-3.3) and,
 * for FL-CAT2 interfaces (Eq. 3.4), the superbee piece, the upwind side or the
 * (component, side) of the limiter minimum, the Rusanov maximum, and for the
 * HLL F^lo its branch and the states that give its wave-speed bounds (the
 * global LF F^lo has alpha = dx / dt, a constant with dt). All else
 * -- the CAT2p recursion of Sec. 2.2, the limiter value inside its piece, the
 * Rusanov speed -- is differentiated. u_n, ubar_np1, ubar_n: device states
 * in the context's layout: FP64 [s][nx]; FP32 compensated pairs
 * [hi(s x nx); lo(s x nx)], the cotangents as compensated values too (the
 * FP32 reverse sweep runs in float, FL-CAT2 interfaces in FP64 on hi + lo).
 * ubar_n must not alias ubar_np1. Uses a context-owned scratch array
 * ((nx+1) x max(2P,4) x s doubles, allocated on first use).
 * Errors: INVALID_ARG, UNSUPPORTED (2D or batched contexts), NOMEM, CUDA. */
int acat_adjoint_step(acat_ctx *ctx, const void *u_n_dev, double dt, const void *ubar_np1_dev,
                      void *ubar_n_dev, void *stream);

/* Forward run that records what the reverse run needs (1D contexts).
 * Takes nsteps CFL steps (as acat_run, without t_end) from u0_dev, which is
 * not modified, and writes u^nsteps to u_out_dev.
 *   every >= 1: checkpoint interval; the state before step n, for every n
 *     with n % every == 0, goes to ckpt_dev + (n / every) * state_bytes, so
 *     ckpt_dev holds ceil(nsteps / every) states (caller-owned).
 *   dts_dev: nsteps doubles (caller-owned), receives the dt of each step.
 * u0_dev, u_out_dev and ckpt_dev must not overlap. Device memory beyond the
 * context's is not allocated. Errors: INVALID_ARG, UNSUPPORTED, CUDA. */
int acat_run_record(acat_ctx *ctx, const void *u0_dev, void *u_out_dev, int nsteps, int every,
                    void *ckpt_dev, double *dts_dev, void *stream);

/* Reverse run over a recorded forward run: ubar_0 = J_1^T ... J_nsteps^T
 * ubar_n, where J_k is the Jacobian of step k at the recorded dt with the
 * discrete choices frozen as in acat_adjoint_step. The states of each
 * checkpoint segment are recomputed from its checkpoint with the recorded dt
 * (bit-identical to the forward run) into a context-owned buffer of every-1
 * states, allocated on first use and grown on demand; then the adjoint steps
 * run in reverse. ckpt_dev, dts_dev, nsteps, every: as given to
 * acat_run_record. ubar_n_dev, ubar_0_dev: device cotangents in the state
 * layout of the context (as acat_adjoint_step); they may be the same buffer.
 * Errors: INVALID_ARG, UNSUPPORTED, NOMEM, CUDA. */
int acat_adjoint_run(acat_ctx *ctx, const void *ckpt_dev, const double *dts_dev, int nsteps, int every,
                     const void *ubar_n_dev, void *ubar_0_dev, void *stream);

/* Largest state, in bytes, that acat_run_noalloc accepts: 8 MiB, i.e.
 * 349525 cells of 1D Euler or 1048576 cells of a scalar law in FP64. */
#define ACAT_NOALLOC_MAX_STATE (8u << 20)

/* acat_run without a context and without any device allocation. The paper
 * has no counterpart: this entry point exists for callers that must not call
 * cudaMalloc, such as a host application that owns all device memory through
 * its own pool and forbids other allocations, a plugin loaded into one, or
 * code whose latency budget cannot absorb an allocation.
 *   p           the problem, as for acat_create (1D, FP64 only).
 *   u_dev       the state, advanced nsteps steps in place; its size
 *               (s * nx * 8 bytes) must not exceed ACAT_NOALLOC_MAX_STATE,
 *               else ACAT_ERR_TOO_LARGE is returned before any device work.
 *   t_end, t_dev  as for acat_run.
 *   status_dev  (nullable, device) receives the status bits of the run.
 * Scratch (dt and time slots, status word, the ping-pong work buffer) lives
 * in one static device array of 256 B + ACAT_NOALLOC_MAX_STATE inside the
 * library, held by every GPU that loads the library until the process exits.
 * The first call on a device uploads the weight tables (once per device,
 * shared with acat_create); make that call before any stream capture. Every
 * call asks the runtime for the array's device address, which allocates
 * nothing. All calls
 * share the array, and it keeps the last call's contents (its slots are
 * cleared at the start of each call). Calls that overlap on the GPU race on
 * it, so issue them on one stream. Steps are launched one by one (no graph).
 * Errors: as acat_create and acat_run, plus ACAT_ERR_TOO_LARGE. */
int acat_run_noalloc(const acat_params *p, void *u_dev, int nsteps, double t_end, void *stream,
                     double *t_dev, unsigned *status_dev);

/* Reads and returns the sticky device status bits (synchronises ctx's
 * work). Returns ACAT_ERR_NONPHYSICAL when any bit is set. */
int acat_status(acat_ctx *ctx, unsigned *flags_out);

/* Clears the sticky status bits. */
int acat_clear_status(acat_ctx *ctx);

/* Human-readable text of an ACAT_ERR_* code (static storage). */
const char *acat_strerror(int code);

/* Kernel launches issued by this context since creation (step kernels,
 * dt reductions and graph-replayed kernels each count one per launch). */
int64_t acat_launch_count(const acat_ctx *ctx);

/* Measured peak of the CUDA-core FMA pipe on the current device, in
 * FLOP/s (FMA = 2 flops): precision 0 FP64, 1 FP32. Runs a dependent-chain
 * FMA kernel that fills every SM; used as the roofline denominator of the
 * arithmetic-bound step. Returns a negative number on error. */
double acat_measure_fma_peak(int precision, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* ACAT_H */
