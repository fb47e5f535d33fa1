// acat_internal.h -- declarations shared by the translation units of libacat.
#pragma once

#include <cstdint>

#define ACAT_MAXP 4
#define ACAT_MAXN 8

// Differentiation-weight tables (built on the host in exact arithmetic by
// weights.cpp, kept in __constant__ memory on each device). Index p is the
// half-width, node and time-level indices r run over 0..2p-1 for the offsets
// r - p + 1.
struct AcatTables {
  double g1[ACAT_MAXP + 1][ACAT_MAXN][ACAT_MAXN];      // gamma^{1,j}_{p,r}   [p][j][r]
  double gk[ACAT_MAXP + 1][ACAT_MAXN][ACAT_MAXN];      // gamma^{k,0}_{p,r}   [p][k][r]
  double gh[ACAT_MAXP + 1][ACAT_MAXN];                 // flux weights, Eq. 2.14
  double gd[ACAT_MAXP + 1][ACAT_MAXN];                 // gamma^{2p-1,1/2}, binomial
  double taylor[ACAT_MAXP + 1][ACAT_MAXN][ACAT_MAXN];  // r^l / l!            [p][r][l]
  double fact[ACAT_MAXP + 1];                          // (2p-1)!
  double invfact[ACAT_MAXN + 1];                       // 1 / k!
  // the same weights rounded to float, for the FP32 recursion
  float g1f[ACAT_MAXP + 1][ACAT_MAXN][ACAT_MAXN];
  float gkf[ACAT_MAXP + 1][ACAT_MAXN][ACAT_MAXN];
  float ghf[ACAT_MAXP + 1][ACAT_MAXN];
  float taylorf[ACAT_MAXP + 1][ACAT_MAXN][ACAT_MAXN];
  float invfactf[ACAT_MAXN + 1];
};

void acat_build_tables(AcatTables *T);

// Arguments of one 1D step launch (passed by value).
struct Step1DArgs {
  const void *u_in;           // FP64: double[s][N]; FP32: float hi[s][N], lo[s][N]
  void *u_out;
  int N;                      // cells
  int bc;                     // ACAT_BC_*
  int limiter_form;
  int psi2_mod;               // 1: psi~^2 in place of psi^2
  int lo_flux;                // F^lo: ACAT_LO_*
  int slot;                   // step index mod 3 (dt-reduction slots)
  int lpn;                    // FP32 1D: lanes per stencil node (1, or 2 for P = 2, 4)
  int nw;                     // FP32 1D fused step: warps per CTA (8, or 7; 0 reads as 8)
  double dx, cfl;
  double dt_fixed;            // > 0: imposed dt
  const double *dt_in;        // device: imposed dt (nullable; takes precedence)
  double t_end;               // > 0: clip t at t_end
  double gamma, adv, eps, thr;
  double fact_tau[ACAT_MAXP + 1];
  float epsf, rf;             // float eps and thr / (1 - thr) of the filtered decision
  float factf[ACAT_MAXP + 1];
  float advf, gammaf, gm1f;   // adv, gamma, gamma - 1 rounded to float (FP32 path)
  unsigned long long *smax;   // 3 slots: max wave speed as ordered double bits
  double *tslot;              // 3 slots: simulated time (nullable)
  int8_t *orders;             // N+1 order codes (nullable)
  double *dt_out;             // dt used (nullable)
  unsigned *status;           // sticky status bits
  double *flux_buf;           // FP64 single instance: [S][N+1] CTA-edge fluxes, and
  int *cnt;                   // one hand-off counter per CTA boundary (both nullable: the
                              // fused 8-warp step kernel runs instead of the small-CTA one)
};

// Work description of a batch of independent 1D instances (ragged sizes),
// concatenated along the cell index: u[c][M] with instance b at cells
// offs[b]..offs[b+1]-1.
struct TileRef {
  int b;     // instance
  int tile;  // tile index within the instance (first cell tile * T)
};
struct BatchArgs {
  const long long *offs;      // B+1 cell offsets
  const TileRef *tiles;       // work list
  long long ntiles;
  int B;
  long long M;                // total cells (component stride)
  double xlen;                // x1 - x0 (each instance spans the domain)
  unsigned long long *smax;   // 3 x B wave-speed slots
  double *t;                  // 3 x B time slots
  double *dt_out;             // B (nullable)
  double *lam;                // B: dt / dx of each instance for this step (k_batch_dt)
  float *lamf;                // B: the same rounded to float (FP32 path)
  int *next;                  // tile queue of the step kernel (k_batch_dt sets it to 0)
  int8_t *orders;             // M + B order codes (nullable), instance b at offs[b] + b
  int nw;                     // warps per CTA (4, 8 or 16); tiles of acat_cells_per_tile_1d(P, prec, nw, lpn) cells
  int cps;                    // CTAs per SM (<= 0: the kernel's occupancy)
  int lpn;                    // lanes per stencil node (1; FP32 with P = 2, 4: 1 or 2)
};

// One batched step: the per-instance dt kernel, then the step kernel (two
// launches; returns 0 or a cudaError_t value).
int acat_launch_batch1d(int P, int flux, int prec, const Step1DArgs &a, const BatchArgs &bt,
                        void *stream);
constexpr int ACAT_BATCH_LAUNCHES_PER_STEP = 2;
// Cells per tile of the batched kernel of precision prec with nw warps per
// CTA and lpn lanes per stencil node (0: unsupported).
int acat_cells_per_tile_1d(int P, int prec, int nw, int lpn);
// Resident CTAs per SM of the batched kernel with nw warps and lpn lanes per
// node (-1: unsupported shape).
int acat_batch_occupancy(int P, int flux, int prec, int nw, int lpn);

int acat_launch_smax_batch(int flux, int prec, const Step1DArgs &a, const BatchArgs &bt, void *stream);

// Arguments of one 2D step launch (passed by value). State u[c][y][x].
struct Step2DArgs {
  const void *u_in;
  void *u_out;
  int NX, NY;
  int bc;
  int limiter_form;
  int psi2_mod;
  int lo_flux;
  int rect_2d;                // 1: rectangular blocks S_{p1,p2} (FP64, high-order kernel)
  int slot;                   // step index mod 3
  double dx, dy, cfl;
  double dt_fixed, t_end;
  double gamma, adv[2], eps, thr;
  double fact_tau[ACAT_MAXP + 1];
  float epsf, rf;
  float factf[ACAT_MAXP + 1];
  float advf[2], gammaf, gm1f;  // adv, gamma, gamma - 1 rounded to float (FP32 path)
  unsigned long long *smax;   // 3 slots x 2 directions: [slot][dir]
  double *tslot;              // 3 slots (nullable)
  int8_t *ord_x;              // NY x (NX+1) (nullable)
  int8_t *ord_y;              // (NY+1) x NX (nullable)
  double *dt_out;
  unsigned *status;
};

int acat_launch_step2d(int P, int flux, int prec, const Step2DArgs &a, void *stream);
int acat_launch_smax2d(int flux, int prec, const Step2DArgs &a, void *stream);
int acat_upload_tables_1d(const AcatTables *T);
int acat_upload_tables_adj(const AcatTables *T);
int acat_upload_tables_batch(const AcatTables *T);
int acat_adjoint_slots(int P);
// Adjoint of one 1D step (a.u_in = u^n, dt from a.dt_in or a.dt_fixed): ubar0 from ubar1.
// FP64: double states and cotangents, double contrib; FP32: compensated float pairs, float contrib.
int acat_launch_adjoint1d(int P, int flux, int prec, const Step1DArgs &a, const void *ubar1, void *contrib,
                          void *ubar0, void *stream);
int acat_upload_tables_2d(const AcatTables *T);

// Initial wave-speed reduction into smax[slot] (and t = 0 into tslot[slot]).
int acat_launch_smax1d(int flux, int prec, const Step1DArgs &a, void *stream);
// One 1D step; returns 0 or a cudaError_t value.
int acat_launch_step1d(int P, int flux, int prec, const Step1DArgs &a, void *stream);
int acat_upload_tables_current_device();
// acat_upload_tables_current_device once per device (dev must be current);
// returns an acat error code.
int acat_ensure_tables(int dev);
int acat_cells_per_cta_1d(int P, int prec);
// CTAs of the small-CTA FP64 step (boundary counters it needs: that many).
int acat_fine_ctas_1d(int P, long N);
double acat_fma_peak_run(int precision, void *stream);
