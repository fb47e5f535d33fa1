/*
 * acat_oracle.h -- public interface of the ACAT CPU oracle.
 *
 * TEST INFRASTRUCTURE. The oracle is a plain, slow FP64 restatement of the
 * Adaptive Compact Approximate Taylor (ACAT) method of Carrillo, Macca, Pares,
 * Russo and Zorio (arXiv 2007.01416). It exists to check the CUDA library and
 * shares no code, header, table or constant generator with it: only the test
 * suite, the package smoke check and the benchmark's CPU-baseline leg load it.
 *
 * Layout conventions (shared with nothing; the Python wrapper follows them):
 *   1D state  u[c*nx + i]            c = 0..s-1, i = 0..nx-1   (SoA)
 *   2D state  u[(c*ny + y)*nx + x]                               (SoA)
 *   1D interfaces m = 0..nx; interface m lies between cells m-1 and m.
 *   2D x-interfaces (m = 0..nx, y = 0..ny-1) stored at [y*(nx+1) + m];
 *      y-interfaces (x = 0..nx-1, m = 0..ny) stored at [m*nx + x].
 *   order codes: p_s in 2..P when the admissible set is non-empty, 1 when the
 *   FL-CAT2 flux was used (Sec. 3, Eq. 3.3).
 */
#ifndef ACAT_ORACLE_H
#define ACAT_ORACLE_H

#include <stdint.h>

#define OR_MAXP 4
#define OR_MAXN (2 * OR_MAXP)
#define OR_MAXS 4

enum { OR_LINEAR = 0, OR_BURGERS = 1, OR_EULER1D = 2, OR_EULER2D = 3 };
enum { OR_PERIODIC = 0, OR_TRANSMISSIVE = 1 };

typedef struct {
  int flux;          /* OR_LINEAR, OR_BURGERS, OR_EULER1D, OR_EULER2D          */
  int P;             /* maximal half-width, 1..4 (P = 1: FL-CAT2 only)          */
  int nx, ny;        /* cells; ny = 1 for 1D                                    */
  int bc;            /* OR_PERIODIC or OR_TRANSMISSIVE                          */
  int tau_factorial; /* 1: tau_p = ((2p-1)! Delta)^2 as printed in Eq. 3.12     */
  int limiter_form;  /* 0: Roe-speed side (Eq. 3.6) for scalar laws, min form
                        (Eq. 3.7) for systems; 1: min form everywhere          */
  int psi2_mod;      /* 1: the modified indicator psi~^2 of Sec. 3.2 (maximum of
                        the two lateral-weight splits that include the central
                        difference) in place of psi^2                          */
  int lo_flux;       /* robust first-order flux F^lo of Eq. 3.4: 0 Rusanov
                        (local LF), 1 global LF (alpha = dx / dt), 2 HLL        */
  int rect_2d;       /* 2D stencils: 0 square blocks S_{p1} for F and S_{p2}
                        for G; 1 one rectangular block S_{p1,p2} per anchor
                        (Sec. 4, end), with p = 1 for a direction on FL-CAT2  */
  double gamma;      /* ratio of specific heats (Euler)                         */
  double adv[2];     /* linear advection speeds a, b                            */
  double cfl;
  double x0, x1, y0, y1;
  double psi_tol;    /* p is admissible when psi^p >= 1 - psi_tol              */
  double eps;        /* epsilon of the lateral weights, Eq. 3.8                 */
} or_params;

int or_fornberg(int p, int k, double q, double *w);
int or_flux_weights(int p, double *w);
int or_nvars(const or_params *P);

void or_flux_x(const or_params *P, const double *u, double *f);
void or_flux_y(const or_params *P, const double *u, double *f);
void or_cell_flux_1d(const or_params *P, const double *u, double *f);

double or_dt_1d(const or_params *P, const double *u);
double or_dt_2d(const or_params *P, const double *u);

int or_cat_flux_1d(const or_params *P, int p, const double *us, double dt,
                   double dx, double *F);
int or_cat_flux_2d(const or_params *P, int p, const double *ub, double dt,
                   double dx, double dy, double *F, double *G);
int or_cat_flux_2d_rect(const or_params *P, int p1, int p2, const double *ub, double dt,
                        double dx, double dy, double *F, double *G);

int or_step_1d(const or_params *P, const double *u, double *u_out,
               double *dt_io, int8_t *orders, double *psi, double *flux);
int or_fluxes_1d_at(const or_params *P, const double *u, double dt, int n,
                    const int32_t *ifaces, double *F, int8_t *orders);
int or_step_1d_cells(const or_params *P, const double *u, double dt, int n,
                     const int32_t *cells, double *out);
int or_step_1d_z(const or_params *P, const double *u_re, const double *u_im,
                 double dt, double *out_re, double *out_im);

int or_step_2d(const or_params *P, const double *u, double *u_out,
               double *dt_io, int8_t *ord_x, int8_t *ord_y);
int or_step_2d_cells(const or_params *P, const double *u, double dt, int n,
                     const int32_t *cx, const int32_t *cy, double *out);

void or_set_threads(int n);
int or_get_threads(void);

#endif
