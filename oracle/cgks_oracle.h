/*
 * CGKS-5 CPU oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow FP64 implementation of the per-stage sweep of the fifth-order
 * compact gas-kinetic scheme (reconstruction on the standard reference cell
 * with the GENO blend, the GKS time-dependent interface flux at Gauss points,
 * and the two-stage fourth-order update of averages, gradients and line
 * derivatives).  Only the test-suite, the smoke check and the CPU-baseline leg
 * of the benchmark may load it; the product path never does.  It shares no
 * code, headers or tables with the CUDA library.
 *
 * State layout (same as the library's public layout): SoA
 *   state[(f * nv + v) * ncell + cell],  cell = i + nx*(j + ny*k)
 * with f = 0 the cell average, f = 1..dim the cell-averaged gradient
 * (physical coordinates) and f = 1+dim.. the line-averaged derivatives
 * (difference of the two paired face Gauss-point values divided by the
 * physical distance between them), line s = axis*gpf + k.
 */
#ifndef CGKS_ORACLE_H
#define CGKS_ORACLE_H
#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int dim;            /* 2 or 3 */
  int n[3];           /* cells per axis (n[2] ignored for dim 2) */
  const double* nodes;/* (n0+1)(n1+1)(n2+1)*dim node coordinates, i fastest; NULL = uniform box */
  double lo[3], hi[3];/* box used when nodes == NULL */
  double gamma;       /* specific heat ratio */
  double mu;          /* dynamic viscosity (0 = inviscid) */
  double prandtl;     /* Prandtl number (heat-flux correction when mu > 0) */
  int tau_mode;       /* 0: tau = 0; 1: inviscid shock-capturing tau; 2: viscous tau */
  double cfl;         /* CFL number */
  double dt_fixed;    /* > 0: use this time step instead of the CFL rule */
  int linear;         /* 1: force chi = 1 (linear CGKS-5) */
  double c_chi;       /* path-function constant C in chi = tanh(C alpha)/tanh(C) */
  int bc[6];          /* per domain face -x,+x,-y,+y,-z,+z: 0 periodic, 1 outflow,
                         2 slip wall, 3 no-slip wall (walls: axis-aligned meshes),
                         4 inflow (a fixed state) */
  double bc_state[6][5]; /* inflow faces: conservative state (rho, m..., rho E) */
} orc_desc;

typedef struct orc_ctx orc_ctx;

orc_ctx* orc_create(const orc_desc* d);
void orc_destroy(orc_ctx* c);
int orc_nfields(const orc_ctx* c);
long orc_ncells(const orc_ctx* c);
int orc_set_state(orc_ctx* c, const double* s, double t);
int orc_get_state(const orc_ctx* c, double* s, double* t);
/* initial data: the points at which primitive values (rho, U, V[, W], p) are needed */
long orc_num_init_points(const orc_ctx* c);
void orc_init_points(const orc_ctx* c, double* pts);          /* npts*dim */
int orc_init_from_prims(orc_ctx* c, const double* prim);       /* npts*nv */
double orc_compute_dt(orc_ctx* c);
/* threads of the OpenMP loops from now on (n <= 0: unchanged); returns the
   number in use.  Results do not depend on it. */
int orc_set_threads(int n);
int orc_step(orc_ctx* c, int nsteps, double* dt_last);
/* one step with a given time step */
int orc_step_dt(orc_ctx* c, double dt);
/* cell-wise chi of the first stage of the last step, [v][cell] */
int orc_get_chi(const orc_ctx* c, double* chi);
long orc_positivity_fallbacks(const orc_ctx* c);

/* learned troubled-cell selector (not in the paper; reference for the
   library's fused selector): params = SEL_NPARAM floats (W1[32][16] b1
   W2[32][32] b2 W3[32][32] b3 w4[32] b4), NULL switches it off; a cell whose
   BF16-emulated logit reaches thr_skip takes chi = 1 for every variable */
int orc_set_selector(orc_ctx* c, const float* params, float thr_skip, float thr_lo);
int orc_selector_stats(const orc_ctx* c, long* nskip, long* nunsure, double* margin);
int orc_selector_features(const orc_ctx* c, float* out);
int orc_selector_logits(const float* params, const float* feat, long n, float* out);
int orc_selector_nparam(void);
/* metric quantities: volume per cell and sum over faces of the area vectors */
int orc_get_metrics(const orc_ctx* c, double* vol, double* closure /* ncell*dim */);

/* ---- unit-level entry points used by the pins ---- */
int orc_basis_size(int dim);
int orc_data_size(int dim);
/* reconstruction matrix M (nb x nd, row-major) and basis exponents (nb x 3) */
int orc_recon_matrix(int dim, double* M, int* exps);
/* one cell in reference space: data (nd) -> values and reference gradients at
   all face Gauss points (ngp x (1+dim)), plus chi; linear: 0 takes chi from
   the GENO path function, 1 forces chi = 1 (the fifth-order polynomial),
   2 forces chi = 0 (the weighted linear sub-stencil polynomials alone) */
int orc_recon_reference(int dim, const double* data, int linear, double c_chi,
                        double* out, double* chi);
/* the P4 polynomial coefficients for a data vector */
int orc_recon_coeffs(int dim, const double* data, double* a);
/* reference-frame Gram matrices of the smoothness indicators (nb x nb) */
int orc_gram(int dim, double* GH, double* GL);
/* linear sub-stencil polynomial gradients for face neighbour m (dim) */
int orc_linear_sub(int dim, int m, const double* data, double* b);
/* local-frame GKS interface solution at one point.
   W*: nv conservative (normal momentum first), dW*: dim x nv derivatives along
   the local axes.  out: Fn, Ft, QL0, QLt, QR0, QRt (6*nv). */
int orc_gks_point(int dim, double gamma, double mu, double prandtl, int tau_mode,
                  double dt, const double* WL, const double* dWL,
                  const double* WR, const double* dWR, double* out);
/* normalised Maxwellian moments <u^n> (full, u>0, u<0), n = 0..6 */
int orc_moments_u(double U, double lam, double* full, double* pos, double* neg);
/* micro-slope a solving <a psi psi> = b for a Maxwellian (rho, U[dim], lam) */
int orc_micro_slope(int dim, double gamma, const double* prim_rho_u_lam, const double* b, double* a);
/* S2O4 combinations (temporal discretisation section): the intermediate state
   from (Q^n, L^n, dL^n/dt) and the new state from (Q^n, L^n, dL^n/dt) and the
   time derivative of L at the intermediate state */
double orc_s2o4_stage1(double Q, double dt, double L, double Lt);
double orc_s2o4_stage2(double Q, double dt, double L, double Lt, double Lt_star);

#ifdef __cplusplus
}
#endif
#endif
