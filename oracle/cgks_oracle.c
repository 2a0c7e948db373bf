/*
 * CGKS-5 CPU oracle -- TEST INFRASTRUCTURE ONLY (see cgks_oracle.h).
 *
 * Plain FP64 C, OpenMP over independent cells/faces only.  Every function
 * cites the passage of the paper (arXiv 2508.08965) it follows.  Where the
 * paper is silent the reading used is stated at the spot and collected in the
 * project's design notes.  Nothing here is shared with the CUDA library: the
 * reconstruction matrix is obtained at run time from this file's own
 * constrained least-squares (KKT) solve in long double, the micro-slopes from
 * a generic Gaussian elimination on the Maxwellian moment matrix, and the
 * fluxes from generic moment sums.
 */
#include "cgks_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <stdint.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define NB3 34 /* quartic zero-mean basis size in 3-D (Eq. base, 1 <= |d| <= 4) */
#define ND3 73 /* data vector size in 3-D (Eq. stencil-5) */
#define MAXV 5
#define MAXGP 24

/* ------------------------------------------------------------------------ */
/* 1. Small dense solver: Gaussian elimination with partial pivoting.        */
/* ------------------------------------------------------------------------ */
static int solve_ld(int n, int nrhs, long double* A, long double* B) {
  for (int c = 0; c < n; ++c) {
    int p = c;
    for (int r = c + 1; r < n; ++r)
      if (fabsl(A[r * n + c]) > fabsl(A[p * n + c])) p = r;
    if (A[p * n + c] == 0.0L) return -1;
    if (p != c) {
      for (int k = 0; k < n; ++k) { long double t = A[c * n + k]; A[c * n + k] = A[p * n + k]; A[p * n + k] = t; }
      for (int k = 0; k < nrhs; ++k) { long double t = B[c * nrhs + k]; B[c * nrhs + k] = B[p * nrhs + k]; B[p * nrhs + k] = t; }
    }
    for (int r = c + 1; r < n; ++r) {
      long double f = A[r * n + c] / A[c * n + c];
      if (f == 0.0L) continue;
      for (int k = c; k < n; ++k) A[r * n + k] -= f * A[c * n + k];
      for (int k = 0; k < nrhs; ++k) B[r * nrhs + k] -= f * B[c * nrhs + k];
    }
  }
  for (int c = n - 1; c >= 0; --c) {
    for (int k = 0; k < nrhs; ++k) {
      long double s = B[c * nrhs + k];
      for (int j = c + 1; j < n; ++j) s -= A[c * n + j] * B[j * nrhs + k];
      B[c * nrhs + k] = s / A[c * n + c];
    }
  }
  return 0;
}

static int solve_d(int n, double* A, double* b) {
  long double AL[25], BL[5];
  for (int i = 0; i < n * n; ++i) AL[i] = A[i];
  for (int i = 0; i < n; ++i) BL[i] = b[i];
  int r = solve_ld(n, 1, AL, BL);
  for (int i = 0; i < n; ++i) b[i] = (double)BL[i];
  return r;
}

/* ------------------------------------------------------------------------ */
/* 2. Reference cell: basis (Eq. base), stencil (Sec. 3.2), Gauss points.    */
/*    The standard cell is the unit cube [0,1]^dim (Sec. 4); its centroid is */
/*    1/2 and h = 1, so delta = xi - 1/2.  Neighbours are unit cubes at      */
/*    integer offsets (the universal-matrix reading of Sec. 4).              */
/* ------------------------------------------------------------------------ */
static const double GQ = 0.28867513459481288225; /* 1/(2 sqrt 3): 2-point Gauss on [-1/2,1/2] */

typedef struct {
  int dim, nv, nb, nd, ne, ntau, gpf, ngp, nlines, nf;
  int exps[NB3][3];
  double mean[NB3];
  int face_off[6][3];
  int edge_off[12][3];
  double tau[12][2][3]; /* edge directional derivative directions */
  /* data index bases */
  int d_face, d_edge, d_fgrad, d_etau, d_line;
  /* reference positions of face Gauss points: gp = (2*axis+side)*gpf + k */
  double gp_pos[MAXGP][3];
  /* tables */
  double M[NB3][ND3];       /* P4 coefficients a = M d */
  double M1[6][3][ND3];     /* linear sub-stencil gradients b_m = M1[m] d */
  double GH[NB3][NB3], GL[NB3][NB3];
  double pv[MAXGP][NB3];    /* p_b at face Gauss points */
  double pd[MAXGP][3][NB3]; /* d p_b / d xi_k at face Gauss points */
  int ok;
} ref_t;

static ref_t REF[4];

static double fact(int n) { double f = 1; for (int i = 2; i <= n; ++i) f *= i; return f; }

/* int_a^b t^e / e! dt */
static double I1(int e, double a, double b) {
  return (pow(b, e + 1) - pow(a, e + 1)) / fact(e + 1);
}

/* tangential axes of a face normal to `axis` (increasing order) */
static void tang_axes(int dim, int axis, int* ta) {
  int c = 0;
  for (int k = 0; k < dim; ++k) if (k != axis) ta[c++] = k;
}

/* average over the unit cell at offset o of p_b (zero-mean basis, Eq. base) */
static double avg_basis(const ref_t* R, int b, const int* o) {
  double v = 1.0;
  for (int i = 0; i < R->dim; ++i) v *= I1(R->exps[b][i], o[i] - 0.5, o[i] + 0.5);
  return v - R->mean[b];
}

/* average over the unit cell at offset o of d p_b / d xi_k */
static double avg_dbasis(const ref_t* R, int b, int k, const int* o) {
  if (R->exps[b][k] == 0) return 0.0;
  double v = 1.0;
  for (int i = 0; i < R->dim; ++i) {
    int e = R->exps[b][i] - (i == k ? 1 : 0);
    v *= I1(e, o[i] - 0.5, o[i] + 0.5);
  }
  return v;
}

static double eval_basis(const ref_t* R, int b, const double* dl) {
  double v = 1.0;
  for (int i = 0; i < R->dim; ++i) v *= pow(dl[i], R->exps[b][i]) / fact(R->exps[b][i]);
  return v - R->mean[b];
}

static double eval_dbasis(const ref_t* R, int b, int k, const double* dl) {
  if (R->exps[b][k] == 0) return 0.0;
  double v = 1.0;
  for (int i = 0; i < R->dim; ++i) {
    int e = R->exps[b][i] - (i == k ? 1 : 0);
    v *= pow(dl[i], e) / fact(e);
  }
  return v;
}

/* reference delta of face Gauss point (axis, side, k): side 0 is xi_axis = 0 */
static void gp_delta(int dim, int axis, int side, int k, double* dl) {
  int ta[2];
  tang_axes(dim, axis, ta);
  dl[0] = dl[1] = dl[2] = 0.0;
  dl[axis] = side ? 0.5 : -0.5;
  if (dim == 2) {
    dl[ta[0]] = (k & 1) ? GQ : -GQ;
  } else {
    dl[ta[0]] = (k & 1) ? GQ : -GQ;
    dl[ta[1]] = (k & 2) ? GQ : -GQ;
  }
}

/* Constrained least squares of Eq. (compact-big-ref) with h1' = 2, h2' = 1,
   h3' = 3: averages of the face neighbours hold exactly, all other rows in the
   least-squares sense.  Solved once through its KKT system. */
static int build_ref(int dim) {
  ref_t* R = &REF[dim];
  memset(R, 0, sizeof(*R));
  R->dim = dim;
  R->nv = dim + 2;
  R->gpf = dim == 3 ? 4 : 2;
  R->ngp = 2 * dim * R->gpf;
  R->nlines = dim * R->gpf;
  R->nf = 1 + dim + R->nlines;
  /* basis: 1 <= |d| <= 4 */
  int nb = 0;
  for (int deg = 1; deg <= 4; ++deg)
    for (int e0 = deg; e0 >= 0; --e0)
      for (int e1 = deg - e0; e1 >= 0; --e1) {
        int e2 = deg - e0 - e1;
        if (dim == 2 && e2 != 0) continue;
        R->exps[nb][0] = e0; R->exps[nb][1] = e1; R->exps[nb][2] = e2;
        ++nb;
      }
  R->nb = nb;
  for (int b = 0; b < nb; ++b) {
    double m = 1.0;
    for (int i = 0; i < dim; ++i) m *= I1(R->exps[b][i], -0.5, 0.5);
    R->mean[b] = m;
  }
  /* face neighbours m = 2*axis + side, side 0 -> offset -1 */
  for (int m = 0; m < 2 * dim; ++m) {
    for (int i = 0; i < 3; ++i) R->face_off[m][i] = 0;
    R->face_off[m][m / 2] = (m & 1) ? 1 : -1;
  }
  /* edge neighbours (3-D: share an edge, Sec. 3.2) or corner neighbours (2-D) */
  int ne = 0;
  for (int p = 0; p < dim; ++p)
    for (int q = p + 1; q < dim; ++q)
      for (int sp = -1; sp <= 1; sp += 2)
        for (int sq = -1; sq <= 1; sq += 2) {
          int* o = R->edge_off[ne];
          o[0] = o[1] = o[2] = 0;
          o[p] = sp; o[q] = sq;
          /* tau_1 along the shared edge, tau_2 toward the neighbour centroid
             (Sec. 3.3); in 2-D only the diagonal tau_2 exists */
          double t2[3] = {0, 0, 0};
          t2[p] = sp / sqrt(2.0); t2[q] = sq / sqrt(2.0);
          if (dim == 3) {
            double t1[3] = {0, 0, 0};
            t1[3 - p - q] = 1.0;
            memcpy(R->tau[ne][0], t1, sizeof t1);
            memcpy(R->tau[ne][1], t2, sizeof t2);
          } else {
            memcpy(R->tau[ne][0], t2, sizeof t2);
          }
          ++ne;
        }
  R->ne = ne;
  R->ntau = dim == 3 ? 2 : 1;
  R->d_face = 1;
  R->d_edge = R->d_face + 2 * dim;
  R->d_fgrad = R->d_edge + ne;
  R->d_etau = R->d_fgrad + 2 * dim * dim;
  R->d_line = R->d_etau + ne * R->ntau;
  R->nd = R->d_line + R->nlines;
  int nd = R->nd;
  for (int a = 0; a < 2 * dim; ++a)
    for (int k = 0; k < R->gpf; ++k) {
      int gp = a * R->gpf + k;
      gp_delta(dim, a / 2, a & 1, k, R->gp_pos[gp]);
    }

  /* rows: equality rows C (face averages), LS rows A with weights */
  const int neq = 2 * dim;
  const int nls = ne + 2 * dim * dim + ne * R->ntau + R->nlines;
  double* A = calloc((size_t)nls * nb, sizeof(double));
  double* W = calloc(nls, sizeof(double));
  double* RA = calloc((size_t)nls * nd, sizeof(double)); /* rhs as linear map of d */
  double* C = calloc((size_t)neq * nb, sizeof(double));
  double* RC = calloc((size_t)neq * nd, sizeof(double));
  for (int m = 0; m < neq; ++m) {
    for (int b = 0; b < nb; ++b) C[m * nb + b] = avg_basis(R, b, R->face_off[m]);
    RC[m * nd + R->d_face + m] = 1.0;
    RC[m * nd + 0] = -1.0;
  }
  int r = 0;
  for (int n = 0; n < ne; ++n, ++r) { /* edge averages, weight 1 */
    for (int b = 0; b < nb; ++b) A[r * nb + b] = avg_basis(R, b, R->edge_off[n]);
    RA[r * nd + R->d_edge + n] = 1.0;
    RA[r * nd + 0] = -1.0;
    W[r] = 1.0;
  }
  for (int m = 0; m < 2 * dim; ++m) /* face-neighbour gradients, h1' = 2 */
    for (int k = 0; k < dim; ++k, ++r) {
      for (int b = 0; b < nb; ++b) A[r * nb + b] = avg_dbasis(R, b, k, R->face_off[m]);
      RA[r * nd + R->d_fgrad + m * dim + k] = 1.0;
      W[r] = 2.0;
    }
  for (int n = 0; n < ne; ++n) /* edge directional derivatives, h2' = 1 */
    for (int t = 0; t < R->ntau; ++t, ++r) {
      for (int b = 0; b < nb; ++b) {
        double s = 0.0;
        for (int k = 0; k < dim; ++k) s += R->tau[n][t][k] * avg_dbasis(R, b, k, R->edge_off[n]);
        A[r * nb + b] = s;
      }
      RA[r * nd + R->d_etau + n * R->ntau + t] = 1.0;
      W[r] = 1.0;
    }
  for (int d = 0; d < dim; ++d) /* own line differences, h3' = 3 */
    for (int k = 0; k < R->gpf; ++k, ++r) {
      double lo[3], hi[3];
      gp_delta(dim, d, 0, k, lo);
      gp_delta(dim, d, 1, k, hi);
      for (int b = 0; b < nb; ++b) A[r * nb + b] = eval_basis(R, b, hi) - eval_basis(R, b, lo);
      RA[r * nd + R->d_line + d * R->gpf + k] = 1.0;
      W[r] = 3.0;
    }
  /* KKT: [A^T W^2 A, C^T; C, 0] [a; mu] = [A^T W^2 RA; RC] d */
  int nk = nb + neq;
  long double* K = calloc((size_t)nk * nk, sizeof(long double));
  long double* B = calloc((size_t)nk * nd, sizeof(long double));
  for (int i = 0; i < nb; ++i) {
    for (int j = 0; j < nb; ++j) {
      long double s = 0;
      for (int q = 0; q < nls; ++q) s += (long double)W[q] * W[q] * A[q * nb + i] * A[q * nb + j];
      K[i * nk + j] = s;
    }
    for (int m = 0; m < neq; ++m) { K[i * nk + nb + m] = C[m * nb + i]; K[(nb + m) * nk + i] = C[m * nb + i]; }
    for (int c = 0; c < nd; ++c) {
      long double s = 0;
      for (int q = 0; q < nls; ++q) s += (long double)W[q] * W[q] * A[q * nb + i] * RA[q * nd + c];
      B[i * nd + c] = s;
    }
  }
  for (int m = 0; m < neq; ++m)
    for (int c = 0; c < nd; ++c) B[(nb + m) * nd + c] = RC[m * nd + c];
  int st = solve_ld(nk, nd, K, B);
  for (int i = 0; i < nb; ++i)
    for (int c = 0; c < nd; ++c) R->M[i][c] = (double)B[i * nd + c];
  free(K); free(B); free(A); free(W); free(RA); free(C); free(RC);
  if (st) return st;

  /* linear sub-stencil polynomials, Eq. (compact-sub-2): the face neighbour
     average exactly, the lines perpendicular to the connecting line (all
     lines not along that axis) in the least-squares sense */
  for (int m = 0; m < 2 * dim; ++m) {
    int ax = m / 2;
    int nl = 0;
    double AL[12][3];
    int li[12];
    for (int d = 0; d < dim; ++d) {
      if (d == ax) continue;
      for (int k = 0; k < R->gpf; ++k) {
        double lo[3], hi[3];
        gp_delta(dim, d, 0, k, lo);
        gp_delta(dim, d, 1, k, hi);
        for (int j = 0; j < dim; ++j) AL[nl][j] = hi[j] - lo[j];
        li[nl] = R->d_line + d * R->gpf + k;
        ++nl;
      }
    }
    int n1 = dim + 1;
    long double K1[16] = {0}, B1[4 * ND3];
    memset(B1, 0, sizeof B1);
    for (int i = 0; i < dim; ++i) {
      for (int j = 0; j < dim; ++j) {
        long double s = 0;
        for (int q = 0; q < nl; ++q) s += (long double)AL[q][i] * AL[q][j];
        K1[i * n1 + j] = s;
      }
      for (int q = 0; q < nl; ++q) B1[i * nd + li[q]] += AL[q][i];
      /* equality row: average of P over the neighbour = Q_{1,m} */
      double ci = R->face_off[m][i]; /* average of delta_i over the neighbour */
      K1[i * n1 + dim] = ci;
      K1[dim * n1 + i] = ci;
    }
    B1[dim * nd + R->d_face + m] = 1.0;
    B1[dim * nd + 0] = -1.0;
    if (solve_ld(n1, nd, K1, B1)) return -2;
    for (int i = 0; i < dim; ++i)
      for (int c = 0; c < nd; ++c) R->M1[m][i][c] = (double)B1[i * nd + c];
  }

  /* Gram matrices of the smoothness indicators: IS^H sums the squared
     integrals of every derivative D^l P, 1 <= |l| <= 4, over the unit cell;
     IS^L keeps |l| = 1 (GENO path function, Sec. 3.3) */
  for (int b = 0; b < nb; ++b)
    for (int c = 0; c < nb; ++c) {
      double sh = 0, sl = 0;
      for (int l0 = 0; l0 <= 4; ++l0)
        for (int l1 = 0; l1 <= 4; ++l1)
          for (int l2 = 0; l2 <= (dim == 3 ? 4 : 0); ++l2) {
            int l[3] = {l0, l1, l2};
            int ord = l0 + l1 + l2;
            if (ord < 1 || ord > 4) continue;
            double v = 1.0;
            for (int i = 0; i < dim && v != 0.0; ++i) {
              int p = R->exps[b][i] - l[i], q = R->exps[c][i] - l[i];
              if (p < 0 || q < 0) { v = 0.0; break; }
              v *= I1(p + q, -0.5, 0.5) * fact(p + q) / (fact(p) * fact(q));
            }
            sh += v;
            if (ord == 1) sl += v;
          }
      R->GH[b][c] = sh;
      R->GL[b][c] = sl;
    }
  for (int gp = 0; gp < R->ngp; ++gp)
    for (int b = 0; b < nb; ++b) {
      R->pv[gp][b] = eval_basis(R, b, R->gp_pos[gp]);
      for (int k = 0; k < dim; ++k) R->pd[gp][k][b] = eval_dbasis(R, b, k, R->gp_pos[gp]);
    }
  R->ok = 1;
  return 0;
}

static const ref_t* get_ref(int dim) {
  if (dim != 2 && dim != 3) return NULL;
  ref_t* R = &REF[dim];
  if (!R->ok) {
#pragma omp critical(orc_ref)
    { if (!R->ok) build_ref(dim); }
  }
  return R->ok ? R : NULL;
}

/* ------------------------------------------------------------------------ */
/* 3. Nonlinear reconstruction at the face Gauss points, Eq. (weno-new).     */
/* ------------------------------------------------------------------------ */
/* d: data vector of one variable in the reference frame.
   out[gp*(1+dim) + 0] = value, out[gp*(1+dim) + 1 + k] = d/dxi_k.
   chi_force < 0: use GENO; otherwise use this chi. */
static void recon_var(const ref_t* R, const double* d, double chi_force, double c_chi,
                      double* out, double* chi_out) {
  const int dim = R->dim, nb = R->nb, nd = R->nd;
  double a[NB3];
  for (int b = 0; b < nb; ++b) {
    double s = 0;
    for (int c = 0; c < nd; ++c) s += R->M[b][c] * d[c];
    a[b] = s;
  }
  double bm[6][3], ism[6];
  for (int m = 0; m < 2 * dim; ++m) {
    ism[m] = 0;
    for (int k = 0; k < dim; ++k) {
      double s = 0;
      for (int c = 0; c < nd; ++c) s += R->M1[m][k][c] * d[c];
      bm[m][k] = s;
      ism[m] += s * s; /* IS_m = integral of |grad P_m^1|^2 over the unit cell */
    }
  }
  double chi;
  if (chi_force >= 0.0) {
    chi = chi_force;
  } else {
    double ish = 0, isl = 0;
    for (int b = 0; b < nb; ++b)
      for (int c = 0; c < nb; ++c) {
        ish += a[b] * R->GH[b][c] * a[c];
        isl += a[b] * R->GL[b][c] * a[c];
      }
    const double eps = 1e-15;
    double ist = ish - isl; /* IS^tau = IS^H - IS^L (reading of the GENO path function) */
    if (ist < 0) ist = 0;
    double rh = ist / (ish + eps), rl = ist / (isl + eps);
    double ah = 1.0 + rh * rh, al = 1.0 + rl * rl; /* r = 2 */
    double alpha = 2.0 * ah / (ah + al);
    chi = tanh(c_chi * alpha) / tanh(c_chi);
  }
  /* linear weights d_m = 1/(2 dim), omega_bar = d_m / (IS_m + eps)^5 */
  double wb[6], ws = 0;
  for (int m = 0; m < 2 * dim; ++m) {
    wb[m] = (1.0 / (2 * dim)) / pow(ism[m] + 1e-15, 5);
    ws += wb[m];
  }
  for (int gp = 0; gp < R->ngp; ++gp) {
    double v4 = d[0], g4[3] = {0, 0, 0};
    for (int b = 0; b < nb; ++b) {
      v4 += a[b] * R->pv[gp][b];
      for (int k = 0; k < dim; ++k) g4[k] += a[b] * R->pd[gp][k][b];
    }
    double v1 = 0, g1[3] = {0, 0, 0};
    for (int m = 0; m < 2 * dim; ++m) {
      double w = wb[m] / ws;
      double pm = d[0];
      for (int k = 0; k < dim; ++k) pm += bm[m][k] * R->gp_pos[gp][k];
      v1 += w * pm;
      for (int k = 0; k < dim; ++k) g1[k] += w * bm[m][k];
    }
    out[gp * (1 + dim)] = chi * v4 + (1.0 - chi) * v1;
    for (int k = 0; k < dim; ++k) out[gp * (1 + dim) + 1 + k] = chi * g4[k] + (1.0 - chi) * g1[k];
  }
  if (chi_out) *chi_out = chi;
}

/* ------------------------------------------------------------------------ */
/* 4. Gas kinetics (Sec. 2): Maxwellian moments, micro-slopes, interface    */
/*    distribution Eq. (flux), its time integrals and moments.               */
/* ------------------------------------------------------------------------ */
typedef struct {
  double rho, U[3], lam;
  double mu_full[9], mu_pos[9], mu_neg[9]; /* <u^n>, normal direction */
  double mv[9], mw[9];                     /* <v^n>, <w^n> full space */
  double mxi[3];                           /* <xi^(2k)> for k = 0, 1, 2 */
} maxw_t;

enum { FULL = 0, POS = 1, NEG = 2 };

/* moments of (lam/pi)^{1/2} exp(-lam (u-U)^2): recurrences of the Gaussian
   integrals, half spaces through erfc */
static void moments_1d(double U, double lam, double* full, double* pos, double* neg) {
  full[0] = 1.0;
  full[1] = U;
  pos[0] = 0.5 * erfc(-sqrt(lam) * U);
  neg[0] = 0.5 * erfc(sqrt(lam) * U);
  double e = 0.5 * exp(-lam * U * U) / sqrt(M_PI * lam);
  pos[1] = U * pos[0] + e;
  neg[1] = U * neg[0] - e;
  for (int n = 0; n + 2 <= 8; ++n) {
    full[n + 2] = U * full[n + 1] + (n + 1) / (2.0 * lam) * full[n];
    pos[n + 2] = U * pos[n + 1] + (n + 1) / (2.0 * lam) * pos[n];
    neg[n + 2] = U * neg[n + 1] + (n + 1) / (2.0 * lam) * neg[n];
  }
}

/* internal degrees of freedom N: (5-3 gamma)/(gamma-1) in 3-D (Sec. 2),
   (4-2 gamma)/(gamma-1) for the 2-D reduction */
static double n_internal(int dim, double gamma) {
  return dim == 3 ? (5.0 - 3.0 * gamma) / (gamma - 1.0) : (4.0 - 2.0 * gamma) / (gamma - 1.0);
}

static void maxw_from_cons(int dim, double gamma, const double* W, maxw_t* g) {
  memset(g, 0, sizeof(*g));
  g->rho = W[0];
  double ke = 0;
  for (int i = 0; i < dim; ++i) { g->U[i] = W[1 + i] / W[0]; ke += g->U[i] * W[1 + i]; }
  double p = (gamma - 1.0) * (W[dim + 1] - 0.5 * ke);
  g->lam = W[0] / (2.0 * p);
  moments_1d(g->U[0], g->lam, g->mu_full, g->mu_pos, g->mu_neg);
  double dummy1[9], dummy2[9];
  moments_1d(g->U[1], g->lam, g->mv, dummy1, dummy2);
  if (dim == 3) moments_1d(g->U[2], g->lam, g->mw, dummy1, dummy2);
  else { for (int i = 0; i < 9; ++i) g->mw[i] = 0; g->mw[0] = 1.0; }
  double K = n_internal(dim, gamma);
  g->mxi[0] = 1.0;
  g->mxi[1] = K / (2.0 * g->lam);
  g->mxi[2] = (K * K + 2.0 * K) / (4.0 * g->lam * g->lam);
}

/* psi components as polynomials: terms (coef, pu, pv, pw, pxi2) */
typedef struct { double c; int e[4]; } term_t;
typedef struct { int n; term_t t[4]; } poly_t;

static void psi_polys(int dim, poly_t* psi) {
  memset(psi, 0, sizeof(poly_t) * MAXV);
  psi[0].n = 1; psi[0].t[0].c = 1.0;
  for (int i = 0; i < dim; ++i) { psi[1 + i].n = 1; psi[1 + i].t[0].c = 1.0; psi[1 + i].t[0].e[i] = 1; }
  poly_t* pe = &psi[dim + 1];
  pe->n = dim + 1;
  for (int i = 0; i < dim; ++i) { pe->t[i].c = 0.5; pe->t[i].e[i] = 2; }
  pe->t[dim].c = 0.5; pe->t[dim].e[3] = 1;
}

static double mono(const maxw_t* g, int region, const int* e) {
  const double* mu = region == FULL ? g->mu_full : (region == POS ? g->mu_pos : g->mu_neg);
  return mu[e[0]] * g->mv[e[1]] * g->mw[e[2]] * g->mxi[e[3]];
}

/* out_i = < (a . psi) u^x0 v^x1 w^x2 psi_i >  (a == NULL: the factor is 1) */
static void mom_psi(int dim, const maxw_t* g, int region, const double* a, const int* x, double* out) {
  poly_t psi[MAXV];
  psi_polys(dim, psi);
  const int nv = dim + 2;
  for (int i = 0; i < nv; ++i) {
    double s = 0;
    for (int j = 0; j < (a ? nv : 1); ++j) {
      double aj = a ? a[j] : 1.0;
      if (aj == 0.0) continue;
      for (int p = 0; p < psi[j].n; ++p)
        for (int q = 0; q < psi[i].n; ++q) {
          int e[4];
          for (int k = 0; k < 4; ++k) e[k] = psi[j].t[p].e[k] + psi[i].t[q].e[k] + (k < 3 ? x[k] : 0);
          s += aj * psi[j].t[p].c * psi[i].t[q].c * mono(g, region, e);
        }
    }
    out[i] = s;
  }
}

/* micro-slope: solve <psi psi^T> a = b (full-space Maxwellian moments) */
static int slope(int dim, const maxw_t* g, const double* b, double* a) {
  const int nv = dim + 2;
  double Mm[25];
  int zero[3] = {0, 0, 0};
  for (int j = 0; j < nv; ++j) {
    double e[MAXV] = {0}, col[MAXV];
    e[j] = 1.0;
    mom_psi(dim, g, FULL, e, zero, col);
    for (int i = 0; i < nv; ++i) Mm[i * nv + j] = col[i];
  }
  for (int i = 0; i < nv; ++i) a[i] = b[i];
  return solve_d(nv, Mm, a);
}

/* time integrals over [0, delta] of the six coefficient functions of
   Eq. (flux): 1-e^{-t/tau}, (t+tau)e^{-t/tau}-tau, t-tau+tau e^{-t/tau},
   e^{-t/tau}, -(tau+t)e^{-t/tau}, -tau e^{-t/tau}; exact limits at tau = 0 */
static void time_coefs(double tau, double dl, double* c) {
  if (tau <= 0.0) {
    c[0] = dl; c[1] = 0.0; c[2] = 0.5 * dl * dl; c[3] = 0.0; c[4] = 0.0; c[5] = 0.0;
    return;
  }
  double em = -expm1(-dl / tau); /* 1 - e^{-dl/tau} */
  double ex = exp(-dl / tau);
  c[0] = dl - tau * em;
  c[1] = 2.0 * tau * tau - tau * (dl + 2.0 * tau) * ex - tau * dl;
  c[2] = 0.5 * dl * dl - tau * dl + tau * tau * em;
  c[3] = tau * em;
  c[4] = -2.0 * tau * tau + tau * (dl + 2.0 * tau) * ex;
  c[5] = -tau * tau * em;
}

/* The GKS interface solution in the local frame (x normal to the face).
   Readings: the equilibrium g0 and its slopes come from the kinetic collision
   of the left and right states (half-space moments); the interface values for
   the derivative update follow the two-sided model of the temporal
   discretisation section with tau0 = 5 |pl-pr|/(pl+pr) dt. */
static int gks_point(int dim, double gamma, double mu, double prandtl, int tau_mode, double dt,
                     const double* WL, const double* dWL, const double* WR, const double* dWR,
                     double* out) {
  const int nv = dim + 2;
  int zero[3] = {0, 0, 0};
  maxw_t gl, gr, g0;
  maxw_from_cons(dim, gamma, WL, &gl);
  maxw_from_cons(dim, gamma, WR, &gr);
  if (!(gl.rho > 0) || !(gr.rho > 0) || !(gl.lam > 0) || !(gr.lam > 0)) return -4;
  double W0[MAXV], t1[MAXV], t2[MAXV];
  mom_psi(dim, &gl, POS, NULL, zero, t1);
  mom_psi(dim, &gr, NEG, NULL, zero, t2);
  for (int i = 0; i < nv; ++i) W0[i] = gl.rho * t1[i] + gr.rho * t2[i];
  maxw_from_cons(dim, gamma, W0, &g0);
  if (!(g0.lam > 0)) return -4;
  /* micro-slopes along each local axis */
  double al[3][MAXV], ar[3][MAXV], a0[3][MAXV];
  for (int j = 0; j < dim; ++j) {
    double b[MAXV];
    for (int i = 0; i < nv; ++i) b[i] = dWL[j * nv + i] / gl.rho;
    slope(dim, &gl, b, al[j]);
    for (int i = 0; i < nv; ++i) b[i] = dWR[j * nv + i] / gr.rho;
    slope(dim, &gr, b, ar[j]);
    mom_psi(dim, &gl, POS, al[j], zero, t1);
    mom_psi(dim, &gr, NEG, ar[j], zero, t2);
    double dW0[MAXV];
    for (int i = 0; i < nv; ++i) dW0[i] = (gl.rho * t1[i] + gr.rho * t2[i]) / g0.rho;
    slope(dim, &g0, dW0, a0[j]);
  }
  /* time slopes from the compatibility condition <(a.u + A) psi> = 0 */
  double bl[MAXV] = {0}, br[MAXV] = {0}, b0[MAXV] = {0};
  double Al[MAXV], Ar[MAXV], A0[MAXV];
  for (int j = 0; j < dim; ++j) {
    int x[3] = {0, 0, 0};
    x[j] = 1;
    mom_psi(dim, &gl, FULL, al[j], x, t1);
    for (int i = 0; i < nv; ++i) bl[i] -= t1[i];
    mom_psi(dim, &gr, FULL, ar[j], x, t1);
    for (int i = 0; i < nv; ++i) br[i] -= t1[i];
    mom_psi(dim, &g0, FULL, a0[j], x, t1);
    for (int i = 0; i < nv; ++i) b0[i] -= t1[i];
  }
  slope(dim, &gl, bl, Al);
  slope(dim, &gr, br, Ar);
  slope(dim, &g0, b0, A0);
  /* collision time (Sec. 6): tau modes 0 (smooth, tau = 0), 1 (inviscid), 2 (viscous) */
  double pl = gl.rho / (2.0 * gl.lam), pr = gr.rho / (2.0 * gr.lam), p0 = g0.rho / (2.0 * g0.lam);
  double jump = fabs((pl - pr) / (pl + pr));
  double tau = 0.0;
  if (tau_mode == 1) tau = 0.05 * dt + 5.0 * jump * dt;
  else if (tau_mode == 2) tau = mu / p0 + 5.0 * jump * dt;
  /* f^n = (4 fbar(dt/2) - fbar(dt))/dt, f_t^n = 4 (fbar(dt) - 2 fbar(dt/2))/dt^2 */
  double cf[6], ch[6], cn[6], ct[6];
  time_coefs(tau, dt, cf);
  time_coefs(tau, 0.5 * dt, ch);
  for (int i = 0; i < 6; ++i) {
    cn[i] = (4.0 * ch[i] - cf[i]) / dt;
    ct[i] = 4.0 * (cf[i] - 2.0 * ch[i]) / (dt * dt);
  }
  /* moments of the six parts: u psi for fluxes (and psi for the heat-flux fix) */
  double Fp[6][MAXV], Qp[6][MAXV];
  for (int pass = 0; pass < 2; ++pass) {
    int xu[3] = {pass == 0 ? 1 : 0, 0, 0};
    double (*P)[MAXV] = pass == 0 ? Fp : Qp;
    double s1[MAXV], s2[MAXV];
    mom_psi(dim, &g0, FULL, NULL, xu, s1);
    for (int i = 0; i < nv; ++i) P[0][i] = g0.rho * s1[i];
    for (int i = 0; i < nv; ++i) P[1][i] = 0.0;
    for (int j = 0; j < dim; ++j) {
      int x[3] = {xu[0], 0, 0};
      x[j] += 1;
      mom_psi(dim, &g0, FULL, a0[j], x, s1);
      for (int i = 0; i < nv; ++i) P[1][i] += g0.rho * s1[i];
    }
    mom_psi(dim, &g0, FULL, A0, xu, s1);
    for (int i = 0; i < nv; ++i) P[2][i] = g0.rho * s1[i];
    mom_psi(dim, &gl, POS, NULL, xu, s1);
    mom_psi(dim, &gr, NEG, NULL, xu, s2);
    for (int i = 0; i < nv; ++i) P[3][i] = gl.rho * s1[i] + gr.rho * s2[i];
    for (int i = 0; i < nv; ++i) P[4][i] = 0.0;
    for (int j = 0; j < dim; ++j) {
      int x[3] = {xu[0], 0, 0};
      x[j] += 1;
      mom_psi(dim, &gl, POS, al[j], x, s1);
      mom_psi(dim, &gr, NEG, ar[j], x, s2);
      for (int i = 0; i < nv; ++i) P[4][i] += gl.rho * s1[i] + gr.rho * s2[i];
    }
    mom_psi(dim, &gl, POS, Al, xu, s1);
    mom_psi(dim, &gr, NEG, Ar, xu, s2);
    for (int i = 0; i < nv; ++i) P[5][i] = gl.rho * s1[i] + gr.rho * s2[i];
  }
  double* Fn = out;
  double* Ft = out + nv;
  for (int i = 0; i < nv; ++i) {
    double sn = 0, st = 0;
    for (int p = 0; p < 6; ++p) {
      sn += cn[p] * Fp[p][i];
      st += ct[p] * Fp[p][i];
    }
    Fn[i] = sn; Ft[i] = st;
  }
  /* Prandtl-number fix for viscous flow: F_E += (1/Pr - 1) q, q the heat flux
     about the interface velocity of the non-equilibrium part f - g, where
     g = g0 (1 + A0 t) is the equilibrium at the interface.  g contributes its
     part 0 (g0) to f^n and its part 2 (A0 g0) to f_t^n with weight one, so q
     is taken from the part sums with those weights lowered by one.  (The
     heat flux of g0 about its own velocity vanishes; that of A0 g0 about the
     fixed interface velocity does not: it is the work (E + p) dU/dt of the
     equilibrium's own evolution.) */
  if (mu > 0.0 && prandtl > 0.0 && prandtl != 1.0) {
    for (int pass = 0; pass < 2; ++pass) {
      const double* cw = pass == 0 ? cn : ct;
      const int peq = pass == 0 ? 0 : 2;
      double F[MAXV], Q[MAXV]; /* u psi- and psi-moments of the non-equilibrium part */
      for (int i = 0; i < nv; ++i) {
        double sf = 0, sq = 0;
        for (int p = 0; p < 6; ++p) {
          const double c = p == peq ? cw[p] - 1.0 : cw[p];
          sf += c * Fp[p][i];
          sq += c * Qp[p][i];
        }
        F[i] = sf; Q[i] = sq;
      }
      double uf = 0, uq = 0, u2 = 0;
      for (int i = 0; i < dim; ++i) { uf += g0.U[i] * F[1 + i]; uq += g0.U[i] * Q[1 + i]; u2 += g0.U[i] * g0.U[i]; }
      double q = (F[dim + 1] - uf + 0.5 * u2 * F[0]) - g0.U[0] * (Q[dim + 1] - uq + 0.5 * u2 * Q[0]);
      (pass == 0 ? Fn : Ft)[dim + 1] += (1.0 / prandtl - 1.0) * q;
    }
  }
  /* interface values: Q^e = W0 + t (dQ/dt)_0, Q_0^{l,r} = W_{l,r} + t (dQ/dt)_{l,r},
     blended with e^{-dt/tau0} */
  double tau0 = 5.0 * jump * dt;
  double w = tau0 > 0.0 ? exp(-dt / tau0) : 0.0;
  double* QL0 = out + 2 * nv;
  double* QLt = out + 3 * nv;
  double* QR0 = out + 4 * nv;
  double* QRt = out + 5 * nv;
  for (int i = 0; i < nv; ++i) {
    double dq0 = g0.rho * b0[i], dql = gl.rho * bl[i], dqr = gr.rho * br[i];
    QL0[i] = (1.0 - w) * W0[i] + w * WL[i];
    QLt[i] = (1.0 - w) * dq0 + w * dql;
    QR0[i] = (1.0 - w) * W0[i] + w * WR[i];
    QRt[i] = (1.0 - w) * dq0 + w * dqr;
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* 5. Mesh metrics (Sec. 4 and Appendix).                                   */
/* ------------------------------------------------------------------------ */
typedef struct {
  double J0[3][3];      /* columns: N2-N1, N3-N1, N4-N1 */
  double JinvT[3][3];   /* (J0^T)^{-1} */
  double vol;
  double area[MAXGP][3];/* area vector (quadrature weight included) of each face Gauss point,
                           pointing toward +xi_axis */
  double tang[MAXGP][3];/* first tangent of the face at the Gauss point */
  double pos[MAXGP][3]; /* physical Gauss point */
  double len[12];       /* |x_G(s,2) - x_G(s,1)| */
} cellgeo_t;

struct orc_ctx {
  orc_desc d;
  const ref_t* R;
  int dim, nv, nf, n[3];
  long ncell;
  double* nodes;
  cellgeo_t* geo;
  double* U;      /* state */
  double* chi;    /* [v][cell] */
  double t;
  long npos_fallback;
  /* work */
  double* gpv;    /* per cell: ngp x nv x (1+dim) physical values/gradients */
  double* fx;     /* per face point: 6 nv */
  double* fxlo;   /* low boundary faces of non-periodic axes */
  double* L1; double* Lt1; double* D1; double* L2; double* Lt2; double* Dt;
  int err;
  struct selector* sel; /* learned troubled-cell selector, or NULL */
  long nskip, nunsure;  /* selector decisions since orc_set_selector */
  double margin;        /* smallest |logit - threshold| seen */
};

static long cidx(const orc_ctx* c, int i, int j, int k) {
  return i + (long)c->n[0] * (j + (long)c->n[1] * k);
}

static void node_at(const orc_ctx* c, int i, int j, int k, double* x) {
  const int dim = c->dim;
  if (!c->nodes) {
    int ii[3] = {i, j, k};
    for (int d = 0; d < dim; ++d) x[d] = c->d.lo[d] + (c->d.hi[d] - c->d.lo[d]) * ii[d] / c->n[d];
    return;
  }
  long nx = c->n[0] + 1, ny = c->n[1] + 1;
  long id = i + nx * (j + ny * (long)k);
  for (int d = 0; d < dim; ++d) x[d] = c->nodes[id * dim + d];
}

/* trilinear (bilinear in 2-D) map of the cell and its Jacobian at xi */
static void cell_map(const orc_ctx* c, int ci, int cj, int ck, const double* xi, double* x, double J[3][3]) {
  const int dim = c->dim;
  for (int a = 0; a < 3; ++a) { x[a] = 0; for (int b = 0; b < 3; ++b) J[a][b] = 0; }
  int nvtx = dim == 3 ? 8 : 4;
  for (int v = 0; v < nvtx; ++v) {
    int o[3] = {v & 1, (v >> 1) & 1, (v >> 2) & 1};
    double X[3];
    node_at(c, ci + o[0], cj + o[1], ck + o[2], X);
    double w[3], dw[3];
    for (int a = 0; a < dim; ++a) { w[a] = o[a] ? xi[a] : 1.0 - xi[a]; dw[a] = o[a] ? 1.0 : -1.0; }
    double wt = 1.0;
    for (int a = 0; a < dim; ++a) wt *= w[a];
    for (int a = 0; a < dim; ++a) {
      x[a] += wt * X[a];
      for (int b = 0; b < dim; ++b) {
        double dwb = dw[b];
        for (int e = 0; e < dim; ++e) if (e != b) dwb *= w[e];
        J[a][b] += dwb * X[a];
      }
    }
  }
}

static double det3(double J[3][3], int dim) {
  if (dim == 2) return J[0][0] * J[1][1] - J[0][1] * J[1][0];
  return J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) - J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
         J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
}

static void build_geo(orc_ctx* c) {
  const int dim = c->dim;
  const ref_t* R = c->R;
  static const double g3x[3] = {-0.77459666924148337704, 0.0, 0.77459666924148337704};
  static const double g3w[3] = {5.0 / 9.0, 8.0 / 9.0, 5.0 / 9.0};
#pragma omp parallel for schedule(static)
  for (long id = 0; id < c->ncell; ++id) {
    int i = id % c->n[0], j = (id / c->n[0]) % c->n[1], k = dim == 3 ? id / ((long)c->n[0] * c->n[1]) : 0;
    cellgeo_t* G = &c->geo[id];
    memset(G, 0, sizeof(*G));
    double N1[3] = {0}, Nk[3] = {0};
    node_at(c, i, j, k, N1);
    for (int a = 0; a < dim; ++a) {
      int o[3] = {0, 0, 0};
      o[a] = 1;
      node_at(c, i + o[0], j + o[1], k + o[2], Nk);
      for (int r = 0; r < dim; ++r) G->J0[r][a] = Nk[r] - N1[r];
    }
    /* (J0^T)^{-1} by cofactors */
    double J[3][3] = {{0}};
    for (int r = 0; r < 3; ++r) for (int s = 0; s < 3; ++s) J[r][s] = G->J0[r][s];
    if (dim == 2) J[2][2] = 1.0;
    double det = det3(J, 3);
    double inv[3][3];
    inv[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) / det;
    inv[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
    inv[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
    inv[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) / det;
    inv[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
    inv[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
    inv[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) / det;
    inv[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
    inv[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
    for (int r = 0; r < 3; ++r) for (int s = 0; s < 3; ++s) G->JinvT[r][s] = inv[s][r];
    /* volume: Gauss quadrature of det(dX/dxi) over the reference cell (Appendix) */
    double vol = 0;
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b)
        for (int e = 0; e < (dim == 3 ? 3 : 1); ++e) {
          double xi[3] = {0.5 + 0.5 * g3x[a], 0.5 + 0.5 * g3x[b], dim == 3 ? 0.5 + 0.5 * g3x[e] : 0.0};
          double x[3], Jm[3][3];
          cell_map(c, i, j, k, xi, x, Jm);
          double w = 0.125 * g3w[a] * g3w[b] * (dim == 3 ? g3w[e] : 2.0);
          if (dim == 2) w = 0.25 * g3w[a] * g3w[b];
          vol += w * det3(Jm, dim);
        }
    G->vol = vol;
    /* face Gauss points: area vectors from the surface map, weight 1/gpf */
    for (int f = 0; f < 2 * dim; ++f) {
      int ax = f / 2, side = f & 1;
      int ta[2];
      tang_axes(dim, ax, ta);
      for (int q = 0; q < R->gpf; ++q) {
        int gp = f * R->gpf + q;
        double xi[3];
        for (int a = 0; a < 3; ++a) xi[a] = R->gp_pos[gp][a] + 0.5;
        xi[ax] = side;
        double x[3], Jm[3][3];
        cell_map(c, i, j, k, xi, x, Jm);
        for (int a = 0; a < 3; ++a) G->pos[gp][a] = a < dim ? x[a] : 0.0;
        double w = 1.0 / R->gpf;
        if (dim == 3) {
          double ta0[3] = {Jm[0][ta[0]], Jm[1][ta[0]], Jm[2][ta[0]]};
          double tb0[3] = {Jm[0][ta[1]], Jm[1][ta[1]], Jm[2][ta[1]]};
          double cr[3] = {ta0[1] * tb0[2] - ta0[2] * tb0[1], ta0[2] * tb0[0] - ta0[0] * tb0[2],
                          ta0[0] * tb0[1] - ta0[1] * tb0[0]};
          double sg = (ax == 1) ? -1.0 : 1.0; /* (axis, ta0, ta1) odd permutation for axis 1 */
          for (int a = 0; a < 3; ++a) { G->area[gp][a] = sg * w * cr[a]; G->tang[gp][a] = ta0[a]; }
        } else {
          double tv[2] = {Jm[0][ta[0]], Jm[1][ta[0]]};
          double sg = (ax == 0) ? 1.0 : -1.0;
          G->area[gp][0] = sg * w * tv[1];
          G->area[gp][1] = -sg * w * tv[0];
          G->area[gp][2] = 0.0;
          G->tang[gp][0] = tv[0]; G->tang[gp][1] = tv[1]; G->tang[gp][2] = 0.0;
        }
      }
    }
    for (int ax = 0; ax < dim; ++ax)
      for (int q = 0; q < R->gpf; ++q) {
        int glo = (2 * ax) * R->gpf + q, ghi = (2 * ax + 1) * R->gpf + q;
        double s = 0;
        for (int a = 0; a < dim; ++a) { double dd = G->pos[ghi][a] - G->pos[glo][a]; s += dd * dd; }
        G->len[ax * R->gpf + q] = sqrt(s);
      }
  }
}

/* ------------------------------------------------------------------------ */
/* 6. Context, state and initial data.                                      */
/* ------------------------------------------------------------------------ */
/* boundary kinds of orc_desc.bc */
enum { BC_PERIODIC = 0, BC_OUTFLOW = 1, BC_SLIP = 2, BC_NOSLIP = 3, BC_INFLOW = 4 };

orc_ctx* orc_create(const orc_desc* d) {
  const ref_t* R = get_ref(d->dim);
  if (!R) return NULL;
  for (int f = 0; f < 2 * d->dim; ++f) {
    if (d->bc[f] < BC_PERIODIC || d->bc[f] > BC_INFLOW) return NULL;
    /* a mirror is a reflection only on a box; inflow faces likewise on boxes */
    if ((d->bc[f] == BC_SLIP || d->bc[f] == BC_NOSLIP || d->bc[f] == BC_INFLOW) && d->nodes) return NULL;
    if ((d->bc[f] == BC_PERIODIC) != (d->bc[f ^ 1] == BC_PERIODIC)) return NULL;
  }
  orc_ctx* c = calloc(1, sizeof(orc_ctx));
  c->d = *d;
  if (d->dim == 2) c->d.bc[4] = c->d.bc[5] = BC_PERIODIC;
  c->R = R;
  c->dim = d->dim;
  c->nv = R->nv;
  c->nf = R->nf;
  c->n[0] = d->n[0]; c->n[1] = d->n[1]; c->n[2] = d->dim == 3 ? d->n[2] : 1;
  c->ncell = (long)c->n[0] * c->n[1] * c->n[2];
  if (d->nodes) {
    long nn = (long)(c->n[0] + 1) * (c->n[1] + 1) * (d->dim == 3 ? c->n[2] + 1 : 1);
    c->nodes = malloc(sizeof(double) * nn * d->dim);
    memcpy(c->nodes, d->nodes, sizeof(double) * nn * d->dim);
  }
  c->d.nodes = NULL;
  c->geo = malloc(sizeof(cellgeo_t) * c->ncell);
  build_geo(c);
  long nst = (long)c->nf * c->nv * c->ncell;
  c->U = calloc(nst, sizeof(double));
  c->chi = calloc((size_t)c->nv * c->ncell, sizeof(double));
  c->gpv = calloc((size_t)c->ncell * R->ngp * c->nv * (1 + c->dim), sizeof(double));
  c->fx = calloc((size_t)c->ncell * c->dim * R->gpf * 6 * c->nv, sizeof(double));
  c->fxlo = calloc((size_t)c->ncell * c->dim * R->gpf * 6 * c->nv, sizeof(double));
  long nd = (long)(c->nf - 1) * c->nv * c->ncell;
  c->L1 = calloc((size_t)c->nv * c->ncell, sizeof(double));
  c->Lt1 = calloc((size_t)c->nv * c->ncell, sizeof(double));
  c->L2 = calloc((size_t)c->nv * c->ncell, sizeof(double));
  c->Lt2 = calloc((size_t)c->nv * c->ncell, sizeof(double));
  c->D1 = calloc(nd, sizeof(double));
  c->Dt = calloc(nd, sizeof(double));
  if (c->d.c_chi <= 0) c->d.c_chi = 100.0;
  return c;
}

void orc_destroy(orc_ctx* c) {
  if (!c) return;
  free(c->nodes); free(c->geo); free(c->U); free(c->chi); free(c->gpv); free(c->fx); free(c->fxlo);
  free(c->sel);
  free(c->L1); free(c->Lt1); free(c->L2); free(c->Lt2); free(c->D1); free(c->Dt);
  free(c);
}

int orc_nfields(const orc_ctx* c) { return c->nf; }
long orc_ncells(const orc_ctx* c) { return c->ncell; }

int orc_set_state(orc_ctx* c, const double* s, double t) {
  memcpy(c->U, s, sizeof(double) * c->nf * c->nv * c->ncell);
  c->t = t;
  return 0;
}

int orc_get_state(const orc_ctx* c, double* s, double* t) {
  memcpy(s, c->U, sizeof(double) * c->nf * c->nv * c->ncell);
  if (t) *t = c->t;
  return 0;
}

static const double G5X[5] = {-0.90617984593866399280, -0.53846931010568309104, 0.0,
                              0.53846931010568309104, 0.90617984593866399280};
static const double G5W[5] = {0.23692688505618908751, 0.47862867049936646804, 0.56888888888888888889,
                              0.47862867049936646804, 0.23692688505618908751};

static int nvolpts(int dim) { return dim == 3 ? 125 : 25; }

long orc_num_init_points(const orc_ctx* c) {
  return c->ncell * (nvolpts(c->dim) + c->R->ngp);
}

/* per cell: 5-point Gauss per axis in the reference cell (mapped), then the
   face Gauss points */
void orc_init_points(const orc_ctx* c, double* pts) {
  const int dim = c->dim, npc = nvolpts(dim) + c->R->ngp;
#pragma omp parallel for schedule(static)
  for (long id = 0; id < c->ncell; ++id) {
    int i = id % c->n[0], j = (id / c->n[0]) % c->n[1], k = dim == 3 ? id / ((long)c->n[0] * c->n[1]) : 0;
    double* p = pts + id * npc * dim;
    int q = 0;
    for (int a = 0; a < 5; ++a)
      for (int b = 0; b < 5; ++b)
        for (int e = 0; e < (dim == 3 ? 5 : 1); ++e, ++q) {
          double xi[3] = {0.5 + 0.5 * G5X[dim == 3 ? e : b], 0.5 + 0.5 * G5X[dim == 3 ? b : a],
                          dim == 3 ? 0.5 + 0.5 * G5X[a] : 0.0};
          double x[3], J[3][3];
          cell_map(c, i, j, k, xi, x, J);
          for (int r = 0; r < dim; ++r) p[q * dim + r] = x[r];
        }
    for (int g = 0; g < c->R->ngp; ++g, ++q)
      for (int r = 0; r < dim; ++r) p[q * dim + r] = c->geo[id].pos[g][r];
  }
}

static void prim_to_cons(int dim, double gamma, const double* pr, double* W) {
  double rho = pr[0], ke = 0;
  W[0] = rho;
  for (int i = 0; i < dim; ++i) { W[1 + i] = rho * pr[1 + i]; ke += pr[1 + i] * pr[1 + i]; }
  W[dim + 1] = pr[dim + 1] / (gamma - 1.0) + 0.5 * rho * ke;
}

/* averages by Gauss quadrature of the mapped cell; gradients and line
   derivatives by the discrete face-point definitions of Eqs. (derivative) and
   (derivative-l) applied to the exact point values */
int orc_init_from_prims(orc_ctx* c, const double* prim) {
  const int dim = c->dim, nv = c->nv, npc = nvolpts(dim) + c->R->ngp;
  const ref_t* R = c->R;
  const long N = c->ncell;
#pragma omp parallel for schedule(static)
  for (long id = 0; id < N; ++id) {
    int i = id % c->n[0], j = (id / c->n[0]) % c->n[1], k = dim == 3 ? id / ((long)c->n[0] * c->n[1]) : 0;
    const double* pr = prim + id * npc * nv;
    double sum[MAXV] = {0}, wsum = 0;
    int q = 0;
    for (int a = 0; a < 5; ++a)
      for (int b = 0; b < 5; ++b)
        for (int e = 0; e < (dim == 3 ? 5 : 1); ++e, ++q) {
          int ix = dim == 3 ? e : b, iy = dim == 3 ? b : a, iz = a;
          double xi[3] = {0.5 + 0.5 * G5X[ix], 0.5 + 0.5 * G5X[iy], dim == 3 ? 0.5 + 0.5 * G5X[iz] : 0.0};
          double x[3], J[3][3];
          cell_map(c, i, j, k, xi, x, J);
          double w = G5W[ix] * G5W[iy] * (dim == 3 ? G5W[iz] : 1.0) * det3(J, dim);
          double W[MAXV];
          prim_to_cons(dim, c->d.gamma, pr + q * nv, W);
          for (int v = 0; v < nv; ++v) sum[v] += w * W[v];
          wsum += w;
        }
    double Wg[MAXGP][MAXV];
    for (int g = 0; g < R->ngp; ++g, ++q) prim_to_cons(dim, c->d.gamma, pr + q * nv, Wg[g]);
    const cellgeo_t* G = &c->geo[id];
    for (int v = 0; v < nv; ++v) {
      c->U[(0 * nv + v) * N + id] = sum[v] / wsum;
      for (int kk = 0; kk < dim; ++kk) {
        double s = 0;
        for (int g = 0; g < R->ngp; ++g) {
          double sgn = ((g / R->gpf) & 1) ? 1.0 : -1.0;
          s += sgn * Wg[g][v] * G->area[g][kk];
        }
        c->U[((1 + kk) * nv + v) * N + id] = s / G->vol;
      }
      for (int ax = 0; ax < dim; ++ax)
        for (int qq = 0; qq < R->gpf; ++qq) {
          int glo = (2 * ax) * R->gpf + qq, ghi = (2 * ax + 1) * R->gpf + qq;
          int s = ax * R->gpf + qq;
          c->U[((1 + dim + s) * nv + v) * N + id] = (Wg[ghi][v] - Wg[glo][v]) / G->len[s];
        }
    }
  }
  c->t = 0.0;
  return 0;
}

int orc_get_metrics(const orc_ctx* c, double* vol, double* closure) {
  const int dim = c->dim;
  for (long id = 0; id < c->ncell; ++id) {
    vol[id] = c->geo[id].vol;
    for (int a = 0; a < dim; ++a) {
      double s = 0;
      for (int g = 0; g < c->R->ngp; ++g) {
        double sgn = ((g / c->R->gpf) & 1) ? 1.0 : -1.0;
        s += sgn * c->geo[id].area[g][a];
      }
      closure[id * dim + a] = s;
    }
  }
  return 0;
}

int orc_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* 7. Time step (Sec. 6): CFL 0.5, convective limit summed over directions */
/*    and the viscous limit CFL h^2/(3 nu).                                  */
/* ------------------------------------------------------------------------ */
double orc_compute_dt(orc_ctx* c) {
  if (c->d.dt_fixed > 0) return c->d.dt_fixed;
  const int dim = c->dim, nv = c->nv, gpf = c->R->gpf;
  const long N = c->ncell;
  double dtmin = 1e300;
#pragma omp parallel for reduction(min : dtmin) schedule(static)
  for (long id = 0; id < N; ++id) {
    const cellgeo_t* G = &c->geo[id];
    double W[MAXV];
    for (int v = 0; v < nv; ++v) W[v] = c->U[v * N + id];
    double rho = W[0], ke = 0, U[3];
    for (int i = 0; i < dim; ++i) { U[i] = W[1 + i] / rho; ke += U[i] * W[1 + i]; }
    double p = (c->d.gamma - 1.0) * (W[dim + 1] - 0.5 * ke);
    double snd = sqrt(c->d.gamma * p / rho);
    /* reading of the CFL rule: dt = CFL / sum_d (|U.n_d| + c)/h_d per cell,
       which reproduces the printed accuracy table of Sec. 6.1 */
    double hmin = 1e300, rate = 0.0;
    for (int ax = 0; ax < dim; ++ax) {
      double A0[3] = {0, 0, 0}, A1[3] = {0, 0, 0};
      for (int q = 0; q < gpf; ++q)
        for (int a = 0; a < dim; ++a) { A0[a] += G->area[(2 * ax) * gpf + q][a]; A1[a] += G->area[(2 * ax + 1) * gpf + q][a]; }
      double s0 = 0, s1 = 0, nn[3], ns = 0;
      for (int a = 0; a < dim; ++a) { s0 += A0[a] * A0[a]; s1 += A1[a] * A1[a]; nn[a] = A0[a] + A1[a]; ns += nn[a] * nn[a]; }
      double S = 0.5 * (sqrt(s0) + sqrt(s1));
      double h = G->vol / S;
      double un = 0;
      for (int a = 0; a < dim; ++a) un += U[a] * nn[a] / sqrt(ns);
      rate += (fabs(un) + snd) / h;
      if (h < hmin) hmin = h;
    }
    double dtc = 1.0 / rate;
    if (c->d.mu > 0) {
      double tv = hmin * hmin * rho / (3.0 * c->d.mu);
      if (tv < dtc) dtc = tv;
    }
    if (dtc < dtmin) dtmin = dtc;
  }
  return c->d.cfl * dtmin;
}

/* ------------------------------------------------------------------------ */
/* 8. One stage: reconstruction, interface solution, accumulation.          */
/* ------------------------------------------------------------------------ */

/* Boundaries (reading of the ghost-cell treatment): beyond a periodic face
   the index wraps; beyond an outflow face it is clamped (the ghost copies the
   boundary cell); beyond a wall it is mirrored and the ghost carries the
   mirror image of the cell's data: reflecting axis a negates the normal
   momentum (slip) or every momentum component (no-slip), and negates
   derivatives along a.  Beyond an inflow face the ghost holds the face's
   fixed state with zero gradients (*inflow = 1 + that face; the index is
   clamped and unused for values). */
static long nbr_bc3(const orc_ctx* c, long id, const int* o, int* mirror, int* noslip, int* inflow) {
  int ii[3] = {(int)(id % c->n[0]), (int)((id / c->n[0]) % c->n[1]),
               c->dim == 3 ? (int)(id / ((long)c->n[0] * c->n[1])) : 0};
  *mirror = 0;
  *noslip = 0;
  *inflow = 0;
  for (int a = 0; a < c->dim; ++a) {
    int x = ii[a] + o[a];
    if (x < 0 || x >= c->n[a]) {
      const int f = 2 * a + (x < 0 ? 0 : 1);
      int bc = c->d.bc[f];
      if (bc == BC_PERIODIC) x = (x + c->n[a]) % c->n[a];
      else if (bc == BC_OUTFLOW) x = x < 0 ? 0 : c->n[a] - 1;
      else if (bc == BC_INFLOW) {
        x = x < 0 ? 0 : c->n[a] - 1;
        if (!*inflow) *inflow = 1 + f;
      } else {
        x = x < 0 ? -1 - x : 2 * c->n[a] - 1 - x;
        *mirror |= 1 << a;
        if (bc == BC_NOSLIP) *noslip |= 1 << a;
      }
    }
    ii[a] = x;
  }
  return cidx(c, ii[0], ii[1], ii[2]);
}

static long nbr_bc(const orc_ctx* c, long id, const int* o, int* mirror, int* noslip) {
  int inf;
  return nbr_bc3(c, id, o, mirror, noslip, &inf);
}

static long nbr(const orc_ctx* c, long id, const int* o) {
  int m, ns;
  return nbr_bc(c, id, o, &m, &ns);
}

static double mirror_sign(int dim, int v, int k, int mirror, int noslip);
#define mirror_sign_fwd mirror_sign

/* value (k < 0) or physical gradient component k of variable v at the
   neighbour of cell id at offset o, through the boundaries */
static double nbr_field(const orc_ctx* c, const double* S, long id, const int* o, int v, int k) {
  int mi, ns, inf;
  const long nb = nbr_bc3(c, id, o, &mi, &ns, &inf);
  if (inf) return k < 0 ? c->d.bc_state[inf - 1][v] : 0.0;
  const long N = c->ncell;
  const double x = S[((long)(k < 0 ? 0 : 1 + k) * c->nv + v) * N + nb];
  return mirror_sign_fwd(c->dim, v, k, mi, ns) * x;
}

/* sign of variable v (and of its derivative along axis k, k < 0: the value)
   in the mirror image across the axes in `mirror` */
static double mirror_sign(int dim, int v, int k, int mirror, int noslip) {
  double s = 1.0;
  for (int a = 0; a < dim; ++a) {
    if (!((mirror >> a) & 1)) continue;
    int mom = v >= 1 && v <= dim;
    if (mom && (((noslip >> a) & 1) || v == 1 + a)) s = -s;
    if (k == a) s = -s;
  }
  return s;
}

/* rho > 0 and p > 0 at every face Gauss point of one cell's reconstruction */
static int gp_states_physical(const ref_t* R, double gamma, double ref[MAXV][MAXGP * 4]) {
  const int dim = R->dim;
  for (int gp = 0; gp < R->ngp; ++gp) {
    double rho = ref[0][gp * (1 + dim)], ke = 0;
    for (int i = 0; i < dim; ++i) { double m = ref[1 + i][gp * (1 + dim)]; ke += m * m; }
    double p = (gamma - 1.0) * (ref[dim + 1][gp * (1 + dim)] - 0.5 * ke / rho);
    if (!(rho > 0) || !(p > 0)) return 0;
  }
  return 1;
}

/* ------------------------------------------------------------------------ */
/* Learned troubled-cell selector (not in the paper; test reference for the */
/* library's fused selector).  Per cell, 16 features from the face-neighbour */
/* averages and the cell's own line derivatives, computed in float with the */
/* rounding of each operation fixed; a 16-32-32-32-1 ReLU network evaluated */
/* with BF16 inputs and weights and float sums; skip (chi = 1 for every      */
/* variable) when the logit reaches thr_skip.                                */
/* ------------------------------------------------------------------------ */
#define SEL_NF 16
#define SEL_H 32
#define SEL_NPARAM (SEL_H * SEL_NF + SEL_H + 2 * (SEL_H * SEL_H + SEL_H) + SEL_H + 1)

struct selector {
  float p[SEL_NPARAM]; /* W1[32][16] b1[32] W2[32][32] b2 W3[32][32] b3 w4[32] b4 */
  float thr_skip, thr_lo;
};

/* features of cell id of state S: per variable class (density, momentum,
   energy) the largest normalised face jump J, corner (edge-neighbour) jump E,
   second-difference ratio R, spread of the line differences S and their
   mismatch with the central difference C, and over all variables the largest
   normalised jump G of a gradient component between the cell and a face
   neighbour; J, E, S, C, G mapped by x/(1+x).  Normalising by the scale is a
   multiplication by its float reciprocal (J, E, S, G) or a division (R, C). */
static void sel_features(const orc_ctx* c, const double* S, long id, float* f) {
  const int dim = c->dim, nv = c->nv, gpf = c->R->gpf;
  const long N = c->ncell;
  const cellgeo_t* G = &c->geo[id];
  float q0[MAXV];
  for (int v = 0; v < nv; ++v) q0[v] = (float)S[(long)v * N + id];
  float fj[3] = {0, 0, 0}, fe[3] = {0, 0, 0}, fr[3] = {0, 0, 0}, fs[3] = {0, 0, 0}, fc[3] = {0, 0, 0};
  float fg = 0.0f;
  for (int v = 0; v < nv; ++v) {
    const int cls = v == 0 ? 0 : (v == nv - 1 ? 2 : 1);
    float scale = fabsf(q0[v]);
    if (cls == 1) scale = scale + sqrtf(fabsf(q0[0]) * fabsf(q0[nv - 1]));
    const float inv = 1.0f / scale;
    for (int a = 0; a < dim; ++a) {
      float qn[2];
      for (int sd = 0; sd < 2; ++sd) {
        int o[3] = {0, 0, 0};
        o[a] = sd ? 1 : -1;
        qn[sd] = (float)nbr_field(c, S, id, o, v, -1);
        for (int k = 0; k < dim; ++k) {
          const float gm = (float)nbr_field(c, S, id, o, v, k);
          const float g0 = (float)S[((long)(1 + k) * nv + v) * N + id];
          const float gd = (fabsf(gm - g0) * (float)G->len[k * gpf]) * inv;
          fg = fmaxf(fg, gd);
        }
      }
      const float dm = q0[v] - qn[0], dp = qn[1] - q0[v];
      const float adm = fabsf(dm), adp = fabsf(dp);
      const float J = fmaxf(adm, adp) * inv;
      const float den = (adm + adp) + 1e-7f * scale;
      const float Rr = fabsf(dp - dm) / den;
      float lsum = 0.0f, lmin = 0.0f, lmax = 0.0f;
      for (int k = 0; k < gpf; ++k) {
        const int sl = a * gpf + k;
        const float lh = (float)S[((long)(1 + dim + sl) * nv + v) * N + id] * (float)G->len[sl];
        lsum = lsum + lh;
        if (k == 0 || lh < lmin) lmin = lh;
        if (k == 0 || lh > lmax) lmax = lh;
      }
      const float lhm = lsum * (1.0f / (float)gpf);
      const float sp = (lmax - lmin) * inv;
      const float cd = (dp + dm) * 0.5f;
      const float Cm = fabsf(lhm - cd) / den;
      fj[cls] = fmaxf(fj[cls], J);
      fr[cls] = fmaxf(fr[cls], Rr);
      fs[cls] = fmaxf(fs[cls], sp);
      fc[cls] = fmaxf(fc[cls], Cm);
      /* edge neighbours across axes a < b */
      for (int b = a + 1; b < dim; ++b)
        for (int sg = 0; sg < 4; ++sg) {
          int o[3] = {0, 0, 0};
          o[a] = (sg & 1) ? 1 : -1;
          o[b] = (sg & 2) ? 1 : -1;
          const float q = (float)nbr_field(c, S, id, o, v, -1);
          fe[cls] = fmaxf(fe[cls], fabsf(q - q0[v]) * inv);
        }
    }
  }
  for (int k = 0; k < 3; ++k) {
    f[5 * k + 0] = fj[k] / (1.0f + fj[k]);
    f[5 * k + 1] = fe[k] / (1.0f + fe[k]);
    f[5 * k + 2] = fr[k];
    f[5 * k + 3] = fs[k] / (1.0f + fs[k]);
    f[5 * k + 4] = fc[k] / (1.0f + fc[k]);
  }
  f[15] = fg / (1.0f + fg);
}

/* round a float to the nearest bfloat16 (ties to even), kept as a float */
static float bf16r(float x) {
  uint32_t u;
  memcpy(&u, &x, 4);
  u += 0x7FFFu + ((u >> 16) & 1u);
  u &= 0xFFFF0000u;
  memcpy(&x, &u, 4);
  return x;
}

static float sel_logit(const struct selector* sl, const float* feat) {
  const float* W1 = sl->p;
  const float* b1 = W1 + SEL_H * SEL_NF;
  const float* W2 = b1 + SEL_H;
  const float* b2 = W2 + SEL_H * SEL_H;
  const float* W3 = b2 + SEL_H;
  const float* b3 = W3 + SEL_H * SEL_H;
  const float* w4 = b3 + SEL_H;
  const float b4 = w4[SEL_H];
  float x[SEL_NF], h1[SEL_H], h2[SEL_H], h3[SEL_H];
  for (int k = 0; k < SEL_NF; ++k) x[k] = bf16r(feat[k]);
  for (int o = 0; o < SEL_H; ++o) {
    float acc = 0.0f;
    for (int k = 0; k < SEL_NF; ++k) acc = acc + bf16r(W1[o * SEL_NF + k]) * x[k];
    const float z = acc + b1[o];
    h1[o] = bf16r(z > 0.0f ? z : 0.0f);
  }
  for (int o = 0; o < SEL_H; ++o) {
    float acc = 0.0f;
    for (int k = 0; k < SEL_H; ++k) acc = acc + bf16r(W2[o * SEL_H + k]) * h1[k];
    const float z = acc + b2[o];
    h2[o] = bf16r(z > 0.0f ? z : 0.0f);
  }
  for (int o = 0; o < SEL_H; ++o) {
    float acc = 0.0f;
    for (int k = 0; k < SEL_H; ++k) acc = acc + bf16r(W3[o * SEL_H + k]) * h2[k];
    const float z = acc + b3[o];
    h3[o] = bf16r(z > 0.0f ? z : 0.0f);
  }
  float acc = 0.0f;
  for (int k = 0; k < SEL_H; ++k) acc = acc + bf16r(w4[k]) * h3[k];
  return acc + b4;
}

/* reconstruct all variables of one cell at its face Gauss points, physical
   gradients (reverse transform of Sec. 4); positivity fallback forces chi = 0 */
static void recon_cell(orc_ctx* c, const double* S, long id, int record_chi) {
  const ref_t* R = c->R;
  const int dim = c->dim, nv = c->nv, nd = R->nd;
  const long N = c->ncell;
  const cellgeo_t* G = &c->geo[id];
  double dat[MAXV][ND3];
  for (int v = 0; v < nv; ++v) {
    double* d = dat[v];
    d[0] = S[(0 * nv + v) * N + id];
    for (int m = 0; m < 2 * dim; ++m) {
      d[R->d_face + m] = nbr_field(c, S, id, R->face_off[m], v, -1);
      /* reference-frame gradient J0^T (grad Q)_{1,m} with the target's J0 */
      for (int k = 0; k < dim; ++k) {
        double s = 0;
        for (int r = 0; r < dim; ++r) s += G->J0[r][k] * nbr_field(c, S, id, R->face_off[m], v, r);
        d[R->d_fgrad + m * dim + k] = s;
      }
    }
    for (int n = 0; n < R->ne; ++n) {
      d[R->d_edge + n] = nbr_field(c, S, id, R->edge_off[n], v, -1);
      double g[3];
      for (int k = 0; k < dim; ++k) {
        double s = 0;
        for (int r = 0; r < dim; ++r) s += G->J0[r][k] * nbr_field(c, S, id, R->edge_off[n], v, r);
        g[k] = s;
      }
      for (int t = 0; t < R->ntau; ++t) {
        double s = 0;
        for (int k = 0; k < dim; ++k) s += R->tau[n][t][k] * g[k];
        d[R->d_etau + n * R->ntau + t] = s;
      }
    }
    for (int s = 0; s < R->nlines; ++s)
      d[R->d_line + s] = S[((1 + dim + s) * nv + v) * N + id] * G->len[s];
  }
  double ref[MAXV][MAXGP * 4];
  double chi[MAXV];
  double force = c->d.linear ? 1.0 : -1.0;
  if (c->sel && !c->d.linear) {
    float feat[SEL_NF];
    sel_features(c, S, id, feat);
    const float lg = sel_logit(c->sel, feat);
    const double mg = fmin(fabs((double)lg - c->sel->thr_skip), fabs((double)lg - c->sel->thr_lo));
#pragma omp critical(orc_selector)
    {
      if (lg >= c->sel->thr_skip) c->nskip++;
      else if (lg > c->sel->thr_lo) c->nunsure++;
      if (mg < c->margin) c->margin = mg;
    }
    if (lg >= c->sel->thr_skip) force = 1.0; /* skip the adaptive weights: P4 alone */
  }
  for (int v = 0; v < nv; ++v) recon_var(R, dat[v], force, c->d.c_chi, ref[v], &chi[v]);
  /* positivity of the reconstructed Gauss-point states */
  int bad = !gp_states_physical(R, c->d.gamma, ref);
  if (bad) {
#pragma omp atomic
    c->npos_fallback++;
    for (int v = 0; v < nv; ++v) recon_var(R, dat[v], 0.0, c->d.c_chi, ref[v], &chi[v]);
    bad = !gp_states_physical(R, c->d.gamma, ref);
    if (bad) {
      /* last resort: first order, the cell average with zero gradient */
      for (int v = 0; v < nv; ++v)
        for (int gp = 0; gp < R->ngp; ++gp) {
          ref[v][gp * (1 + dim)] = dat[v][0];
          for (int k = 0; k < dim; ++k) ref[v][gp * (1 + dim) + 1 + k] = 0.0;
        }
    }
  }
  if (record_chi)
    for (int v = 0; v < nv; ++v) c->chi[(long)v * N + id] = chi[v];
  double* out = c->gpv + id * R->ngp * nv * (1 + dim);
  for (int gp = 0; gp < R->ngp; ++gp)
    for (int v = 0; v < nv; ++v) {
      double* o = out + (gp * nv + v) * (1 + dim);
      o[0] = ref[v][gp * (1 + dim)];
      for (int k = 0; k < dim; ++k) {
        double s = 0;
        for (int r = 0; r < dim; ++r) s += G->JinvT[k][r] * ref[v][gp * (1 + dim) + 1 + r];
        o[1 + k] = s;
      }
    }
}

/* local orthonormal frame: n from the area vector, t1 from the face tangent */
static void frame(int dim, const double* A, const double* T, double Rm[3][3]) {
  double an = 0;
  for (int a = 0; a < dim; ++a) an += A[a] * A[a];
  an = sqrt(an);
  double n[3] = {0, 0, 0};
  for (int a = 0; a < dim; ++a) n[a] = A[a] / an;
  memset(Rm, 0, sizeof(double) * 9);
  if (dim == 2) {
    Rm[0][0] = n[0]; Rm[0][1] = n[1];
    Rm[1][0] = -n[1]; Rm[1][1] = n[0];
    return;
  }
  double tn = T[0] * n[0] + T[1] * n[1] + T[2] * n[2];
  double t1[3] = {T[0] - tn * n[0], T[1] - tn * n[1], T[2] - tn * n[2]};
  double tl = sqrt(t1[0] * t1[0] + t1[1] * t1[1] + t1[2] * t1[2]);
  for (int a = 0; a < 3; ++a) t1[a] /= tl;
  double t2[3] = {n[1] * t1[2] - n[2] * t1[1], n[2] * t1[0] - n[0] * t1[2], n[0] * t1[1] - n[1] * t1[0]};
  for (int a = 0; a < 3; ++a) { Rm[0][a] = n[a]; Rm[1][a] = t1[a]; Rm[2][a] = t2[a]; }
}

static void rotate_in(int dim, double Rm[3][3], const double* o /* nv*(1+dim) */, int nv, double* W, double* dW) {
  /* values */
  double g[MAXV][3];
  for (int v = 0; v < nv; ++v) {
    W[v] = o[v * (1 + dim)];
    for (int k = 0; k < dim; ++k) g[v][k] = o[v * (1 + dim) + 1 + k];
  }
  double m[3];
  for (int i = 0; i < dim; ++i) { m[i] = 0; for (int a = 0; a < dim; ++a) m[i] += Rm[i][a] * W[1 + a]; }
  for (int i = 0; i < dim; ++i) W[1 + i] = m[i];
  /* gradients: rotate the momentum components, then take directional derivatives */
  double gr[MAXV][3];
  for (int k = 0; k < dim; ++k) {
    gr[0][k] = g[0][k];
    gr[dim + 1][k] = g[dim + 1][k];
    for (int i = 0; i < dim; ++i) { double s = 0; for (int a = 0; a < dim; ++a) s += Rm[i][a] * g[1 + a][k]; gr[1 + i][k] = s; }
  }
  for (int j = 0; j < dim; ++j)
    for (int v = 0; v < nv; ++v) {
      double s = 0;
      for (int k = 0; k < dim; ++k) s += Rm[j][k] * gr[v][k];
      dW[j * nv + v] = s;
    }
}

static void rotate_out(int dim, double Rm[3][3], double* F) {
  double m[3];
  for (int a = 0; a < dim; ++a) { m[a] = 0; for (int i = 0; i < dim; ++i) m[a] += Rm[i][a] * F[1 + i]; }
  for (int a = 0; a < dim; ++a) F[1 + a] = m[a];
}

/* A wall face (adiabatic; the paper's non-slip adiabatic wall and its slip
   counterpart) lets no mass and no energy through, and the gas on it moves
   along the wall (slip) or rests (no-slip): the flux from the mirrored states
   keeps its momentum part, its mass and energy parts are zero, and the
   interface values carry zero normal (slip) or zero total (no-slip) momentum. */
static void wall_face(int dim, int ax, int bc, int nv, double* out) {
  out[0] = out[nv] = 0.0;
  out[dim + 1] = out[nv + dim + 1] = 0.0;
  for (int p = 2; p < 6; ++p)
    for (int i = 0; i < dim; ++i)
      if (bc == BC_NOSLIP || i == ax) out[p * nv + 1 + i] = 0.0;
}

static int stage(orc_ctx* c, const double* S, double dt, double* Lout, double* Ltout, double* Dn, double* Dtn,
                 int record_chi) {
  const ref_t* R = c->R;
  const int dim = c->dim, nv = c->nv, gpf = R->gpf, ngp = R->ngp;
  const long N = c->ncell;
  const int stride = ngp * nv * (1 + dim);
  int err = 0;
#pragma omp parallel for schedule(dynamic, 64)
  for (long id = 0; id < N; ++id) recon_cell(c, S, id, record_chi);
  /* interface solutions: face (axis, cell L) between L and its +axis
     neighbour; at a non-periodic face the missing side is the mirror image
     (wall) or a copy (outflow) of the interior side's Gauss-point state */
#pragma omp parallel for schedule(dynamic, 64) reduction(| : err)
  for (long id = 0; id < N; ++id) {
    int ii[3] = {(int)(id % c->n[0]), (int)((id / c->n[0]) % c->n[1]),
                 dim == 3 ? (int)(id / ((long)c->n[0] * c->n[1])) : 0};
    for (int ax = 0; ax < dim; ++ax) {
      int o[3] = {0, 0, 0};
      o[ax] = 1;
      long rid = nbr(c, id, o);
      const int hi_bnd = ii[ax] == c->n[ax] - 1 && c->d.bc[2 * ax + 1] != BC_PERIODIC;
      const int lo_bnd = ii[ax] == 0 && c->d.bc[2 * ax] != BC_PERIODIC;
      for (int q = 0; q < gpf; ++q) {
        int gl = (2 * ax + 1) * gpf + q, gr = (2 * ax) * gpf + q;
        for (int pass = 0; pass < 1 + lo_bnd; ++pass) {
          /* pass 0: the high face of this cell; pass 1: its low boundary face */
          const int gown = pass == 0 ? gl : gr;
          const double* A = c->geo[id].area[gown];
          double Rm[3][3];
          frame(dim, A, c->geo[id].tang[gown], Rm);
          double st_in[MAXV * 4], st_bc[MAXV * 4];
          const double* own = c->gpv + id * stride + gown * nv * (1 + dim);
          const int bnd = pass == 0 ? hi_bnd : 1;
          const int bc = c->d.bc[2 * ax + (pass == 0 ? 1 : 0)];
          if (bnd && bc == BC_INFLOW) {
            const int f = 2 * ax + (pass == 0 ? 1 : 0);
            for (int v = 0; v < nv; ++v)
              for (int k = -1; k < dim; ++k) st_bc[v * (1 + dim) + 1 + k] = k < 0 ? c->d.bc_state[f][v] : 0.0;
          } else if (bnd) {
            int mi = bc == BC_OUTFLOW ? 0 : 1 << ax, ns = bc == BC_NOSLIP ? 1 << ax : 0;
            for (int v = 0; v < nv; ++v)
              for (int k = -1; k < dim; ++k)
                st_bc[v * (1 + dim) + 1 + k] = mirror_sign(dim, v, k, mi, ns) * own[v * (1 + dim) + 1 + k];
          }
          const double* sl = pass == 0 ? own : st_bc;
          const double* sr = pass == 0 ? (bnd ? st_bc : c->gpv + rid * stride + gr * nv * (1 + dim)) : own;
          double WL[MAXV], dWL[3 * MAXV], WR[MAXV], dWR[3 * MAXV];
          rotate_in(dim, Rm, sl, nv, WL, dWL);
          rotate_in(dim, Rm, sr, nv, WR, dWR);
          double* out = pass == 0 ? c->fx + ((id * dim + ax) * gpf + q) * 6 * nv
                                  : c->fxlo + ((id * dim + ax) * gpf + q) * 6 * nv;
          int st = gks_point(dim, c->d.gamma, c->d.mu, c->d.prandtl, c->d.tau_mode, dt, WL, dWL, WR, dWR, out);
          if (st) err |= 1;
          for (int p = 0; p < 6; ++p) rotate_out(dim, Rm, out + p * nv);
          if (bnd && (bc == BC_SLIP || bc == BC_NOSLIP)) wall_face(dim, ax, bc, nv, out);
        }
      }
    }
  }
  if (err) return -4;
  /* accumulate per cell: L = -(1/|Omega|) sum F.n dS (Eq. semi with Gauss
     quadrature); gradients by Gauss' theorem (Eq. derivative); line
     derivatives by Eq. (derivative-l) */
#pragma omp parallel for schedule(static)
  for (long id = 0; id < N; ++id) {
    const cellgeo_t* G = &c->geo[id];
    double Lc[MAXV] = {0}, Ltc[MAXV] = {0};
    double qn[MAXGP][MAXV], qt[MAXGP][MAXV];
    const int ii0 = (int)(id % c->n[0]), ii1 = (int)((id / c->n[0]) % c->n[1]);
    const int ii2 = dim == 3 ? (int)(id / ((long)c->n[0] * c->n[1])) : 0;
    const int iis[3] = {ii0, ii1, ii2};
    for (int ax = 0; ax < dim; ++ax) {
      int o[3] = {0, 0, 0};
      o[ax] = -1;
      long lid = nbr(c, id, o);
      const int lo_bnd = iis[ax] == 0 && c->d.bc[2 * ax] != BC_PERIODIC;
      for (int q = 0; q < gpf; ++q) {
        /* high face: this cell is the left side */
        const double* fh = c->fx + ((id * dim + ax) * gpf + q) * 6 * nv;
        const double* Ah = G->area[(2 * ax + 1) * gpf + q];
        double sh = 0;
        for (int a = 0; a < dim; ++a) sh += Ah[a] * Ah[a];
        sh = sqrt(sh);
        /* low face: this cell is the right side of the face owned by lid, or of
           its own boundary face */
        const double* fl = lo_bnd ? c->fxlo + ((id * dim + ax) * gpf + q) * 6 * nv
                                  : c->fx + ((lid * dim + ax) * gpf + q) * 6 * nv;
        const double* Al = lo_bnd ? G->area[(2 * ax) * gpf + q] : c->geo[lid].area[(2 * ax + 1) * gpf + q];
        double sl = 0;
        for (int a = 0; a < dim; ++a) sl += Al[a] * Al[a];
        sl = sqrt(sl);
        for (int v = 0; v < nv; ++v) {
          Lc[v] += -fh[v] * sh + fl[v] * sl;
          Ltc[v] += -fh[nv + v] * sh + fl[nv + v] * sl;
          qn[(2 * ax + 1) * gpf + q][v] = fh[2 * nv + v];
          qt[(2 * ax + 1) * gpf + q][v] = fh[3 * nv + v];
          qn[(2 * ax) * gpf + q][v] = fl[4 * nv + v];
          qt[(2 * ax) * gpf + q][v] = fl[5 * nv + v];
        }
      }
    }
    for (int v = 0; v < nv; ++v) {
      Lout[(long)v * N + id] = Lc[v] / G->vol;
      Ltout[(long)v * N + id] = Ltc[v] / G->vol;
      for (int pass = 0; pass < 2; ++pass) {
        double (*qq)[MAXV] = pass == 0 ? qn : qt;
        double* D = pass == 0 ? Dn : Dtn;
        if (!D) continue;
        for (int k = 0; k < dim; ++k) {
          double s = 0;
          for (int g = 0; g < ngp; ++g) {
            double sgn = ((g / gpf) & 1) ? 1.0 : -1.0;
            s += sgn * qq[g][v] * G->area[g][k];
          }
          D[((long)k * nv + v) * N + id] = s / G->vol;
        }
        for (int ax = 0; ax < dim; ++ax)
          for (int q = 0; q < gpf; ++q) {
            int s = ax * gpf + q;
            D[((long)(dim + s) * nv + v) * N + id] =
                (qq[(2 * ax + 1) * gpf + q][v] - qq[(2 * ax) * gpf + q][v]) / G->len[s];
          }
      }
    }
  }
  return 0;
}

/* S2O4 (temporal discretisation section) */
double orc_s2o4_stage1(double Q, double dt, double L, double Lt) {
  return Q + 0.5 * dt * L + 0.125 * dt * dt * Lt;
}
double orc_s2o4_stage2(double Q, double dt, double L, double Lt, double Lt_star) {
  return Q + dt * L + dt * dt / 6.0 * (Lt + 2.0 * Lt_star);
}

static int step_impl(orc_ctx* c, int nsteps, double dt_given, double* dt_last) {
  const int nv = c->nv, nf = c->nf;
  const long N = c->ncell;
  const long nderiv = (long)(nf - 1) * nv * N;
  double* Us = malloc(sizeof(double) * nf * nv * N);
  double* Dt2 = malloc(sizeof(double) * nderiv);
  int rc = 0;
  for (int s = 0; s < nsteps && !rc; ++s) {
    double dt = dt_given > 0 ? dt_given : orc_compute_dt(c);
    if (!(dt > 0) || !isfinite(dt)) { rc = -4; break; }
    /* stage 1 from U^n */
    rc = stage(c, c->U, dt, c->L1, c->Lt1, c->D1, c->Dt, 1);
    if (rc) break;
    for (long i = 0; i < (long)nv * N; ++i) Us[i] = orc_s2o4_stage1(c->U[i], dt, c->L1[i], c->Lt1[i]);
    /* interface values evolve as Q* = Q^n + dt/2 (dQ/dt)^n, so the derivative
       fields take the same linear combination */
    for (long i = 0; i < nderiv; ++i) Us[nv * N + i] = c->D1[i] + 0.5 * dt * c->Dt[i];
    /* stage 2 from U* */
    rc = stage(c, Us, dt, c->L2, c->Lt2, NULL, Dt2, 0);
    if (rc) break;
    for (long i = 0; i < (long)nv * N; ++i) c->U[i] = orc_s2o4_stage2(c->U[i], dt, c->L1[i], c->Lt1[i], c->Lt2[i]);
    for (long i = 0; i < nderiv; ++i) c->U[nv * N + i] = c->D1[i] + dt * Dt2[i];
    c->t += dt;
    if (dt_last) *dt_last = dt;
  }
  free(Us);
  free(Dt2);
  return rc;
}

int orc_step(orc_ctx* c, int nsteps, double* dt_last) { return step_impl(c, nsteps, 0.0, dt_last); }
int orc_step_dt(orc_ctx* c, double dt) { return step_impl(c, 1, dt, NULL); }

int orc_set_selector(orc_ctx* c, const float* params, float thr_skip, float thr_lo) {
  free(c->sel);
  c->sel = NULL;
  c->nskip = c->nunsure = 0;
  c->margin = 1e300;
  if (!params) return 0;
  c->sel = malloc(sizeof(struct selector));
  memcpy(c->sel->p, params, sizeof(float) * SEL_NPARAM);
  c->sel->thr_skip = thr_skip;
  c->sel->thr_lo = thr_lo;
  return 0;
}

int orc_selector_stats(const orc_ctx* c, long* nskip, long* nunsure, double* margin) {
  *nskip = c->nskip;
  *nunsure = c->nunsure;
  *margin = c->margin;
  return 0;
}

/* features of every cell of the current state, [cell][16] */
int orc_selector_features(const orc_ctx* c, float* out) {
#pragma omp parallel for schedule(static)
  for (long id = 0; id < c->ncell; ++id) sel_features(c, c->U, id, out + id * SEL_NF);
  return 0;
}

/* the emulated BF16 logit of given features (unit-level) */
int orc_selector_logits(const float* params, const float* feat, long n, float* out) {
  struct selector sl;
  memcpy(sl.p, params, sizeof(float) * SEL_NPARAM);
  for (long i = 0; i < n; ++i) out[i] = sel_logit(&sl, feat + i * SEL_NF);
  return 0;
}

int orc_selector_nparam(void) { return SEL_NPARAM; }

int orc_get_chi(const orc_ctx* c, double* chi) {
  memcpy(chi, c->chi, sizeof(double) * c->nv * c->ncell);
  return 0;
}
long orc_positivity_fallbacks(const orc_ctx* c) { return c->npos_fallback; }

/* ------------------------------------------------------------------------ */
/* 9. Unit-level entry points.                                              */
/* ------------------------------------------------------------------------ */
int orc_basis_size(int dim) { const ref_t* R = get_ref(dim); return R ? R->nb : -1; }
int orc_data_size(int dim) { const ref_t* R = get_ref(dim); return R ? R->nd : -1; }

int orc_recon_matrix(int dim, double* M, int* exps) {
  const ref_t* R = get_ref(dim);
  if (!R) return -1;
  for (int b = 0; b < R->nb; ++b) {
    for (int c = 0; c < R->nd; ++c) M[b * R->nd + c] = R->M[b][c];
    for (int k = 0; k < 3; ++k) exps[b * 3 + k] = R->exps[b][k];
  }
  return 0;
}

int orc_recon_reference(int dim, const double* data, int linear, double c_chi, double* out, double* chi) {
  const ref_t* R = get_ref(dim);
  if (!R) return -1;
  const double chi_force = linear == 1 ? 1.0 : (linear == 2 ? 0.0 : -1.0);
  recon_var(R, data, chi_force, c_chi > 0 ? c_chi : 100.0, out, chi);
  return 0;
}

int orc_recon_coeffs(int dim, const double* data, double* a) {
  const ref_t* R = get_ref(dim);
  if (!R) return -1;
  for (int b = 0; b < R->nb; ++b) {
    double s = 0;
    for (int c = 0; c < R->nd; ++c) s += R->M[b][c] * data[c];
    a[b] = s;
  }
  return 0;
}

int orc_gram(int dim, double* GH, double* GL) {
  const ref_t* R = get_ref(dim);
  if (!R) return -1;
  for (int b = 0; b < R->nb; ++b)
    for (int c = 0; c < R->nb; ++c) { GH[b * R->nb + c] = R->GH[b][c]; GL[b * R->nb + c] = R->GL[b][c]; }
  return 0;
}

int orc_linear_sub(int dim, int m, const double* data, double* b) {
  const ref_t* R = get_ref(dim);
  if (!R || m < 0 || m >= 2 * dim) return -1;
  for (int k = 0; k < dim; ++k) {
    double s = 0;
    for (int c = 0; c < R->nd; ++c) s += R->M1[m][k][c] * data[c];
    b[k] = s;
  }
  return 0;
}

int orc_gks_point(int dim, double gamma, double mu, double prandtl, int tau_mode, double dt, const double* WL,
                  const double* dWL, const double* WR, const double* dWR, double* out) {
  return gks_point(dim, gamma, mu, prandtl, tau_mode, dt, WL, dWL, WR, dWR, out);
}

int orc_moments_u(double U, double lam, double* full, double* pos, double* neg) {
  double f[9], p[9], n[9];
  moments_1d(U, lam, f, p, n);
  for (int i = 0; i < 7; ++i) { full[i] = f[i]; pos[i] = p[i]; neg[i] = n[i]; }
  return 0;
}

int orc_micro_slope(int dim, double gamma, const double* prim, const double* b, double* a) {
  maxw_t g;
  memset(&g, 0, sizeof g);
  g.rho = prim[0];
  for (int i = 0; i < dim; ++i) g.U[i] = prim[1 + i];
  g.lam = prim[dim + 1];
  double d1[9], d2[9];
  moments_1d(g.U[0], g.lam, g.mu_full, g.mu_pos, g.mu_neg);
  moments_1d(g.U[1], g.lam, g.mv, d1, d2);
  if (dim == 3) moments_1d(g.U[2], g.lam, g.mw, d1, d2);
  else { memset(g.mw, 0, sizeof g.mw); g.mw[0] = 1.0; }
  double K = n_internal(dim, gamma);
  g.mxi[0] = 1.0; g.mxi[1] = K / (2.0 * g.lam); g.mxi[2] = (K * K + 2.0 * K) / (4.0 * g.lam * g.lam);
  return slope(dim, &g, b, a);
}
