/*
 * Device arithmetic of the CGKS-5 sweep (arXiv 2508.08965).
 *
 * Per-cell / per-face / per-point routines are CGKS_HD functions; the kernels
 * in cgks_kernels.cuh are thin wrappers that map threads onto them.
 *
 * Storage (all SoA over cells, FP64):
 *   state   [(f*NV + v)*ncell + cell]                         (public layout)
 *   gpL/gpR [((ax*GPF + k)*NV + v)*(1+DIM) + comp][ncell]      face Gauss-point states,
 *           L = the face's low cell at its high face, R = the high cell at its low face;
 *           face (ax, c) lies between cell c and its +ax neighbour; comp 0 value,
 *           1..DIM physical gradient
 *   flux    [((ax*GPF + k)*6 + part)*NV + v][ncell]            parts: F^n, F_t^n, Q^l(0),
 *           (dQ/dt)^l, Q^r(0), (dQ/dt)^r, all in the global frame, per unit area
 */
#pragma once
#include <math.h>
#include <stdint.h>

#ifndef CGKS_HD
#define CGKS_HD __host__ __device__ __forceinline__
#endif

#include "cgks_tables.h"

namespace cgks {

/* ---------------- compile-time sizes ---------------- */
template <int DIM> struct Sz;
template <> struct Sz<2> {
  static constexpr int NB = T2_NB, ND = T2_ND, NGP = T2_NGP, GPF = 2, NE = 4, NTAU = 1, NV = 4, NL = 4, NF = 7;
};
template <> struct Sz<3> {
  static constexpr int NB = T3_NB, ND = T3_ND, NGP = T3_NGP, GPF = 4, NE = 12, NTAU = 2, NV = 5, NL = 12, NF = 16;
};

template <int DIM> CGKS_HD double tabM(int b, int c) {
  if constexpr (DIM == 3) return T3_M[b][c]; else return T2_M[b][c];
}
template <int DIM> CGKS_HD double tabGH(int b, int c) {
  if constexpr (DIM == 3) return T3_GH[b][c]; else return T2_GH[b][c];
}
template <int DIM> CGKS_HD double tabGL(int b, int c) {
  if constexpr (DIM == 3) return T3_GL[b][c]; else return T2_GL[b][c];
}
template <int DIM> CGKS_HD double tabPV(int g, int b) {
  if constexpr (DIM == 3) return T3_PV[g][b]; else return T2_PV[g][b];
}
template <int DIM> CGKS_HD double tabPD(int g, int k, int b) {
  if constexpr (DIM == 3) return T3_PD[g][k][b]; else return T2_PD[g][k][b];
}

/* 2-point Gauss on [-1/2, 1/2] */
#define CGKS_GQ 0.28867513459481288225

/* reference position delta of face Gauss point gp = (2*ax+side)*GPF + k */
template <int DIM> CGKS_HD double gp_delta(int gp, int a) {
  const int GPF = Sz<DIM>::GPF;
  int f = gp / GPF, k = gp % GPF, ax = f / 2, side = f & 1;
  if (a == ax) return side ? 0.5 : -0.5;
  int t = 0;  /* rank of `a` among the tangential axes */
  for (int q = 0; q < a; ++q) if (q != ax) ++t;
  int bit = (t == 0) ? (k & 1) : (k & 2);
  return bit ? CGKS_GQ : -CGKS_GQ;
}

/* ---------------- mesh description ---------------- */
/* curvilinear metric record per cell, SoA [field][ncell] */
template <int DIM> struct Met {
  static constexpr int J0 = 0;                         /* 9: J0[r][c] */
  static constexpr int JIT = 9;                        /* 9: (J0^T)^{-1}[r][c] */
  static constexpr int VOL = 18;                       /* 1 */
  static constexpr int AREA = 19;                      /* NGP*3: own face Gauss-point area vectors (+xi) */
  static constexpr int TANG = AREA + Sz<DIM>::NGP * 3; /* DIM*GPF*3: first tangent of the high faces */
  static constexpr int LEN = TANG + DIM * Sz<DIM>::GPF * 3; /* NL: line lengths */
  static constexpr int N = LEN + Sz<DIM>::NL;
};

struct DevGeo {
  int n[3];
  long ncell;
  int curvi;          /* 0: uniform box with spacing h */
  double h[3];
  const double* met;  /* curvilinear metrics (Met<DIM>), or null */
};

struct Phys {
  double gamma, mu, prandtl, cfl, c_chi;
  int tau_mode, linear;
};

CGKS_HD long cell_index(const DevGeo& g, int i, int j, int k) {
  return i + (long)g.n[0] * (j + (long)g.n[1] * k);
}
CGKS_HD void cell_ijk(const DevGeo& g, long c, int& i, int& j, int& k) {
  i = (int)(c % g.n[0]);
  long r = c / g.n[0];
  j = (int)(r % g.n[1]);
  k = (int)(r / g.n[1]);
}
/* periodic neighbour */
CGKS_HD long nbr(const DevGeo& g, int i, int j, int k, int ox, int oy, int oz) {
  int a = i + ox, b = j + oy, c = k + oz;
  a = a < 0 ? a + g.n[0] : (a >= g.n[0] ? a - g.n[0] : a);
  b = b < 0 ? b + g.n[1] : (b >= g.n[1] ? b - g.n[1] : b);
  c = c < 0 ? c + g.n[2] : (c >= g.n[2] ? c - g.n[2] : c);
  return cell_index(g, a, b, c);
}

template <int DIM> CGKS_HD double met_J0(const DevGeo& g, long c, int r, int q) {
  if (!g.curvi) return r == q ? g.h[r] : 0.0;
  return g.met[(long)(Met<DIM>::J0 + r * 3 + q) * g.ncell + c];
}
template <int DIM> CGKS_HD double met_JiT(const DevGeo& g, long c, int r, int q) {
  if (!g.curvi) return r == q ? 1.0 / g.h[r] : 0.0;
  return g.met[(long)(Met<DIM>::JIT + r * 3 + q) * g.ncell + c];
}
template <int DIM> CGKS_HD double met_vol(const DevGeo& g, long c) {
  if (!g.curvi) return DIM == 3 ? g.h[0] * g.h[1] * g.h[2] : g.h[0] * g.h[1];
  return g.met[(long)Met<DIM>::VOL * g.ncell + c];
}
/* area vector component a of the cell's own face Gauss point gp (pointing to +xi_ax) */
template <int DIM> CGKS_HD double met_area(const DevGeo& g, long c, int gp, int a) {
  if (!g.curvi) {
    const int ax = gp / Sz<DIM>::GPF / 2;
    if (a != ax) return 0.0;
    double s = 1.0;
    for (int q = 0; q < DIM; ++q) if (q != ax) s *= g.h[q];
    return s / Sz<DIM>::GPF;
  }
  return g.met[(long)(Met<DIM>::AREA + gp * 3 + a) * g.ncell + c];
}
template <int DIM> CGKS_HD double met_tang(const DevGeo& g, long c, int ax, int k, int a) {
  if (!g.curvi) {
    int t0 = ax == 0 ? 1 : 0;
    return a == t0 ? 1.0 : 0.0;
  }
  return g.met[(long)(Met<DIM>::TANG + (ax * Sz<DIM>::GPF + k) * 3 + a) * g.ncell + c];
}
template <int DIM> CGKS_HD double met_len(const DevGeo& g, long c, int s) {
  if (!g.curvi) return g.h[s / Sz<DIM>::GPF];
  return g.met[(long)(Met<DIM>::LEN + s) * g.ncell + c];
}

/* ===================================================================== */
/* (a) reconstruction of one variable of one cell                        */
/* ===================================================================== */
/* Loads the data vector of Eq. (compact-big-ref) in the order of the
   generated tables, forms a = M d, the linear sub-stencil gradients of
   Eq. (compact-sub-2) (closed form: the face-neighbour difference along the
   connecting axis, the mean of the four (two) line differences along each
   other axis), the GENO weights, and writes the blended value and physical
   gradient at every face Gauss point.  chi_force >= 0 overrides chi.
   Returns chi. */
template <int DIM>
CGKS_HD double recon_var(const double* __restrict__ U, const DevGeo& g, const Phys& ph, long c, int ci, int cj,
                         int ck, int v, double chi_force, double* __restrict__ gpL, double* __restrict__ gpR) {
  typedef Sz<DIM> S;
  const long N = g.ncell;
  const int NV = S::NV;
  double a[S::NB];
#pragma unroll
  for (int b = 0; b < S::NB; ++b) a[b] = 0.0;
  double J0[3][3];
#pragma unroll
  for (int r = 0; r < DIM; ++r)
#pragma unroll
    for (int q = 0; q < DIM; ++q) J0[r][q] = met_J0<DIM>(g, c, r, q);

  const double q0 = U[(long)v * N + c];
#pragma unroll
  for (int b = 0; b < S::NB; ++b) a[b] += tabM<DIM>(b, 0) * q0;
  int col = 1;
  double qf[2 * DIM];
  /* face neighbours -x,+x,-y,+y(,-z,+z): average and J0^T grad */
#pragma unroll
  for (int m = 0; m < 2 * DIM; ++m) {
    int o[3] = {0, 0, 0};
    o[m / 2] = (m & 1) ? 1 : -1;
    long nb = nbr(g, ci, cj, ck, o[0], o[1], o[2]);
    double q = U[(long)v * N + nb];
    qf[m] = q;
#pragma unroll
    for (int b = 0; b < S::NB; ++b) a[b] += tabM<DIM>(b, col) * q;
    ++col;
    double gp[3];
#pragma unroll
    for (int r = 0; r < DIM; ++r) gp[r] = U[((long)(1 + r) * NV + v) * N + nb];
#pragma unroll
    for (int kk = 0; kk < DIM; ++kk) {
      double s = 0.0;
#pragma unroll
      for (int r = 0; r < DIM; ++r) s += J0[r][kk] * gp[r];
#pragma unroll
      for (int b = 0; b < S::NB; ++b) a[b] += tabM<DIM>(b, col) * s;
      ++col;
    }
  }
  /* edge (3-D) / corner (2-D) neighbours, offsets in (oz, oy, ox) order */
#pragma unroll
  for (int oz = (DIM == 3 ? -1 : 0); oz <= (DIM == 3 ? 1 : 0); ++oz)
#pragma unroll
    for (int oy = -1; oy <= 1; ++oy)
#pragma unroll
      for (int ox = -1; ox <= 1; ++ox) {
        int nzc = (ox != 0) + (oy != 0) + (oz != 0);
        if (nzc != 2) continue;
        long nb = nbr(g, ci, cj, ck, ox, oy, oz);
        double q = U[(long)v * N + nb];
#pragma unroll
        for (int b = 0; b < S::NB; ++b) a[b] += tabM<DIM>(b, col) * q;
        ++col;
        double gp[3], gr[3];
#pragma unroll
        for (int r = 0; r < DIM; ++r) gp[r] = U[((long)(1 + r) * NV + v) * N + nb];
#pragma unroll
        for (int kk = 0; kk < DIM; ++kk) {
          double s = 0.0;
#pragma unroll
          for (int r = 0; r < DIM; ++r) s += J0[r][kk] * gp[r];
          gr[kk] = s;
        }
        int o[3] = {ox, oy, oz};
        if (DIM == 3) { /* along the shared edge: the axis with zero offset */
          int ze = ox == 0 ? 0 : (oy == 0 ? 1 : 2);
          double d = gr[ze];
#pragma unroll
          for (int b = 0; b < S::NB; ++b) a[b] += tabM<DIM>(b, col) * d;
          ++col;
        }
        { /* toward the neighbour centroid (un-normalised offset vector) */
          double d = 0.0;
#pragma unroll
          for (int kk = 0; kk < DIM; ++kk) d += o[kk] * gr[kk];
#pragma unroll
          for (int b = 0; b < S::NB; ++b) a[b] += tabM<DIM>(b, col) * d;
          ++col;
        }
      }
  /* own line differences (reference frame): stored derivative x length */
  double lsum[3] = {0.0, 0.0, 0.0};
#pragma unroll
  for (int s = 0; s < S::NL; ++s) {
    double d = U[((long)(1 + DIM + s) * NV + v) * N + c] * met_len<DIM>(g, c, s);
    lsum[s / S::GPF] += d;
#pragma unroll
    for (int b = 0; b < S::NB; ++b) a[b] += tabM<DIM>(b, col) * d;
    ++col;
  }

  /* GENO path function (Sec. 3.3) */
  double chi;
  if (chi_force >= 0.0) {
    chi = chi_force;
  } else {
    double ish = 0.0, isl = 0.0;
#pragma unroll
    for (int b = 0; b < S::NB; ++b) {
      double th = 0.0, tl = 0.0;
#pragma unroll
      for (int q = 0; q < S::NB; ++q) {
        th += tabGH<DIM>(b, q) * a[q];
        tl += tabGL<DIM>(b, q) * a[q];
      }
      ish += a[b] * th;
      isl += a[b] * tl;
    }
    const double eps = 1e-15;
    double ist = ish - isl;
    if (ist < 0.0) ist = 0.0;
    double rh = ist / (ish + eps), rl = ist / (isl + eps);
    double ah = 1.0 + rh * rh, al = 1.0 + rl * rl;
    double alpha = 2.0 * ah / (ah + al);
    chi = tanh(ph.c_chi * alpha) / tanh(ph.c_chi);
  }
  /* linear sub-stencil polynomials and their WENO weights (d_m = 1/(2 dim)) */
  double bbar[3] = {0.0, 0.0, 0.0};
  {
    double bm[2 * DIM][3], wb[2 * DIM], ws = 0.0;
#pragma unroll
    for (int m = 0; m < 2 * DIM; ++m) {
      int ax = m / 2;
      double sg = (m & 1) ? 1.0 : -1.0;
      double is = 0.0;
#pragma unroll
      for (int kk = 0; kk < DIM; ++kk) {
        double bv = (kk == ax) ? sg * (qf[m] - q0) : lsum[kk] * (1.0 / S::GPF);
        bm[m][kk] = bv;
        is += bv * bv;
      }
      double t = is + 1e-15;
      double t2 = t * t;
      wb[m] = (1.0 / (2 * DIM)) / (t2 * t2 * t);
      ws += wb[m];
    }
#pragma unroll
    for (int m = 0; m < 2 * DIM; ++m) {
      double w = wb[m] / ws;
#pragma unroll
      for (int kk = 0; kk < DIM; ++kk) bbar[kk] += w * bm[m][kk];
    }
  }
  double JiT[3][3];
#pragma unroll
  for (int r = 0; r < DIM; ++r)
#pragma unroll
    for (int q = 0; q < DIM; ++q) JiT[r][q] = met_JiT<DIM>(g, c, r, q);
  /* blended values at the face Gauss points, Eq. (weno-new) */
#pragma unroll 1
  for (int gp = 0; gp < S::NGP; ++gp) {
    double v4 = q0, g4[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int b = 0; b < S::NB; ++b) {
      v4 += a[b] * tabPV<DIM>(gp, b);
#pragma unroll
      for (int kk = 0; kk < DIM; ++kk) g4[kk] += a[b] * tabPD<DIM>(gp, kk, b);
    }
    double v1 = q0;
#pragma unroll
    for (int kk = 0; kk < DIM; ++kk) v1 += bbar[kk] * gp_delta<DIM>(gp, kk);
    double val = chi * v4 + (1.0 - chi) * v1;
    double gref[3];
#pragma unroll
    for (int kk = 0; kk < DIM; ++kk) gref[kk] = chi * g4[kk] + (1.0 - chi) * bbar[kk];
    int f = gp / S::GPF, k = gp % S::GPF, ax = f / 2, side = f & 1;
    double* dst;
    long cell;
    if (side) {
      dst = gpL;
      cell = c;
    } else {
      dst = gpR;
      int o[3] = {0, 0, 0};
      o[ax] = -1;
      cell = nbr(g, ci, cj, ck, o[0], o[1], o[2]);
    }
    long base = ((long)((ax * S::GPF + k) * NV + v) * (1 + DIM)) * N + cell;
    dst[base] = val;
#pragma unroll
    for (int kk = 0; kk < DIM; ++kk) {
      double s = 0.0;
#pragma unroll
      for (int r = 0; r < DIM; ++r) s += JiT[kk][r] * gref[r];
      dst[base + (long)(1 + kk) * N] = s;
    }
  }
  return chi;
}

/* positivity of the reconstructed Gauss-point states of a cell (C18 reading:
   the states just written by this thread are read back) */
template <int DIM>
CGKS_HD bool cell_states_physical(const DevGeo& g, const Phys& ph, long c, int ci, int cj, int ck,
                                  const double* __restrict__ gpL, const double* __restrict__ gpR) {
  typedef Sz<DIM> S;
  const long N = g.ncell;
  for (int gp = 0; gp < S::NGP; ++gp) {
    int f = gp / S::GPF, k = gp % S::GPF, ax = f / 2, side = f & 1;
    const double* src;
    long cell;
    if (side) {
      src = gpL;
      cell = c;
    } else {
      src = gpR;
      int o[3] = {0, 0, 0};
      o[ax] = -1;
      cell = nbr(g, ci, cj, ck, o[0], o[1], o[2]);
    }
    double w[S::NV];
    for (int v = 0; v < S::NV; ++v) w[v] = src[((long)((ax * S::GPF + k) * S::NV + v) * (1 + DIM)) * N + cell];
    double ke = 0.0;
    for (int i = 0; i < DIM; ++i) ke += w[1 + i] * w[1 + i];
    double p = (ph.gamma - 1.0) * (w[DIM + 1] - 0.5 * ke / w[0]);
    if (!(w[0] > 0.0) || !(p > 0.0)) return false;
  }
  return true;
}

/* ===================================================================== */
/* (b) gas-kinetic interface solution at one Gauss point (Sec. 2)        */
/* ===================================================================== */
template <int DIM> struct Maxw {
  double rho, U[3], lam;
};

/* normalised moments <u^n> (normal direction, full or half space), <v^n>,
   <w^n> (full), <xi^2>, <xi^4> */
struct Mom {
  double u[7], v[7], w[7], xi2, xi4;
};

CGKS_HD void mom1d_full(double U, double lam, double* m) {
  m[0] = 1.0;
  m[1] = U;
  for (int n = 0; n + 2 < 7; ++n) m[n + 2] = U * m[n + 1] + (n + 1) / (2.0 * lam) * m[n];
}

/* region: 0 full, 1 u > 0, 2 u < 0 */
template <int DIM>
CGKS_HD void moments(const Maxw<DIM>& g, double K, int region, Mom& T) {
  if (region == 0) {
    mom1d_full(g.U[0], g.lam, T.u);
  } else {
    double sl = sqrt(g.lam);
    double e = 0.5 * exp(-g.lam * g.U[0] * g.U[0]) / sqrt(3.14159265358979323846 * g.lam);
    if (region == 1) {
      T.u[0] = 0.5 * erfc(-sl * g.U[0]);
      T.u[1] = g.U[0] * T.u[0] + e;
    } else {
      T.u[0] = 0.5 * erfc(sl * g.U[0]);
      T.u[1] = g.U[0] * T.u[0] - e;
    }
    for (int n = 0; n + 2 < 7; ++n) T.u[n + 2] = g.U[0] * T.u[n + 1] + (n + 1) / (2.0 * g.lam) * T.u[n];
  }
  mom1d_full(g.U[1], g.lam, T.v);
  if (DIM == 3) {
    mom1d_full(g.U[2], g.lam, T.w);
  } else {
    T.w[0] = 1.0;
    for (int n = 1; n < 7; ++n) T.w[n] = 0.0;
  }
  T.xi2 = K / (2.0 * g.lam);
  T.xi4 = (K * K + 2.0 * K) / (4.0 * g.lam * g.lam);
}

/* <u^a v^b w^c psi> */
template <int DIM>
CGKS_HD void mpsi(const Mom& T, int a, int b, int c, double* o) {
  double m0 = T.u[a] * T.v[b] * T.w[c];
  o[0] = m0;
  o[1] = T.u[a + 1] * T.v[b] * T.w[c];
  o[2] = T.u[a] * T.v[b + 1] * T.w[c];
  double e = T.u[a + 2] * T.v[b] * T.w[c] + T.u[a] * T.v[b + 2] * T.w[c] + m0 * T.xi2;
  if (DIM == 3) {
    o[3] = T.u[a] * T.v[b] * T.w[c + 1];
    e += T.u[a] * T.v[b] * T.w[c + 2];
  }
  o[DIM + 1] = 0.5 * e;
}

/* <xi^2 u^a v^b w^c psi> */
template <int DIM>
CGKS_HD void mpsi_xi2(const Mom& T, int a, int b, int c, double* o) {
  double m0 = T.u[a] * T.v[b] * T.w[c];
  o[0] = m0 * T.xi2;
  o[1] = T.u[a + 1] * T.v[b] * T.w[c] * T.xi2;
  o[2] = T.u[a] * T.v[b + 1] * T.w[c] * T.xi2;
  double e = (T.u[a + 2] * T.v[b] * T.w[c] + T.u[a] * T.v[b + 2] * T.w[c]) * T.xi2 + m0 * T.xi4;
  if (DIM == 3) {
    o[3] = T.u[a] * T.v[b] * T.w[c + 1] * T.xi2;
    e += T.u[a] * T.v[b] * T.w[c + 2] * T.xi2;
  }
  o[DIM + 1] = 0.5 * e;
}

/* <(al . psi) u^a v^b w^c psi> */
template <int DIM>
CGKS_HD void mapsi(const Mom& T, const double* al, int a, int b, int c, double* o) {
  const int NV = DIM + 2;
  double t[NV], e[NV];
  mpsi<DIM>(T, a, b, c, t);
  for (int i = 0; i < NV; ++i) o[i] = al[0] * t[i];
  mpsi<DIM>(T, a + 1, b, c, t);
  for (int i = 0; i < NV; ++i) o[i] += al[1] * t[i];
  mpsi<DIM>(T, a, b + 1, c, t);
  for (int i = 0; i < NV; ++i) o[i] += al[2] * t[i];
  if (DIM == 3) {
    mpsi<DIM>(T, a, b, c + 1, t);
    for (int i = 0; i < NV; ++i) o[i] += al[3] * t[i];
  }
  mpsi<DIM>(T, a + 2, b, c, e);
  mpsi<DIM>(T, a, b + 2, c, t);
  for (int i = 0; i < NV; ++i) e[i] += t[i];
  if (DIM == 3) {
    mpsi<DIM>(T, a, b, c + 2, t);
    for (int i = 0; i < NV; ++i) e[i] += t[i];
  }
  mpsi_xi2<DIM>(T, a, b, c, t);
  for (int i = 0; i < NV; ++i) o[i] += 0.5 * al[NV - 1] * (e[i] + t[i]);
}

/* micro-slope: solve <a psi psi^T> = b in closed form (D = K + dim = 2/(gamma-1)) */
template <int DIM>
CGKS_HD void slope(const Maxw<DIM>& g, double D, const double* b, double* a) {
  double q2 = 0.0, R[3], uR = 0.0;
  for (int i = 0; i < DIM; ++i) {
    q2 += g.U[i] * g.U[i];
    R[i] = b[1 + i] - g.U[i] * b[0];
    uR += g.U[i] * R[i];
  }
  double th = q2 + D / (2.0 * g.lam);
  double Re = 2.0 * b[DIM + 1] - th * b[0];
  double ae = 4.0 * g.lam * g.lam / D * (Re - 2.0 * uR);
  double s = 0.0;
  for (int i = 0; i < DIM; ++i) {
    a[1 + i] = 2.0 * g.lam * R[i] - g.U[i] * ae;
    s += g.U[i] * a[1 + i];
  }
  a[DIM + 1] = ae;
  a[0] = b[0] - s - 0.5 * ae * th;
}

template <int DIM>
CGKS_HD bool maxw_of(const double* W, double gam, Maxw<DIM>& m) {
  m.rho = W[0];
  double ke = 0.0;
  for (int i = 0; i < 3; ++i) m.U[i] = 0.0;
  for (int i = 0; i < DIM; ++i) {
    m.U[i] = W[1 + i] / W[0];
    ke += m.U[i] * W[1 + i];
  }
  double p = (gam - 1.0) * (W[DIM + 1] - 0.5 * ke);
  m.lam = W[0] / (2.0 * p);
  return (W[0] > 0.0) && (p > 0.0);
}

/* time integrals over [0, dl] of the six coefficient functions of Eq. (flux) */
CGKS_HD void tcoef(double tau, double dl, double* c) {
  if (tau <= 0.0) {
    c[0] = dl; c[1] = 0.0; c[2] = 0.5 * dl * dl; c[3] = 0.0; c[4] = 0.0; c[5] = 0.0;
    return;
  }
  double em = -expm1(-dl / tau);
  double ex = exp(-dl / tau);
  c[0] = dl - tau * em;
  c[1] = 2.0 * tau * tau - tau * (dl + 2.0 * tau) * ex - tau * dl;
  c[2] = 0.5 * dl * dl - tau * dl + tau * tau * em;
  c[3] = tau * em;
  c[4] = -2.0 * tau * tau + tau * (dl + 2.0 * tau) * ex;
  c[5] = -tau * tau * em;
}

/* Local frame (x normal): W* values, dW*[j][v] derivatives along local axis j.
   out[part*NV + v], parts F^n, F_t^n, Q^l(0), (dQ/dt)^l, Q^r(0), (dQ/dt)^r.
   Returns false on a non-physical state. */
template <int DIM>
CGKS_HD bool gks_point(const Phys& ph, double dt, const double* WL, const double* dWL, const double* WR,
                       const double* dWR, double* out) {
  const int NV = DIM + 2;
  const double gam = ph.gamma;
  const double D = 2.0 / (gam - 1.0);
  const double K = D - DIM;
  Maxw<DIM> gl, gr, g0;
  if (!maxw_of<DIM>(WL, gam, gl) || !maxw_of<DIM>(WR, gam, gr)) return false;
  Mom Tlp, Trn, Tlf, Trf, T0;
  moments<DIM>(gl, K, 1, Tlp);
  moments<DIM>(gr, K, 2, Trn);
  double W0[NV], t1[NV], t2[NV];
  mpsi<DIM>(Tlp, 0, 0, 0, t1);
  mpsi<DIM>(Trn, 0, 0, 0, t2);
  for (int i = 0; i < NV; ++i) W0[i] = gl.rho * t1[i] + gr.rho * t2[i];
  if (!maxw_of<DIM>(W0, gam, g0)) return false;
  moments<DIM>(g0, K, 0, T0);
  moments<DIM>(gl, K, 0, Tlf);
  moments<DIM>(gr, K, 0, Trf);
  /* spatial micro-slopes of the two sides and of g0 */
  double al[DIM][NV], ar[DIM][NV], a0[DIM][NV];
  for (int j = 0; j < DIM; ++j) {
    double b[NV];
    for (int i = 0; i < NV; ++i) b[i] = dWL[j * NV + i] / gl.rho;
    slope<DIM>(gl, D, b, al[j]);
    for (int i = 0; i < NV; ++i) b[i] = dWR[j * NV + i] / gr.rho;
    slope<DIM>(gr, D, b, ar[j]);
    mapsi<DIM>(Tlp, al[j], 0, 0, 0, t1);
    mapsi<DIM>(Trn, ar[j], 0, 0, 0, t2);
    for (int i = 0; i < NV; ++i) b[i] = (gl.rho * t1[i] + gr.rho * t2[i]) / g0.rho;
    slope<DIM>(g0, D, b, a0[j]);
  }
  /* time slopes: compatibility <(a.u + A) psi> = 0 */
  double bl[NV], br[NV], b0[NV];
  for (int i = 0; i < NV; ++i) bl[i] = br[i] = b0[i] = 0.0;
  for (int j = 0; j < DIM; ++j) {
    int e0 = j == 0, e1 = j == 1, e2 = j == 2;
    mapsi<DIM>(Tlf, al[j], e0, e1, e2, t1);
    for (int i = 0; i < NV; ++i) bl[i] -= t1[i];
    mapsi<DIM>(Trf, ar[j], e0, e1, e2, t1);
    for (int i = 0; i < NV; ++i) br[i] -= t1[i];
    mapsi<DIM>(T0, a0[j], e0, e1, e2, t1);
    for (int i = 0; i < NV; ++i) b0[i] -= t1[i];
  }
  double Al[NV], Ar[NV], A0[NV];
  slope<DIM>(gl, D, bl, Al);
  slope<DIM>(gr, D, br, Ar);
  slope<DIM>(g0, D, b0, A0);
  /* collision time (Sec. 6) */
  double pl = gl.rho / (2.0 * gl.lam), pr = gr.rho / (2.0 * gr.lam), p0 = g0.rho / (2.0 * g0.lam);
  double jump = fabs((pl - pr) / (pl + pr));
  double tau = 0.0;
  if (ph.tau_mode == 1) tau = 0.05 * dt + 5.0 * jump * dt;
  else if (ph.tau_mode == 2) tau = ph.mu / p0 + 5.0 * jump * dt;
  double cf[6], chf[6], cn[6], ct[6];
  tcoef(tau, dt, cf);
  tcoef(tau, 0.5 * dt, chf);
  for (int i = 0; i < 6; ++i) {
    cn[i] = (4.0 * chf[i] - cf[i]) / dt;
    ct[i] = 4.0 * (cf[i] - 2.0 * chf[i]) / (dt * dt);
  }
  const bool prfix = ph.mu > 0.0 && ph.prandtl > 0.0 && ph.prandtl != 1.0;
  double Fn[NV], Ft[NV], Qn[NV], Qt[NV];
  for (int i = 0; i < NV; ++i) Fn[i] = Ft[i] = Qn[i] = Qt[i] = 0.0;
  for (int pass = 0; pass < (prfix ? 2 : 1); ++pass) {
    const int xu = pass == 0 ? 1 : 0; /* u-moment for fluxes, none for Q */
    double* An = pass == 0 ? Fn : Qn;
    double* At = pass == 0 ? Ft : Qt;
    double part[NV], s1[NV], s2[NV];
    /* g0 */
    mpsi<DIM>(T0, xu, 0, 0, s1);
    for (int i = 0; i < NV; ++i) { part[i] = g0.rho * s1[i]; An[i] += cn[0] * part[i]; At[i] += ct[0] * part[i]; }
    for (int i = 0; i < NV; ++i) part[i] = 0.0;
    for (int j = 0; j < DIM; ++j) {
      mapsi<DIM>(T0, a0[j], xu + (j == 0), j == 1, j == 2, s1);
      for (int i = 0; i < NV; ++i) part[i] += g0.rho * s1[i];
    }
    for (int i = 0; i < NV; ++i) { An[i] += cn[1] * part[i]; At[i] += ct[1] * part[i]; }
    mapsi<DIM>(T0, A0, xu, 0, 0, s1);
    for (int i = 0; i < NV; ++i) { part[i] = g0.rho * s1[i]; An[i] += cn[2] * part[i]; At[i] += ct[2] * part[i]; }
    /* g_l H(u) + g_r (1 - H(u)) */
    mpsi<DIM>(Tlp, xu, 0, 0, s1);
    mpsi<DIM>(Trn, xu, 0, 0, s2);
    for (int i = 0; i < NV; ++i) {
      part[i] = gl.rho * s1[i] + gr.rho * s2[i];
      An[i] += cn[3] * part[i];
      At[i] += ct[3] * part[i];
    }
    for (int i = 0; i < NV; ++i) part[i] = 0.0;
    for (int j = 0; j < DIM; ++j) {
      mapsi<DIM>(Tlp, al[j], xu + (j == 0), j == 1, j == 2, s1);
      mapsi<DIM>(Trn, ar[j], xu + (j == 0), j == 1, j == 2, s2);
      for (int i = 0; i < NV; ++i) part[i] += gl.rho * s1[i] + gr.rho * s2[i];
    }
    for (int i = 0; i < NV; ++i) { An[i] += cn[4] * part[i]; At[i] += ct[4] * part[i]; }
    mapsi<DIM>(Tlp, Al, xu, 0, 0, s1);
    mapsi<DIM>(Trn, Ar, xu, 0, 0, s2);
    for (int i = 0; i < NV; ++i) {
      part[i] = gl.rho * s1[i] + gr.rho * s2[i];
      An[i] += cn[5] * part[i];
      At[i] += ct[5] * part[i];
    }
  }
  if (prfix) { /* heat-flux correction F_E += (1/Pr - 1) q about the interface velocity */
    for (int pass = 0; pass < 2; ++pass) {
      double* F = pass == 0 ? Fn : Ft;
      double* Q = pass == 0 ? Qn : Qt;
      double uf = 0.0, uq = 0.0, u2 = 0.0;
      for (int i = 0; i < DIM; ++i) {
        uf += g0.U[i] * F[1 + i];
        uq += g0.U[i] * Q[1 + i];
        u2 += g0.U[i] * g0.U[i];
      }
      double q = (F[DIM + 1] - uf + 0.5 * u2 * F[0]) - g0.U[0] * (Q[DIM + 1] - uq + 0.5 * u2 * Q[0]);
      F[DIM + 1] += (1.0 / ph.prandtl - 1.0) * q;
    }
  }
  /* interface values for the derivative update (temporal discretisation section) */
  double tau0 = 5.0 * jump * dt;
  double w = tau0 > 0.0 ? exp(-dt / tau0) : 0.0;
  for (int i = 0; i < NV; ++i) {
    out[i] = Fn[i];
    out[NV + i] = Ft[i];
    double dq0 = g0.rho * b0[i];
    out[2 * NV + i] = (1.0 - w) * W0[i] + w * WL[i];
    out[3 * NV + i] = (1.0 - w) * dq0 + w * gl.rho * bl[i];
    out[4 * NV + i] = (1.0 - w) * W0[i] + w * WR[i];
    out[5 * NV + i] = (1.0 - w) * dq0 + w * gr.rho * br[i];
  }
  return true;
}

/* local orthonormal frame rows (n, t1, t2): n along the area vector, t1 from
   the face tangent (3-D); t = (-n_y, n_x) in 2-D */
template <int DIM>
CGKS_HD void face_frame(const double* A, const double* T, double R[3][3]) {
  double an = 0.0;
  for (int a = 0; a < DIM; ++a) an += A[a] * A[a];
  an = sqrt(an);
  double n[3] = {0.0, 0.0, 0.0};
  for (int a = 0; a < DIM; ++a) n[a] = A[a] / an;
  for (int r = 0; r < 3; ++r) for (int q = 0; q < 3; ++q) R[r][q] = 0.0;
  if (DIM == 2) {
    R[0][0] = n[0]; R[0][1] = n[1];
    R[1][0] = -n[1]; R[1][1] = n[0];
    return;
  }
  double tn = T[0] * n[0] + T[1] * n[1] + T[2] * n[2];
  double t1[3] = {T[0] - tn * n[0], T[1] - tn * n[1], T[2] - tn * n[2]};
  double tl = sqrt(t1[0] * t1[0] + t1[1] * t1[1] + t1[2] * t1[2]);
  for (int a = 0; a < 3; ++a) t1[a] /= tl;
  double t2[3] = {n[1] * t1[2] - n[2] * t1[1], n[2] * t1[0] - n[0] * t1[2], n[0] * t1[1] - n[1] * t1[0]};
  for (int a = 0; a < 3; ++a) { R[0][a] = n[a]; R[1][a] = t1[a]; R[2][a] = t2[a]; }
}

/* global-frame Gauss-point state (value + gradient per variable) -> local frame */
template <int DIM>
CGKS_HD void to_local(const double R[3][3], const double* st /* NV*(1+DIM) */, double* W, double* dW) {
  const int NV = DIM + 2;
  double gv[NV][3];
  for (int v = 0; v < NV; ++v) {
    W[v] = st[v * (1 + DIM)];
    for (int k = 0; k < DIM; ++k) gv[v][k] = st[v * (1 + DIM) + 1 + k];
  }
  double m[3];
  for (int i = 0; i < DIM; ++i) {
    m[i] = 0.0;
    for (int a = 0; a < DIM; ++a) m[i] += R[i][a] * W[1 + a];
  }
  for (int i = 0; i < DIM; ++i) W[1 + i] = m[i];
  double gr[NV][3];
  for (int k = 0; k < DIM; ++k) {
    gr[0][k] = gv[0][k];
    gr[NV - 1][k] = gv[NV - 1][k];
    for (int i = 0; i < DIM; ++i) {
      double s = 0.0;
      for (int a = 0; a < DIM; ++a) s += R[i][a] * gv[1 + a][k];
      gr[1 + i][k] = s;
    }
  }
  for (int j = 0; j < DIM; ++j)
    for (int v = 0; v < NV; ++v) {
      double s = 0.0;
      for (int k = 0; k < DIM; ++k) s += R[j][k] * gr[v][k];
      dW[j * NV + v] = s;
    }
}

template <int DIM>
CGKS_HD void to_global(const double R[3][3], double* F) {
  double m[3];
  for (int a = 0; a < DIM; ++a) {
    m[a] = 0.0;
    for (int i = 0; i < DIM; ++i) m[a] += R[i][a] * F[1 + i];
  }
  for (int a = 0; a < DIM; ++a) F[1 + a] = m[a];
}

/* one face Gauss point: gather, rotate, solve, rotate back, store */
template <int DIM>
CGKS_HD bool flux_point(const DevGeo& g, const Phys& ph, double dt, int ax, int k, long c,
                        const double* __restrict__ gpL, const double* __restrict__ gpR, double* __restrict__ flux) {
  typedef Sz<DIM> S;
  const int NV = S::NV;
  const long N = g.ncell;
  double sl[NV * (1 + DIM)], sr[NV * (1 + DIM)];
  long base = (long)((ax * S::GPF + k) * NV) * (1 + DIM);
  for (int q = 0; q < NV * (1 + DIM); ++q) {
    sl[q] = gpL[(base + q) * N + c];
    sr[q] = gpR[(base + q) * N + c];
  }
  double A[3], T[3];
  int gp = (2 * ax + 1) * S::GPF + k;
  for (int a = 0; a < 3; ++a) {
    A[a] = a < DIM ? met_area<DIM>(g, c, gp, a) : 0.0;
    T[a] = a < DIM ? met_tang<DIM>(g, c, ax, k, a) : 0.0;
  }
  double R[3][3];
  face_frame<DIM>(A, T, R);
  double WL[NV], dWL[DIM * NV], WR[NV], dWR[DIM * NV], out[6 * NV];
  to_local<DIM>(R, sl, WL, dWL);
  to_local<DIM>(R, sr, WR, dWR);
  bool ok = gks_point<DIM>(ph, dt, WL, dWL, WR, dWR, out);
  for (int p = 0; p < 6; ++p) to_global<DIM>(R, out + p * NV);
  long fb = (long)((ax * S::GPF + k) * 6) * NV;
  for (int q = 0; q < 6 * NV; ++q) flux[(fb + q) * N + c] = out[q];
  return ok;
}

/* ===================================================================== */
/* (c) accumulation and S2O4 update of one cell                          */
/* ===================================================================== */
/* stage 1: Uout = U* ; stash = {Q^n + dt L + dt^2/6 L_t ; D(Q^n(x_G))}
   stage 2: Uout = U^{n+1} = {stash + dt^2/3 L_t* ; stash_D + dt D((dQ/dt)*(x_G))} */
template <int DIM>
CGKS_HD void update_cell(const DevGeo& g, double dt, int stage, long c, int ci, int cj, int ck,
                         const double* __restrict__ Uin, const double* __restrict__ flux,
                         double* __restrict__ stash, double* __restrict__ Uout) {
  typedef Sz<DIM> S;
  const int NV = S::NV, GPF = S::GPF;
  const long N = g.ncell;
  const double vol = met_vol<DIM>(g, c);
  long lo[3];
  for (int ax = 0; ax < DIM; ++ax) {
    int o[3] = {0, 0, 0};
    o[ax] = -1;
    lo[ax] = nbr(g, ci, cj, ck, o[0], o[1], o[2]);
  }
  for (int v = 0; v < NV; ++v) {
    double L = 0.0, Lt = 0.0;
    double qn[S::NGP], qt[S::NGP];
    for (int ax = 0; ax < DIM; ++ax) {
      for (int k = 0; k < GPF; ++k) {
        long fb = (long)((ax * GPF + k) * 6) * NV + v;
        int ghi = (2 * ax + 1) * GPF + k, glo = (2 * ax) * GPF + k;
        double sh = 0.0, sl = 0.0;
        for (int a = 0; a < DIM; ++a) {
          double ah = met_area<DIM>(g, c, ghi, a);
          double al = met_area<DIM>(g, lo[ax], ghi, a);
          sh += ah * ah;
          sl += al * al;
        }
        sh = sqrt(sh);
        sl = sqrt(sl);
        L += -flux[(fb + 0 * NV) * N + c] * sh + flux[(fb + 0 * NV) * N + lo[ax]] * sl;
        Lt += -flux[(fb + 1 * NV) * N + c] * sh + flux[(fb + 1 * NV) * N + lo[ax]] * sl;
        qn[ghi] = flux[(fb + 2 * NV) * N + c];
        qt[ghi] = flux[(fb + 3 * NV) * N + c];
        qn[glo] = flux[(fb + 4 * NV) * N + lo[ax]];
        qt[glo] = flux[(fb + 5 * NV) * N + lo[ax]];
      }
    }
    L /= vol;
    Lt /= vol;
    const long iavg = (long)v * N + c;
    if (stage == 1) {
      double q = Uin[iavg];
      Uout[iavg] = q + 0.5 * dt * L + 0.125 * dt * dt * Lt;
      stash[iavg] = q + dt * L + dt * dt / 6.0 * Lt;
    } else {
      Uout[iavg] = stash[iavg] + dt * dt / 3.0 * Lt;
    }
    /* derivative fields: gradient (Gauss' theorem) and line derivatives */
    for (int f = 1; f < S::NF; ++f) {
      double dn = 0.0, dtv = 0.0;
      if (f <= DIM) {
        int kk = f - 1;
        for (int gp = 0; gp < S::NGP; ++gp) {
          double sgn = ((gp / GPF) & 1) ? 1.0 : -1.0;
          double A = met_area<DIM>(g, c, gp, kk);
          dn += sgn * qn[gp] * A;
          dtv += sgn * qt[gp] * A;
        }
        dn /= vol;
        dtv /= vol;
      } else {
        int s = f - 1 - DIM, ax = s / GPF, k = s % GPF;
        double len = met_len<DIM>(g, c, s);
        dn = (qn[(2 * ax + 1) * GPF + k] - qn[(2 * ax) * GPF + k]) / len;
        dtv = (qt[(2 * ax + 1) * GPF + k] - qt[(2 * ax) * GPF + k]) / len;
      }
      const long idx = ((long)f * NV + v) * N + c;
      if (stage == 1) {
        Uout[idx] = dn + 0.5 * dt * dtv;
        stash[idx] = dn;
      } else {
        Uout[idx] = stash[idx] + dt * dtv;
      }
    }
  }
}

/* ===================================================================== */
/* time step                                                             */
/* ===================================================================== */
/* returns the per-cell rate r with dt = CFL / max r (convective rate summed
   over directions, viscous rate 3 nu / h_min^2) */
template <int DIM>
CGKS_HD double cell_rate(const DevGeo& g, const Phys& ph, const double* __restrict__ U, long c) {
  const long N = g.ncell;
  double W[DIM + 2];
  for (int v = 0; v < DIM + 2; ++v) W[v] = U[(long)v * N + c];
  double rho = W[0], ke = 0.0, Uv[3];
  for (int i = 0; i < DIM; ++i) {
    Uv[i] = W[1 + i] / rho;
    ke += Uv[i] * W[1 + i];
  }
  double p = (ph.gamma - 1.0) * (W[DIM + 1] - 0.5 * ke);
  double snd = sqrt(ph.gamma * p / rho);
  double vol = met_vol<DIM>(g, c);
  double rate = 0.0, hmin = 1e300;
  for (int ax = 0; ax < DIM; ++ax) {
    double A0[3] = {0.0, 0.0, 0.0}, A1[3] = {0.0, 0.0, 0.0};
    for (int k = 0; k < Sz<DIM>::GPF; ++k)
      for (int a = 0; a < DIM; ++a) {
        A0[a] += met_area<DIM>(g, c, (2 * ax) * Sz<DIM>::GPF + k, a);
        A1[a] += met_area<DIM>(g, c, (2 * ax + 1) * Sz<DIM>::GPF + k, a);
      }
    double s0 = 0.0, s1 = 0.0, nn[3], ns = 0.0;
    for (int a = 0; a < DIM; ++a) {
      s0 += A0[a] * A0[a];
      s1 += A1[a] * A1[a];
      nn[a] = A0[a] + A1[a];
      ns += nn[a] * nn[a];
    }
    double h = vol / (0.5 * (sqrt(s0) + sqrt(s1)));
    double un = 0.0;
    for (int a = 0; a < DIM; ++a) un += Uv[a] * nn[a] / sqrt(ns);
    rate += (fabs(un) + snd) / h;
    if (h < hmin) hmin = h;
  }
  if (ph.mu > 0.0) {
    double rv = 3.0 * ph.mu / (rho * hmin * hmin);
    if (rv > rate) rate = rv;
  }
  if (!(rho > 0.0) || !(p > 0.0) || !(rate == rate)) rate = 1e300; /* flags a bad state */
  return rate;
}

}  // namespace cgks
