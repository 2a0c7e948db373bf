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
template <int DIM, typename T = double> CGKS_HD T gp_delta(int gp, int a) {
  const int GPF = Sz<DIM>::GPF;
  int f = gp / GPF, k = gp % GPF, ax = f / 2, side = f & 1;
  if (a == ax) return side ? T(0.5) : T(-0.5);
  int t = 0;  /* rank of `a` among the tangential axes */
  for (int q = 0; q < a; ++q) if (q != ax) ++t;
  int bit = (t == 0) ? (k & 1) : (k & 2);
  return bit ? T(CGKS_GQ) : T(-CGKS_GQ);
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
  double ih[3];       /* 1/h */
  float hf[3], ihf[3]; /* the same in FP32, so FP32 kernels need no conversions */
  const double* met;  /* curvilinear metrics (Met<DIM>), or null */
  const float* rmet;  /* curvilinear: FP32 CFL metric per cell (RateMet<DIM>), or null */
  int bcm;            /* boundary kind (BcKind) of domain face f = -x,+x,-y,+y,-z,+z in bits
                         3f..3f+2: shifts, not an array, so that no copy of DevGeo is
                         indexed at run time (which would put it in local memory) */
  const double* bcq;  /* inflow faces: conservative states [face][5] (device), followed by
                         their exact FP32 hi and lo parts [face][5] each (bcq_hi, bcq_lo);
                         or null when no face is an inflow */
  long nplane;        /* slots of the low-boundary face array per (axis, Gauss point):
                         the largest ncell / n[axis] over non-periodic axes, else 0 */
};

/* boundary kinds (the values of the public CGKS_BC_* codes) */
enum BcKind { BC_PERIODIC = 0, BC_OUTFLOW = 1, BC_SLIP = 2, BC_NOSLIP = 3, BC_INFLOW = 4 };
CGKS_HD int geo_bc(const DevGeo& g, int f) { return (g.bcm >> (3 * f)) & 7; }
constexpr int BCQ_DOUBLES = 60; /* size of one inflow-state block in doubles: 30 + 2 x 30 floats */
CGKS_HD const float* bcq_hi(const DevGeo& g) { return reinterpret_cast<const float*>(g.bcq + 30); }
CGKS_HD const float* bcq_lo(const DevGeo& g) { return reinterpret_cast<const float*>(g.bcq + 30) + 30; }
/* host: one block of inflow states (BCQ_DOUBLES doubles) from the
   descriptor's [face][5] states: the FP64 values, then their exact FP32 hi
   and lo parts */
inline void pack_bcq(const double (&st)[6][5], double* out) {
  float* h = reinterpret_cast<float*>(out + 30);
  float* l = h + 30;
  for (int q = 0; q < 30; ++q) {
    const double x = st[q / 5][q % 5];
    out[q] = x;
    h[q] = (float)x;
    l[q] = (float)(x - (double)h[q]);
  }
}
CGKS_HD bool bc_wall(int bc) { return bc == BC_SLIP || bc == BC_NOSLIP; }

/* FP32 CFL metric of a curvilinear cell, [k * ncell + cell]: per axis the
   direction w = n/(|n| h) and 1/h (n the mean face normal, h = vol / mean
   face area), then the smallest h */
template <int DIM> struct RateMet {
  static constexpr int W = 0;            /* DIM*DIM: w[ax][a] */
  static constexpr int IH = DIM * DIM;   /* DIM: 1/h per axis */
  static constexpr int HMIN = IH + DIM;  /* 1 */
  static constexpr int N = HMIN + 1;
};

struct Phys {
  double gamma, mu, prandtl, cfl, c_chi;
  int tau_mode, linear;
  /* FP32 copies and the heat-flux-fix switch (mu > 0 and Pr != 1) */
  float gammaf, muf, prandtlf, c_chif;
  int prfix;
  /* test hook: bytes added to what the flux's TMA barrier expects, so that
     it never completes and the bounded wait runs out (0 in normal use) */
  int stall_tx;
};

/* the physics constants in T */
template <typename T> CGKS_HD T ph_gamma(const Phys& p) { if constexpr (sizeof(T) == 4) return p.gammaf; else return p.gamma; }
template <typename T> CGKS_HD T ph_mu(const Phys& p) { if constexpr (sizeof(T) == 4) return p.muf; else return p.mu; }
template <typename T> CGKS_HD T ph_pr(const Phys& p) { if constexpr (sizeof(T) == 4) return p.prandtlf; else return p.prandtl; }
template <typename T> CGKS_HD T ph_cchi(const Phys& p) { if constexpr (sizeof(T) == 4) return p.c_chif; else return p.c_chi; }
template <typename T> CGKS_HD T geo_h(const DevGeo& g, int a) { if constexpr (sizeof(T) == 4) return g.hf[a]; else return g.h[a]; }
template <typename T> CGKS_HD T geo_ih(const DevGeo& g, int a) { if constexpr (sizeof(T) == 4) return g.ihf[a]; else return g.ih[a]; }

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

/* neighbour through the domain boundaries: periodic faces wrap, outflow
   faces clamp (the ghost copies the boundary cell), walls mirror the index
   and the ghost holds the mirror image of the cell.  *mm receives the axes
   mirrored (bits 0-2) and which of them are no-slip walls (bits 3-5). */
CGKS_HD long nbr_bc(const DevGeo& g, int i, int j, int k, int ox, int oy, int oz, int* mm) {
  int x[3] = {i + ox, j + oy, k + oz};
  int m = 0;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (x[a] < 0 || x[a] >= g.n[a]) {
      const int hi = x[a] >= g.n[a] ? 1 : 0;
      const int bc = geo_bc(g, 2 * a + hi);
      if (bc == BC_PERIODIC) x[a] += hi ? -g.n[a] : g.n[a];
      else if (bc == BC_OUTFLOW || bc == BC_INFLOW) x[a] = hi ? g.n[a] - 1 : 0;
      else {
        x[a] = hi ? 2 * g.n[a] - 1 - x[a] : -1 - x[a];
        m |= (1 << a) | (bc == BC_NOSLIP ? (8 << a) : 0);
      }
    }
  }
  *mm = m;
  return cell_index(g, x[0], x[1], x[2]);
}

/* The stencil neighbours of one cell, resolved once: the linear-index
   offsets of the -1 and +1 neighbours along each axis (through the
   boundaries as nbr_bc resolves them) and their mirror bits, so that a
   neighbour (ox, oy, oz) in {-1, 0, 1}^DIM costs additions only.  Beyond an
   inflow face the neighbour is the face's fixed state: bit 6 + axis of mm
   (the index is clamped and not read for values). */
constexpr int MM_INFLOW = 0x1C0;
template <int DIM> struct NbrOff {
  int lo[3], hi[3];
  int mlo, mhi; /* nbr_bc's mm format plus inflow bits; the bits of different axes are disjoint */
  CGKS_HD void setup(const DevGeo& g, int ci, int cj, int ck) {
    const int x[3] = {ci, cj, ck};
    int stride = 1;
    mlo = mhi = 0;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      const int n = g.n[a];
      const int bits = (1 << a);
      if (x[a] > 0) lo[a] = -stride;
      else {
        const int bc = geo_bc(g, 2 * a);
        lo[a] = bc == BC_PERIODIC ? (n - 1) * stride : 0;
        if (bc_wall(bc)) mlo |= bits | (bc == BC_NOSLIP ? bits << 3 : 0);
        if (bc == BC_INFLOW) mlo |= bits << 6;
      }
      if (x[a] < n - 1) hi[a] = stride;
      else {
        const int bc = geo_bc(g, 2 * a + 1);
        hi[a] = bc == BC_PERIODIC ? -(n - 1) * stride : 0;
        if (bc_wall(bc)) mhi |= bits | (bc == BC_NOSLIP ? bits << 3 : 0);
        if (bc == BC_INFLOW) mhi |= bits << 6;
      }
      stride *= n;
    }
  }
  /* WALL = false: the mesh has no wall, no neighbour is a mirror image */
  template <bool WALL> CGKS_HD long at(long c, int ox, int oy, int oz, int* mm) const {
    long i = c;
    int m = 0;
    if (ox < 0) { i += lo[0]; m |= mlo & 0x49; } else if (ox > 0) { i += hi[0]; m |= mhi & 0x49; }
    if (oy < 0) { i += lo[1]; m |= mlo & 0x92; } else if (oy > 0) { i += hi[1]; m |= mhi & 0x92; }
    if (DIM == 3) {
      if (oz < 0) { i += lo[2]; m |= mlo & 0x124; } else if (oz > 0) { i += hi[2]; m |= mhi & 0x124; }
    }
    *mm = WALL ? m : 0;
    return i;
  }
  /* the inflow face a neighbour with inflow bits in mm lies beyond: the
     first such axis, on the side of the offset */
  CGKS_HD static int inflow_face(int mm, int ox, int oy, int oz) {
    if (mm & 0x40) return ox < 0 ? 0 : 1;
    if (mm & 0x80) return oy < 0 ? 2 : 3;
    return oz < 0 ? 4 : 5;
  }
};

/* true if a neighbour of cell (ci, cj, ck) lies beyond a wall or inflow face
   (the cell touches such a face); elsewhere the plain neighbour path applies */
template <int DIM> CGKS_HD bool touches_wall(const DevGeo& g, int ci, int cj, int ck) {
  const int x[3] = {ci, cj, ck};
  bool t = false;
#pragma unroll
  for (int a = 0; a < DIM; ++a) {
    t |= x[a] == 0 && geo_bc(g, 2 * a) >= BC_SLIP;
    t |= x[a] == g.n[a] - 1 && geo_bc(g, 2 * a + 1) >= BC_SLIP;
  }
  return t;
}

/* 1 if variable v changes sign in the mirror image across the axes of mm:
   the momentum component along a mirrored axis, and every momentum
   component at a no-slip mirror; a derivative along a mirrored axis changes
   sign once more (mirror_odd ^ ((mm >> axis) & 1)) */
template <int DIM> CGKS_HD int mirror_odd(int v, int mm) {
  if (!mm || v < 1 || v > DIM) return 0;
  int f = 0;
#pragma unroll
  for (int a = 0; a < DIM; ++a)
    if ((mm >> a) & 1) f ^= (v == 1 + a || ((mm >> (3 + a)) & 1)) ? 1 : 0;
  return f;
}

/* index of the cell (i, j, k) within its boundary plane normal to axis ax */
CGKS_HD long plane_index(const DevGeo& g, int ax, int i, int j, int k) {
  if (ax == 0) return j + (long)g.n[1] * k;
  if (ax == 1) return i + (long)g.n[0] * k;
  return i + (long)g.n[0] * j;
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

/* math wrappers so that the same code serves FP64 and FP32 */
CGKS_HD double cg_erfc(double x) { return erfc(x); }
CGKS_HD float cg_erfc(float x) { return erfcf(x); }
CGKS_HD double cg_exp(double x) { return exp(x); }
CGKS_HD float cg_exp(float x) { return expf(x); }
CGKS_HD double cg_expm1(double x) { return expm1(x); }
CGKS_HD float cg_expm1(float x) { return expm1f(x); }
CGKS_HD double cg_sqrt(double x) { return sqrt(x); }
CGKS_HD float cg_sqrt(float x) { return sqrtf(x); }
#if defined(__CUDA_ARCH__)
CGKS_HD double cg_rsqrt(double x) { return rsqrt(x); }
CGKS_HD float cg_rsqrt(float x) { return rsqrtf(x); }
#else
CGKS_HD double cg_rsqrt(double x) { return 1.0 / sqrt(x); }
CGKS_HD float cg_rsqrt(float x) { return 1.0f / sqrtf(x); }
#endif
CGKS_HD double cg_fabs(double x) { return fabs(x); }
CGKS_HD float cg_fabs(float x) { return fabsf(x); }
CGKS_HD double cg_fma(double a, double b, double c) { return fma(a, b, c); }
CGKS_HD float cg_fma(float a, float b, float c) { return fmaf(a, b, c); }
/* a b + c d and a b + c d + e f, evaluated left to right (the paired type
   overloads them with compensated dot products) */
CGKS_HD double cg_dot2(double a, double b, double c, double d) { return a * b + c * d; }
CGKS_HD float cg_dot2(float a, float b, float c, float d) { return a * b + c * d; }
CGKS_HD double cg_dot3(double a, double b, double c, double d, double e, double f) { return a * b + c * d + e * f; }
CGKS_HD float cg_dot3(float a, float b, float c, float d, float e, float f) { return a * b + c * d + e * f; }
/* a b + c (the paired type overloads it with one renormalisation) */
CGKS_HD double cg_madd(double a, double b, double c) { return a * b + c; }
CGKS_HD float cg_madd(float a, float b, float c) { return a * b + c; }
/* a value renormalised before its sign is read (the paired type overloads
   it; plain types are their own normal form) */
CGKS_HD double cg_norm(double x) { return x; }
CGKS_HD float cg_norm(float x) { return x; }
#include "cgks_pair.cuh"
CGKS_HD double cg_tanh(double x) { return tanh(x); }
CGKS_HD float cg_tanh(float x) { return tanhf(x); }

/* ===================================================================== */
/* (a) reconstruction of one variable of one cell                        */
/* ===================================================================== */
#include "cgks_recon_gen.cuh"

/* data access of the reconstruction of variable v of cell c.  Averages are
   handed over relative to the cell's own average: the reconstruction depends
   on differences only, so the large offsets never enter T arithmetic.  FP64:
   differences of the FP64 averages.  FP32: every average is also kept as an
   exact pair hi + lo of FP32 numbers (written by the update), so the
   difference is (hi_k - hi_0) + (lo_k - lo_0), computed in FP32 without the
   FP64 pipe.  Gradients are mapped to the target's reference frame with J0^T
   (Sec. 4; CURVI = false: J0 = diag(h)); line differences are the stored
   derivatives times the line length.  der: [(f-1)][v][cell] in T, f >= 1.
   WALL: neighbours beyond a wall are mirror images (signs by mirror_odd). */
template <typename T, int DIM, bool CURVI, bool WALL> struct ReconLd {
  const double* __restrict__ avgp;  /* FP64 averages [v][cell] (FP64 form) */
  const float* __restrict__ avh;    /* hi and lo parts [v][cell] (FP32 form) */
  const float* __restrict__ avl;
  const T* __restrict__ der;
  DevGeo g;
  long c;
  int ci, cj, ck, v;
  NbrOff<DIM> nb;
  double q0d;
  float q0h, q0l;
  T J0[3][3];
  CGKS_HD void init_q0() {
    if constexpr (sizeof(T) == 4) {
      q0h = avh[(long)v * g.ncell + c];
      q0l = avl[(long)v * g.ncell + c];
      q0d = 0.0;
    } else {
      q0d = avgp[(long)v * g.ncell + c];
    }
  }
  CGKS_HD T q0() const { return T(0); }
  /* branch-free: beyond an inflow face the (base, index) of the one load
     switch to the face's state, a mirror image flips the loaded value, so a
     stencil's loads issue together */
  CGKS_HD T avg(int ox, int oy, int oz) const {
    int mm;
    long i = (long)v * g.ncell + nb.template at<WALL>(c, ox, oy, oz, &mm);
    const bool inflow = WALL && (mm & MM_INFLOW);
    const bool odd = WALL && !inflow && mirror_odd<DIM>(v, mm);
    if (inflow) i = NbrOff<DIM>::inflow_face(mm, ox, oy, oz) * 5 + v;
    if constexpr (sizeof(T) == 4) {
      const float* ph = inflow ? bcq_hi(g) : avh;
      const float* pl = inflow ? bcq_lo(g) : avl;
      float h = ph[i], l = pl[i];
      if (odd) {
        h = -h;
        l = -l;
      }
      return (h - q0h) + (l - q0l);
    } else {
      double a = (inflow ? g.bcq : avgp)[i];
      if (odd) a = -a;
      return T(a - q0d);
    }
  }
  /* the full value q0 + rel at a Gauss point, stored in T */
  CGKS_HD T full(T rel) const {
    if constexpr (sizeof(T) == 4) return q0h + (q0l + rel);
    else return T(q0d + double(rel));
  }
  CGKS_HD void grefv(int ox, int oy, int oz, T* out) const {
    int mm;
    const long ni = nb.template at<WALL>(c, ox, oy, oz, &mm);
    T gp[3];
#pragma unroll
    for (int r = 0; r < DIM; ++r) gp[r] = der[((long)r * (DIM + 2) + v) * g.ncell + ni];
    if (WALL && (mm & MM_INFLOW)) {
#pragma unroll
      for (int r = 0; r < DIM; ++r) gp[r] = T(0);
    } else if (WALL && mm) {
      const int f = mirror_odd<DIM>(v, mm);
#pragma unroll
      for (int r = 0; r < DIM; ++r)
        if (f ^ ((mm >> r) & 1)) gp[r] = -gp[r];
    }
    if constexpr (CURVI) {
#pragma unroll
      for (int k = 0; k < DIM; ++k) {
        T s = T(0);
#pragma unroll
        for (int r = 0; r < DIM; ++r) s += J0[r][k] * gp[r];
        out[k] = s;
      }
    } else {
#pragma unroll
      for (int k = 0; k < DIM; ++k) out[k] = geo_h<T>(g, k) * gp[k];
    }
  }
  CGKS_HD T line(int s) const {
    const T len = CURVI ? T(met_len<DIM>(g, c, s)) : geo_h<T>(g, s / Sz<DIM>::GPF);
    return der[((long)(DIM + s) * (DIM + 2) + v) * g.ncell + c] * len;
  }
};

/* FP64 path: whether the path function certainly saturates, chi = 1 to the
   last bit, judged from the smoothness indicators evaluated in FP32 (64
   times the FP64 rate on GB300) with a rigorous rounding margin, so that the
   FP64 indicators are only formed where chi may be below 1.  With
   r_L = IS^tau / (IS^L + eps) and r_H = IS^tau / (IS^H + eps) <= 1, the
   blend parameter is alpha = 2 (1 + r_H^2) / (2 + r_H^2 + r_L^2) >=
   2 / (3 + r_L^2); tanh(C alpha) rounds to exactly 1 = tanh(C) once
   C alpha >= 25 (1 - tanh(25) < 1e-21), which holds when
   r_L^2 <= 2 C / 25 - 3.  IS^tau = a^T (GH - GL) a and IS^L = a^T GL a are
   bounded from their FP32 values with 2e-5 times the forms of the absolute
   values (the FP32 error of these sums of at most ~100 terms is below 7e-6
   of that, the FP64 one far below).  FP32 form: never (its indicators are
   FP32 already). */
template <int DIM> CGKS_HD bool geno_saturates_f32v(const float* af, double C) {
  const double r2 = 2.0 * C / 25.0 - 3.0 - 0.2;
  if (!(r2 > 0.0)) return false;
  typedef Sz<DIM> S;
  float aa[S::NB];
#pragma unroll
  for (int b = 0; b < S::NB; ++b) aa[b] = fabsf(af[b]);
  float ist, isl, ista, isla;
  if constexpr (DIM == 3) {
    ist = gen_ist_3d<float>(af);
    isl = gen_isl_3d<float>(af);
    ista = gen_ista_3d<float>(aa);
    isla = gen_isla_3d<float>(aa);
  } else {
    ist = gen_ist_2d<float>(af);
    isl = gen_isl_2d<float>(af);
    ista = gen_ista_2d<float>(aa);
    isla = gen_isla_2d<float>(aa);
  }
  const float ist_ub = fmaxf(ist + 2e-5f * ista, 0.f);
  const float isl_lb = fmaxf(isl - 2e-5f * isla, 0.f) + 1e-15f;
  return ist_ub <= sqrtf((float)r2) * isl_lb; /* false for inf / NaN */
}
template <typename T, int DIM> CGKS_HD bool geno_saturates_fp32(const T* a, double C) {
  if constexpr (sizeof(T) == 4) {
    return false;
  } else {
    typedef Sz<DIM> S;
    float af[S::NB];
#pragma unroll
    for (int b = 0; b < S::NB; ++b) af[b] = (float)a[b];
    return geno_saturates_f32v<DIM>(af, C);
  }
}
/* the GENO path function chi (Sec. 3.3) from the reconstruction's
   coefficients a, evaluated in T */
template <typename T, int DIM> CGKS_HD T geno_chi(const T* a, const Phys& ph) {
  T ish, isl;
  if constexpr (DIM == 3) {
    ish = gen_ish_3d<T>(a);
    isl = gen_isl_3d<T>(a);
  } else {
    ish = gen_ish_2d<T>(a);
    isl = gen_isl_2d<T>(a);
  }
  const T eps = T(1e-15);
  T ist = ish - isl;
  if (ist < T(0)) ist = T(0);
  const T rh = ist / (ish + eps), rl = ist / (isl + eps);
  const T ah = T(1) + rh * rh, al = T(1) + rl * rl;
  const T alpha = T(2) * ah / (ah + al);
  return cg_tanh(ph_cchi<T>(ph) * alpha) / cg_tanh(ph_cchi<T>(ph));
}

/* the blended gradient bbar of the linear sub-stencil polynomials with their
   WENO weights (d_m = 1/(2 dim)):
   omega_m = (IS_m + eps)^-5 / sum_m' (IS_m' + eps)^-5, evaluated through the
   ratios (IS_min + eps)/(IS_m + eps) <= 1, which stays finite in FP32. */
template <typename T, int DIM, class Ld> CGKS_HD void substencil_bbar(const Ld& ld, T* bbar) {
  typedef Sz<DIM> S;
  T lsum[3] = {T(0), T(0), T(0)};
#pragma unroll
  for (int s = 0; s < S::NL; ++s) lsum[s / S::GPF] += ld.line(s);
  T bm[2 * DIM][3], tis[2 * DIM];
#pragma unroll
  for (int m = 0; m < 2 * DIM; ++m) {
    const int ax = m / 2;
    int o[3] = {0, 0, 0};
    o[ax] = (m & 1) ? 1 : -1;
    const T qf = ld.avg(o[0], o[1], o[2]);
    const T sg = (m & 1) ? T(1) : T(-1);
    T is = T(0);
#pragma unroll
    for (int kk = 0; kk < DIM; ++kk) {
      const T bv = (kk == ax) ? sg * qf : lsum[kk] * (T(1) / T(S::GPF));
      bm[m][kk] = bv;
      is += bv * bv;
    }
    tis[m] = is + T(1e-15);
  }
  T tmin = tis[0];
#pragma unroll
  for (int m = 1; m < 2 * DIM; ++m) tmin = tis[m] < tmin ? tis[m] : tmin;
  T wb[2 * DIM], ws = T(0);
#pragma unroll
  for (int m = 0; m < 2 * DIM; ++m) {
    const T r = tmin / tis[m];
    const T r2 = r * r;
    wb[m] = r2 * r2 * r;
    ws += wb[m];
  }
  const T iws = T(1) / ws;
#pragma unroll
  for (int m = 0; m < 2 * DIM; ++m) {
    const T w = wb[m] * iws;
#pragma unroll
    for (int kk = 0; kk < DIM; ++kk) bbar[kk] += w * bm[m][kk];
  }
}

/* Reconstruction of Eq. (compact-big-ref) on the reference cell: a = M d by the
   generated symmetry-reduced code, the linear sub-stencil gradients of
   Eq. (compact-sub-2) (closed form: the face-neighbour difference along the
   connecting axis, the mean of the line differences along each other axis),
   the GENO weights, and the blended value and physical gradient at every
   face Gauss point (Eq. weno-new, reverse transform of Sec. 4), stored in T.
   chi_force >= 0 overrides chi.  Returns chi. */
template <typename T, int DIM, bool CURVI, bool WALL>
CGKS_HD T recon_var(const double* __restrict__ avg, const float* __restrict__ avh, const float* __restrict__ avl,
                    const T* __restrict__ der, const DevGeo& g, const Phys& ph, long c, int ci, int cj, int ck, int v,
                    T chi_force, T* __restrict__ gpL, T* __restrict__ gpR) {
  typedef Sz<DIM> S;
  const long N = g.ncell;
  constexpr int NV = S::NV;
  ReconLd<T, DIM, CURVI, WALL> ld;
  ld.avgp = avg;
  ld.avh = avh;
  ld.avl = avl;
  ld.der = der;
  ld.g = g;
  ld.c = c;
  ld.ci = ci;
  ld.cj = cj;
  ld.ck = ck;
  ld.v = v;
  ld.nb.setup(g, ci, cj, ck);
  ld.init_q0();
  if constexpr (CURVI) {
#pragma unroll
    for (int r = 0; r < DIM; ++r)
#pragma unroll
      for (int q = 0; q < DIM; ++q) ld.J0[r][q] = T(met_J0<DIM>(g, c, r, q));
  }
  T a[S::NB];
  if constexpr (DIM == 3) gen_coeffs_3d<T>(ld, a);
  else gen_coeffs_2d<T>(ld, a);

  /* GENO path function (Sec. 3.3) */
  T chi;
  if (chi_force >= T(0)) {
    chi = chi_force;
  } else if (geno_saturates_fp32<T, DIM>(a, ph_cchi<double>(ph))) {
    chi = T(1); /* exactly what the FP64 evaluation below gives */
  } else {
    chi = geno_chi<T, DIM>(a, ph);
  }
  /* chi == 1 (forced, or the path function saturated in T): the blend is
     the fifth-order polynomial alone, bit for bit, and the sub-stencil
     polynomials are not needed */
  const bool lin = chi == T(1);
  T bbar[3] = {T(0), T(0), T(0)};
  if (!lin) substencil_bbar<T, DIM>(ld, bbar);
  T JiT[3][3];
  if constexpr (CURVI) {
#pragma unroll
    for (int r = 0; r < DIM; ++r)
#pragma unroll
      for (int q = 0; q < DIM; ++q) JiT[r][q] = T(met_JiT<DIM>(g, c, r, q));
  }
  T mean4;
  if constexpr (DIM == 3) mean4 = gen_mean_3d<T>(a);
  else mean4 = gen_mean_2d<T>(a);
  /* blended values at the face Gauss points, Eq. (weno-new), axis by axis.
     The FP32 form on Cartesian meshes takes every axis through one copy of
     the axis-0 transform on the coefficients relabelled by pi (pi(0) = ax,
     the tangential axes in order; gen_perm), the transform's derivative j
     being the physical derivative pi(j): one copy instead of three keeps
     the code the instruction cache must hold, and the registers, to a third
     (TGV 128^3 reconstruction 1.75 -> 1.58 ms, spills 192 -> 0 B).  In
     FP64 the relabelling selects cost more than they save (25.9 -> 26.9 ms),
     and curvilinear meshes take their gradient through (J0^T)^-1 by its
     physical components: both keep a copy per axis. */
  constexpr bool RELABEL = !CURVI && sizeof(T) == 4;
#pragma unroll 1
  for (int ax = 0; ax < DIM; ++ax) {
    T pv[2 * S::GPF], pg[2 * S::GPF][DIM];
    int pi[3] = {0, 1, 2};
    T ihc[3], bbc[3];
    if constexpr (!RELABEL) {
      if constexpr (DIM == 3) {
        if (ax == 0) gen_gp_3d_ax0<T>(a, pv, pg);
        else if (ax == 1) gen_gp_3d_ax1<T>(a, pv, pg);
        else gen_gp_3d_ax2<T>(a, pv, pg);
      } else {
        if (ax == 0) gen_gp_2d_ax0<T>(a, pv, pg);
        else gen_gp_2d_ax1<T>(a, pv, pg);
      }
    } else {
      pi[0] = ax;
      pi[1] = ax == 0 ? 1 : 0;
      pi[2] = ax == 2 ? 1 : 2;
#pragma unroll
      for (int j = 0; j < DIM; ++j) { /* by selects: pi is a run-time relabelling */
        ihc[j] = pi[j] == 0 ? geo_ih<T>(g, 0) : (pi[j] == 1 ? geo_ih<T>(g, 1) : geo_ih<T>(g, DIM - 1));
        bbc[j] = pi[j] == 0 ? bbar[0] : (pi[j] == 1 ? bbar[1] : bbar[DIM - 1]);
      }
      T ar[S::NB];
      if constexpr (DIM == 3) {
        gen_perm_3d<T>(a, ax, ar);
        gen_gp_3d_ax0<T>(ar, pv, pg);
      } else {
        gen_perm_2d<T>(a, ax, ar);
        gen_gp_2d_ax0<T>(ar, pv, pg);
      }
    }
    int o[3] = {0, 0, 0};
    o[ax] = -1;
    const long clo = nbr(g, ci, cj, ck, o[0], o[1], o[2]);
#pragma unroll
    for (int i = 0; i < 2 * S::GPF; ++i) {
      const int side = i / S::GPF, k = i % S::GPF;
      const int gp = (2 * ax + side) * S::GPF + k;
      T rel, gref[3];
      if (lin) {
        rel = pv[i] - mean4;
#pragma unroll
        for (int kk = 0; kk < DIM; ++kk) gref[kk] = pg[i][kk];
      } else {
        T v1 = T(0);
#pragma unroll
        for (int kk = 0; kk < DIM; ++kk) v1 += bbar[kk] * gp_delta<DIM, T>(gp, kk);
        rel = chi * (pv[i] - mean4) + (T(1) - chi) * v1;
#pragma unroll
        for (int kk = 0; kk < DIM; ++kk)
          gref[kk] = chi * pg[i][kk] + (T(1) - chi) * (RELABEL ? bbc[kk] : bbar[kk]);
      }
      T* dst = side ? gpL : gpR;
      const long cell = side ? c : clo;
      const long b = ((long)((ax * S::GPF + k) * NV + v) * (1 + DIM)) * N + cell;
      dst[b] = ld.full(rel);
#pragma unroll
      for (int kk = 0; kk < DIM; ++kk) {
        if constexpr (CURVI) {
          T sg = T(0);
#pragma unroll
          for (int r = 0; r < DIM; ++r) sg += JiT[kk][r] * gref[r];
          dst[b + (long)(1 + kk) * N] = sg;
        } else if constexpr (RELABEL) { /* derivative kk is the physical derivative pi(kk) */
          dst[b + (long)(1 + pi[kk]) * N] = gref[kk] * ihc[kk];
        } else {
          dst[b + (long)(1 + kk) * N] = gref[kk] * geo_ih<T>(g, kk);
        }
      }
    }
  }
  return chi;
}

/* recon_var on Cartesian meshes in FP64 storage with its Gauss-point
   transform on the FP32 pipe: a = M d in FP64 (in unnormalised pairs the
   map's straight-line code outgrows the instruction cache and runs no
   faster; nor does splitting its neighbour groups between the two
   pipes), the coefficients converted to pairs (fpacc) on the integer pipe,
   then the GENO screen (from their leading floats), the mean and the
   Gauss-point values and gradients in pairs, rounded once to FP64 when
   stored.  Where the screen cannot certify chi = 1, chi and the sub-stencil
   gradient come from the FP64 code on the coefficients rounded back to
   double, and the blend is FP64.  Same steps and readings as recon_var;
   results agree with it to the pairs' rounding (relative 2^-47 per
   coefficient). */
template <int DIM, bool WALL>
CGKS_HD double recon_var_pair(const double* __restrict__ avg, const double* __restrict__ der, const DevGeo& g,
                              const Phys& ph, long c, int ci, int cj, int ck, int v, double chi_force,
                              double* __restrict__ gpL, double* __restrict__ gpR) {
  typedef Sz<DIM> S;
  const long N = g.ncell;
  constexpr int NV = S::NV;
  ReconLd<double, DIM, false, WALL> ld;
  ld.avgp = avg;
  ld.avh = nullptr;
  ld.avl = nullptr;
  ld.der = der;
  ld.g = g;
  ld.c = c;
  ld.ci = ci;
  ld.cj = cj;
  ld.ck = ck;
  ld.v = v;
  ld.nb.setup(g, ci, cj, ck);
  ld.init_q0();
  fpacc ap[S::NB];
  {
    double a[S::NB];
    if constexpr (DIM == 3) gen_coeffs_3d<double>(ld, a);
    else gen_coeffs_2d<double>(ld, a);
#pragma unroll
    for (int b = 0; b < S::NB; ++b) ap[b] = fpacc_from_double(a[b]);
  }

  double chi;
  if (chi_force >= 0.0) {
    chi = chi_force;
  } else {
    float af[S::NB];
#pragma unroll
    for (int b = 0; b < S::NB; ++b) {
      ap[b] = fpacc_norm(ap[b]);
      af[b] = ap[b].hi;
    }
    if (geno_saturates_f32v<DIM>(af, ph_cchi<double>(ph))) {
      chi = 1.0;
    } else {
      double a[S::NB];
#pragma unroll
      for (int b = 0; b < S::NB; ++b) a[b] = fpacc_to_double(ap[b]);
      chi = geno_chi<double, DIM>(a, ph);
    }
  }
  const bool lin = chi == 1.0;
  double bbar[3] = {0.0, 0.0, 0.0};
  if (!lin) substencil_bbar<double, DIM>(ld, bbar);
  fpacc mean4;
  if constexpr (DIM == 3) mean4 = gen_mean_3d<fpacc>(ap);
  else mean4 = gen_mean_2d<fpacc>(ap);
  fpacc ih[3];
#pragma unroll
  for (int a = 0; a < DIM; ++a) ih[a] = fpacc_from_double(g.ih[a]);
  /* every axis through one copy of the axis-0 transform: the coefficients
     relabelled by pi (pi(0) = ax, the tangential axes in order; gen_perm),
     the transform's derivative j being the physical derivative pi(j) (one
     copy instead of three keeps the code the instruction cache must hold
     to a third) */
#pragma unroll 1
  for (int ax = 0; ax < DIM; ++ax) {
    int pi[3];
    pi[0] = ax;
    pi[1] = ax == 0 ? 1 : 0;
    pi[2] = ax == 2 ? 1 : 2;
    fpacc ihc[DIM];
    double ihd[DIM], bbc[DIM];
#pragma unroll
    for (int j = 0; j < DIM; ++j) { /* by selects: pi is a run-time relabelling */
      ihc[j] = pi[j] == 0 ? ih[0] : (pi[j] == 1 ? ih[1] : ih[DIM - 1]);
      ihd[j] = pi[j] == 0 ? g.ih[0] : (pi[j] == 1 ? g.ih[1] : g.ih[DIM - 1]);
      bbc[j] = pi[j] == 0 ? bbar[0] : (pi[j] == 1 ? bbar[1] : bbar[DIM - 1]);
    }
    fpacc pv[2 * S::GPF], pg[2 * S::GPF][DIM];
    {
      fpacc ar[S::NB];
      if constexpr (DIM == 3) {
        gen_perm_3d<fpacc>(ap, ax, ar);
        gen_gp_3d_ax0<fpacc>(ar, pv, pg);
      } else {
        gen_perm_2d<fpacc>(ap, ax, ar);
        gen_gp_2d_ax0<fpacc>(ar, pv, pg);
      }
    }
    int o[3] = {0, 0, 0};
    o[ax] = -1;
    const long clo = nbr(g, ci, cj, ck, o[0], o[1], o[2]);
#pragma unroll
    for (int i = 0; i < 2 * S::GPF; ++i) {
      const int side = i / S::GPF, k = i % S::GPF;
      const int gp = (2 * ax + side) * S::GPF + k;
      double* dst = side ? gpL : gpR;
      const long cell = side ? c : clo;
      const long b = ((long)((ax * S::GPF + k) * NV + v) * (1 + DIM)) * N + cell;
      const double rel = fpacc_to_double(pv[i] - mean4);
      if (lin) {
        dst[b] = ld.full(rel);
#pragma unroll
        for (int j = 0; j < DIM; ++j) dst[b + (long)(1 + pi[j]) * N] = fpacc_to_double(pg[i][j] * ihc[j]);
      } else {
        double v1 = 0.0;
#pragma unroll
        for (int kk = 0; kk < DIM; ++kk) v1 += bbar[kk] * gp_delta<DIM, double>(gp, kk);
        dst[b] = ld.full(chi * rel + (1.0 - chi) * v1);
#pragma unroll
        for (int j = 0; j < DIM; ++j)
          dst[b + (long)(1 + pi[j]) * N] = (chi * fpacc_to_double(pg[i][j]) + (1.0 - chi) * bbc[j]) * ihd[j];
      }
    }
  }
  return chi;
}

/* positivity of the reconstructed Gauss-point states of a cell (C18 reading:
   the states just written by this thread are read back) */
template <typename T, int DIM>
CGKS_HD bool cell_states_physical(const DevGeo& g, const Phys& ph, long c, int ci, int cj, int ck,
                                  const T* __restrict__ gpL, const T* __restrict__ gpR) {
  typedef Sz<DIM> S;
  const long N = g.ncell;
  for (int gp = 0; gp < S::NGP; ++gp) {
    int f = gp / S::GPF, k = gp % S::GPF, ax = f / 2, side = f & 1;
    const T* src;
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
    T w[S::NV];
    for (int v = 0; v < S::NV; ++v) w[v] = src[((long)((ax * S::GPF + k) * S::NV + v) * (1 + DIM)) * N + cell];
    T ke = T(0);
    for (int i = 0; i < DIM; ++i) ke += w[1 + i] * w[1 + i];
    const T p = (ph_gamma<T>(ph) - T(1)) * (w[DIM + 1] - T(0.5) * ke / w[0]);
    if (!(w[0] > T(0)) || !(p > T(0))) return false;
  }
  return true;
}

/* ===================================================================== */
/* (b) gas-kinetic interface solution at one Gauss point (Sec. 2)        */
/* ===================================================================== */
enum { REG_FULL = 0, REG_POS = 1, REG_NEG = 2 };

/* Maxwellian of a conservative state: macroscopic scalars plus the two base
   moments <u^0>, <u^1> of the normal direction over the full space or a half
   space (the latter need erfc and exp, so they are kept, not recomputed). */
template <typename T, int DIM> struct MxS {
  T rho, irho, U[3], lam, p, i2l, u0, u1, xi2, xi4;
};
/* normalised 1-D moment tables up to order 6, built from MxS by recurrence */
template <typename T> struct MxT {
  T u[7], v[7], w[7];
};

/* returns false for a non-positive density or pressure */
template <typename T, int DIM>
CGKS_HD bool mx_init(const T* W, T gam, T K, int region, MxS<T, DIM>& m) {
  m.rho = W[0];
  m.irho = T(1) / W[0];
  T ke = T(0);
#pragma unroll
  for (int i = 0; i < 3; ++i) m.U[i] = T(0);
#pragma unroll
  for (int i = 0; i < DIM; ++i) {
    m.U[i] = W[1 + i] * m.irho;
    ke += m.U[i] * W[1 + i];
  }
  m.p = cg_norm((gam - T(1)) * (W[DIM + 1] - T(0.5) * ke));
  if (!(m.rho > T(0)) || !(m.p > T(0))) return false;
  m.i2l = m.p * m.irho; /* 1/(2 lambda) = p/rho */
  m.lam = T(0.5) / m.i2l;
  if (region == REG_FULL) {
    m.u0 = T(1);
    m.u1 = m.U[0];
  } else {
    /* sqrt(lam) and 1/sqrt(pi lam) from one reciprocal square root */
    const T isl = cg_rsqrt(m.lam);
    const T sl = m.lam * isl;
    const T e = T(0.28209479177387814347) * cg_exp(-m.lam * m.U[0] * m.U[0]) * isl; /* 1/(2 sqrt(pi)) */
    if (region == REG_POS) {
      m.u0 = T(0.5) * cg_erfc(-sl * m.U[0]);
      m.u1 = m.U[0] * m.u0 + e;
    } else {
      m.u0 = T(0.5) * cg_erfc(sl * m.U[0]);
      m.u1 = m.U[0] * m.u0 - e;
    }
  }
  m.xi2 = K * m.i2l;
  m.xi4 = (K * K + T(2) * K) * m.i2l * m.i2l;
  return true;
}

template <typename T, int DIM>
CGKS_HD void mx_tables(const MxS<T, DIM>& m, MxT<T>& t) {
  t.u[0] = m.u0;
  t.u[1] = m.u1;
  t.v[0] = T(1);
  t.v[1] = m.U[1];
  t.w[0] = T(1);
  t.w[1] = DIM == 3 ? m.U[2] : T(0);
#pragma unroll
  for (int n = 0; n < 5; ++n) {
    const T c = T(n + 1) * m.i2l;
    t.u[n + 2] = cg_dot2(m.U[0], t.u[n + 1], c, t.u[n]);
    t.v[n + 2] = cg_dot2(m.U[1], t.v[n + 1], c, t.v[n]);
    t.w[n + 2] = DIM == 3 ? cg_dot2(m.U[2], t.w[n + 1], c, t.w[n]) : T(0);
  }
}

/* out_i = < (al . psi) u^A v^B w^C psi_i >, psi = (1, u, v[, w], (u^2+v^2[+w^2]+xi^2)/2).
   Factorised over the three velocity directions: with P = al . psi and
   G(p, q, r) = < P u^p v^q w^r >,
     G(p,q,r) = u_p T(q,r) + (a1 u_{p+1} + ae/2 u_{p+2}) v_q w_r,
     T(q,r)   = v_q S(r) + (a2 v_{q+1} + ae/2 v_{q+2}) w_r,
     S(r)     = (a0 + ae/2 <xi^2>) w_r + a3 w_{r+1} + ae/2 w_{r+2},
   out_0..DIM are G at (A,B,C) and its unit shifts, and
   out_{DIM+1} = (G(A+2,B,C) + G(A,B+2,C) + G(A,B,C+2) + <xi^2> G(A,B,C)
                 + ae/2 (<xi^4> - <xi^2>^2) u_A v_B w_C) / 2.
   The same slope's moments at several (A, B, C) share their S, T and G
   terms once inlined into one scope, which is how the callers use it. */
template <typename T, int DIM> struct PolyMom {
  const MxT<T>& t;
  T a0x, a1, a2, a3, ah, xi2, xi4;
  CGKS_HD PolyMom(const MxS<T, DIM>& s, const MxT<T>& m, const T* al) : t(m) {
    ah = T(0.5) * al[DIM + 1];
    a0x = al[0] + ah * s.xi2;
    a1 = al[1];
    a2 = al[2];
    a3 = DIM == 3 ? al[DIM == 3 ? 3 : 0] : T(0);
    xi2 = s.xi2;
    xi4 = s.xi4;
  }
  template <int R> CGKS_HD T S() const {
    if constexpr (DIM == 3) return cg_dot3(a0x, t.w[R], a3, t.w[R + 1], ah, t.w[R + 2]);
    else return R == 0 ? a0x : T(0);
  }
  template <int R> CGKS_HD T W() const {
    if constexpr (DIM == 3) return t.w[R];
    else return R == 0 ? T(1) : T(0);
  }
  template <int Q, int R> CGKS_HD T Tq() const {
    return cg_dot2(t.v[Q], S<R>(), cg_dot2(a2, t.v[Q + 1], ah, t.v[Q + 2]), W<R>());
  }
  template <int P, int Q, int R> CGKS_HD T G() const {
    return cg_dot2(t.u[P], Tq<Q, R>(), cg_dot2(a1, t.u[P + 1], ah, t.u[P + 2]), t.v[Q] * W<R>());
  }
  template <int A, int B, int C> CGKS_HD void out(T* o) const {
    const T g0 = G<A, B, C>();
    o[0] = g0;
    o[1] = G<A + 1, B, C>();
    o[2] = G<A, B + 1, C>();
    T gs = G<A + 2, B, C>() + G<A, B + 2, C>();
    if constexpr (DIM == 3) {
      o[3] = G<A, B, C + 1>();
      gs += G<A, B, C + 2>();
    }
    const T e = cg_madd(ah * (xi4 - xi2 * xi2), t.u[A] * t.v[B] * W<C>(), cg_madd(xi2, g0, gs));
    o[DIM + 1] = T(0.5) * e;
  }
};

template <typename T, int DIM, int A, int B, int C>
CGKS_HD void mvec(const MxS<T, DIM>& s, const MxT<T>& m, const T* al, T* out) {
  PolyMom<T, DIM>(s, m, al).template out<A, B, C>(out);
}

/* <u^A psi> */
template <typename T, int DIM, int A>
CGKS_HD void mpsi_u(const MxS<T, DIM>& s, const MxT<T>& m, T* out) {
  out[0] = m.u[A];
  out[1] = m.u[A + 1];
  out[2] = m.u[A] * m.v[1];
  T c2 = m.v[2] + s.xi2;
  if constexpr (DIM == 3) {
    out[3] = m.u[A] * m.w[1];
    c2 += m.w[2];
  }
  out[DIM + 1] = T(0.5) * cg_madd(m.u[A], c2, m.u[A + 2]);
}

/* micro-slope: solve <a psi psi^T> = b in closed form (D = K + dim = 2/(gamma-1)) */
template <typename T, int DIM>
CGKS_HD void slope_solve(const MxS<T, DIM>& g, T D, T iD, const T* b, T* a) {
  T q2 = T(0), R[3], uR = T(0);
#pragma unroll
  for (int i = 0; i < DIM; ++i) {
    q2 = cg_madd(g.U[i], g.U[i], q2);
    R[i] = cg_madd(-g.U[i], b[0], b[1 + i]);
    uR = cg_madd(g.U[i], R[i], uR);
  }
  const T th = cg_madd(D, g.i2l, q2);
  const T Re = cg_madd(-th, b[0], T(2) * b[DIM + 1]);
  const T ae = T(4) * g.lam * g.lam * iD * (Re - T(2) * uR);
  const T l2 = T(2) * g.lam;
  T s = T(0);
#pragma unroll
  for (int i = 0; i < DIM; ++i) {
    a[1 + i] = cg_dot2(l2, R[i], -g.U[i], ae);
    s = cg_madd(g.U[i], a[1 + i], s);
  }
  a[DIM + 1] = ae;
  a[0] = cg_madd(T(-0.5) * ae, th, b[0] - s);
}

/* Euler flux along local axis j of a Maxwellian state, and its Jacobian
   applied to dW: for a Maxwellian, rho <(a.psi) u_j psi> = (dF_j/dW) dW when
   rho <a psi> = dW, which replaces the compatibility moments */
template <typename T, int DIM>
CGKS_HD void euler_flux(const MxS<T, DIM>& g, const T* W, int j, T* F) {
  const T H = (W[DIM + 1] + g.p) * g.irho;
  const T mj = W[1 + j];
  F[0] = mj;
#pragma unroll
  for (int i = 0; i < DIM; ++i) F[1 + i] = mj * g.U[i] + (i == j ? g.p : T(0));
  F[DIM + 1] = H * mj;
}

template <typename T, int DIM>
CGKS_HD void euler_jvp(const MxS<T, DIM>& g, T gam, const T* W, int j, const T* dW, T* out) {
  const T H = (W[DIM + 1] + g.p) * g.irho;
  T q2 = T(0), um = T(0);
#pragma unroll
  for (int i = 0; i < DIM; ++i) {
    q2 += g.U[i] * g.U[i];
    um += g.U[i] * dW[1 + i];
  }
  const T dp = (gam - T(1)) * (dW[DIM + 1] - um + T(0.5) * q2 * dW[0]);
  /* by selects: j may be a run-time loop index (an indexed register array
     would go to local memory) */
  const T uj = j == 0 ? g.U[0] : (j == 1 ? g.U[1] : g.U[DIM - 1]);
  const T dmj = j == 0 ? dW[1] : (j == 1 ? dW[2] : dW[DIM]);
  out[0] = dmj;
#pragma unroll
  for (int i = 0; i < DIM; ++i) {
    const T o = cg_dot3(uj, dW[1 + i], g.U[i], dmj, -(uj * g.U[i]), dW[0]);
    out[1 + i] = i == j ? o + dp : o;
  }
  out[DIM + 1] = cg_dot2(uj, dW[DIM + 1] + dp, H, dmj - uj * dW[0]);
}

/* time integrals over [0, dl] of the six coefficient functions of Eq. (flux),
   given em = 1 - e^{-dl/tau} and ex = e^{-dl/tau} */
template <typename T>
CGKS_HD void tcoef(T tau, T dl, T em, T ex, T* c) {
  if (tau <= T(0)) {
    c[0] = dl; c[1] = T(0); c[2] = T(0.5) * dl * dl; c[3] = T(0); c[4] = T(0); c[5] = T(0);
    return;
  }
  c[0] = dl - tau * em;
  c[1] = T(2) * tau * tau - tau * (dl + T(2) * tau) * ex - tau * dl;
  c[2] = T(0.5) * dl * dl - tau * dl + tau * tau * em;
  c[3] = tau * em;
  c[4] = T(-2) * tau * tau + tau * (dl + T(2) * tau) * ex;
  c[5] = -tau * tau * em;
}

/* qw . o: the psi-moment vector o of a distribution part weighted into its
   moment of the peculiar energy about the interface velocity U,
   qw = (|U|^2/2, -U, 1), which is all the heat-flux fix needs of it */
template <typename T, int DIM> CGKS_HD T qdot(const T* qw, const T* o) {
  T q = qw[DIM + 1] * o[DIM + 1];
#pragma unroll
  for (int i = 0; i <= DIM; ++i) q = cg_madd(qw[i], o[i], q);
  return q;
}

/* one side (the left half Maxwellian for u > 0 or the right one for u < 0):
   its slopes along each local axis, its share of the g0 slopes dW0, its
   compatibility right-hand side and time slope, and its flux parts 4 and 5
   (and their psi-moments for the heat-flux fix) */
template <typename T, int DIM, int J>
CGKS_HD void side_dir(const MxS<T, DIM>& s, const MxT<T>& t, T gam, T D, T iD, const T* W, const T* dWj,
                      const T* cn, const T* ct, bool prfix, T* Fn, T* Ft, const T* qw, T& qn, T& qt, T* bs,
                      T* dW0j) {
  constexpr int NV = DIM + 2;
  constexpr int E0 = J == 0, E1 = J == 1, E2 = J == 2;
  T b[NV], a[NV], t1[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) b[i] = dWj[i] * s.irho;
  slope_solve<T, DIM>(s, D, iD, b, a);
  mvec<T, DIM, 0, 0, 0>(s, t, a, t1);
#pragma unroll
  for (int i = 0; i < NV; ++i) dW0j[i] = cg_madd(s.rho, t1[i], dW0j[i]);
  euler_jvp<T, DIM>(s, gam, W, J, dWj, t1);
#pragma unroll
  for (int i = 0; i < NV; ++i) bs[i] = cg_madd(-t1[i], s.irho, bs[i]);
  mvec<T, DIM, 1 + E0, E1, E2>(s, t, a, t1);
  const T crn = cn[4] * s.rho, crt = ct[4] * s.rho;
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    Fn[i] = cg_madd(crn, t1[i], Fn[i]);
    Ft[i] = cg_madd(crt, t1[i], Ft[i]);
  }
  if (prfix) {
    mvec<T, DIM, E0, E1, E2>(s, t, a, t1);
    const T q = qdot<T, DIM>(qw, t1);
    qn = cg_madd(crn, q, qn);
    qt = cg_madd(crt, q, qt);
  }
}

template <typename T, int DIM, class Ld>
CGKS_HD void side_all(const MxS<T, DIM>& s, const MxT<T>& t, T gam, T D, T iD, const T* W, const Ld& ld, int side,
                      const T* cn, const T* ct, bool prfix, T* Fn, T* Ft, const T* qw, T& qn, T& qt, T* bs,
                      T* dW0) {
  constexpr int NV = DIM + 2;
#pragma unroll
  for (int i = 0; i < NV; ++i) bs[i] = T(0);
  T dWj[NV];
  ld.grad(side, 0, dWj);
  side_dir<T, DIM, 0>(s, t, gam, D, iD, W, dWj, cn, ct, prfix, Fn, Ft, qw, qn, qt, bs, dW0);
  ld.grad(side, 1, dWj);
  side_dir<T, DIM, 1>(s, t, gam, D, iD, W, dWj, cn, ct, prfix, Fn, Ft, qw, qn, qt, bs, dW0 + NV);
  if constexpr (DIM == 3) {
    ld.grad(side, 2, dWj);
    side_dir<T, DIM, 2>(s, t, gam, D, iD, W, dWj, cn, ct, prfix, Fn, Ft, qw, qn, qt, bs, dW0 + 2 * NV);
  }
  T A[NV], t1[NV];
  slope_solve<T, DIM>(s, D, iD, bs, A);
  mvec<T, DIM, 1, 0, 0>(s, t, A, t1);
  const T crn = cn[5] * s.rho, crt = ct[5] * s.rho;
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    Fn[i] = cg_madd(crn, t1[i], Fn[i]);
    Ft[i] = cg_madd(crt, t1[i], Ft[i]);
  }
  if (prfix) {
    mvec<T, DIM, 0, 0, 0>(s, t, A, t1);
    const T q = qdot<T, DIM>(qw, t1);
    qn = cg_madd(crn, q, qn);
    qt = cg_madd(crt, q, qt);
  }
}

/* g0 along local axis j: slope from dW0_j, flux part 1 and the compatibility
   right-hand side (whose psi-moment is the Euler Jacobian product) */
template <typename T, int DIM, int J>
CGKS_HD void g0_dir(const MxS<T, DIM>& z, const MxT<T>& t, T gam, T D, T iD, const T* W0, const T* dW0j,
                    const T* cn, const T* ct, bool prfix, T* Fn, T* Ft, const T* qw, T& qn, T& qt, T* b0) {
  constexpr int NV = DIM + 2;
  constexpr int E0 = J == 0, E1 = J == 1, E2 = J == 2;
  T b[NV], a[NV], t1[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) b[i] = dW0j[i] * z.irho;
  slope_solve<T, DIM>(z, D, iD, b, a);
  mvec<T, DIM, 1 + E0, E1, E2>(z, t, a, t1);
  const T crn = cn[1] * z.rho, crt = ct[1] * z.rho;
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    Fn[i] = cg_madd(crn, t1[i], Fn[i]);
    Ft[i] = cg_madd(crt, t1[i], Ft[i]);
  }
  euler_jvp<T, DIM>(z, gam, W0, J, dW0j, t1);
#pragma unroll
  for (int i = 0; i < NV; ++i) b0[i] = cg_madd(-t1[i], z.irho, b0[i]);
  if (prfix) {
    const T q = qdot<T, DIM>(qw, t1);
    qn = cg_madd(cn[1], q, qn);
    qt = cg_madd(ct[1], q, qt);
  }
}

/* The interface solution in the local frame (x normal to the face).
   WL, WR: conservative states (normal momentum first); dWL, dWR: DIM x NV
   derivatives along the local axes.  out[part*NV + v], parts F^n, F_t^n,
   Q^l(0), (dQ/dt)^l, Q^r(0), (dQ/dt)^r.  Returns false on a non-physical state.
   Readings: g0 and its slopes from the kinetic collision of the two half
   Maxwellians; f^n, f_t^n from the time integrals over dt and dt/2; the
   interface values of the two-sided model with tau0 = 5|pl-pr|/(pl+pr) dt. */
template <typename T, int DIM, class Ld>
CGKS_HD bool gks_point_ld(const Phys& ph, T dt, const T* WL, const T* WR, const Ld& ld, T* out) {
  constexpr int NV = DIM + 2;
  const T gam = ph_gamma<T>(ph);
  const T D = T(2) / (gam - T(1));
  const T iD = T(0.5) * (gam - T(1));
  const T K = D - T(DIM);
  MxS<T, DIM> l, r, z;
  /* equilibrium state W0 and flux part 3 from the two half Maxwellians (the
     moment tables are rebuilt for the slope parts below: keeping both sides'
     tables live spills 250 B per thread in FP64 3-D and measured no faster) */
  T W0[NV], H3[NV], t1[NV], t2[NV];
  if constexpr (cg_same<T, fpair>::value) {
    /* the paired solve: one rolled copy for both sides (see the side loop) */
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      W0[i] = T(0);
      H3[i] = T(0);
    }
#pragma unroll 1
    for (int side = 0; side < 2; ++side) {
      T W[NV];
#pragma unroll
      for (int i = 0; i < NV; ++i) W[i] = side ? WR[i] : WL[i];
      MxS<T, DIM> m;
      if (!mx_init<T, DIM>(W, gam, K, side ? REG_NEG : REG_POS, m)) return false;
      MxT<T> t;
      mx_tables<T, DIM>(m, t);
      mpsi_u<T, DIM, 0>(m, t, t1);
      mpsi_u<T, DIM, 1>(m, t, t2);
#pragma unroll
      for (int i = 0; i < NV; ++i) {
        W0[i] = cg_madd(m.rho, t1[i], W0[i]);
        H3[i] = cg_madd(m.rho, t2[i], H3[i]);
      }
      if (side) r = m;
      else l = m;
    }
  } else {
    if (!mx_init<T, DIM>(WL, gam, K, REG_POS, l) || !mx_init<T, DIM>(WR, gam, K, REG_NEG, r)) return false;
    MxT<T> t;
    mx_tables<T, DIM>(l, t);
    mpsi_u<T, DIM, 0>(l, t, t1);
    mpsi_u<T, DIM, 1>(l, t, t2);
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      W0[i] = l.rho * t1[i];
      H3[i] = l.rho * t2[i];
    }
    mx_tables<T, DIM>(r, t);
    mpsi_u<T, DIM, 0>(r, t, t1);
    mpsi_u<T, DIM, 1>(r, t, t2);
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      W0[i] += r.rho * t1[i];
      H3[i] += r.rho * t2[i];
    }
  }
  if (!mx_init<T, DIM>(W0, gam, K, REG_FULL, z)) return false;
  /* collision time (Sec. 6) and the time-integral coefficients */
  const T jump = cg_fabs((l.p - r.p) / (l.p + r.p));
  T tau = T(0);
  if (ph.tau_mode == 1) tau = T(0.05) * dt + T(5) * jump * dt;
  else if (ph.tau_mode == 2) tau = ph_mu<T>(ph) / z.p + T(5) * jump * dt;
  T cn[6], ct[6];
  {
    /* one expm1 serves both intervals: with eh = 1 - e^{-dt/(2 tau)},
       1 - e^{-dt/tau} = eh (2 - eh) and e^{-dt/tau} = (1 - eh)^2 */
    T cf[6], chf[6];
    const T eh = tau > T(0) ? -cg_expm1(T(-0.5) * dt / tau) : T(0);
    const T xh = T(1) - eh;
    tcoef<T>(tau, dt, eh * (T(2) - eh), xh * xh, cf);
    tcoef<T>(tau, T(0.5) * dt, eh, xh, chf);
    const T idt = T(1) / dt;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      cn[i] = (T(4) * chf[i] - cf[i]) * idt;
      ct[i] = T(4) * (cf[i] - T(2) * chf[i]) * idt * idt;
    }
  }
  const bool prfix = ph.prfix != 0;
  T Fn[NV], Ft[NV], bl[NV], br[NV], b0[NV], dW0[DIM * NV];
  /* the heat-flux fix needs of the psi-moments Q of f^n and f_t^n only their
     peculiar-energy moment about the interface velocity, qw . Q */
  T qw[NV];
  {
    T u2 = T(0);
#pragma unroll
    for (int i = 0; i < DIM; ++i) {
      qw[1 + i] = -z.U[i];
      u2 += z.U[i] * z.U[i];
    }
    qw[0] = T(0.5) * u2;
    qw[DIM + 1] = T(1);
  }
  euler_flux<T, DIM>(z, W0, 0, t1); /* part 0: rho0 <u psi> of g0 */
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    Fn[i] = cg_dot2(cn[0], t1[i], cn[3], H3[i]);
    Ft[i] = cg_dot2(ct[0], t1[i], ct[3], H3[i]);
    b0[i] = T(0);
  }
  T qn = T(0), qt = T(0);
  if (prfix) {
    const T q = qdot<T, DIM>(qw, W0);
    qn = (cn[0] + cn[3]) * q;
    qt = (ct[0] + ct[3]) * q;
  }
#pragma unroll
  for (int i = 0; i < DIM * NV; ++i) dW0[i] = T(0);
  if constexpr (cg_same<T, fpair>::value) {
    /* the paired solve: one copy of the per-side code, run for the left and
       then the right side (its straight-line code is what the instruction
       fetch of this kernel waits on); same order, same results */
#pragma unroll 1
    for (int side = 0; side < 2; ++side) {
      const MxS<T, DIM> s = side ? r : l;
      T W[NV], bs[NV];
#pragma unroll
      for (int i = 0; i < NV; ++i) W[i] = side ? WR[i] : WL[i];
      MxT<T> t;
      mx_tables<T, DIM>(s, t);
      side_all<T, DIM>(s, t, gam, D, iD, W, ld, side, cn, ct, prfix, Fn, Ft, qw, qn, qt, bs, dW0);
#pragma unroll
      for (int i = 0; i < NV; ++i) {
        if (side) br[i] = bs[i];
        else bl[i] = bs[i];
      }
    }
  } else {
    MxT<T> t;
    mx_tables<T, DIM>(l, t);
    side_all<T, DIM>(l, t, gam, D, iD, WL, ld, 0, cn, ct, prfix, Fn, Ft, qw, qn, qt, bl, dW0);
    mx_tables<T, DIM>(r, t);
    side_all<T, DIM>(r, t, gam, D, iD, WR, ld, 1, cn, ct, prfix, Fn, Ft, qw, qn, qt, br, dW0);
  }
  {
    MxT<T> t;
    mx_tables<T, DIM>(z, t);
    if constexpr (cg_same<T, fpair>::value) {
      /* the paired solve: the three directions as one rolled loop (the
         direction's slopes picked by selects, its flux moments by
         warp-uniform branches); same order, same results */
#pragma unroll 1
      for (int j = 0; j < DIM; ++j) {
        T dj[NV], b[NV], a[NV], t1[NV];
#pragma unroll
        for (int i = 0; i < NV; ++i) {
          dj[i] = j == 0 ? dW0[i] : (j == 1 ? dW0[NV + i] : dW0[(DIM - 1) * NV + i]);
          b[i] = dj[i] * z.irho;
        }
        slope_solve<T, DIM>(z, D, iD, b, a);
        if (j == 0) mvec<T, DIM, 2, 0, 0>(z, t, a, t1);
        else if (DIM == 2 || j == 1) mvec<T, DIM, 1, 1, 0>(z, t, a, t1);
        else mvec<T, DIM, 1, 0, DIM == 3 ? 1 : 0>(z, t, a, t1);
        const T crn = cn[1] * z.rho, crt = ct[1] * z.rho;
#pragma unroll
        for (int i = 0; i < NV; ++i) {
          Fn[i] = cg_madd(crn, t1[i], Fn[i]);
          Ft[i] = cg_madd(crt, t1[i], Ft[i]);
        }
        euler_jvp<T, DIM>(z, gam, W0, j, dj, t1);
#pragma unroll
        for (int i = 0; i < NV; ++i) b0[i] = cg_madd(-t1[i], z.irho, b0[i]);
        if (prfix) {
          const T q = qdot<T, DIM>(qw, t1);
          qn = cg_madd(cn[1], q, qn);
          qt = cg_madd(ct[1], q, qt);
        }
      }
    } else {
      g0_dir<T, DIM, 0>(z, t, gam, D, iD, W0, dW0, cn, ct, prfix, Fn, Ft, qw, qn, qt, b0);
      g0_dir<T, DIM, 1>(z, t, gam, D, iD, W0, dW0 + NV, cn, ct, prfix, Fn, Ft, qw, qn, qt, b0);
      if constexpr (DIM == 3) g0_dir<T, DIM, 2>(z, t, gam, D, iD, W0, dW0 + 2 * NV, cn, ct, prfix, Fn, Ft, qw, qn, qt, b0);
    }
  }
  /* part 2: rho0 <A0 u psi> = (dF_x/dW)(rho0 b0), psi-moment rho0 b0 */
#pragma unroll
  for (int i = 0; i < NV; ++i) t2[i] = z.rho * b0[i];
  euler_jvp<T, DIM>(z, gam, W0, 0, t2, t1);
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    Fn[i] = cg_madd(cn[2], t1[i], Fn[i]);
    Ft[i] = cg_madd(ct[2], t1[i], Ft[i]);
  }
  if (prfix) { /* heat-flux correction F_E += (1/Pr - 1) q about the interface velocity,
                  q = qw . F - U_x qw . Q of the non-equilibrium part f - g0 (1 + A0 t):
                  g0 adds no heat flux to f^n; A0 g0 (part 2, weight one in f_t^n)
                  is taken out of the time derivative's */
    const T q2 = qdot<T, DIM>(qw, t2);
    qn += cn[2] * q2;
    qt += ct[2] * q2;
    const T f = T(1) / ph_pr<T>(ph) - T(1);
    const T hn = qdot<T, DIM>(qw, Fn) - z.U[0] * qn;
    const T ht = qdot<T, DIM>(qw, Ft) - z.U[0] * qt - (qdot<T, DIM>(qw, t1) - z.U[0] * q2);
    Fn[DIM + 1] += f * hn;
    Ft[DIM + 1] += f * ht;
  }
  /* interface values for the derivative update (temporal discretisation section) */
  const T tau0 = T(5) * jump * dt;
  const T w = tau0 > T(0) ? cg_exp(-dt / tau0) : T(0);
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    out[i] = Fn[i];
    out[NV + i] = Ft[i];
    const T dq0 = z.rho * b0[i];
    out[2 * NV + i] = cg_dot2(T(1) - w, W0[i], w, WL[i]);
    out[3 * NV + i] = cg_dot2(T(1) - w, dq0, w * l.rho, bl[i]);
    out[4 * NV + i] = cg_dot2(T(1) - w, W0[i], w, WR[i]);
    out[5 * NV + i] = cg_dot2(T(1) - w, dq0, w * r.rho, br[i]);
  }
  return true;
}

/* derivative loader over local arrays dWL, dWR (DIM x NV each) */
template <typename T, int DIM> struct ArrLd {
  const T* dL;
  const T* dR;
  CGKS_HD void grad(int side, int j, T* o) const {
    const T* src = (side == 0 ? dL : dR) + j * (DIM + 2);
    for (int i = 0; i < DIM + 2; ++i) o[i] = src[i];
  }
};

template <typename T, int DIM>
CGKS_HD bool gks_point(const Phys& ph, T dt, const T* WL, const T* dWL, const T* WR, const T* dWR, T* out) {
  ArrLd<T, DIM> ld{dWL, dWR};
  return gks_point_ld<T, DIM>(ph, dt, WL, WR, ld, out);
}

/* derivative loader of the Cartesian path: reads the local-frame derivative of
   side 0 (left, gl) or 1 (right, gr) along local axis j, through the
   signed-permutation frame.  Component q of a side's Gauss-point state is at
   [(base + q) * N + c]: the global face-major arrays (base of the face, N =
   cells, c = slot), or a thread's staged copy in shared memory (base 0, N =
   the block size, c = the thread) */
template <typename T, int DIM, typename C = T> struct CartLd {
  const T* gl;
  const T* gr;
  long base, N, c;
  int p[3], s[3];
  CGKS_HD void grad(int side, int j, C* o) const {
    const T* src = side == 0 ? gl : gr;
#pragma unroll
    for (int v = 0; v < DIM + 2; ++v) {
      int vg = v, sv = 1;
      if (v >= 1 && v <= DIM) { vg = 1 + p[v - 1]; sv = s[v - 1]; }
      o[v] = C(T(sv * s[j]) * src[(base + vg * (1 + DIM) + 1 + p[j]) * N + c]);
    }
  }
};

/* asynchronous copy of one element global -> shared (cp.async, sm_80 on):
   the copies of a thread stay in flight together until async_wait_all */
template <typename T> __device__ __forceinline__ void async_copy(T* dst_smem, const T* src) {
#if defined(__CUDA_ARCH__)
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst_smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(d), "l"(src), "n"(sizeof(T)) : "memory");
#else
  *dst_smem = *src;
#endif
}
__device__ __forceinline__ void async_wait_all() {
#if defined(__CUDA_ARCH__)
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
#endif
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

/* Cartesian face frames as signed permutations: local axis i = s[i] e_{p[i]}.
   They equal face_frame for axis-aligned faces: (x,y,z), (y,x,-z), (z,x,y);
   2-D: (x,y), (y,-x). */
template <int DIM>
CGKS_HD void cart_frame(int ax, int* p, int* s) {
  if (DIM == 2) {
    p[0] = ax; p[1] = 1 - ax; s[0] = 1; s[1] = ax == 0 ? 1 : -1;
    return;
  }
  if (ax == 0) { p[0] = 0; p[1] = 1; p[2] = 2; s[0] = s[1] = s[2] = 1; }
  else if (ax == 1) { p[0] = 1; p[1] = 0; p[2] = 2; s[0] = 1; s[1] = 1; s[2] = -1; }
  else { p[0] = 2; p[1] = 0; p[2] = 1; s[0] = s[1] = s[2] = 1; }
}

/* global-frame Gauss-point state (value + gradient per variable) -> local frame */
template <typename T, int DIM>
CGKS_HD void to_local(const double R[3][3], const T* st /* NV*(1+DIM) */, T* W, T* dW) {
  const int NV = DIM + 2;
  T gv[NV][3];
  for (int v = 0; v < NV; ++v) {
    W[v] = st[v * (1 + DIM)];
    for (int k = 0; k < DIM; ++k) gv[v][k] = st[v * (1 + DIM) + 1 + k];
  }
  T m[3];
  for (int i = 0; i < DIM; ++i) {
    m[i] = T(0);
    for (int a = 0; a < DIM; ++a) m[i] += T(R[i][a]) * W[1 + a];
  }
  for (int i = 0; i < DIM; ++i) W[1 + i] = m[i];
  T gr[NV][3];
  for (int k = 0; k < DIM; ++k) {
    gr[0][k] = gv[0][k];
    gr[NV - 1][k] = gv[NV - 1][k];
    for (int i = 0; i < DIM; ++i) {
      T s = T(0);
      for (int a = 0; a < DIM; ++a) s += T(R[i][a]) * gv[1 + a][k];
      gr[1 + i][k] = s;
    }
  }
  for (int j = 0; j < DIM; ++j)
    for (int v = 0; v < NV; ++v) {
      T s = T(0);
      for (int k = 0; k < DIM; ++k) s += T(R[j][k]) * gr[v][k];
      dW[j * NV + v] = s;
    }
}

template <typename T, int DIM>
CGKS_HD void to_global(const double R[3][3], T* F) {
  T m[3];
  for (int a = 0; a < DIM; ++a) {
    m[a] = T(0);
    for (int i = 0; i < DIM; ++i) m[a] += T(R[i][a]) * F[1 + i];
  }
  for (int a = 0; a < DIM; ++a) F[1 + a] = m[a];
}

/* one face Gauss point: gather, rotate, solve, rotate back, store.
   CURVI selects at compile time between the Cartesian signed-permutation
   frames and general face frames.  Cartesian: with sm (this thread's slot of
   a [2][NV (1+DIM)][ns] shared array, ns = the block size) the point's two
   Gauss-point states are first copied there asynchronously, all 2 NV (1+DIM)
   loads in flight at once, and the solve reads them from shared memory.
   C is the type the solve computes in: T, or fpair for the paired form,
   which converts the loaded (curvilinear: rotated) states and rounds the
   results back to T. */
template <typename T, int DIM, bool CURVI, typename C = T>
CGKS_HD bool flux_point(const DevGeo& g, const Phys& ph, T dt, int ax, int k, long c,
                        const T* __restrict__ gpL, const T* __restrict__ gpR, T* __restrict__ flux,
                        T* sm = nullptr, int ns = 0, bool staged = false) {
  typedef Sz<DIM> S;
  constexpr int NV = S::NV;
  const long N = g.ncell;
  const long base = (long)((ax * S::GPF + k) * NV) * (1 + DIM);
  if constexpr (!CURVI) {
    /* value and momentum: W_loc[1+i] = s_i m_{p_i}; derivative along local j:
       s_j d/dx_{p_j} of the local variable (loaded when its side needs it) */
    constexpr int NQ = NV * (1 + DIM);
    C WL[NV], WR[NV], out[6 * NV];
    CartLd<T, DIM, C> ld;
    if (sm) {
      if (!staged) { /* else the block's tile is in shared memory already (TMA) */
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
          async_copy(sm + (long)q * ns, gpL + (base + q) * N + c);
          async_copy(sm + (long)(NQ + q) * ns, gpR + (base + q) * N + c);
        }
        async_wait_all();
      }
      ld.gl = sm;
      ld.gr = sm + (long)NQ * ns;
      ld.base = 0;
      ld.N = ns;
      ld.c = 0;
    } else {
      ld.gl = gpL;
      ld.gr = gpR;
      ld.base = base;
      ld.N = N;
      ld.c = c;
    }
    cart_frame<DIM>(ax, ld.p, ld.s);
    const int* p = ld.p;
    const int* s = ld.s;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      int vg = v, sv = 1;
      if (v >= 1 && v <= DIM) { vg = 1 + p[v - 1]; sv = s[v - 1]; }
      const long b = (ld.base + vg * (1 + DIM)) * ld.N + ld.c;
      WL[v] = C(T(sv) * ld.gl[b]);
      WR[v] = C(T(sv) * ld.gr[b]);
    }
    bool ok = gks_point_ld<C, DIM>(ph, C(dt), WL, WR, ld, out);
    const long fb = (long)((ax * S::GPF + k) * 6) * NV;
#pragma unroll
    for (int part = 0; part < 6; ++part) {
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        int vg = v, sv = 1;
        if (v >= 1 && v <= DIM) { vg = 1 + p[v - 1]; sv = s[v - 1]; }
        flux[(fb + part * NV + vg) * N + c] = T(sv) * to_storage<T>(out[part * NV + v]);
      }
    }
    return ok;
  } else {
  T WL[NV], WR[NV], out[6 * NV];
  T dWL[DIM * NV], dWR[DIM * NV];
  T sl[NV * (1 + DIM)], sr[NV * (1 + DIM)];
  for (int q = 0; q < NV * (1 + DIM); ++q) {
    sl[q] = gpL[(base + q) * N + c];
    sr[q] = gpR[(base + q) * N + c];
  }
  double A[3], Tt[3];
  int gp = (2 * ax + 1) * S::GPF + k;
  for (int a = 0; a < 3; ++a) {
    A[a] = a < DIM ? met_area<DIM>(g, c, gp, a) : 0.0;
    Tt[a] = a < DIM ? met_tang<DIM>(g, c, ax, k, a) : 0.0;
  }
  double R[3][3];
  face_frame<DIM>(A, Tt, R);
  to_local<T, DIM>(R, sl, WL, dWL);
  to_local<T, DIM>(R, sr, WR, dWR);
  bool ok;
  if constexpr (cg_same<C, T>::value) {
    ok = gks_point<T, DIM>(ph, dt, WL, dWL, WR, dWR, out);
  } else {
    /* the rotation stays in the storage type; the solve computes in C */
    C cWL[NV], cWR[NV], cdL[DIM * NV], cdR[DIM * NV], cout[6 * NV];
    for (int i = 0; i < NV; ++i) {
      cWL[i] = C(WL[i]);
      cWR[i] = C(WR[i]);
    }
    for (int i = 0; i < DIM * NV; ++i) {
      cdL[i] = C(dWL[i]);
      cdR[i] = C(dWR[i]);
    }
    ok = gks_point<C, DIM>(ph, C(dt), cWL, cdL, cWR, cdR, cout);
    for (int i = 0; i < 6 * NV; ++i) out[i] = to_storage<T>(cout[i]);
  }
  for (int p = 0; p < 6; ++p) to_global<T, DIM>(R, out + p * NV);
  const long fb = (long)((ax * S::GPF + k) * 6) * NV;
  for (int q = 0; q < 6 * NV; ++q) flux[(fb + q) * N + c] = out[q];
  return ok;
  }
}

/* ---- boundary faces ---------------------------------------------------- */
/* In the face frame (local axis 0 = the wall normal) the mirror image of a
   state negates the normal momentum (every momentum component at a no-slip
   wall) and derivatives along the normal; an outflow image is a copy. */
template <int DIM> CGKS_HD int image_odd(int kind, int v, int j /* -1: the value */) {
  if (kind == BC_OUTFLOW) return 0;
  const int f = (v == 1 || (kind == BC_NOSLIP && v >= 1 && v <= DIM)) ? 1 : 0;
  return f ^ (j == 0 ? 1 : 0);
}

/* derivative loader of a boundary face: the real side's derivatives from
   global memory (CartLd), the image side's from the same with image_odd */
template <typename T, int DIM> struct BndLd {
  CartLd<T, DIM> cl;
  int real, kind;
  CGKS_HD void grad(int side, int j, T* o) const {
    if (side != real && kind == BC_INFLOW) {
#pragma unroll
      for (int v = 0; v < DIM + 2; ++v) o[v] = T(0);
      return;
    }
    cl.grad(real, j, o);
    if (side != real) {
#pragma unroll
      for (int v = 0; v < DIM + 2; ++v)
        if (image_odd<DIM>(kind, v, j)) o[v] = -o[v];
    }
  }
};

/* A wall face (adiabatic: the paper's non-slip adiabatic wall and its slip
   counterpart) passes no mass and no energy, and the gas on it slides along
   the wall (slip) or rests (no-slip): in the face frame the mass and energy
   parts of F and F_t are zero and the interface values (parts 2..5) carry no
   normal (slip) or no (no-slip) momentum */
template <typename T, int DIM> CGKS_HD void wall_face_local(int kind, T* out) {
  constexpr int NV = DIM + 2;
  out[0] = out[NV - 1] = T(0);
  out[NV] = out[2 * NV - 1] = T(0);
#pragma unroll
  for (int part = 2; part < 6; ++part)
#pragma unroll
    for (int i = 1; i <= DIM; ++i)
      if (i == 1 || kind == BC_NOSLIP) out[part * NV + i] = T(0);
}

/* One Gauss point of a domain-boundary face: the GKS problem between the
   Gauss-point state of the boundary cell (side `real`: 0 = it is the left
   state, at the high boundary; 1 = the right state, at the low boundary),
   read from face slot c, and its image; the result goes to
   out[(part * NV + var) * ns + oidx] of the point's block.  Curvilinear
   meshes take outflow only (the image is a copy); the frame comes from the
   area vector of Gauss point fgp of cell fc. */
template <typename T, int DIM, bool CURVI>
CGKS_HD bool flux_bnd_point(const DevGeo& g, const Phys& ph, T dt, int ax, int k, long c, long fc, int fgp,
                            int real, int kind, const T* __restrict__ gpL, const T* __restrict__ gpR,
                            T* __restrict__ out_arr, long ns, long oidx) {
  typedef Sz<DIM> S;
  constexpr int NV = S::NV;
  const long N = g.ncell;
  const long base = (long)((ax * S::GPF + k) * NV) * (1 + DIM);
  const long fb = (long)((ax * S::GPF + k) * 6) * NV;
  T WL[NV], WR[NV], out[6 * NV];
  const T* src = real ? gpR : gpL;
  if constexpr (!CURVI) {
    BndLd<T, DIM> ld;
    ld.cl.gl = gpL;
    ld.cl.gr = gpR;
    ld.cl.base = base;
    ld.cl.N = N;
    ld.cl.c = c;
    ld.real = real;
    ld.kind = kind;
    cart_frame<DIM>(ax, ld.cl.p, ld.cl.s);
    const int* p = ld.cl.p;
    const int* sg = ld.cl.s;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      int vg = v, sv = 1;
      if (v >= 1 && v <= DIM) { vg = 1 + p[v - 1]; sv = sg[v - 1]; }
      const T w = T(sv) * src[(base + vg * (1 + DIM)) * N + c];
      const int face = 2 * ax + (real ? 0 : 1);
      const T wi = kind == BC_INFLOW ? T(sv) * T(g.bcq[face * 5 + vg]) : (image_odd<DIM>(kind, v, -1) ? -w : w);
      WL[v] = real ? wi : w;
      WR[v] = real ? w : wi;
    }
    bool ok = gks_point_ld<T, DIM>(ph, dt, WL, WR, ld, out);
    if (bc_wall(kind)) wall_face_local<T, DIM>(kind, out);
#pragma unroll
    for (int part = 0; part < 6; ++part) {
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        int vg = v, sv = 1;
        if (v >= 1 && v <= DIM) { vg = 1 + p[v - 1]; sv = sg[v - 1]; }
        out_arr[(fb + part * NV + vg) * ns + oidx] = T(sv) * out[part * NV + v];
      }
    }
    return ok;
  } else {
    T dW[DIM * NV];
    T st[NV * (1 + DIM)];
    for (int q = 0; q < NV * (1 + DIM); ++q) st[q] = src[(base + q) * N + c];
    double A[3], Tt[3];
    for (int a = 0; a < 3; ++a) {
      A[a] = a < DIM ? met_area<DIM>(g, fc, fgp, a) : 0.0;
      Tt[a] = a < DIM ? met_tang<DIM>(g, fc, ax, k, a) : 0.0;
    }
    double R[3][3];
    face_frame<DIM>(A, Tt, R);
    to_local<T, DIM>(R, st, WL, dW);
    bool ok;
    if (kind == BC_INFLOW) {
      /* the fixed state, zero derivatives, on the image side */
      const int face = 2 * ax + (real ? 0 : 1);
      T sq[NV * (1 + DIM)], Wq[NV], dq[DIM * NV];
      for (int v = 0; v < NV; ++v) {
        sq[v * (1 + DIM)] = T(g.bcq[face * 5 + v]);
        for (int k2 = 0; k2 < DIM; ++k2) sq[v * (1 + DIM) + 1 + k2] = T(0);
      }
      to_local<T, DIM>(R, sq, Wq, dq);
      ok = real ? gks_point<T, DIM>(ph, dt, Wq, dq, WL, dW, out) : gks_point<T, DIM>(ph, dt, WL, dW, Wq, dq, out);
    } else {
      for (int v = 0; v < NV; ++v) WR[v] = WL[v];
      ok = gks_point<T, DIM>(ph, dt, WL, dW, WR, dW, out);
    }
    for (int part = 0; part < 6; ++part) to_global<T, DIM>(R, out + part * NV);
    for (int q = 0; q < 6 * NV; ++q) out_arr[(fb + q) * ns + oidx] = out[q];
    return ok;
  }
}

/* ===================================================================== */
/* (c) accumulation and S2O4 update of one cell                          */
/* ===================================================================== */
/* S2O4 update of variable v of cell c (temporal discretisation section):
   stage 1: out = U* ; stash = {Q^n + dt L + dt^2/6 L_t ; D(Q^n(x_G))}
   stage 2: out = U^{n+1} = {stash + dt^2/3 L_t* ; stash_D + dt D((dQ/dt)*(x_G))}
   L = -(1/|Omega|) sum_faces sum_k F.n S (Eq. semi with Gauss quadrature); the
   gradient by Gauss' theorem (Eq. derivative) and the line derivatives by
   Eq. (derivative-l) from the interface values of each side.  CURVI = false:
   axis-aligned cells, where both reduce to differences divided by h. */
/* the step's FP64 coefficients of the S2O4 update, formed once when dt is
   set (stage_coef) instead of by every thread of the update (the same
   products, in the same order): stage 1: U* = Q + h1 L + e1 Lt and the stash
   Q + dt L + s1 Lt; stage 2: U = stash + t2 Lt */
struct StageCoef {
  double dt, h1, e1, s1, t2;
};
CGKS_HD StageCoef stage_coef(double dt) {
  StageCoef k;
  k.dt = dt;
  k.h1 = 0.5 * dt;
  k.e1 = 0.125 * dt * dt;
  k.s1 = dt * dt / 6.0;
  k.t2 = dt * dt / 3.0;
  return k;
}

/* a stored value as double: floats exactly, on the integer pipe (the FP32
   form's update is bound by its FP64 pipe, which would convert them) */
template <typename T> CGKS_HD double to_f64(const T& x) { return double(x); }
CGKS_HD double to_f64(float x) { return fp_f2d_exact(x); }

template <typename T, int DIM, bool CURVI>
CGKS_HD void update_var(const DevGeo& g, const StageCoef& kc, int stage, long c, int ci, int cj, int ck, int v,
                        const double* __restrict__ avg_in, const T* __restrict__ flux, const T* __restrict__ fxb,
                        double* __restrict__ stash_avg, T* __restrict__ stash_der, double* __restrict__ avg_out,
                        T* __restrict__ der_out, float* __restrict__ avh_out, float* __restrict__ avl_out) {
  typedef Sz<DIM> S;
  constexpr int NV = S::NV, GPF = S::GPF;
  const long N = g.ncell;
  const double dt = kc.dt;
  const T tdt = T(dt), hdt = T(0.5) * tdt;
  T ivol = T(1);
  if constexpr (CURVI) ivol = T(1.0 / met_vol<DIM>(g, c));
  /* L and dL/dt accumulate in FP64 from per-face sums in T: both cells of a
     face form the same face sum in the same order, so the face enters them
     with exactly opposite values and domain sums are conserved to FP64
     rounding */
  double L = 0.0, Lt = 0.0;
  T gn[3] = {T(0), T(0), T(0)}, gt[3] = {T(0), T(0), T(0)};
#pragma unroll
  for (int ax = 0; ax < DIM; ++ax) {
    int o[3] = {0, 0, 0};
    o[ax] = -1;
    const long lo = nbr(g, ci, cj, ck, o[0], o[1], o[2]);
    /* the low face of a cell on a non-periodic low boundary lives in fxb */
    const int cc[3] = {ci, cj, ck};
    const bool lowb = geo_bc(g, 2 * ax) != BC_PERIODIC && cc[ax] == 0;
    const T* __restrict__ fsrc = lowb ? fxb : flux;
    const long fs = lowb ? g.nplane : N;
    const long fi = lowb ? plane_index(g, ax, ci, cj, ck) : lo;
    const T ih = CURVI ? T(1) : geo_ih<T>(g, ax);
    T sh_f = T(0), sl_f = T(0), sth_f = T(0), stl_f = T(0); /* face sums, high and low face */
#pragma unroll
    for (int k = 0; k < GPF; ++k) {
      const long fb = (long)((ax * GPF + k) * 6) * NV + v;
      const int ghi = (2 * ax + 1) * GPF + k, glo = (2 * ax) * GPF + k;
      const T fh = flux[(fb + 0 * NV) * N + c], fl = fsrc[(fb + 0 * NV) * fs + fi];
      const T fth = flux[(fb + 1 * NV) * N + c], ftl = fsrc[(fb + 1 * NV) * fs + fi];
      const T qnh = flux[(fb + 2 * NV) * N + c], qth = flux[(fb + 3 * NV) * N + c];
      const T qnl = fsrc[(fb + 4 * NV) * fs + fi], qtl = fsrc[(fb + 5 * NV) * fs + fi];
      if constexpr (CURVI) {
        T a2 = T(0), b2 = T(0);
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
          const T ah = T(met_area<DIM>(g, c, ghi, a));
          const T al = T(lowb ? met_area<DIM>(g, c, glo, a) : met_area<DIM>(g, lo, ghi, a));
          a2 += ah * ah;
          b2 += al * al;
          /* Gauss' theorem with the cell's own outward area vectors */
          const T Al = T(met_area<DIM>(g, c, glo, a));
          gn[a] += qnh * ah - qnl * Al;
          gt[a] += qth * ah - qtl * Al;
        }
        const T sh = cg_sqrt(a2), sl = cg_sqrt(b2);
        sh_f += fh * sh;
        sl_f += fl * sl;
        sth_f += fth * sh;
        stl_f += ftl * sl;
      } else {
        sh_f += fh;
        sl_f += fl;
        sth_f += fth;
        stl_f += ftl;
      }
      /* line derivative s = ax*GPF + k, Eq. (derivative-l) */
      const int s2 = ax * GPF + k;
      const T il = CURVI ? T(1.0 / met_len<DIM>(g, c, s2)) : ih;
      const T ln = (qnh - qnl) * il, lt = (qth - qtl) * il;
      if constexpr (!CURVI) {
        gn[ax] += ln;
        gt[ax] += lt;
      }
      const long idx = ((long)(DIM + s2) * NV + v) * N + c;
      if (stage == 1) {
        der_out[idx] = ln + hdt * lt;
        stash_der[idx] = ln;
      } else {
        der_out[idx] = stash_der[idx] + tdt * lt;
      }
    }
    const double w = CURVI ? 1.0 : g.ih[ax] * (1.0 / GPF);
    L += w * (to_f64(sl_f) - to_f64(sh_f));
    Lt += w * (to_f64(stl_f) - to_f64(sth_f));
  }
  if constexpr (CURVI) {
    const double iv = 1.0 / met_vol<DIM>(g, c);
    L *= iv;
    Lt *= iv;
  }
  /* cell averages accumulate in FP64 across the S2O4 stages */
  const long iavg = (long)v * N + c;
  const double Ld = L, Ltd = Lt;
  double out;
  if (stage == 1) {
    const double q = avg_in[iavg];
    out = q + kc.h1 * Ld + kc.e1 * Ltd;
    stash_avg[iavg] = q + dt * Ld + kc.s1 * Ltd;
  } else {
    out = stash_avg[iavg] + kc.t2 * Ltd;
  }
  avg_out[iavg] = out;
  if constexpr (sizeof(T) == 4) {
    const float h = float(out);
    avh_out[iavg] = h;
    avl_out[iavg] = float(out - fp_f2d_exact(h));
  }
  /* gradient: Gauss' theorem (Eq. derivative); on an axis-aligned cell the
     mean of the line derivatives */
#pragma unroll
  for (int kk = 0; kk < DIM; ++kk) {
    const T dn = CURVI ? gn[kk] * ivol : gn[kk] * T(1.0 / GPF);
    const T dtv = CURVI ? gt[kk] * ivol : gt[kk] * T(1.0 / GPF);
    const long idx = ((long)kk * NV + v) * N + c;
    if (stage == 1) {
      der_out[idx] = dn + hdt * dtv;
      stash_der[idx] = dn;
    } else {
      der_out[idx] = stash_der[idx] + tdt * dtv;
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
  const double rho = W[0], irho = 1.0 / rho;
  double ke = 0.0, Uv[3];
  for (int i = 0; i < DIM; ++i) {
    Uv[i] = W[1 + i] * irho;
    ke += Uv[i] * W[1 + i];
  }
  const double p = (ph.gamma - 1.0) * (W[DIM + 1] - 0.5 * ke);
  const double snd = sqrt(ph.gamma * p * irho);
  double rate = 0.0, hmin = 1e300;
  if (!g.curvi) {
    for (int ax = 0; ax < DIM; ++ax) {
      rate += (fabs(Uv[ax]) + snd) * g.ih[ax];
      hmin = g.h[ax] < hmin ? g.h[ax] : hmin;
    }
  } else {
    const double vol = met_vol<DIM>(g, c);
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
      const double h = vol / (0.5 * (sqrt(s0) + sqrt(s1)));
      double un = 0.0;
      for (int a = 0; a < DIM; ++a) un += Uv[a] * nn[a] / sqrt(ns);
      rate += (fabs(un) + snd) / h;
      if (h < hmin) hmin = h;
    }
  }
  if (ph.mu > 0.0) {
    const double rv = 3.0 * ph.mu * irho / (hmin * hmin);
    if (rv > rate) rate = rv;
  }
  if (!(rho > 0.0) || !(p > 0.0) || !(rate == rate)) rate = 1e300; /* flags a bad state */
  return rate;
}

/* Bounds on the FP64 rate of cell_rate from the FP32 averages W: the FP32
   rate r with its relative error bound eta.  The inputs carry a relative
   error of at most 2^-24 (one rounding from FP64) and about 20 further
   roundings follow; the pressure, a difference, amplifies those by up to
   E/(E - ke/2).  eta = 64 u (2 + E/(E - ke/2)) covers the whole with a wide
   margin.  Where FP32 cannot decide (a non-positive or non-finite value, or
   eta >= 1/4) the bounds are [0, inf): the cell is always evaluated in FP64
   and never raises the threshold. */
template <int DIM>
__device__ __forceinline__ void cell_rate_bounds_f32(const DevGeo& g, const Phys& ph, const float* W, long c,
                                                     float* lo, float* hi) {
  const float rho = W[0], irho = 1.0f / rho;
  float ke = 0.0f, Uv[3];
#pragma unroll
  for (int i = 0; i < DIM; ++i) {
    Uv[i] = W[1 + i] * irho;
    ke = fmaf(Uv[i], W[1 + i], ke);
  }
  const float pe = W[DIM + 1] - 0.5f * ke;
  const float p = (ph.gammaf - 1.0f) * pe;
  const float snd = sqrtf(ph.gammaf * p * irho);
  float rate = 0.0f, hmin;
  if (!g.curvi) {
    hmin = g.hf[0];
#pragma unroll
    for (int ax = 0; ax < DIM; ++ax) {
      rate = fmaf(fabsf(Uv[ax]) + snd, g.ihf[ax], rate);
      hmin = fminf(hmin, g.hf[ax]);
    }
  } else {
    const long N = g.ncell;
#pragma unroll
    for (int ax = 0; ax < DIM; ++ax) {
      float un = 0.0f;
#pragma unroll
      for (int a = 0; a < DIM; ++a) un = fmaf(Uv[a], g.rmet[(RateMet<DIM>::W + ax * DIM + a) * N + c], un);
      rate += fabsf(un);
      rate = fmaf(snd, g.rmet[(RateMet<DIM>::IH + ax) * N + c], rate);
    }
    hmin = g.rmet[RateMet<DIM>::HMIN * N + c];
  }
  if (ph.muf > 0.0f) rate = fmaxf(rate, 3.0f * ph.muf * irho / (hmin * hmin));
  const float eta = 64.0f * 5.9604645e-8f * (2.0f + W[DIM + 1] / pe);
  if (!(rho > 0.0f) || !(p > 0.0f) || !(rate <= 1.0e37f) || !(eta < 0.25f)) {
    *lo = 0.0f;
    *hi = __int_as_float(0x7f800000);
    return;
  }
  *lo = rate * (1.0f - eta);
  *hi = rate * (1.0f + eta);
}

}  // namespace cgks
