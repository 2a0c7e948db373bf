// Host build of the library's device routines, for CPU tests.
//
// The CUDA kernels of paper_2508_08965_gb300/csrc/cgks_kernels.cuh are
// compiled here as plain C++ and run one work item at a time (blockDim = 1,
// one "block" per item), with host stand-ins for the few CUDA intrinsics
// they use: exact IEEE single operations for the __f*_rn intrinsics,
// sequential atomics, and warp votes that see the calling lane only.  This
// checks the arithmetic of the kernels against the oracle without a GPU; it
// says nothing about their parallel execution, which the GPU tests cover.
// Built with -ffp-contract=off so that no multiply-add is fused behind the
// source's back.
#define CGKS_HD inline
#define CGKS_TABLE static const
#define CGKS_GTABLE static const
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

struct HostDim {
  unsigned x, y, z;
};
static HostDim blockIdx, blockDim, threadIdx, gridDim;
#define __global__ inline
#define __shared__
#define __launch_bounds__(...)
#define __noinline__
#define __host__
#ifndef __device__
#define __device__
#endif
#define __forceinline__ inline
#define __grid_constant__
static inline long long __double_as_longlong(double d) { long long r; memcpy(&r, &d, 8); return r; }
static inline double __longlong_as_double(long long d) { double r; memcpy(&r, &d, 8); return r; }
static inline unsigned __float_as_uint(float f) { unsigned r; memcpy(&r, &f, 4); return r; }
static inline float __uint_as_float(unsigned u) { float r; memcpy(&r, &u, 4); return r; }
static inline float __int_as_float(int u) { float r; memcpy(&r, &u, 4); return r; }
static inline unsigned long long atomicMax(unsigned long long* p, unsigned long long v) { auto o = *p; if (v > o) *p = v; return o; }
static inline unsigned atomicMax(unsigned* p, unsigned v) { auto o = *p; if (v > o) *p = v; return o; }
static inline int atomicAdd(int* p, int v) { int o = *p; *p += v; return o; }
static inline unsigned long long atomicAdd(unsigned long long* p, unsigned long long v) { auto o = *p; *p += v; return o; }
template <typename U> static inline U atomicAdd(U* p, U v) { U o = *p; *p += v; return o; }
static inline int atomicOr(int* p, int v) { int o = *p; *p |= v; return o; }
static inline void __syncthreads() {}
static inline int __syncthreads_or(int p) { return p; }
static inline void __syncwarp(unsigned = 0xffffffffu) {}
static inline unsigned __ballot_sync(unsigned, int p) { return p ? 1u : 0u; }
static inline bool __any_sync(unsigned, bool p) { return p; }
template <typename U> static inline U __shfl_xor_sync(unsigned, U v, int) { return v; }
static inline int __popc(unsigned x) { return __builtin_popcount(x); }
template <typename U> static inline U __ldg(const U* p) { return *p; }
static inline float __fadd_rn(float a, float b) { return a + b; }
static inline float __fsub_rn(float a, float b) { return a - b; }
static inline float __fmul_rn(float a, float b) { return a * b; }
static inline float __fdiv_rn(float a, float b) { return a / b; }
static inline float __fsqrt_rn(float a) { return sqrtf(a); }
static inline float __frcp_rn(float a) { return 1.0f / a; }
#include "../paper_2508_08965_gb300/csrc/cgks_kernels.cuh"
using namespace cgks;

namespace {

int g_bc[6] = {0, 0, 0, 0, 0, 0};
double g_bcq[BCQ_DOUBLES] = {0};

template <typename T, int DIM, bool CV, typename C = T>
int run_stage(DevGeo& g, Phys& ph, double dt, int stage, double** avg, T** der, double* savg, T* sder,
              std::vector<T>& gpL, std::vector<T>& gpR, std::vector<T>& flux, float** avh, float** avl,
              std::vector<T>& fxb) {
  const long N = g.ncell;
  const int in = stage == 1 ? 0 : 1, out = stage == 1 ? 1 : 0;
  int st[ST_N] = {0};
  std::vector<double> chi((size_t)Sz<DIM>::NV * N);
  DtState dts{};
  set_dt(dts, dt);
  blockDim.x = 1;
  threadIdx.x = 0;
  for (long t = 0; t < N; ++t) {
    blockIdx.x = (unsigned)t;
    /* the paired form (C = fpair) also reconstructs with the paired
       Gauss-point transform on Cartesian meshes, as the library does */
    k_recon<T, DIM, CV, true, !CV && cg_same<C, fpair>::value>(avg[in], avh[in], avl[in], der[in], g, ph, gpL.data(),
                                                                 gpR.data(), chi.data(), 0, st, SelectorDev{});
  }
  for (long t = 0; t < (long)DIM * Sz<DIM>::GPF * N; ++t) {
    blockIdx.x = (unsigned)t;
    k_flux<T, DIM, CV, C>(g, ph, &dts, gpL.data(), gpR.data(), flux.data(), st, CUtensorMap{}, CUtensorMap{});
  }
  for (long t = 0; t < 2L * DIM * Sz<DIM>::GPF * g.nplane; ++t) {
    blockIdx.x = (unsigned)t;
    k_flux_bnd<T, DIM, CV>(g, ph, &dts, gpL.data(), gpR.data(), flux.data(), fxb.data(), st);
  }
  for (long t = 0; t < (long)Sz<DIM>::NV * N; ++t) {
    blockIdx.x = (unsigned)t;
    k_update<T, DIM, CV>(g, &dts, stage, avg[in], flux.data(), fxb.data(), savg, sder, avg[out], der[out], avh[out],
                         avl[out]);
  }
  return (st[ST_FLUX] || st[ST_NONPHYS]) ? 1 : 0;
}

template <int DIM>
void geometry(DevGeo& g, const int* n, const double* lo, const double* hi) {
  for (int a = 0; a < 3; ++a) {
    g.n[a] = a < DIM ? n[a] : 1;
    g.h[a] = a < DIM ? (hi[a] - lo[a]) / n[a] : 1.0;
    g.ih[a] = 1.0 / g.h[a];
    g.hf[a] = (float)g.h[a];
    g.ihf[a] = (float)g.ih[a];
  }
  g.ncell = (long)g.n[0] * g.n[1] * g.n[2];
  g.curvi = 0;
  g.met = nullptr;
  g.bcq = g_bcq;
  g.bcm = 0;
  g.nplane = 0;
  for (int f = 0; f < 2 * DIM; ++f) {
    g.bcm |= g_bc[f] << (3 * f);
    if (g_bc[f]) g.nplane = std::max(g.nplane, g.ncell / g.n[f / 2]);
  }
}

template <typename T, int DIM, typename C = T>
int run(const int* n, const double* lo, const double* hi, const double* nodes, const double* phys, double* U,
        int nsteps, double* dt_out) {
  DevGeo g{};
  geometry<DIM>(g, n, lo, hi);
  std::vector<double> met;
  if (nodes) {
    met.resize((size_t)Met<DIM>::N * g.ncell);
    for (long c = 0; c < g.ncell; ++c) metrics_cell<DIM>(nodes, g, c, met.data());
    g.curvi = 1;
    g.met = met.data();
  }
  /* phys: gamma, mu, prandtl, cfl, c_chi, tau_mode, linear, dt_fixed */
  const double gamma = phys[0], mu = phys[1], pr = phys[2], cfl = phys[3], cchi = phys[4], dt_fixed = phys[7];
  Phys ph{gamma, mu, pr, cfl, cchi, (int)phys[5], (int)phys[6], (float)gamma, (float)mu, (float)pr, (float)cchi,
          (mu > 0 && pr > 0 && pr != 1.0) ? 1 : 0};
  const long N = g.ncell;
  const int NV = Sz<DIM>::NV, NF = Sz<DIM>::NF, GPF = Sz<DIM>::GPF;
  const size_t navg = (size_t)NV * N, nder = (size_t)(NF - 1) * NV * N;
  std::vector<double> A0(U, U + navg), A1(navg), SA(navg);
  std::vector<T> D0(nder), D1(nder), SD(nder);
  for (size_t i = 0; i < nder; ++i) D0[i] = T(U[navg + i]);
  std::vector<T> gpL((size_t)DIM * GPF * NV * (1 + DIM) * N), gpR(gpL.size()), fx((size_t)DIM * GPF * 6 * NV * N);
  std::vector<T> fxb((size_t)DIM * GPF * 6 * NV * std::max(g.nplane, 1L));
  double* avg[2] = {A0.data(), A1.data()};
  T* der[2] = {D0.data(), D1.data()};
  std::vector<float> H0(navg), L0(navg), H1(navg), L1(navg);
  for (size_t i = 0; i < navg; ++i) {
    H0[i] = float(A0[i]);
    L0[i] = float(A0[i] - double(H0[i]));
  }
  float* avh[2] = {H0.data(), H1.data()};
  float* avl[2] = {L0.data(), L1.data()};
  for (int s = 0; s < nsteps; ++s) {
    double dt = dt_fixed;
    if (!(dt > 0)) {
      double rmax = 0;
      for (long c = 0; c < N; ++c) rmax = std::max(rmax, cell_rate<DIM>(g, ph, avg[0], c));
      dt = cfl / rmax;
    }
    int bad = 0;
    if (g.curvi) {
      bad |= run_stage<T, DIM, true, C>(g, ph, dt, 1, avg, der, SA.data(), SD.data(), gpL, gpR, fx, avh, avl, fxb);
      bad |= run_stage<T, DIM, true, C>(g, ph, dt, 2, avg, der, SA.data(), SD.data(), gpL, gpR, fx, avh, avl, fxb);
    } else {
      bad |= run_stage<T, DIM, false, C>(g, ph, dt, 1, avg, der, SA.data(), SD.data(), gpL, gpR, fx, avh, avl, fxb);
      bad |= run_stage<T, DIM, false, C>(g, ph, dt, 2, avg, der, SA.data(), SD.data(), gpL, gpR, fx, avh, avl, fxb);
    }
    if (bad) return -4;
    *dt_out = dt;
  }
  for (size_t i = 0; i < navg; ++i) U[i] = A0[i];
  for (size_t i = 0; i < nder; ++i) U[navg + i] = double(D0[i]);
  return 0;
}

template <int DIM>
void features(const int* n, const double* lo, const double* hi, const double* U, int prec, float* out) {
  DevGeo g{};
  geometry<DIM>(g, n, lo, hi);
  const long N = g.ncell;
  const int NV = DIM + 2, NF = Sz<DIM>::NF;
  std::vector<float> hf((size_t)NV * N), df((size_t)(NF - 1) * NV * N);
  for (size_t i = 0; i < hf.size(); ++i) hf[i] = (float)U[i];
  for (size_t i = 0; i < df.size(); ++i) df[i] = (float)U[(size_t)NV * N + i];
  for (long c = 0; c < N; ++c) {
    int i, j, k;
    cell_ijk(g, c, i, j, k);
    if (prec) selector_features<DIM, true>(hf.data(), df.data(), g, c, i, j, k, out + c * SEL_NF);
    else selector_features<DIM, true>(U, U + (size_t)NV * N, g, c, i, j, k, out + c * SEL_NF);
  }
}

}  // namespace

extern "C" {
/* boundary kinds per face and the inflow states [face][5] of the next runs */
void host_set_bc(const int* bc, const double* states) {
  double st[6][5];
  for (int f = 0; f < 6; ++f) {
    g_bc[f] = bc[f];
    for (int v = 0; v < 5; ++v) st[f][v] = states[5 * f + v];
  }
  pack_bcq(st, g_bcq);
}
/* nsteps S2O4 steps of the public-layout state U (in place); precision 0:
   FP64 kernels, 1: the FP32 form, 2: FP64 with the paired-FP32 interface
   flux.  Returns 0, or -4 on a non-physical state */
int host_run(int dim, int precision, const int* n, const double* lo, const double* hi, const double* nodes,
             const double* phys, double* U, int nsteps, double* dt_out) {
  if (dim == 3) {
    if (precision == 1) return run<float, 3>(n, lo, hi, nodes, phys, U, nsteps, dt_out);
    if (precision == 2) return run<double, 3, fpair>(n, lo, hi, nodes, phys, U, nsteps, dt_out);
    return run<double, 3>(n, lo, hi, nodes, phys, U, nsteps, dt_out);
  }
  if (precision == 1) return run<float, 2>(n, lo, hi, nodes, phys, U, nsteps, dt_out);
  if (precision == 2) return run<double, 2, fpair>(n, lo, hi, nodes, phys, U, nsteps, dt_out);
  return run<double, 2>(n, lo, hi, nodes, phys, U, nsteps, dt_out);
}
/* the face Gauss-point transforms of the generated code: for random
   coefficients, the largest relative difference between axis ax's own
   transform and the axis-0 transform of the relabelled coefficients
   (gen_perm), with the derivative j of the latter read as the physical
   derivative pi(j) */
double host_gp_perm_check(int dim, unsigned seed) {
  unsigned long long x = 0x9e3779b97f4a7c15ull ^ seed;
  auto rnd = [&]() {
    x ^= x << 13;
    x ^= x >> 7;
    x ^= x << 17;
    return (double)(x >> 11) * (2.0 / 9007199254740992.0) - 1.0;
  };
  double worst = 0.0;
  for (int it = 0; it < 200; ++it) {
    double a[34], o[34], v0[8], g0[8][3], v1[8], g1[8][3];
    const int nb = dim == 3 ? 34 : 14, np = dim == 3 ? 8 : 4;
    for (int b = 0; b < nb; ++b) a[b] = rnd();
    for (int ax = 0; ax < dim; ++ax) {
      if (dim == 3) {
        if (ax == 0) gen_gp_3d_ax0<double>(a, v0, g0);
        else if (ax == 1) gen_gp_3d_ax1<double>(a, v0, g0);
        else gen_gp_3d_ax2<double>(a, v0, g0);
        gen_perm_3d<double>(a, ax, o);
        gen_gp_3d_ax0<double>(o, v1, g1);
      } else {
        double g02[4][2], g12[4][2];
        if (ax == 0) gen_gp_2d_ax0<double>(a, v0, g02);
        else gen_gp_2d_ax1<double>(a, v0, g02);
        gen_perm_2d<double>(a, ax, o);
        gen_gp_2d_ax0<double>(o, v1, g12);
        for (int i = 0; i < np; ++i)
          for (int k = 0; k < 2; ++k) {
            g0[i][k] = g02[i][k];
            g1[i][k] = g12[i][k];
          }
      }
      int pi[3] = {ax, 0, 0};
      for (int j = 1, q = 0; q < dim; ++q)
        if (q != ax) pi[j++] = q;
      double scale = 0.0;
      for (int i = 0; i < np; ++i) scale = std::max(scale, std::fabs(v0[i]));
      for (int i = 0; i < np; ++i) {
        worst = std::max(worst, std::fabs(v1[i] - v0[i]) / scale);
        for (int j = 0; j < dim; ++j) worst = std::max(worst, std::fabs(g1[i][j] - g0[i][pi[j]]) / scale);
      }
    }
  }
  return worst;
}
/* the learned selector's 16 features of every cell (uniform boxes) */
void host_features(int dim, const int* n, const double* lo, const double* hi, const double* U, int precision,
                   float* out) {
  if (dim == 3) features<3>(n, lo, hi, U, precision, out);
  else features<2>(n, lo, hi, U, precision, out);
}
}
