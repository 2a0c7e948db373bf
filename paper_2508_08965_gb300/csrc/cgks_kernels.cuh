/*
 * Kernels of the CGKS-5 library: thin thread mappings onto the routines of
 * cgks_device.cuh, plus the metric precompute (Sec. 4 and Appendix), the
 * initial-data kernels and the time-step reduction.
 */
#pragma once
#include <cuda.h> /* CUtensorMap (a type only: maps are encoded through the runtime's driver entry point) */

#include "cgks_device.cuh"
#include "cgks_selector.cuh"

namespace cgks {

/* device status words: [0] non-physical state that chi = 0 cannot cure,
   [1] positivity fallbacks, [2] non-physical interface state,
   [3] non-physical cell in the time-step reduction */
enum { ST_NONPHYS = 0, ST_FALLBACK = 1, ST_FLUX = 2, ST_DT = 3, ST_N = 4 };

/* time-step bookkeeping on the device: [0] rate bits (max), [1] dt, [2] t, [3] t_end */
struct DtState {
  unsigned long long rate_bits; /* FP64 maximum rate (bit pattern; orders like the value) */
  unsigned int lo_bits;         /* FP32 screening: largest lower bound of a cell's rate */
  unsigned int pad;
  double dt, t, t_end, dt_fixed;
  StageCoef k; /* stage_coef(dt), set with dt */
  /* within one cgks_step call: the steps whose output is not known to be
     non-physical, and the time before the last of them (the time to go
     back to when the next step's time step finds that output non-physical) */
  double t_prev;
  int nok, pad2;
};
/* a stage or time-step kernel has flagged a non-physical state */
CGKS_HD bool st_failed(const int* st) { return st[ST_NONPHYS] || st[ST_FLUX] || st[ST_DT]; }
CGKS_HD void set_dt(DtState& d, double dt) {
  d.dt = dt;
  d.k = stage_coef(dt);
}

/* Blocks of 128 threads per SM: FP32 3-D kernels fit 3 (168 registers), FP32
   2-D ones 4 (128 registers; the 2-D reconstruction is latency-bound and
   gains from the extra warps); the FP64 ones keep 2 (they are bound by the
   FP64 pipe, and spill more when capped) */
template <typename T, int DIM = 3> constexpr int min_blocks() { return sizeof(T) == 4 ? (DIM == 2 ? 4 : 3) : 2; }
/* the Cartesian kernels: FP32 fits 4 blocks in 3-D as well (128 registers:
   the flux spills 8 B since its Maxwellian moments are factorised, the
   reconstruction none since its Gauss-point transform runs one relabelled
   copy for all axes; 5 blocks spill and run slower: reconstruction 1.57 ->
   1.65 ms, flux 2.59 -> 3.29 ms at TGV 128^3) and the 2-D flux 5 (96
   registers, no spill); the curvilinear ones, which spill more, keep 3.
   PR: the paired form's 3-D reconstruction runs 3 (168 registers; its
   812 B of spills cost less than the latency the extra warps hide: TGV
   128^3 20.1 -> 19.4 ms per stage; 4 blocks spill 2.2 KB: 20.1 ms) */
template <typename T, int DIM, bool CURVI, bool PR = false> constexpr int recon_min_blocks() {
  return PR && DIM == 3 ? 3 : (sizeof(T) == 4 && DIM == 3 && !CURVI ? 4 : min_blocks<T, DIM>());
}
template <typename T, int DIM, bool CURVI> constexpr int flux_min_blocks() {
  return sizeof(T) == 4 && !CURVI ? (DIM == 2 ? 5 : 4) : min_blocks<T, DIM>();
}

/* first order: every face Gauss-point state of cell c is its cell average
   with zero gradient (stored where recon_var stores them) */
template <typename T, int DIM>
__device__ __noinline__ void first_order_states(const double* __restrict__ avg, const float* __restrict__ avh,
                                                const float* __restrict__ avl, const DevGeo& g, long c, int i, int j,
                                                int k, T* __restrict__ gpL, T* __restrict__ gpR) {
  typedef Sz<DIM> S;
  const long N = g.ncell;
  for (int v = 0; v < S::NV; ++v) {
    T q;
    if constexpr (sizeof(T) == 4) q = avh[(long)v * N + c] + avl[(long)v * N + c];
    else q = T(avg[(long)v * N + c]);
    for (int ax = 0; ax < DIM; ++ax) {
      int o[3] = {0, 0, 0};
      o[ax] = -1;
      const long clo = nbr(g, i, j, k, o[0], o[1], o[2]);
      for (int side = 0; side < 2; ++side)
        for (int kq = 0; kq < S::GPF; ++kq) {
          T* dst = side ? gpL : gpR;
          const long b = ((long)((ax * S::GPF + kq) * S::NV + v) * (1 + DIM)) * N + (side ? c : clo);
          dst[b] = q;
          for (int kk = 0; kk < DIM; ++kk) dst[b + (long)(1 + kk) * N] = T(0);
        }
    }
  }
}

/* reconstruction of all variables of cell c = (i, j, k), with the
   positivity fallbacks (shared by the single-case and batched kernels):
   chi = 0 if a face Gauss-point state has rho <= 0 or p <= 0, then first
   order if that is not enough either */
/* one variable's reconstruction: PR selects the paired linear maps
   (recon_var_pair; FP64 storage, Cartesian meshes) */
template <typename T, int DIM, bool CURVI, bool WALL, bool PR>
__device__ __forceinline__ T recon_var_any(const double* __restrict__ avg, const float* __restrict__ avh,
                                           const float* __restrict__ avl, const T* __restrict__ der,
                                           const DevGeo& g, const Phys& ph, long c, int i, int j, int k, int v,
                                           T force, T* __restrict__ gpL, T* __restrict__ gpR) {
  if constexpr (PR && !CURVI && sizeof(T) == 8)
    return recon_var_pair<DIM, WALL>(avg, der, g, ph, c, i, j, k, v, force, gpL, gpR);
  else
    return recon_var<T, DIM, CURVI, WALL>(avg, avh, avl, der, g, ph, c, i, j, k, v, force, gpL, gpR);
}

template <typename T, int DIM, bool CURVI, bool WALL, bool PR = false>
__device__ __forceinline__ void recon_cell(const double* __restrict__ avg, const float* __restrict__ avh,
                                           const float* __restrict__ avl, const T* __restrict__ der, const DevGeo& g,
                                           const Phys& ph, long c, int i, int j, int k, T* __restrict__ gpL,
                                           T* __restrict__ gpR, double* __restrict__ chi, int record_chi,
                                           int* __restrict__ st, bool skip = false) {
  const int NV = Sz<DIM>::NV;
  /* skip: the learned selector passed this cell (chi = 1, no adaptive weights) */
  const T force = (ph.linear || skip) ? T(1) : T(-1);
  T cs[NV];
#pragma unroll 1
  for (int v = 0; v < NV; ++v)
    cs[v] = recon_var_any<T, DIM, CURVI, WALL, PR>(avg, avh, avl, der, g, ph, c, i, j, k, v, force, gpL, gpR);
  if (!cell_states_physical<T, DIM>(g, ph, c, i, j, k, gpL, gpR)) {
    atomicAdd(&st[ST_FALLBACK], 1);
#pragma unroll 1
    for (int v = 0; v < NV; ++v)
      cs[v] = recon_var_any<T, DIM, CURVI, WALL, PR>(avg, avh, avl, der, g, ph, c, i, j, k, v, T(0), gpL, gpR);
    if (!cell_states_physical<T, DIM>(g, ph, c, i, j, k, gpL, gpR)) {
      first_order_states<T, DIM>(avg, avh, avl, g, c, i, j, k, gpL, gpR);
      if (!cell_states_physical<T, DIM>(g, ph, c, i, j, k, gpL, gpR)) atomicOr(&st[ST_NONPHYS], 1);
    }
  }
  if (record_chi)
    for (int v = 0; v < NV; ++v) chi[(long)v * g.ncell + c] = double(cs[v]);
}

/* whether the calling warp reconstructs with the boundary selects of the
   WALL path (warp-collective).  2-D: only warps with a cell next to a wall or
   inflow face do (the selects cost the latency-bound FP32 form about 40%;
   measured 0.33 -> 0.24 ms on a 1024^2 shock-vortex mesh).  3-D: every warp
   of a WALL mesh: warps run along x, so at 128 cells per row half of them
   touch an x-wall, and a second inlined copy of the 3-D reconstruction cost
   more than it saved (2.67 -> 3.44 ms at 128^3). */
template <bool WALL, int DIM>
__device__ __forceinline__ bool wall_warp(const DevGeo& g, bool active, int i, int j, int k) {
  if constexpr (WALL && DIM == 2) return __any_sync(0xffffffffu, active && touches_wall<DIM>(g, i, j, k));
  else return WALL;
}

/* the selector's decision for the calling lane's cell (warp-collective: all
   lanes call it, inactive ones with active = false); blocks of 128 threads.
   wall: the warp has a cell next to a wall or inflow face (warp-uniform) */
template <typename T, int DIM, bool WALL>
__device__ __forceinline__ bool selector_skip(const SelectorDev& sel, const double* __restrict__ avg,
                                              const float* __restrict__ avh, const T* __restrict__ der,
                                              const DevGeo& g, long c, int i, int j, int k, bool active,
                                              bool wall = WALL) {
  __shared__ uint32_t stage[4][32 * SEL_PITCH];
  float f[SEL_NF];
  if (active) {
    if (WALL && wall) {
      if constexpr (sizeof(T) == 4) selector_features<DIM, WALL>(avh, der, g, c, i, j, k, f);
      else selector_features<DIM, WALL>(avg, der, g, c, i, j, k, f);
    } else {
      if constexpr (sizeof(T) == 4) selector_features<DIM, false>(avh, der, g, c, i, j, k, f);
      else selector_features<DIM, false>(avg, der, g, c, i, j, k, f);
    }
  } else {
#pragma unroll
    for (int q = 0; q < SEL_NF; ++q) f[q] = 0.f;
  }
  return selector_decide(sel, f, active, stage[threadIdx.x >> 5]) == SEL_SKIP;
}

template <typename T, int DIM, bool CURVI, bool WALL, bool PR = false>
__global__ void __launch_bounds__(128, recon_min_blocks<T, DIM, CURVI, PR>())
    k_recon(const double* __restrict__ avg, const float* __restrict__ avh, const float* __restrict__ avl,
            const T* __restrict__ der, DevGeo g, Phys ph, T* __restrict__ gpL, T* __restrict__ gpR,
            double* __restrict__ chi, int record_chi, int* __restrict__ st, SelectorDev sel) {
  long c = blockIdx.x * (long)blockDim.x + threadIdx.x;
  const bool active = c < g.ncell;
  int i = 0, j = 0, k = 0;
  if (active) cell_ijk(g, c, i, j, k);
  const bool wall = wall_warp<WALL, DIM>(g, active, i, j, k);
  bool skip = false;
  if (sel.on && !ph.linear) skip = selector_skip<T, DIM, WALL>(sel, avg, avh, der, g, c, i, j, k, active, wall);
  if (!active) return;
  if (wall) recon_cell<T, DIM, CURVI, WALL, PR>(avg, avh, avl, der, g, ph, c, i, j, k, gpL, gpR, chi, record_chi, st, skip);
  else recon_cell<T, DIM, CURVI, false, PR>(avg, avh, avl, der, g, ph, c, i, j, k, gpL, gpR, chi, record_chi, st, skip);
}

/* features of every cell of a state, [cell][SEL_NF] (training samples) */
template <typename T, int DIM, bool WALL>
__global__ void k_selector_features(const double* __restrict__ avg, const float* __restrict__ avh,
                                    const T* __restrict__ der, DevGeo g, float* __restrict__ out) {
  long c = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (c >= g.ncell) return;
  int i, j, k;
  cell_ijk(g, c, i, j, k);
  float f[SEL_NF];
  if constexpr (sizeof(T) == 4) selector_features<DIM, WALL>(avh, der, g, c, i, j, k, f);
  else selector_features<DIM, WALL>(avg, der, g, c, i, j, k, f);
#pragma unroll
  for (int q = 0; q < SEL_NF; ++q) out[c * SEL_NF + q] = f[q];
}

/* face-point item t = (ax * GPF + k) * N + c of a mesh: the face slot above
   cell c along ax at Gauss point k; slots on a non-periodic high boundary are
   left to the boundary items */
template <typename T, int DIM, bool CURVI, typename C = T>
__device__ __forceinline__ void flux_item(const DevGeo& g, const Phys& ph, double dt, long t, const T* __restrict__ gpL,
                                          const T* __restrict__ gpR, T* __restrict__ flux, int* __restrict__ st,
                                          T* sm = nullptr, int ns = 0, bool staged = false) {
  const long N = g.ncell;
  const long c = t % N;
  const int r = (int)(t / N);
  const int k = r % Sz<DIM>::GPF, ax = r / Sz<DIM>::GPF;
  if (geo_bc(g, 2 * ax + 1) != BC_PERIODIC) {
    int ijk[3];
    cell_ijk(g, c, ijk[0], ijk[1], ijk[2]);
    if (ijk[ax] == g.n[ax] - 1) return;
  }
  if (!flux_point<T, DIM, CURVI, C>(g, ph, T(dt), ax, k, c, gpL, gpR, flux, sm, ns, staged))
    atomicOr(&st[ST_FLUX], 1);
}

/* ---- TMA tiles ----------------------------------------------------------
   The Gauss-point states of the 128 face points of a flux block are, per
   stored quantity q, 128 consecutive values of one row of gpL (and of gpR)
   viewed as a 2-D array [row][cell] (row = (ax * GPF + k) * NQ + q): one
   box of NQ rows x 128 cells each.  One thread loads both boxes with the
   tensor memory accelerator (cp.async.bulk.tensor) into the block's
   staging tile, and the block waits for them on a shared-memory barrier.
   Requires a Cartesian
   mesh whose cell count is a multiple of 128 (a block's points then share
   (ax, k), its first cell is 16-byte aligned in every row, and the row
   pitch is a multiple of 16 bytes); other meshes stage by cp.async. */
__device__ __forceinline__ void tma_bar_init(uint64_t* bar) {
#if defined(__CUDA_ARCH__)
  const unsigned a = (unsigned)__cvta_generic_to_shared(bar);
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(a) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
#endif
}
__device__ __forceinline__ void tma_expect(uint64_t* bar, unsigned bytes) {
#if defined(__CUDA_ARCH__)
  const unsigned a = (unsigned)__cvta_generic_to_shared(bar);
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(a), "r"(bytes) : "memory");
#endif
}
/* box at (x = first cell, y = first row) of the tensor map into dst */
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
#if defined(__CUDA_ARCH__)
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  const unsigned b = (unsigned)__cvta_generic_to_shared(bar);
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n" ::"r"(d),
      "l"((unsigned long long)map), "r"(x), "r"(y), "r"(b)
      : "memory");
#endif
}
/* wait for phase 0 of the barrier; false if it has not completed within
   about a second (the caller then reports CGKS_ETIMEOUT) */
__device__ __forceinline__ bool tma_wait(uint64_t* bar) {
#if defined(__CUDA_ARCH__)
  const unsigned a = (unsigned)__cvta_generic_to_shared(bar);
  const long long t0 = clock64();
  while (true) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], 0;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > 2000000000LL) return false;
  }
#else
  return true;
#endif
}

/* boundary face-point item t = ((side * DIM + ax) * GPF + k) * nplane + plane.
   In a plane normal to ax, c0 is the cell on the low boundary and c1 the one
   on the high boundary; slot c1 holds both c1's high-face state (gpL) and
   c0's low-face state (gpR).  The high face goes to flux at slot c1, the low
   face to fxb. */
template <typename T, int DIM, bool CURVI>
__device__ __forceinline__ void flux_bnd_item(const DevGeo& g, const Phys& ph, double dt, long t,
                                              const T* __restrict__ gpL, const T* __restrict__ gpR,
                                              T* __restrict__ flux, T* __restrict__ fxb, int* __restrict__ st) {
  const long pidx = t % g.nplane;
  int r = (int)(t / g.nplane);
  const int k = r % Sz<DIM>::GPF;
  r /= Sz<DIM>::GPF;
  const int ax = r % DIM, side = r / DIM; /* side 1: high boundary */
  const int bc = geo_bc(g, 2 * ax + side);
  const long N = g.ncell;
  if (bc == BC_PERIODIC || pidx >= N / g.n[ax]) return;
  int ijk[3] = {0, 0, 0};
  const int a0 = ax == 0 ? 1 : 0, a1 = ax == 2 ? 1 : 2;
  ijk[a0] = (int)(pidx % g.n[a0]);
  ijk[a1] = (int)(pidx / g.n[a0]);
  const long c0 = cell_index(g, ijk[0], ijk[1], ijk[2]);
  ijk[ax] = g.n[ax] - 1;
  const long c1 = cell_index(g, ijk[0], ijk[1], ijk[2]);
  bool ok;
  if (side)
    ok = flux_bnd_point<T, DIM, CURVI>(g, ph, T(dt), ax, k, c1, c1, (2 * ax + 1) * Sz<DIM>::GPF + k, 0, bc, gpL,
                                       gpR, flux, N, c1);
  else
    ok = flux_bnd_point<T, DIM, CURVI>(g, ph, T(dt), ax, k, c1, c0, (2 * ax) * Sz<DIM>::GPF + k, 1, bc, gpL, gpR,
                                       fxb, g.nplane, pidx);
  if (!ok) atomicOr(&st[ST_FLUX], 1);
}

/* one thread per face slot and Gauss point (blocks of 128); the Cartesian
   path stages each point's Gauss-point states in shared memory.  C: the
   solve's compute type (fpair: the paired form, FP64 storage, Cartesian or
   curvilinear with the face-frame rotation in FP64) */
template <typename T, int DIM, bool CURVI, typename C = T, bool TMA = false>
__global__ void __launch_bounds__(128, flux_min_blocks<T, DIM, CURVI>()) k_flux(DevGeo g, Phys ph, const DtState* __restrict__ dts,
                                              const T* __restrict__ gpL, const T* __restrict__ gpR,
                                              T* __restrict__ flux, int* __restrict__ st,
                                              const __grid_constant__ CUtensorMap tmL,
                                              const __grid_constant__ CUtensorMap tmR) {
  long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
  const long N = g.ncell;
  if (t >= (long)DIM * Sz<DIM>::GPF * N) return;
  const double dt = dts->dt;
  if (!(dt > 0.0)) return;
  if constexpr (!CURVI) {
    constexpr int NQ = Sz<DIM>::NV * (1 + DIM);
    __shared__ __align__(128) T stage[2 * NQ * 128];
    if constexpr (TMA) { /* every thread of the block is here: 128 | N, 128 | the point count */
      __shared__ __align__(8) uint64_t bar;
      __shared__ int gave_up;
      const long t0 = blockIdx.x * 128L;
      const int r = (int)(t0 / N);
      if (threadIdx.x == 0) {
        /* once a block's wait has given up, later blocks skip theirs, so a
           launch that stalls ends after one wave of waits */
        gave_up = *(volatile int*)&st[ST_FLUX] & 2;
        if (!gave_up) tma_bar_init(&bar);
      }
      __syncthreads();
      if (gave_up) return;
      if (threadIdx.x == 0) {
        tma_expect(&bar, 2u * NQ * 128u * (unsigned)sizeof(T) + (unsigned)ph.stall_tx);
        tma_load_2d(stage, &tmL, (int)(t0 - (long)r * N), r * NQ, &bar);
        tma_load_2d(stage + NQ * 128, &tmR, (int)(t0 - (long)r * N), r * NQ, &bar);
      }
      /* the two copies have landed whether or not the barrier completes
         (only the test hook's extra bytes can hold it back), so a block that
         gives up leaves nothing in flight */
      if (!tma_wait(&bar)) {
        if (threadIdx.x == 0) atomicOr(&st[ST_FLUX], 2);
        return;
      }
      flux_item<T, DIM, CURVI, C>(g, ph, dt, t, gpL, gpR, flux, st, stage + threadIdx.x, 128, true);
    } else {
      flux_item<T, DIM, CURVI, C>(g, ph, dt, t, gpL, gpR, flux, st, stage + threadIdx.x, 128);
    }
  } else {
    flux_item<T, DIM, CURVI, C>(g, ph, dt, t, gpL, gpR, flux, st);
  }
}

/* the faces on the non-periodic domain boundaries (flux_bnd_item) */
template <typename T, int DIM, bool CURVI>
__global__ void __launch_bounds__(128) k_flux_bnd(DevGeo g, Phys ph, const DtState* __restrict__ dts,
                                                  const T* __restrict__ gpL, const T* __restrict__ gpR,
                                                  T* __restrict__ flux, T* __restrict__ fxb, int* __restrict__ st) {
  long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (t >= 2L * DIM * Sz<DIM>::GPF * g.nplane) return;
  const double dt = dts->dt;
  if (!(dt > 0.0)) return;
  flux_bnd_item<T, DIM, CURVI>(g, ph, dt, t, gpL, gpR, flux, fxb, st);
}

/* blocks of 128 per SM for the update, an HBM- and latency-bound kernel:
   as many as fit without spilling (FP32 Cartesian: 64 registers, 16% faster
   than the 72 the compiler picks unbounded) */
template <typename T, int DIM, bool CURVI> constexpr int update_min_blocks() {
  if constexpr (sizeof(T) == 4) return CURVI ? 5 : 8;
  else return CURVI ? (DIM == 3 ? 4 : 6) : (DIM == 3 ? 6 : 10);
}

template <typename T, int DIM, bool CURVI>
__global__ void __launch_bounds__(128, update_min_blocks<T, DIM, CURVI>()) k_update(DevGeo g, const DtState* __restrict__ dts, int stage,
                                                const double* __restrict__ avg_in, const T* __restrict__ flux,
                                                const T* __restrict__ fxb,
                                                double* __restrict__ stash_avg, T* __restrict__ stash_der,
                                                double* __restrict__ avg_out, T* __restrict__ der_out,
                                                float* __restrict__ avh_out, float* __restrict__ avl_out) {
  const long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
  const long N = g.ncell;
  if (t >= (long)Sz<DIM>::NV * N) return;
  const StageCoef kc = dts->k;
  if (!(kc.dt > 0.0)) return;
  const long c = t % N;
  const int v = (int)(t / N);
  int i, j, k;
  cell_ijk(g, c, i, j, k);
  update_var<T, DIM, CURVI>(g, kc, stage, c, i, j, k, v, avg_in, flux, fxb, stash_avg, stash_der, avg_out, der_out,
                            avh_out, avl_out);
}

/* public FP64 layout <-> FP64 averages + derivative fields in T */
template <typename T>
__global__ void k_split(const double* __restrict__ full, double* __restrict__ avg, float* __restrict__ avh,
                        float* __restrict__ avl, T* __restrict__ der, long navg, long nder) {
  long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (t < navg) {
    const double x = full[t];
    avg[t] = x;
    const float h = float(x);
    avh[t] = h;
    avl[t] = float(x - double(h));
  } else if (t < navg + nder) {
    der[t - navg] = T(full[t]);
  }
}
/* the same split restricted to cells [cell0, cell0 + ncells) of every field */
template <typename T>
__global__ void k_split_cells(const double* __restrict__ full, double* __restrict__ avg, float* __restrict__ avh,
                              float* __restrict__ avl, T* __restrict__ der, long N, int nv, int nf, long cell0,
                              long ncells) {
  long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (t >= (long)nf * nv * ncells) return;
  const long cl = t % ncells, fv = t / ncells;
  const long idx = fv * N + cell0 + cl;
  const long navg = (long)nv * N;
  if (idx < navg) {
    const double x = full[idx];
    avg[idx] = x;
    const float h = float(x);
    avh[idx] = h;
    avl[idx] = float(x - double(h));
  } else {
    der[idx - navg] = T(full[idx]);
  }
}
template <typename T>
__global__ void k_join(const double* __restrict__ avg, const T* __restrict__ der, double* __restrict__ full, long navg,
                       long nder) {
  long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (t < navg) full[t] = avg[t];
  else if (t < navg + nder) full[t] = double(der[t - navg]);
}

/* max over cells of the rate; positive doubles order like their bit patterns */
/* The CFL maximum in two passes.  Bounds on every cell's rate from FP32
   arithmetic (cell_rate_bounds_f32) cost a few FP32 operations; pass 1 takes
   the largest lower bound over the mesh, and pass 2 evaluates the FP64 rate
   only where the upper bound reaches it -- the cells that can hold the FP64
   maximum -- so dt equals the FP64 maximum exactly while the FP64 pipe sees a
   handful of cells.  S: the averages the FP32 bounds read (the FP64 averages,
   converted, or the FP32 form's rounded hi parts). */
template <int DIM, typename S>
__device__ __forceinline__ void rate_bounds(const DevGeo& g, const Phys& ph, const S* __restrict__ src, long c,
                                            float* lo, float* hi) {
  float W[DIM + 2];
#pragma unroll
  for (int v = 0; v < DIM + 2; ++v) W[v] = (float)src[(long)v * g.ncell + c];
  cell_rate_bounds_f32<DIM>(g, ph, W, c, lo, hi);
}

template <typename U>
__device__ __forceinline__ U block_max(U x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    U y = __shfl_xor_sync(0xffffffffu, x, o);
    x = y > x ? y : x;
  }
  __shared__ U wmax[8];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) wmax[wid] = x;
  __syncthreads();
  U m = 0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = wmax[w] > m ? wmax[w] : m;
  return m; /* valid in thread 0 */
}

template <int DIM, typename S>
__global__ void __launch_bounds__(256) k_dt_screen(DevGeo g, Phys ph, const S* __restrict__ src,
                                                   DtState* __restrict__ dts) {
  const long c = blockIdx.x * (long)blockDim.x + threadIdx.x;
  float lo = 0.0f, hi;
  if (c < g.ncell) rate_bounds<DIM, S>(g, ph, src, c, &lo, &hi);
  const unsigned int m = block_max<unsigned int>(__float_as_uint(lo));
  if (threadIdx.x == 0) atomicMax(&dts->lo_bits, m);
}

template <int DIM, typename S>
__global__ void __launch_bounds__(256) k_dt_rate(DevGeo g, Phys ph, const S* __restrict__ src,
                                                 const double* __restrict__ U, DtState* __restrict__ dts) {
  const long c = blockIdx.x * (long)blockDim.x + threadIdx.x;
  double r = 0.0;
  if (c < g.ncell) {
    float lo, hi;
    rate_bounds<DIM, S>(g, ph, src, c, &lo, &hi);
    if (hi >= __uint_as_float(dts->lo_bits)) r = cell_rate<DIM>(g, ph, U, c);
  }
  const unsigned long long m = block_max<unsigned long long>((unsigned long long)__double_as_longlong(r));
  if (threadIdx.x == 0) atomicMax(&dts->rate_bits, m);
}

static __global__ void k_dt_reset(DtState* dts) {
  dts->rate_bits = 0ull;
  dts->lo_bits = 0u;
}

/* dt = CFL / max rate, or the fixed step; shortened to reach t_end */
/* in_step: the time step of a step of cgks_step.  Once a kernel has flagged
   a non-physical state the step gets dt = 0, so that its updates (and those
   of every later step of the call) write nothing; when this step's input,
   the previous step's output, is the non-physical one, that step is
   uncounted and the time goes back to before it. */
static __global__ void k_dt_final(Phys ph, DtState* dts, int* st, int in_step) {
  const bool prior = st_failed(st);
  double rate = __longlong_as_double((long long)dts->rate_bits);
  const bool bad = !(rate > 0.0 && rate < 1e299);
  double dt;
  if (dts->dt_fixed > 0.0) dt = dts->dt_fixed;
  else dt = bad ? 0.0 : ph.cfl / rate;
  if (bad) atomicOr(&st[ST_DT], 1);
  if (in_step) {
    if (bad && !prior && dts->nok > 0) {
      dts->nok -= 1;
      dts->t = dts->t_prev;
    }
    if (prior || bad) dt = 0.0;
  }
  if (dts->t_end > 0.0) {
    double rem = dts->t_end - dts->t;
    if (rem < dt) dt = rem > 0.0 ? rem : 0.0;
  }
  set_dt(*dts, dt);
}

/* the end of a step: counted, and the time advanced, unless a kernel of the
   step flagged a non-physical state */
static __global__ void k_time_advance(DtState* dts, const int* st) {
  if (st_failed(st)) return;
  dts->t_prev = dts->t;
  dts->t += dts->dt;
  dts->nok += 1;
}
/* a fresh time-step record at time t (dt_fixed > 0: that step, else CFL);
   a kernel rather than a copy from host memory, so that setting a state
   never waits for the stream */
static __global__ void k_dt_init(DtState* dts, double t, double dt_fixed) {
  DtState d{};
  d.t = t;
  d.dt_fixed = dt_fixed;
  *dts = d;
}

/* ------------------------------------------------------------------ */
/* metrics from node coordinates (Sec. 4 J0, Appendix volume)           */
/* ------------------------------------------------------------------ */
template <int DIM>
CGKS_HD void node_xyz(const double* nodes, const int* n, int i, int j, int k, double* x) {
  long nx = n[0] + 1, ny = n[1] + 1;
  long id = i + nx * (j + ny * (long)k);
  for (int d = 0; d < DIM; ++d) x[d] = nodes[id * DIM + d];
}

/* trilinear (bilinear) map of cell (i,j,k) and its Jacobian at xi in [0,1]^DIM */
template <int DIM>
CGKS_HD void cell_map(const double* nodes, const int* n, int i, int j, int k, const double* xi, double* x,
                      double J[3][3]) {
  for (int a = 0; a < 3; ++a) {
    x[a] = 0.0;
    for (int b = 0; b < 3; ++b) J[a][b] = 0.0;
  }
  const int nvtx = DIM == 3 ? 8 : 4;
  for (int vtx = 0; vtx < nvtx; ++vtx) {
    int o[3] = {vtx & 1, (vtx >> 1) & 1, (vtx >> 2) & 1};
    double X[3];
    node_xyz<DIM>(nodes, n, i + o[0], j + o[1], k + o[2], X);
    double w[3], dw[3];
    for (int a = 0; a < DIM; ++a) {
      w[a] = o[a] ? xi[a] : 1.0 - xi[a];
      dw[a] = o[a] ? 1.0 : -1.0;
    }
    double wt = 1.0;
    for (int a = 0; a < DIM; ++a) wt *= w[a];
    for (int a = 0; a < DIM; ++a) {
      x[a] += wt * X[a];
      for (int b = 0; b < DIM; ++b) {
        double d = dw[b];
        for (int e = 0; e < DIM; ++e)
          if (e != b) d *= w[e];
        J[a][b] += d * X[a];
      }
    }
  }
}

template <int DIM> CGKS_HD double det_dim(const double J[3][3]) {
  if (DIM == 2) return J[0][0] * J[1][1] - J[0][1] * J[1][0];
  return J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) - J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
         J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
}

template <int DIM>
CGKS_HD void metrics_cell(const double* __restrict__ nodes, const DevGeo& g, long c, double* __restrict__ met) {
  typedef Sz<DIM> S;
  typedef Met<DIM> MT;
  const long N = g.ncell;
  int i, j, k;
  cell_ijk(g, c, i, j, k);
  double N1[3], Nk[3];
  node_xyz<DIM>(nodes, g.n, i, j, k, N1);
  double J0[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 1}};
  for (int a = 0; a < DIM; ++a) {
    int o[3] = {0, 0, 0};
    o[a] = 1;
    node_xyz<DIM>(nodes, g.n, i + o[0], j + o[1], k + o[2], Nk);
    for (int r = 0; r < DIM; ++r) J0[r][a] = Nk[r] - N1[r];
  }
  double det = det_dim<3>(J0);
  double inv[3][3];
  inv[0][0] = (J0[1][1] * J0[2][2] - J0[1][2] * J0[2][1]) / det;
  inv[0][1] = (J0[0][2] * J0[2][1] - J0[0][1] * J0[2][2]) / det;
  inv[0][2] = (J0[0][1] * J0[1][2] - J0[0][2] * J0[1][1]) / det;
  inv[1][0] = (J0[1][2] * J0[2][0] - J0[1][0] * J0[2][2]) / det;
  inv[1][1] = (J0[0][0] * J0[2][2] - J0[0][2] * J0[2][0]) / det;
  inv[1][2] = (J0[0][2] * J0[1][0] - J0[0][0] * J0[1][2]) / det;
  inv[2][0] = (J0[1][0] * J0[2][1] - J0[1][1] * J0[2][0]) / det;
  inv[2][1] = (J0[0][1] * J0[2][0] - J0[0][0] * J0[2][1]) / det;
  inv[2][2] = (J0[0][0] * J0[1][1] - J0[0][1] * J0[1][0]) / det;
  for (int r = 0; r < 3; ++r)
    for (int q = 0; q < 3; ++q) {
      met[(long)(MT::J0 + r * 3 + q) * N + c] = (r < DIM && q < DIM) ? J0[r][q] : 0.0;
      met[(long)(MT::JIT + r * 3 + q) * N + c] = (r < DIM && q < DIM) ? inv[q][r] : 0.0;
    }
  /* volume: 3-point Gauss per axis of det(dX/dxi) */
  const double gx[3] = {-0.77459666924148337704, 0.0, 0.77459666924148337704};
  const double gw[3] = {5.0 / 9.0, 8.0 / 9.0, 5.0 / 9.0};
  double vol = 0.0;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b)
      for (int e = 0; e < (DIM == 3 ? 3 : 1); ++e) {
        double xi[3] = {0.5 + 0.5 * gx[a], 0.5 + 0.5 * gx[b], DIM == 3 ? 0.5 + 0.5 * gx[e] : 0.0};
        double x[3], Jm[3][3];
        cell_map<DIM>(nodes, g.n, i, j, k, xi, x, Jm);
        double w = DIM == 3 ? 0.125 * gw[a] * gw[b] * gw[e] : 0.25 * gw[a] * gw[b];
        vol += w * det_dim<DIM>(Jm);
      }
  met[(long)MT::VOL * N + c] = vol;
  double pos[S::NGP][3];
  for (int f = 0; f < 2 * DIM; ++f) {
    int ax = f / 2, side = f & 1;
    int ta[2] = {0, 0}, nt = 0;
    for (int q = 0; q < DIM; ++q)
      if (q != ax) ta[nt++] = q;
    for (int kk = 0; kk < S::GPF; ++kk) {
      int gp = f * S::GPF + kk;
      double xi[3];
      for (int a = 0; a < 3; ++a) xi[a] = a < DIM ? gp_delta<DIM>(gp, a) + 0.5 : 0.0;
      xi[ax] = side;
      double x[3], Jm[3][3];
      cell_map<DIM>(nodes, g.n, i, j, k, xi, x, Jm);
      for (int a = 0; a < 3; ++a) pos[gp][a] = x[a];
      double w = 1.0 / S::GPF;
      double A[3] = {0.0, 0.0, 0.0}, T[3] = {0.0, 0.0, 0.0};
      if (DIM == 3) {
        double u0[3] = {Jm[0][ta[0]], Jm[1][ta[0]], Jm[2][ta[0]]};
        double u1[3] = {Jm[0][ta[1]], Jm[1][ta[1]], Jm[2][ta[1]]};
        double cr[3] = {u0[1] * u1[2] - u0[2] * u1[1], u0[2] * u1[0] - u0[0] * u1[2], u0[0] * u1[1] - u0[1] * u1[0]};
        double sg = ax == 1 ? -1.0 : 1.0;
        for (int a = 0; a < 3; ++a) {
          A[a] = sg * w * cr[a];
          T[a] = u0[a];
        }
      } else {
        double tv[2] = {Jm[0][ta[0]], Jm[1][ta[0]]};
        double sg = ax == 0 ? 1.0 : -1.0;
        A[0] = sg * w * tv[1];
        A[1] = -sg * w * tv[0];
        T[0] = tv[0];
        T[1] = tv[1];
      }
      for (int a = 0; a < 3; ++a) met[(long)(MT::AREA + gp * 3 + a) * N + c] = A[a];
      if (side)
        for (int a = 0; a < 3; ++a) met[(long)(MT::TANG + (ax * S::GPF + kk) * 3 + a) * N + c] = T[a];
    }
  }
  for (int ax = 0; ax < DIM; ++ax)
    for (int kk = 0; kk < S::GPF; ++kk) {
      int glo = (2 * ax) * S::GPF + kk, ghi = (2 * ax + 1) * S::GPF + kk;
      double s = 0.0;
      for (int a = 0; a < DIM; ++a) {
        double d = pos[ghi][a] - pos[glo][a];
        s += d * d;
      }
      met[(long)(MT::LEN + ax * S::GPF + kk) * N + c] = sqrt(s);
    }
}

template <int DIM>
__global__ void k_metrics(const double* __restrict__ nodes, DevGeo g, double* __restrict__ met) {
  long c = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (c >= g.ncell) return;
  metrics_cell<DIM>(nodes, g, c, met);
}

/* ------------------------------------------------------------------ */
/* initial data                                                        */
/* ------------------------------------------------------------------ */
#define CGKS_G5X0 0.90617984593866399280
#define CGKS_G5X1 0.53846931010568309104
CGKS_HD double g5x(int q) {
  return q == 0 ? -CGKS_G5X0 : q == 1 ? -CGKS_G5X1 : q == 2 ? 0.0 : q == 3 ? CGKS_G5X1 : CGKS_G5X0;
}
CGKS_HD double g5w(int q) {
  return (q == 0 || q == 4) ? 0.23692688505618908751 : (q == 1 || q == 3) ? 0.47862867049936646804
                                                                          : 0.56888888888888888889;
}
/* Volume sums of the TGV diagnostics (Sec. 6.2): kinetic energy 1/2 |m|^2/rho,
   mu |curl U|^2 (the velocity gradient from the conservative averages and
   cell-averaged gradients: d_k U_i = (d_k m_i - U_i d_k rho) / rho), mass and
   volume; block partials [block][4], summed in a fixed order by the host */
template <typename T, int DIM>
__global__ void __launch_bounds__(256) k_diagnostics(DevGeo g, const double* __restrict__ avg,
                                                     const T* __restrict__ der, double mu,
                                                     double* __restrict__ part) {
  const long N = g.ncell;
  constexpr int NV = DIM + 2;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (long c = blockIdx.x * (long)blockDim.x + threadIdx.x; c < N; c += (long)gridDim.x * blockDim.x) {
    const double vol = g.curvi ? met_vol<DIM>(g, c) : (DIM == 3 ? g.h[0] * g.h[1] * g.h[2] : g.h[0] * g.h[1]);
    const double rho = avg[c];
    double U[3] = {0.0, 0.0, 0.0}, ke = 0.0;
    for (int i = 0; i < DIM; ++i) {
      U[i] = avg[(long)(1 + i) * N + c] / rho;
      ke += 0.5 * rho * U[i] * U[i];
    }
    double G[3][3] = {{0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}}; /* G[i][k] = d_k U_i */
    for (int k = 0; k < DIM; ++k) {
      const double dr = (double)der[((long)k * NV + 0) * N + c];
      for (int i = 0; i < DIM; ++i) G[i][k] = ((double)der[((long)k * NV + 1 + i) * N + c] - U[i] * dr) / rho;
    }
    double w2;
    if (DIM == 3) {
      const double w0 = G[2][1] - G[1][2], w1 = G[0][2] - G[2][0], wz = G[1][0] - G[0][1];
      w2 = w0 * w0 + w1 * w1 + wz * wz;
    } else {
      const double wz = G[1][0] - G[0][1];
      w2 = wz * wz;
    }
    acc[0] += ke * vol;
    acc[1] += mu * w2 * vol;
    acc[2] += rho * vol;
    acc[3] += vol;
  }
  __shared__ double sh[256][4];
  for (int q = 0; q < 4; ++q) sh[threadIdx.x][q] = acc[q];
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o)
      for (int q = 0; q < 4; ++q) sh[threadIdx.x][q] += sh[threadIdx.x + o][q];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int q = 0; q < 4; ++q) part[blockIdx.x * 4 + q] = sh[0][q];
}

/* FP32 CFL metric of each curvilinear cell (RateMet<DIM>) from the FP64
   metrics, by the same formulas as the curvilinear branch of cell_rate */
template <int DIM>
__global__ void k_rate_metrics(DevGeo g, float* __restrict__ rmet) {
  const long c = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (c >= g.ncell) return;
  const long N = g.ncell;
  const double vol = met_vol<DIM>(g, c);
  double hmin = 1e300;
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
    for (int a = 0; a < DIM; ++a) rmet[(RateMet<DIM>::W + ax * DIM + a) * N + c] = (float)(nn[a] / sqrt(ns) / h);
    rmet[(RateMet<DIM>::IH + ax) * N + c] = (float)(1.0 / h);
    if (h < hmin) hmin = h;
  }
  rmet[RateMet<DIM>::HMIN * N + c] = (float)hmin;
}

template <int DIM> __host__ __device__ constexpr int npts_cell() { return (DIM == 3 ? 125 : 25) + Sz<DIM>::NGP; }

/* physical position of reference point xi of cell (i,j,k) */
template <int DIM>
CGKS_HD void ref_to_phys(const double* nodes, const DevGeo& g, const double* lo, int i, int j, int k,
                            const double* xi, double* x, double* detJ) {
  if (nodes) {
    double J[3][3];
    cell_map<DIM>(nodes, g.n, i, j, k, xi, x, J);
    *detJ = det_dim<DIM>(J);
  } else {
    int ii[3] = {i, j, k};
    double d = 1.0;
    for (int a = 0; a < DIM; ++a) {
      x[a] = lo[a] + (ii[a] + xi[a]) * g.h[a];
      d *= g.h[a];
    }
    *detJ = d;
  }
}

template <int DIM>
CGKS_HD void init_point(const double* __restrict__ nodes, const DevGeo& g, const double* lo3, long cell0, long t,
                        double* __restrict__ pts) {
  const int NP = npts_cell<DIM>();
  long cl = t / NP;
  int q = (int)(t % NP);
  long c = cell0 + cl;
  int i, j, k;
  cell_ijk(g, c, i, j, k);
  double lo[3] = {lo3[0], lo3[1], lo3[2]};
  double xi[3] = {0.0, 0.0, 0.0}, x[3], dj;
  const int NVOL = DIM == 3 ? 125 : 25;
  if (q < NVOL) {
    int qx = q % 5, qy = (q / 5) % 5, qz = q / 25;
    xi[0] = 0.5 + 0.5 * g5x(qx);
    xi[1] = 0.5 + 0.5 * g5x(qy);
    if (DIM == 3) xi[2] = 0.5 + 0.5 * g5x(qz);
  } else {
    int gp = q - NVOL;
    for (int a = 0; a < DIM; ++a) xi[a] = gp_delta<DIM>(gp, a) + 0.5;
  }
  ref_to_phys<DIM>(nodes, g, lo, i, j, k, xi, x, &dj);
  for (int a = 0; a < DIM; ++a) pts[t * DIM + a] = x[a];
}

template <int DIM>
__global__ void k_init_points(const double* __restrict__ nodes, DevGeo g, const double* lo3, long cell0, long ncells,
                              double* __restrict__ pts) {
  long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (t >= ncells * npts_cell<DIM>()) return;
  init_point<DIM>(nodes, g, lo3, cell0, t, pts);
}

template <int DIM>
CGKS_HD void init_cell(const double* __restrict__ nodes, const DevGeo& g, const Phys& ph, const double* lo3, long cell0,
                       long cl, const double* __restrict__ prims, double* __restrict__ U) {
  typedef Sz<DIM> S;
  const int NV = S::NV, NP = npts_cell<DIM>(), NVOL = DIM == 3 ? 125 : 25;
  const long N = g.ncell;
  long c = cell0 + cl;
  int i, j, k;
  cell_ijk(g, c, i, j, k);
  double lo[3] = {lo3[0], lo3[1], lo3[2]};
  const double* pr = prims + cl * NP * NV;
  double sum[NV], wsum = 0.0;
  for (int v = 0; v < NV; ++v) sum[v] = 0.0;
  for (int q = 0; q < NVOL; ++q) {
    int qx = q % 5, qy = (q / 5) % 5, qz = q / 25;
    double xi[3] = {0.5 + 0.5 * g5x(qx), 0.5 + 0.5 * g5x(qy), DIM == 3 ? 0.5 + 0.5 * g5x(qz) : 0.0};
    double x[3], dj;
    ref_to_phys<DIM>(nodes, g, lo, i, j, k, xi, x, &dj);
    double w = g5w(qx) * g5w(qy) * (DIM == 3 ? g5w(qz) : 1.0) * dj;
    const double* p = pr + q * NV;
    double ke = 0.0;
    for (int a = 0; a < DIM; ++a) ke += p[1 + a] * p[1 + a];
    double W[NV];
    W[0] = p[0];
    for (int a = 0; a < DIM; ++a) W[1 + a] = p[0] * p[1 + a];
    W[NV - 1] = p[NV - 1] / (ph.gamma - 1.0) + 0.5 * p[0] * ke;
    for (int v = 0; v < NV; ++v) sum[v] += w * W[v];
    wsum += w;
  }
  for (int v = 0; v < NV; ++v) U[(long)v * N + c] = sum[v] / wsum;
  /* face-point values -> gradient and line derivatives */
  const double vol = met_vol<DIM>(g, c);
  for (int v = 0; v < NV; ++v) {
    double gr[3] = {0.0, 0.0, 0.0};
    double val[S::NGP];
    for (int gp = 0; gp < S::NGP; ++gp) {
      const double* p = pr + (NVOL + gp) * NV;
      double W;
      if (v == 0) W = p[0];
      else if (v < NV - 1) W = p[0] * p[v];
      else {
        double ke = 0.0;
        for (int a = 0; a < DIM; ++a) ke += p[1 + a] * p[1 + a];
        W = p[NV - 1] / (ph.gamma - 1.0) + 0.5 * p[0] * ke;
      }
      val[gp] = W;
      double sgn = ((gp / S::GPF) & 1) ? 1.0 : -1.0;
      for (int a = 0; a < DIM; ++a) gr[a] += sgn * W * met_area<DIM>(g, c, gp, a);
    }
    for (int a = 0; a < DIM; ++a) U[((long)(1 + a) * NV + v) * N + c] = gr[a] / vol;
    for (int s = 0; s < S::NL; ++s) {
      int ax = s / S::GPF, kk = s % S::GPF;
      double d = val[(2 * ax + 1) * S::GPF + kk] - val[(2 * ax) * S::GPF + kk];
      U[((long)(1 + DIM + s) * NV + v) * N + c] = d / met_len<DIM>(g, c, s);
    }
  }
}

template <int DIM>
__global__ void k_init_from_prims(const double* __restrict__ nodes, DevGeo g, Phys ph, const double* lo3, long cell0,
                                  long ncells, const double* __restrict__ prims, double* __restrict__ U) {
  long cl = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (cl >= ncells) return;
  init_cell<DIM>(nodes, g, ph, lo3, cell0, cl, prims, U);
}

}  // namespace cgks
