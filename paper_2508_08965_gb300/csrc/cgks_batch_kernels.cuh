/*
 * Batched kernels: many independent meshes (cases) of uneven size advance
 * together.  Every per-case array lives in one concatenated allocation per
 * kind, case k's part starting at (per-cell size) x cell0 (or x plane0 for
 * the low-boundary faces); inside it the case keeps the single-case layout,
 * so the per-cell and per-face device functions of cgks_device.cuh and
 * cgks_kernels.cuh run unchanged on it.
 *
 * Work is cut into tiles of one block each.  A tile list holds, for the
 * cases that take part in a phase, the prefix sums of their tile counts; a
 * persistent block walks the tiles blockIdx.x, blockIdx.x + gridDim.x, ...,
 * finds its case by binary search and stages the case's descriptor in shared
 * memory.  Grid size (persistent or one block per tile) and the tile shape
 * of the reconstruction are launch parameters, chosen by the host's
 * autotuner.
 */
#ifndef CGKS_BATCH_KERNELS_CUH
#define CGKS_BATCH_KERNELS_CUH

#include "cgks_kernels.cuh"

namespace cgks {

struct BatchCase {
  DevGeo g;
  Phys ph;
  long cell0;  /* first cell of the case in the concatenated cell arrays */
  long plane0; /* first slot of the case in the concatenated low-boundary face array */
};

/* base pointers of the concatenated arrays of one S2O4 stage */
template <typename T> struct BatchArrays {
  const double* avg_in;
  const float* avh_in;
  const float* avl_in;
  const T* der_in;
  double* avg_out;
  float* avh_out;
  float* avl_out;
  T* der_out;
  double* savg;
  T* sder;
  T* gpL;
  T* gpR;
  T* flux;
  T* fxb;
  DtState* dts; /* one per case */
  int* st;
};

/* tiles of one phase: entry e covers tiles [start[e], start[e+1]) of case
   cases[e] */
struct TileList {
  const int* start; /* nentry + 1 */
  const int* cases; /* nentry */
  int nentry;
  int ntile;
};

__device__ __forceinline__ int tile_entry(const TileList& L, int tile) {
  int lo = 0, hi = L.nentry - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (L.start[mid] <= tile) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

/* the block's current tile: its case (staged in shared memory by the
   caller) and the tile's index within the case */
struct TileRef {
  int ci;  /* case index */
  int lt;  /* tile index within the case */
};

__device__ __forceinline__ TileRef stage_tile(const TileList& L, const BatchCase* __restrict__ cases, int tile,
                                              BatchCase* sh_case, TileRef* sh_ref) {
  __syncthreads(); /* the previous tile is done with the shared copy */
  if (threadIdx.x == 0) {
    const int e = tile_entry(L, tile);
    sh_ref->ci = L.cases[e];
    sh_ref->lt = tile - L.start[e];
  }
  __syncthreads();
  const int ci = sh_ref->ci;
  const int* src = reinterpret_cast<const int*>(cases + ci);
  int* dst = reinterpret_cast<int*>(sh_case);
  for (int w = threadIdx.x; w < (int)(sizeof(BatchCase) / sizeof(int)); w += blockDim.x) dst[w] = src[w];
  __syncthreads();
  return *sh_ref;
}

template <int DIM> __host__ __device__ constexpr int batch_nf() { return 1 + DIM + DIM * Sz<DIM>::GPF; }

/* reconstruction: a tile is a tx x ty patch of one (i, j) plane of a case */
template <typename T, int DIM, bool WALL>
__global__ void __launch_bounds__(128, min_blocks<T, DIM>())
    kb_recon(const BatchCase* __restrict__ cases, TileList L, BatchArrays<T> A, int tx, int ty, SelectorDev sel) {
  __shared__ BatchCase sc;
  __shared__ TileRef sr;
  constexpr int NV = Sz<DIM>::NV;
  for (int tile = blockIdx.x; tile < L.ntile; tile += gridDim.x) {
    const TileRef ref = stage_tile(L, cases, tile, &sc, &sr);
    const DevGeo& g = sc.g;
    const int ntx = (g.n[0] + tx - 1) / tx, nty = (g.n[1] + ty - 1) / ty;
    const int i = (ref.lt % ntx) * tx + (int)threadIdx.x % tx;
    const int j = ((ref.lt / ntx) % nty) * ty + (int)threadIdx.x / tx;
    const int k = ref.lt / (ntx * nty);
    const bool active = (int)threadIdx.x < tx * ty && i < g.n[0] && j < g.n[1];
    const Phys& ph = sc.ph;
    const long o = sc.cell0;
    const long c = active ? cell_index(g, i, j, k) : 0;
    const double* avg = A.avg_in + NV * o;
    const float* avh = A.avh_in ? A.avh_in + NV * o : nullptr;
    const T* der = A.der_in + (long)(batch_nf<DIM>() - 1) * NV * o;
    /* every cell of a batch with walls takes the boundary path: which cells
       share a warp depends on the tile shape the tuner picks, and the two
       compiled paths may round differently, so a per-warp choice would make
       the results depend on the tiles */
    const bool wall = WALL;
    bool skip = false;
    if (sel.on && !ph.linear) skip = selector_skip<T, DIM, WALL>(sel, avg, avh, der, g, c, i, j, k, active, wall);
    if (active) {
      const int ngp = DIM * Sz<DIM>::GPF * NV * (1 + DIM);
      const float* avl = A.avl_in ? A.avl_in + NV * o : nullptr;
      T* gl = A.gpL + (long)ngp * o;
      T* gr = A.gpR + (long)ngp * o;
      if (wall) recon_cell<T, DIM, false, WALL>(avg, avh, avl, der, g, ph, c, i, j, k, gl, gr, nullptr, 0, A.st, skip);
      else recon_cell<T, DIM, false, false>(avg, avh, avl, der, g, ph, c, i, j, k, gl, gr, nullptr, 0, A.st, skip);
    }
  }
}

/* interface flux: tiles of blockDim.x = 128 face-point items (flux_item),
   each point's Gauss-point states staged in shared memory */
template <typename T, int DIM>
__global__ void __launch_bounds__(128, flux_min_blocks<T, DIM, false>())
    kb_flux(const BatchCase* __restrict__ cases, TileList L, BatchArrays<T> A) {
  __shared__ BatchCase sc;
  __shared__ TileRef sr;
  constexpr int NV = Sz<DIM>::NV;
  __shared__ T stage[2 * NV * (1 + DIM) * 128];
  for (int tile = blockIdx.x; tile < L.ntile; tile += gridDim.x) {
    const TileRef ref = stage_tile(L, cases, tile, &sc, &sr);
    const long t = (long)ref.lt * blockDim.x + threadIdx.x;
    const DevGeo& g = sc.g;
    const double dt = A.dts[ref.ci].dt;
    if (t < (long)DIM * Sz<DIM>::GPF * g.ncell && dt > 0.0) {
      const long o = sc.cell0;
      const int ngp = DIM * Sz<DIM>::GPF * NV * (1 + DIM);
      const int nfx = DIM * Sz<DIM>::GPF * 6 * NV;
      flux_item<T, DIM, false>(g, sc.ph, dt, t, A.gpL + (long)ngp * o, A.gpR + (long)ngp * o,
                               A.flux + (long)nfx * o, A.st, stage + threadIdx.x, 128);
    }
  }
}

/* boundary faces of the cases with a non-periodic axis (flux_bnd_item) */
template <typename T, int DIM>
__global__ void __launch_bounds__(128) kb_flux_bnd(const BatchCase* __restrict__ cases, TileList L, BatchArrays<T> A) {
  __shared__ BatchCase sc;
  __shared__ TileRef sr;
  constexpr int NV = Sz<DIM>::NV;
  for (int tile = blockIdx.x; tile < L.ntile; tile += gridDim.x) {
    const TileRef ref = stage_tile(L, cases, tile, &sc, &sr);
    const long t = (long)ref.lt * blockDim.x + threadIdx.x;
    const DevGeo& g = sc.g;
    const double dt = A.dts[ref.ci].dt;
    if (t < 2L * DIM * Sz<DIM>::GPF * g.nplane && dt > 0.0) {
      const long o = sc.cell0;
      const int ngp = DIM * Sz<DIM>::GPF * NV * (1 + DIM);
      const int nfx = DIM * Sz<DIM>::GPF * 6 * NV;
      flux_bnd_item<T, DIM, false>(g, sc.ph, dt, t, A.gpL + (long)ngp * o, A.gpR + (long)ngp * o,
                                   A.flux + (long)nfx * o, A.fxb + (long)nfx * sc.plane0, A.st);
    }
  }
}

/* S2O4 update: tiles of blockDim.x (cell, variable) items, item = v * N + c */
template <typename T, int DIM>
__global__ void __launch_bounds__(128)
    kb_update(const BatchCase* __restrict__ cases, TileList L, BatchArrays<T> A, int stage) {
  __shared__ BatchCase sc;
  __shared__ TileRef sr;
  constexpr int NV = Sz<DIM>::NV;
  for (int tile = blockIdx.x; tile < L.ntile; tile += gridDim.x) {
    const TileRef ref = stage_tile(L, cases, tile, &sc, &sr);
    const long t = (long)ref.lt * blockDim.x + threadIdx.x;
    const DevGeo& g = sc.g;
    const StageCoef kc = A.dts[ref.ci].k;
    const double dt = kc.dt;
    if (t < (long)NV * g.ncell && dt > 0.0) {
      const long o = sc.cell0;
      const long c = t % g.ncell;
      const int v = (int)(t / g.ncell);
      int i, j, k;
      cell_ijk(g, c, i, j, k);
      const long nd = (long)(batch_nf<DIM>() - 1) * NV;
      const int nfx = DIM * Sz<DIM>::GPF * 6 * NV;
      update_var<T, DIM, false>(g, kc, stage, c, i, j, k, v, A.avg_in + NV * o, A.flux + (long)nfx * o,
                                A.fxb + (long)nfx * sc.plane0, A.savg + NV * o, A.sder + nd * o,
                                A.avg_out + NV * o, A.der_out + nd * o, A.avh_out ? A.avh_out + NV * o : nullptr,
                                A.avl_out ? A.avl_out + NV * o : nullptr);
    }
  }
}

/* CFL maximum per case, the two passes of k_dt_screen / k_dt_rate over
   tiles of 256 cells; S: the averages the FP32 bounds read */
template <int DIM, typename S>
__global__ void __launch_bounds__(256)
    kb_dt_screen(const BatchCase* __restrict__ cases, TileList L, const S* __restrict__ src, DtState* dts) {
  __shared__ BatchCase sc;
  __shared__ TileRef sr;
  for (int tile = blockIdx.x; tile < L.ntile; tile += gridDim.x) {
    const TileRef ref = stage_tile(L, cases, tile, &sc, &sr);
    const long c = (long)ref.lt * blockDim.x + threadIdx.x;
    const DevGeo& g = sc.g;
    float lo = 0.0f, hi;
    if (c < g.ncell) rate_bounds<DIM, S>(g, sc.ph, src + (DIM + 2) * sc.cell0, c, &lo, &hi);
    const unsigned int m = block_max<unsigned int>(__float_as_uint(lo));
    if (threadIdx.x == 0) atomicMax(&dts[ref.ci].lo_bits, m);
  }
}

template <int DIM, typename S>
__global__ void __launch_bounds__(256) kb_dt_rate(const BatchCase* __restrict__ cases, TileList L,
                                                  const S* __restrict__ src, const double* __restrict__ U,
                                                  DtState* dts) {
  __shared__ BatchCase sc;
  __shared__ TileRef sr;
  for (int tile = blockIdx.x; tile < L.ntile; tile += gridDim.x) {
    const TileRef ref = stage_tile(L, cases, tile, &sc, &sr);
    const long c = (long)ref.lt * blockDim.x + threadIdx.x;
    const DevGeo& g = sc.g;
    double r = 0.0;
    if (c < g.ncell) {
      float lo, hi;
      rate_bounds<DIM, S>(g, sc.ph, src + (DIM + 2) * sc.cell0, c, &lo, &hi);
      if (hi >= __uint_as_float(dts[ref.ci].lo_bits)) r = cell_rate<DIM>(g, sc.ph, U + (DIM + 2) * sc.cell0, c);
    }
    const unsigned long long m = block_max<unsigned long long>((unsigned long long)__double_as_longlong(r));
    if (threadIdx.x == 0) atomicMax(&dts[ref.ci].rate_bits, m);
  }
}

static __global__ void kb_dt_reset(DtState* dts, int ncase) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < ncase) {
    dts[i].rate_bits = 0ull;
    dts[i].lo_bits = 0u;
  }
}

/* per case: dt = CFL / max rate (or the fixed step), shortened to t_end */
static __global__ void kb_dt_final(const BatchCase* __restrict__ cases, DtState* dts, int* st, int ncase) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ncase) return;
  DtState& d = dts[i];
  const double rate = __longlong_as_double((long long)d.rate_bits);
  double dt;
  if (d.dt_fixed > 0.0) dt = d.dt_fixed;
  else dt = (rate > 0.0 && rate < 1e299) ? cases[i].ph.cfl / rate : 0.0;
  if (rate >= 1e299) atomicOr(&st[ST_DT], 1);
  if (d.t_end > 0.0) {
    const double rem = d.t_end - d.t;
    if (rem < dt) dt = rem > 0.0 ? rem : 0.0;
  }
  set_dt(d, dt);
}

static __global__ void kb_time_advance(DtState* dts, int ncase) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < ncase) dts[i].t += dts[i].dt;
}

}  // namespace cgks

#endif
