/*
 * cgks_compute_dt_noalloc: the CFL time step of a caller-held state without
 * any device allocation (see include/cgks.h).
 *
 * Who needs it: callers that must not allocate device memory themselves or
 * through this library -- e.g. an application whose device memory is owned
 * by another allocator that reserved it up front, or a timed loop that cannot
 * afford cudaMalloc/cudaFree (both may synchronise the device).  They pass the
 * state they already hold and receive dt; the work space is a fixed array
 * that exists in every GPU's memory from the moment the library's module is
 * loaded on that GPU until the process exits.
 *
 * The scratch: one partial maximum per thread block (the bit pattern of the
 * largest positive rate, which orders like the double) plus the final
 * result slot.  Every call overwrites the partials it reads and the result
 * slot, so nothing has to start at zero.  All calls share the one array:
 * calls whose kernels overlap on the GPU (different streams without
 * ordering) race on it.
 */
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "../../include/cgks.h"
#include "cgks_device.cuh"

using namespace cgks;

namespace {

constexpr int kThreads = 256;
constexpr int kMaxBlocks = CGKS_DT_NOALLOC_MAX_CELLS / kThreads;
constexpr int kMaxDevices = 64;

/* partial maxima [0, kMaxBlocks) and the result slot kMaxBlocks */
static __device__ __align__(256) unsigned long long g_dt_scratch[kMaxBlocks + 1];

/* device address of g_dt_scratch, looked up once per device with that device current */
unsigned long long* g_scratch_ptr[kMaxDevices] = {nullptr};
std::mutex g_setup_mutex;

template <int DIM>
__global__ void __launch_bounds__(kThreads) k_dt_partial(DevGeo g, Phys ph, const double* __restrict__ U,
                                                         unsigned long long* __restrict__ scratch) {
  long c = blockIdx.x * (long)blockDim.x + threadIdx.x;
  double r = 0.0;
  if (c < g.ncell) r = cell_rate<DIM>(g, ph, U, c);
  unsigned long long bits = (unsigned long long)__double_as_longlong(r);
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long ob = __shfl_xor_sync(0xffffffffu, bits, o);
    bits = ob > bits ? ob : bits;
  }
  __shared__ unsigned long long wmax[kThreads / 32];
  if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = bits;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long m = 0;
    for (int w = 0; w < kThreads / 32; ++w) m = wmax[w] > m ? wmax[w] : m;
    scratch[blockIdx.x] = m;
  }
}

__global__ void __launch_bounds__(kThreads) k_dt_combine(unsigned long long* __restrict__ scratch, int nblocks) {
  unsigned long long m = 0;
  for (int b = threadIdx.x; b < nblocks; b += kThreads) m = scratch[b] > m ? scratch[b] : m;
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long ob = __shfl_xor_sync(0xffffffffu, m, o);
    m = ob > m ? ob : m;
  }
  __shared__ unsigned long long wmax[kThreads / 32];
  if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long r = 0;
    for (int w = 0; w < kThreads / 32; ++w) r = wmax[w] > r ? wmax[w] : r;
    scratch[kMaxBlocks] = r;
  }
}

/* once per device, with that device current */
cgks_status scratch_for_current_device(unsigned long long** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return CGKS_ECUDA;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_dt_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return CGKS_ECUDA;
    }
    g_scratch_ptr[dev] = static_cast<unsigned long long*>(p);
  }
  *out = g_scratch_ptr[dev];
  return CGKS_OK;
}

}  // namespace

extern "C" cgks_status cgks_compute_dt_noalloc(const cgks_mesh_desc* d, const double* dev_state, double* dt_out) {
  if (!d || !dev_state || !dt_out) return CGKS_EINVAL;
  if (d->dim != 2 && d->dim != 3) return CGKS_EINVAL;
  if (d->nodes) return CGKS_EUNSUPPORTED; /* curvilinear metrics would need device memory */
  long ncell = 1;
  for (int a = 0; a < d->dim; ++a) {
    if (d->n[a] < 1) return CGKS_EINVAL;
    ncell *= d->n[a];
    if (ncell > CGKS_DT_NOALLOC_MAX_CELLS) return CGKS_ETOOLARGE;
  }
  if (!(d->gamma > 1.0) || d->mu < 0.0 || !(d->cfl > 0.0)) return CGKS_EINVAL;
  /* the state must be device memory of the current device */
  int cur = 0;
  if (cudaGetDevice(&cur) != cudaSuccess) return CGKS_ECUDA;
  cudaPointerAttributes pa{};
  if (cudaPointerGetAttributes(&pa, dev_state) != cudaSuccess) {
    cudaGetLastError();
    return CGKS_EINVAL;
  }
  if ((pa.type != cudaMemoryTypeDevice && pa.type != cudaMemoryTypeManaged) || pa.device != cur) return CGKS_EINVAL;
  unsigned long long* scratch = nullptr;
  cgks_status s = scratch_for_current_device(&scratch);
  if (s != CGKS_OK) return s;
  DevGeo g{};
  for (int a = 0; a < 3; ++a) {
    g.n[a] = a < d->dim ? d->n[a] : 1;
    g.h[a] = a < d->dim ? (d->hi[a] - d->lo[a]) / d->n[a] : 1.0;
    g.ih[a] = 1.0 / g.h[a];
    g.hf[a] = (float)g.h[a];
    g.ihf[a] = (float)g.ih[a];
  }
  g.ncell = ncell;
  g.curvi = 0;
  g.met = nullptr;
  Phys ph{};
  ph.gamma = d->gamma;
  ph.mu = d->mu;
  ph.cfl = d->cfl;
  cudaStream_t st = (cudaStream_t)d->stream;
  int nblocks = (int)((ncell + kThreads - 1) / kThreads);
  if (d->dim == 3) k_dt_partial<3><<<nblocks, kThreads, 0, st>>>(g, ph, dev_state, scratch);
  else k_dt_partial<2><<<nblocks, kThreads, 0, st>>>(g, ph, dev_state, scratch);
  k_dt_combine<<<1, kThreads, 0, st>>>(scratch, nblocks);
  if (cudaGetLastError() != cudaSuccess) return CGKS_ECUDA;
  unsigned long long bits = 0;
  if (cudaMemcpyAsync(&bits, scratch + kMaxBlocks, sizeof bits, cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return CGKS_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return CGKS_ECUDA;
  double rate;
  memcpy(&rate, &bits, sizeof rate);
  if (!(rate > 0.0) || rate >= 1e299) return CGKS_ENONPHYS;
  *dt_out = d->dt_fixed > 0.0 ? d->dt_fixed : d->cfl / rate;
  return CGKS_OK;
}
