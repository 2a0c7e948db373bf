/*
 * Internal to the library: the context behind the cgks_ctx handle of
 * include/cgks.h, shared by the host API (cgks.cu) and the stage launchers,
 * which live in one translation unit per precision (cgks_stage_f64.cu,
 * cgks_stage_f32.cu) so that they compile in parallel.
 */
#ifndef CGKS_CTX_H
#define CGKS_CTX_H
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/cgks.h"
#include "cgks_kernels.cuh"

namespace cgks_host {

enum KernelId { KID_RECON, KID_FLUX, KID_UPDATE, KID_DT, KID_N };
inline const char* const kKernelNames[KID_N] = {"recon", "flux", "update", "dt"};

struct Prof {
  bool on = false;
  std::vector<cudaEvent_t> pool;
  std::vector<std::pair<int, int>> rec;  /* (kernel id, event index of start) */
  long launches[KID_N] = {0};
  double ms[KID_N] = {0};
};

}  // namespace cgks_host

struct cgks_ctx {
  int dim, nv, nf;
  int n[3];
  long ncell;
  int prec;                 /* 0: FP64; 1: FP32 bulk with FP64 averages */
  bool walls;               /* some face is a wall: reconstruction with mirror images */
  bool pair_flux = false;   /* FP64 storage, interface flux solved in paired FP32 (precision 2) */
  cgks_mesh_desc desc;
  cudaStream_t stream;
  cgks::DevGeo geo;
  cgks::Phys ph;
  double* d_nodes = nullptr;
  double* d_met = nullptr;
  float* d_rmet = nullptr;
  double* d_bcq = nullptr;  /* inflow states [face][5], then their FP32 hi and lo parts */
  double* d_lo = nullptr;
  /* state buffers.  FP64: full public-layout arrays U (current), Us
     (intermediate) and a stash, with the derivative fields right after the
     averages.  FP32: FP64 averages and FP32 derivative fields in separate
     arrays, plus a public-layout FP64 staging buffer for copies in and out. */
  double* U = nullptr;
  double* Us = nullptr;
  double* stash = nullptr;
  double* avg[2] = {nullptr, nullptr};
  void* der[2] = {nullptr, nullptr};
  double* savg = nullptr;
  void* sder = nullptr;
  void* f32 = nullptr;      /* FP32 derivative storage (3 arrays) */
  float* avh[2] = {nullptr, nullptr}; /* FP32 form: exact hi + lo pairs of the averages */
  float* avl[2] = {nullptr, nullptr};
  float* pairs = nullptr;
  void* gpL = nullptr;
  void* gpR = nullptr;
  void* flux = nullptr;
  void* fxb = nullptr;      /* low-boundary faces of the non-periodic axes */
  double* chi = nullptr;
  /* the flux kernel's TMA tiles: gpL and gpR as 2-D arrays [row][cell]
     (boxes of one Gauss point's quantities x 128 cells); tma = false where
     the mesh does not allow them (curvilinear, cell count not a multiple of
     128) or the driver gave no encoder: the flux then stages by cp.async */
  bool tma = false;
  CUtensorMap tmL{}, tmR{};
  cgks::DtState* dts = nullptr;
  int* st = nullptr;
  double t = 0.0;
  std::string err;
  cgks_host::Prof prof;
  /* learned selector (cgks_set_selector): device copy of its parameters */
  cgks::SelectorDev sel{};
  void* sel_buf = nullptr; /* BF16 weights, FP32 biases, two counters */
};


inline long cdiv(long a, long b) { return (a + b - 1) / b; }

/* device copy of a selector's parameters (packed as cgks_set_selector takes
   them) in *buf (allocated on first use): BF16 weights, FP32 biases and two
   zeroed counters; fills *sd and switches it on */
cgks_status selector_upload(void** buf, cgks::SelectorDev* sd, const float* params, float thr_skip, float thr_lo,
                            cudaStream_t stream);

/* ---- profiling: CUDA events around each launch on the context stream ---- */
inline void prof_begin(cgks_ctx* ctx, int kid) {
  if (!ctx->prof.on) return;
  cgks_host::Prof& p = ctx->prof;
  size_t need = p.rec.size() * 2 + 2;
  while (p.pool.size() < need) {
    cudaEvent_t e;
    cudaEventCreate(&e);
    p.pool.push_back(e);
  }
  int idx = (int)p.rec.size() * 2;
  p.rec.push_back({kid, idx});
  cudaEventRecord(p.pool[idx], ctx->stream);
}
inline void prof_end(cgks_ctx* ctx) {
  if (!ctx->prof.on) return;
  cgks_host::Prof& p = ctx->prof;
  cudaEventRecord(p.pool[p.rec.back().second + 1], ctx->stream);
}

/* one S2O4 stage (reconstruction, interface flux, update) of a single-case
   context; WALL: some face of the mesh is a wall (mirror images in the
   reconstruction stencil).  Instantiated in cgks_stage_f64.cu / _f32.cu. */
template <typename T, int DIM, bool CURVI, bool WALL>
void launch_stage(cgks_ctx* ctx, int stage);

#define CGKS_DECLARE_STAGES(T)                                     \
  extern template void launch_stage<T, 2, false, false>(cgks_ctx*, int); \
  extern template void launch_stage<T, 2, false, true>(cgks_ctx*, int);  \
  extern template void launch_stage<T, 2, true, false>(cgks_ctx*, int);  \
  extern template void launch_stage<T, 3, false, false>(cgks_ctx*, int); \
  extern template void launch_stage<T, 3, false, true>(cgks_ctx*, int);  \
  extern template void launch_stage<T, 3, true, false>(cgks_ctx*, int);
CGKS_DECLARE_STAGES(float)
CGKS_DECLARE_STAGES(double)

/* the interface flux of the paired form: FP64 Gauss-point states in, the
   GKS solve in paired-FP32 arithmetic, FP64 fluxes out.  Instantiated in
   cgks_stage_pair.cu (Cartesian) and cgks_stage_pair_curvi.cu. */
template <int DIM, bool CURVI>
void launch_flux_pair(cgks_ctx* ctx, const double* gpL, const double* gpR, double* flux);
extern template void launch_flux_pair<2, false>(cgks_ctx*, const double*, const double*, double*);
extern template void launch_flux_pair<3, false>(cgks_ctx*, const double*, const double*, double*);
extern template void launch_flux_pair<2, true>(cgks_ctx*, const double*, const double*, double*);
extern template void launch_flux_pair<3, true>(cgks_ctx*, const double*, const double*, double*);

/* the reconstruction of the paired form on Cartesian meshes: FP64 averages
   and derivatives in, the linear maps in paired FP32, FP64 Gauss-point
   states out.  Instantiated in cgks_recon_pair.cu. */
template <int DIM, bool WALL>
void launch_recon_pair(cgks_ctx* ctx, int in, int record_chi);
extern template void launch_recon_pair<2, false>(cgks_ctx*, int, int);
extern template void launch_recon_pair<2, true>(cgks_ctx*, int, int);
extern template void launch_recon_pair<3, false>(cgks_ctx*, int, int);
extern template void launch_recon_pair<3, true>(cgks_ctx*, int, int);

#endif
