/*
 * Batched ensemble (include/cgks.h, cgks_batch_*): many independent meshes of
 * uneven size advance together.  All cases share one set of concatenated
 * device arrays and one launch per kernel and phase (cgks_batch_kernels.cuh);
 * a run of nsteps S2O4 steps is captured once as a CUDA graph and replayed,
 * so a whole advance is one graph launch.  Each case keeps its own time step,
 * time, boundaries and physics.  The autotuner times the candidate tile
 * shapes and grid sizes of each phase on the batch itself and keeps the
 * fastest.
 */
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/cgks.h"
#include "cgks_batch_kernels.cuh"

using namespace cgks;

/* defined in cgks.cu */
cgks_status selector_upload(void** buf, cgks::SelectorDev* sd, const float* params, float thr_skip, float thr_lo,
                            cudaStream_t stream);

namespace {

struct List {
  int* d = nullptr; /* device: start[nentry + 1] then cases[nentry] */
  int nentry = 0, ntile = 0;
  TileList view() const {
    TileList t;
    t.start = d;
    t.cases = d ? d + nentry + 1 : nullptr;
    t.nentry = nentry;
    t.ntile = ntile;
    return t;
  }
};

struct Graph {
  int nsteps;
  cudaGraphExec_t exec;
};

long cdivl(long a, long b) { return (a + b - 1) / b; }

}  // namespace

struct cgks_batch {
  int ncase = 0, dim = 2, prec = 0, nv = 4, nf = 7, gpf = 2;
  int nsm = 152;
  cudaStream_t stream = nullptr;
  std::vector<cgks_mesh_desc> desc;
  std::vector<BatchCase> hcase;
  BatchCase* dcase = nullptr;
  long ncell = 0, nplane = 0;
  bool wall = false;
  /* concatenated arrays */
  double* avg = nullptr;  /* avg0 | avg1 | stash, nv * ncell each */
  void* der = nullptr;    /* der0 | der1 | stash, (nf - 1) * nv * ncell each, in T */
  float* pairs = nullptr; /* FP32 form: hi0 | lo0 | hi1 | lo1 */
  void* gp = nullptr;     /* gpL | gpR */
  void* flux = nullptr;
  void* fxb = nullptr;
  DtState* dts = nullptr;
  int* st = nullptr;
  double* staging = nullptr; /* public layout of the largest case */
  double* bcq = nullptr;     /* inflow states per case (cgks::BCQ_DOUBLES each) */
  List l_recon[2], l_flux, l_fbnd, l_upd, l_dt;
  cgks_batch_tiles tiles{};
  std::vector<Graph> graphs;
  SelectorDev sel{};
  void* sel_buf = nullptr;
  std::string err;
};

static cgks_status bfail(cgks_batch* b, cgks_status s, const char* fmt, ...) {
  if (b) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    b->err = buf;
  }
  return s;
}

#define BCK(call)                                                                                    \
  do {                                                                                               \
    cudaError_t e_ = (call);                                                                         \
    if (e_ != cudaSuccess) return bfail(b, CGKS_ECUDA, "%s: %s", #call, cudaGetErrorString(e_));     \
  } while (0)

/* ---- tile lists ---------------------------------------------------------- */
/* work items of case k in a phase, cut into tiles of `per` items; cases with
   no items are left out */
template <class F>
static cgks_status build_list(cgks_batch* b, List& L, F tiles_of) {
  std::vector<int> start, cases;
  long tot = 0;
  for (int k = 0; k < b->ncase; ++k) {
    const long nt = tiles_of(k);
    if (nt <= 0) continue;
    start.push_back((int)tot);
    cases.push_back(k);
    tot += nt;
  }
  if (tot > 0x7fffffffL) return bfail(b, CGKS_ETOOLARGE, "more than 2^31 tiles in one phase");
  start.push_back((int)tot);
  cudaFree(L.d);
  L.d = nullptr;
  L.nentry = (int)cases.size();
  L.ntile = (int)tot;
  if (L.nentry == 0) return CGKS_OK;
  std::vector<int> h(start);
  h.insert(h.end(), cases.begin(), cases.end());
  BCK(cudaMalloc((void**)&L.d, sizeof(int) * h.size()));
  BCK(cudaMemcpyAsync(L.d, h.data(), sizeof(int) * h.size(), cudaMemcpyHostToDevice, b->stream));
  BCK(cudaStreamSynchronize(b->stream));
  return CGKS_OK;
}

static bool case_has_wall(const cgks_mesh_desc& d) {
  for (int f = 0; f < 2 * d.dim; ++f)
    if (d.bc[f] >= CGKS_BC_SLIP_WALL) return true;
  return false;
}

static cgks_status build_lists(cgks_batch* b) {
  const cgks_batch_tiles& t = b->tiles;
  cgks_status s;
  for (int w = 0; w < 2; ++w) {
    s = build_list(b, b->l_recon[w], [&](int k) -> long {
      const DevGeo& g = b->hcase[k].g;
      if (case_has_wall(b->desc[k]) != (w == 1)) return 0;
      return cdivl(g.n[0], t.tile_x) * cdivl(g.n[1], t.tile_y) * g.n[2];
    });
    if (s != CGKS_OK) return s;
  }
  const int gpf = b->gpf, dim = b->dim, nv = b->nv;
  s = build_list(b, b->l_flux, [&](int k) { return cdivl((long)dim * gpf * b->hcase[k].g.ncell, 128); });
  if (s != CGKS_OK) return s;
  s = build_list(b, b->l_fbnd, [&](int k) { return cdivl(2L * dim * gpf * b->hcase[k].g.nplane, 128); });
  if (s != CGKS_OK) return s;
  s = build_list(b, b->l_upd, [&](int k) { return cdivl((long)nv * b->hcase[k].g.ncell, 128); });
  if (s != CGKS_OK) return s;
  return build_list(b, b->l_dt, [&](int k) { return cdivl(b->hcase[k].g.ncell, 256); });
}

/* grid of a phase: blocks_per_sm > 0 makes it persistent (that many blocks
   per SM, never more than there are tiles); 0 gives one block per tile */
static int grid_of(const cgks_batch* b, const List& L, int blocks_per_sm) {
  if (L.ntile == 0) return 0;
  if (blocks_per_sm <= 0) return L.ntile;
  return std::max(1, std::min(L.ntile, blocks_per_sm * b->nsm));
}

/* ---- one step ------------------------------------------------------------ */
template <typename T, int DIM>
static BatchArrays<T> arrays(cgks_batch* b, int stage) {
  const long na = (long)b->nv * b->ncell, nd = (long)(b->nf - 1) * b->nv * b->ncell;
  const int in = stage == 1 ? 0 : 1, out = stage == 1 ? 1 : 0;
  T* der = (T*)b->der;
  T* gp = (T*)b->gp;
  const long ngp = (long)DIM * Sz<DIM>::GPF * Sz<DIM>::NV * (1 + DIM) * b->ncell;
  BatchArrays<T> A;
  A.avg_in = b->avg + in * na;
  A.avg_out = b->avg + out * na;
  A.savg = b->avg + 2 * na;
  A.der_in = der + in * nd;
  A.der_out = der + out * nd;
  A.sder = der + 2 * nd;
  A.avh_in = b->pairs ? b->pairs + (2 * in) * na : nullptr;
  A.avl_in = b->pairs ? b->pairs + (2 * in + 1) * na : nullptr;
  A.avh_out = b->pairs ? b->pairs + (2 * out) * na : nullptr;
  A.avl_out = b->pairs ? b->pairs + (2 * out + 1) * na : nullptr;
  A.gpL = gp;
  A.gpR = gp + ngp;
  A.flux = (T*)b->flux;
  A.fxb = (T*)b->fxb;
  A.dts = b->dts;
  A.st = b->st;
  return A;
}

template <typename T, int DIM>
static void enqueue_dt(cgks_batch* b) {
  const int nc = b->ncase;
  kb_dt_reset<<<(int)cdivl(nc, 128), 128, 0, b->stream>>>(b->dts, nc);
  const int g = grid_of(b, b->l_dt, b->tiles.update_blocks);
  if (b->pairs) {
    kb_dt_screen<DIM, float><<<g, 256, 0, b->stream>>>(b->dcase, b->l_dt.view(), b->pairs, b->dts);
    kb_dt_rate<DIM, float><<<g, 256, 0, b->stream>>>(b->dcase, b->l_dt.view(), b->pairs, b->avg, b->dts);
  } else {
    kb_dt_screen<DIM, double><<<g, 256, 0, b->stream>>>(b->dcase, b->l_dt.view(), b->avg, b->dts);
    kb_dt_rate<DIM, double><<<g, 256, 0, b->stream>>>(b->dcase, b->l_dt.view(), b->avg, b->avg, b->dts);
  }
  kb_dt_final<<<(int)cdivl(nc, 128), 128, 0, b->stream>>>(b->dcase, b->dts, b->st, nc);
}

/* phases of one stage: 0 reconstruction, 1 interface flux, 2 update; -1 all */
template <typename T, int DIM>
static void enqueue_stage(cgks_batch* b, int stage, int phase = -1) {
  const BatchArrays<T> A = arrays<T, DIM>(b, stage);
  const cgks_batch_tiles& t = b->tiles;
  if (phase < 0 || phase == 0) {
    const int tpb = 128;
    if (b->l_recon[0].ntile)
      kb_recon<T, DIM, false><<<grid_of(b, b->l_recon[0], t.recon_blocks), tpb, 0, b->stream>>>(
          b->dcase, b->l_recon[0].view(), A, t.tile_x, t.tile_y, b->sel);
    if (b->l_recon[1].ntile)
      kb_recon<T, DIM, true><<<grid_of(b, b->l_recon[1], t.recon_blocks), tpb, 0, b->stream>>>(
          b->dcase, b->l_recon[1].view(), A, t.tile_x, t.tile_y, b->sel);
  }
  if (phase < 0 || phase == 1) {
    kb_flux<T, DIM><<<grid_of(b, b->l_flux, t.flux_blocks), 128, 0, b->stream>>>(b->dcase, b->l_flux.view(), A);
    if (b->l_fbnd.ntile)
      kb_flux_bnd<T, DIM><<<grid_of(b, b->l_fbnd, t.flux_blocks), 128, 0, b->stream>>>(b->dcase,
                                                                                       b->l_fbnd.view(), A);
  }
  if (phase < 0 || phase == 2)
    kb_update<T, DIM><<<grid_of(b, b->l_upd, t.update_blocks), 128, 0, b->stream>>>(b->dcase, b->l_upd.view(), A,
                                                                                    stage);
}

template <typename T, int DIM>
static void enqueue_step(cgks_batch* b) {
  enqueue_dt<T, DIM>(b);
  enqueue_stage<T, DIM>(b, 1);
  enqueue_stage<T, DIM>(b, 2);
  kb_time_advance<<<(int)cdivl(b->ncase, 128), 128, 0, b->stream>>>(b->dts, b->ncase);
}

static void enqueue_steps(cgks_batch* b, int nsteps) {
  for (int s = 0; s < nsteps; ++s) {
    if (b->prec == 0) {
      if (b->dim == 3) enqueue_step<double, 3>(b);
      else enqueue_step<double, 2>(b);
    } else {
      if (b->dim == 3) enqueue_step<float, 3>(b);
      else enqueue_step<float, 2>(b);
    }
  }
}

static void drop_graphs(cgks_batch* b) {
  for (auto& g : b->graphs) cudaGraphExecDestroy(g.exec);
  b->graphs.clear();
}

static cgks_status check_batch_status(cgks_batch* b) {
  int st[ST_N];
  BCK(cudaMemcpyAsync(st, b->st, sizeof st, cudaMemcpyDeviceToHost, b->stream));
  BCK(cudaStreamSynchronize(b->stream));
  if (st[ST_NONPHYS] || st[ST_FLUX] || st[ST_DT]) {
    int z[ST_N] = {0, st[ST_FALLBACK], 0, 0};
    BCK(cudaMemcpyAsync(b->st, z, sizeof z, cudaMemcpyHostToDevice, b->stream));
    BCK(cudaStreamSynchronize(b->stream));
    return bfail(b, CGKS_ENONPHYS, "non-physical state in some case (recon %d, interface %d, cell %d)",
                 st[ST_NONPHYS], st[ST_FLUX], st[ST_DT]);
  }
  return CGKS_OK;
}

extern "C" {

cgks_status cgks_batch_create(const cgks_mesh_desc* descs, int ncase, void* stream, cgks_batch** out) {
  if (!descs || ncase < 1 || !out) return CGKS_EINVAL;
  const int dim = descs[0].dim, prec = descs[0].precision;
  for (int k = 0; k < ncase; ++k) {
    const cgks_mesh_desc& d = descs[k];
    if (d.dim != dim || d.precision != prec) return CGKS_EINVAL;
    if (d.dim != 2 && d.dim != 3) return CGKS_EINVAL;
    if (prec != 0 && prec != 1) return CGKS_EUNSUPPORTED;
    if (d.nodes) return CGKS_EUNSUPPORTED; /* uniform boxes only */
    for (int a = 0; a < dim; ++a)
      if (d.n[a] < 3) return CGKS_EINVAL;
    for (int f = 0; f < 2 * dim; ++f) {
      if (d.bc[f] < CGKS_BC_PERIODIC || d.bc[f] > CGKS_BC_INFLOW) return CGKS_EINVAL;
      if ((d.bc[f] == CGKS_BC_PERIODIC) != (d.bc[f ^ 1] == CGKS_BC_PERIODIC)) return CGKS_EINVAL;
    }
    if (!(d.gamma > 1.0) || d.mu < 0.0 || !(d.cfl > 0.0) || d.tau_mode < 0 || d.tau_mode > 2) return CGKS_EINVAL;
  }
  cgks_batch* b = new cgks_batch();
  b->ncase = ncase;
  b->dim = dim;
  b->prec = prec;
  b->nv = dim + 2;
  b->gpf = dim == 3 ? 4 : 2;
  b->nf = 1 + dim + dim * b->gpf;
  b->stream = (cudaStream_t)stream;
  b->desc.assign(descs, descs + ncase);
  int dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, dev);
  b->hcase.resize(ncase);
  long maxcell = 0;
  for (int k = 0; k < ncase; ++k) {
    const cgks_mesh_desc& d = descs[k];
    BatchCase& C = b->hcase[k];
    memset(&C, 0, sizeof C);
    DevGeo& g = C.g;
    for (int a = 0; a < 3; ++a) {
      g.n[a] = a < dim ? d.n[a] : 1;
      g.h[a] = a < dim ? (d.hi[a] - d.lo[a]) / d.n[a] : 1.0;
      g.ih[a] = 1.0 / g.h[a];
      g.hf[a] = (float)g.h[a];
      g.ihf[a] = (float)g.ih[a];
    }
    g.ncell = (long)g.n[0] * g.n[1] * g.n[2];
    g.curvi = 0;
    g.met = nullptr;
    g.rmet = nullptr;
    g.bcm = 0;
    g.nplane = 0;
    for (int f = 0; f < 2 * dim; ++f) {
      g.bcm |= d.bc[f] << (3 * f);
      if (d.bc[f] != CGKS_BC_PERIODIC) g.nplane = std::max(g.nplane, g.ncell / g.n[f / 2]);
    }
    if (case_has_wall(d)) b->wall = true;
    Phys& ph = C.ph;
    ph.gamma = d.gamma;
    ph.mu = d.mu;
    ph.prandtl = d.prandtl;
    ph.cfl = d.cfl;
    ph.c_chi = d.c_chi > 0.0 ? d.c_chi : 100.0;
    ph.tau_mode = d.tau_mode;
    ph.linear = d.linear;
    ph.gammaf = (float)ph.gamma;
    ph.muf = (float)ph.mu;
    ph.prandtlf = (float)ph.prandtl;
    ph.c_chif = (float)ph.c_chi;
    ph.prfix = (ph.mu > 0.0 && ph.prandtl > 0.0 && ph.prandtl != 1.0) ? 1 : 0;
    C.cell0 = b->ncell;
    C.plane0 = b->nplane;
    b->ncell += g.ncell;
    b->nplane += g.nplane;
    maxcell = std::max(maxcell, g.ncell);
  }
  const long N = b->ncell, nv = b->nv, nd = (long)(b->nf - 1) * nv;
  const size_t rsz = prec == 0 ? sizeof(double) : sizeof(float);
  const long ngp = (long)dim * b->gpf * nv * (1 + dim), nfx = (long)dim * b->gpf * 6 * nv;
#define BALLOC(p, sz)                                     \
  do {                                                    \
    if (cudaMalloc((void**)&(p), (sz)) != cudaSuccess) {  \
      cudaGetLastError();                                 \
      cgks_batch_destroy(b);                              \
      return CGKS_ENOMEM;                                 \
    }                                                     \
  } while (0)
  BALLOC(b->dcase, sizeof(BatchCase) * ncase);
  BALLOC(b->avg, sizeof(double) * 3 * nv * N);
  BALLOC(b->der, rsz * 3 * nd * N);
  if (prec == 1) BALLOC(b->pairs, sizeof(float) * 4 * nv * N);
  BALLOC(b->gp, rsz * 2 * ngp * N);
  BALLOC(b->flux, rsz * nfx * N);
  BALLOC(b->fxb, rsz * nfx * std::max(b->nplane, 1L));
  BALLOC(b->dts, sizeof(DtState) * ncase);
  BALLOC(b->st, sizeof(int) * ST_N);
  BALLOC(b->staging, sizeof(double) * (nd + nv) * maxcell);
  BALLOC(b->bcq, sizeof(double) * cgks::BCQ_DOUBLES * ncase);
#undef BALLOC
  {
    std::vector<double> hq(cgks::BCQ_DOUBLES * (size_t)ncase);
    for (int k = 0; k < ncase; ++k) {
      cgks::pack_bcq(descs[k].bc_state, &hq[cgks::BCQ_DOUBLES * (size_t)k]);
      b->hcase[k].g.bcq = b->bcq + cgks::BCQ_DOUBLES * (size_t)k;
    }
    if (cudaMemcpy(b->bcq, hq.data(), sizeof(double) * hq.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
      cgks_batch_destroy(b);
      return CGKS_ECUDA;
    }
  }
  std::vector<DtState> d0(ncase);
  for (int k = 0; k < ncase; ++k) {
    memset(&d0[k], 0, sizeof(DtState));
    d0[k].dt_fixed = descs[k].dt_fixed;
  }
  cgks_status s = CGKS_OK;
  if (cudaMemcpyAsync(b->dcase, b->hcase.data(), sizeof(BatchCase) * ncase, cudaMemcpyHostToDevice, b->stream) !=
          cudaSuccess ||
      cudaMemcpyAsync(b->dts, d0.data(), sizeof(DtState) * ncase, cudaMemcpyHostToDevice, b->stream) !=
          cudaSuccess ||
      cudaMemsetAsync(b->st, 0, sizeof(int) * ST_N, b->stream) != cudaSuccess ||
      cudaMemsetAsync(b->avg, 0, sizeof(double) * 3 * nv * N, b->stream) != cudaSuccess ||
      cudaMemsetAsync(b->der, 0, rsz * 3 * nd * N, b->stream) != cudaSuccess ||
      (b->pairs && cudaMemsetAsync(b->pairs, 0, sizeof(float) * 4 * nv * N, b->stream) != cudaSuccess) ||
      cudaStreamSynchronize(b->stream) != cudaSuccess)
    s = CGKS_ECUDA;
  /* default tiles until the autotuner runs */
  b->tiles.tile_x = 32;
  b->tiles.tile_y = 4;
  b->tiles.recon_blocks = 0;
  b->tiles.flux_blocks = 0;
  b->tiles.update_blocks = 0;
  if (s == CGKS_OK) s = build_lists(b);
  if (s != CGKS_OK) {
    cgks_batch_destroy(b);
    return s;
  }
  *out = b;
  return CGKS_OK;
}

void cgks_batch_destroy(cgks_batch* b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  else cudaDeviceSynchronize();
  drop_graphs(b);
  List* ls[] = {&b->l_recon[0], &b->l_recon[1], &b->l_flux, &b->l_fbnd, &b->l_upd, &b->l_dt};
  for (List* l : ls) cudaFree(l->d);
  cudaFree(b->dcase);
  cudaFree(b->avg);
  cudaFree(b->der);
  cudaFree(b->pairs);
  cudaFree(b->gp);
  cudaFree(b->flux);
  cudaFree(b->fxb);
  cudaFree(b->dts);
  cudaFree(b->st);
  cudaFree(b->staging);
  cudaFree(b->bcq);
  cudaFree(b->sel_buf);
  delete b;
}

int cgks_batch_num_cases(const cgks_batch* b) { return b ? b->ncase : -1; }
long cgks_batch_num_cells(const cgks_batch* b) { return b ? b->ncell : -1; }

cgks_status cgks_batch_set_state(cgks_batch* b, int k, const double* src, int is_device, double t) {
  if (!b || !src || k < 0 || k >= b->ncase) return CGKS_EINVAL;
  const BatchCase& C = b->hcase[k];
  const long N = C.g.ncell, nv = b->nv, nd = (long)(b->nf - 1) * nv;
  const long na_tot = nv * b->ncell;
  const cudaMemcpyKind kind = is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  if (b->prec == 0) {
    BCK(cudaMemcpyAsync(b->avg + nv * C.cell0, src, sizeof(double) * nv * N, kind, b->stream));
    BCK(cudaMemcpyAsync((double*)b->der + nd * C.cell0, src + nv * N, sizeof(double) * nd * N, kind, b->stream));
  } else {
    BCK(cudaMemcpyAsync(b->staging, src, sizeof(double) * (nv + nd) * N, kind, b->stream));
    k_split<float><<<(int)cdivl((nv + nd) * N, 256), 256, 0, b->stream>>>(
        b->staging, b->avg + nv * C.cell0, b->pairs + nv * C.cell0, b->pairs + na_tot + nv * C.cell0,
        (float*)b->der + nd * C.cell0, nv * N, nd * N);
    BCK(cudaGetLastError());
  }
  DtState h;
  BCK(cudaMemcpyAsync(&h, b->dts + k, sizeof h, cudaMemcpyDeviceToHost, b->stream));
  BCK(cudaStreamSynchronize(b->stream));
  h.t = t;
  cgks::set_dt(h, 0.0);
  h.t_end = 0.0;
  BCK(cudaMemcpyAsync(b->dts + k, &h, sizeof h, cudaMemcpyHostToDevice, b->stream));
  BCK(cudaStreamSynchronize(b->stream));
  return CGKS_OK;
}

cgks_status cgks_batch_get_state(cgks_batch* b, int k, double* dst, int is_device, double* t) {
  if (!b || !dst || k < 0 || k >= b->ncase) return CGKS_EINVAL;
  const BatchCase& C = b->hcase[k];
  const long N = C.g.ncell, nv = b->nv, nd = (long)(b->nf - 1) * nv;
  const cudaMemcpyKind kind = is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (b->prec == 0) {
    BCK(cudaMemcpyAsync(dst, b->avg + nv * C.cell0, sizeof(double) * nv * N, kind, b->stream));
    BCK(cudaMemcpyAsync(dst + nv * N, (double*)b->der + nd * C.cell0, sizeof(double) * nd * N, kind, b->stream));
  } else {
    k_join<float><<<(int)cdivl((nv + nd) * N, 256), 256, 0, b->stream>>>(b->avg + nv * C.cell0,
                                                                          (const float*)b->der + nd * C.cell0,
                                                                          b->staging, nv * N, nd * N);
    BCK(cudaGetLastError());
    BCK(cudaMemcpyAsync(dst, b->staging, sizeof(double) * (nv + nd) * N, kind, b->stream));
  }
  if (t) {
    DtState h;
    BCK(cudaMemcpyAsync(&h, b->dts + k, sizeof h, cudaMemcpyDeviceToHost, b->stream));
    BCK(cudaStreamSynchronize(b->stream));
    *t = h.t;
  }
  BCK(cudaStreamSynchronize(b->stream));
  return CGKS_OK;
}

cgks_status cgks_batch_times(cgks_batch* b, double* t, double* dt_last) {
  if (!b) return CGKS_EINVAL;
  std::vector<DtState> h(b->ncase);
  BCK(cudaMemcpyAsync(h.data(), b->dts, sizeof(DtState) * b->ncase, cudaMemcpyDeviceToHost, b->stream));
  BCK(cudaStreamSynchronize(b->stream));
  for (int k = 0; k < b->ncase; ++k) {
    if (t) t[k] = h[k].t;
    if (dt_last) dt_last[k] = h[k].dt;
  }
  return CGKS_OK;
}

cgks_status cgks_batch_step(cgks_batch* b, int nsteps, int use_graph) {
  if (!b || nsteps < 0) return CGKS_EINVAL;
  if (nsteps == 0) return CGKS_OK;
  if (!use_graph) {
    enqueue_steps(b, nsteps);
    BCK(cudaGetLastError());
    return check_batch_status(b);
  }
  cudaGraphExec_t exec = nullptr;
  for (auto& g : b->graphs)
    if (g.nsteps == nsteps) exec = g.exec;
  if (!exec) {
    if (!b->stream) return bfail(b, CGKS_EINVAL, "graph capture needs a non-default stream");
    cudaGraph_t graph = nullptr;
    BCK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    enqueue_steps(b, nsteps);
    cudaError_t e = cudaStreamEndCapture(b->stream, &graph);
    if (e != cudaSuccess) return bfail(b, CGKS_ECUDA, "graph capture: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return bfail(b, CGKS_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
    b->graphs.push_back({nsteps, exec});
  }
  BCK(cudaGraphLaunch(exec, b->stream));
  return check_batch_status(b);
}

cgks_status cgks_batch_get_tiles(const cgks_batch* b, cgks_batch_tiles* out) {
  if (!b || !out) return CGKS_EINVAL;
  *out = b->tiles;
  return CGKS_OK;
}

cgks_status cgks_batch_set_tiles(cgks_batch* b, const cgks_batch_tiles* t) {
  if (!b || !t) return CGKS_EINVAL;
  if (t->tile_x < 1 || t->tile_y < 1 || t->tile_x * t->tile_y > 128 || t->recon_blocks < 0 || t->flux_blocks < 0 ||
      t->update_blocks < 0 || t->recon_blocks > 64 || t->flux_blocks > 64 || t->update_blocks > 64)
    return CGKS_EINVAL;
  const bool relist = t->tile_x != b->tiles.tile_x || t->tile_y != b->tiles.tile_y;
  b->tiles = *t;
  drop_graphs(b);
  return relist ? build_lists(b) : CGKS_OK;
}

/* Autotuner.  Times, on the batch's own data, each phase of stage 1 (which
   reads the current state and writes only the intermediate arrays, so the
   state is left as it was) under each candidate: tile shapes and persistent
   or one-block-per-tile grids for the reconstruction, grid sizes for the
   interface flux and the update.  Keeps the fastest per phase. */
cgks_status cgks_batch_tune(cgks_batch* b, int reps, cgks_batch_tiles* chosen, double* ms_best) {
  if (!b) return CGKS_EINVAL;
  if (reps < 1) reps = 3;
  if (!b->stream) return bfail(b, CGKS_EINVAL, "the autotuner needs a non-default stream");
  cudaEvent_t e0, e1;
  BCK(cudaEventCreate(&e0));
  BCK(cudaEventCreate(&e1));
  auto run_dt = [&]() {
    if (b->prec == 0) {
      if (b->dim == 3) enqueue_dt<double, 3>(b);
      else enqueue_dt<double, 2>(b);
    } else {
      if (b->dim == 3) enqueue_dt<float, 3>(b);
      else enqueue_dt<float, 2>(b);
    }
  };
  auto run_phase = [&](int phase) {
    if (b->prec == 0) {
      if (b->dim == 3) enqueue_stage<double, 3>(b, 1, phase);
      else enqueue_stage<double, 2>(b, 1, phase);
    } else {
      if (b->dim == 3) enqueue_stage<float, 3>(b, 1, phase);
      else enqueue_stage<float, 2>(b, 1, phase);
    }
  };
  auto time_phase = [&](int phase, float* ms) -> cgks_status {
    run_phase(phase); /* warm-up */
    BCK(cudaEventRecord(e0, b->stream));
    for (int r = 0; r < reps; ++r) run_phase(phase);
    BCK(cudaEventRecord(e1, b->stream));
    BCK(cudaEventSynchronize(e1));
    BCK(cudaGetLastError());
    BCK(cudaEventElapsedTime(ms, e0, e1));
    *ms /= reps;
    return CGKS_OK;
  };
  run_dt();
  for (int ph = 0; ph < 3; ++ph) run_phase(ph); /* inputs of every phase */
  cgks_batch_tiles best = b->tiles;
  cgks_status s = CGKS_OK;
  float total = 0.f;
  /* reconstruction: tile shape x grid */
  {
    const int shapes[][2] = {{128, 1}, {64, 2}, {32, 4}, {16, 8}, {8, 16}};
    const int grids[] = {0, 1, 2, 3, 4};
    float bm = 1e30f;
    for (auto& sh : shapes) {
      if (sh[1] > 1 && b->dim >= 2) {
        bool fits = false; /* a shape taller than every case is pointless */
        for (auto& C : b->hcase) fits |= C.g.n[1] >= sh[1];
        if (!fits) continue;
      }
      for (int gsz : grids) {
        cgks_batch_tiles t = best;
        t.tile_x = sh[0];
        t.tile_y = sh[1];
        t.recon_blocks = gsz;
        if ((s = cgks_batch_set_tiles(b, &t)) != CGKS_OK) goto done;
        float ms;
        if ((s = time_phase(0, &ms)) != CGKS_OK) goto done;
        if (ms < bm) {
          bm = ms;
          best.tile_x = t.tile_x;
          best.tile_y = t.tile_y;
          best.recon_blocks = t.recon_blocks;
        }
      }
    }
    if ((s = cgks_batch_set_tiles(b, &best)) != CGKS_OK) goto done;
    total += bm;
  }
  /* interface flux and update: grid sizes */
  for (int ph = 1; ph <= 2; ++ph) {
    const int grids[] = {0, 1, 2, 3, 4, 6, 8};
    float bm = 1e30f;
    int bg = 0;
    for (int gsz : grids) {
      cgks_batch_tiles t = best;
      if (ph == 1) t.flux_blocks = gsz;
      else t.update_blocks = gsz;
      if ((s = cgks_batch_set_tiles(b, &t)) != CGKS_OK) goto done;
      float ms;
      if ((s = time_phase(ph, &ms)) != CGKS_OK) goto done;
      if (ms < bm) {
        bm = ms;
        bg = gsz;
      }
    }
    if (ph == 1) best.flux_blocks = bg;
    else best.update_blocks = bg;
    total += bm;
  }
  s = cgks_batch_set_tiles(b, &best);
done:
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (s == CGKS_OK) {
    if (chosen) *chosen = b->tiles;
    if (ms_best) *ms_best = total;
  }
  return s;
}

cgks_status cgks_batch_set_selector(cgks_batch* b, const float* params, float thr_skip, float thr_lo) {
  if (!b) return CGKS_EINVAL;
  drop_graphs(b); /* the graphs hold the selector by value */
  if (!params) {
    b->sel.on = 0;
    return CGKS_OK;
  }
  if (!(thr_lo <= thr_skip)) return CGKS_EINVAL;
  cgks_status s = selector_upload(&b->sel_buf, &b->sel, params, thr_skip, thr_lo, b->stream);
  if (s != CGKS_OK) return bfail(b, s, "selector upload failed");
  return CGKS_OK;
}

cgks_status cgks_batch_selector_stats(cgks_batch* b, unsigned long long* skips, unsigned long long* unsure) {
  if (!b) return CGKS_EINVAL;
  unsigned long long h[2 * SEL_SLOTS] = {0};
  if (b->sel.counts) {
    BCK(cudaMemcpyAsync(h, b->sel.counts, sizeof h, cudaMemcpyDeviceToHost, b->stream));
    BCK(cudaStreamSynchronize(b->stream));
  }
  unsigned long long a = 0, u = 0;
  for (int i = 0; i < SEL_SLOTS; ++i) {
    a += h[2 * i];
    u += h[2 * i + 1];
  }
  if (skips) *skips = a;
  if (unsure) *unsure = u;
  return CGKS_OK;
}

cgks_status cgks_batch_last_error(const cgks_batch* b, char* msg, size_t cap) {
  if (!b || !msg || cap == 0) return CGKS_EINVAL;
  snprintf(msg, cap, "%s", b->err.c_str());
  return CGKS_OK;
}

}  // extern "C"
