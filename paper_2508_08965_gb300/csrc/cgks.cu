/*
 * Host side of the CGKS-5 C-ABI (include/cgks.h): context, device memory,
 * step orchestration and per-kernel event timing.  All arithmetic of the
 * scheme runs in the kernels of cgks_kernels.cuh.
 */
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <utility>

#include <cstdarg>
#include <cstdio>
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/cgks.h"
#include "cgks_kernels.cuh"
#include "cgks_ctx.h"

using namespace cgks;
using namespace cgks_host;

static cgks_status fail(cgks_ctx* c, cgks_status s, const char* fmt, ...) {
  if (c) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    c->err = buf;
  }
  return s;
}

#define CK(call)                                                                          \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess) return fail(ctx, CGKS_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)


static void prof_fold(cgks_ctx* ctx) {
  Prof& p = ctx->prof;
  if (p.rec.empty()) return;
  cudaStreamSynchronize(ctx->stream);
  for (auto& r : p.rec) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, p.pool[r.second], p.pool[r.second + 1]);
    p.ms[r.first] += ms;
    p.launches[r.first] += 1;
  }
  p.rec.clear();
}

template <int DIM>
static cgks_status run_stage(cgks_ctx* ctx, int stage) {
  const bool cv = ctx->geo.curvi != 0;
  const bool wall = ctx->walls;
  if (ctx->prec == 0) {
    if (cv) launch_stage<double, DIM, true, false>(ctx, stage);
    else if (wall) launch_stage<double, DIM, false, true>(ctx, stage);
    else launch_stage<double, DIM, false, false>(ctx, stage);
  } else {
    if (cv) launch_stage<float, DIM, true, false>(ctx, stage);
    else if (wall) launch_stage<float, DIM, false, true>(ctx, stage);
    else launch_stage<float, DIM, false, false>(ctx, stage);
  }
  CK(cudaGetLastError());
  return CGKS_OK;
}

template <int DIM>
static cgks_status run_dt(cgks_ctx* ctx, const double* avg, const float* avh, int in_step) {
  prof_begin(ctx, KID_DT);
  const long nb = cdiv(ctx->ncell, 256);
  k_dt_reset<<<1, 1, 0, ctx->stream>>>(ctx->dts);
  if (avh) {
    k_dt_screen<DIM, float><<<nb, 256, 0, ctx->stream>>>(ctx->geo, ctx->ph, avh, ctx->dts);
    k_dt_rate<DIM, float><<<nb, 256, 0, ctx->stream>>>(ctx->geo, ctx->ph, avh, avg, ctx->dts);
  } else {
    k_dt_screen<DIM, double><<<nb, 256, 0, ctx->stream>>>(ctx->geo, ctx->ph, avg, ctx->dts);
    k_dt_rate<DIM, double><<<nb, 256, 0, ctx->stream>>>(ctx->geo, ctx->ph, avg, avg, ctx->dts);
  }
  k_dt_final<<<1, 1, 0, ctx->stream>>>(ctx->ph, ctx->dts, ctx->st, in_step);
  prof_end(ctx);
  CK(cudaGetLastError());
  return CGKS_OK;
}

/* The state arrays of index 0 hold the current state; both stages write
   into those of index 1 (stage 2 reads only the stash, so it can overwrite
   U*), and the two sets swap roles after every step.  A step thus never
   overwrites its own input, which is what lets a failed call return the
   last good state (cgks_step). */
static void swap_state(cgks_ctx* ctx) {
  std::swap(ctx->avg[0], ctx->avg[1]);
  std::swap(ctx->der[0], ctx->der[1]);
  std::swap(ctx->avh[0], ctx->avh[1]);
  std::swap(ctx->avl[0], ctx->avl[1]);
  if (ctx->prec == 0) std::swap(ctx->U, ctx->Us); /* the public-layout state is avg[0], der[0] */
}

template <int DIM>
static cgks_status run_step(cgks_ctx* ctx) {
  cgks_status s;
  if ((s = run_dt<DIM>(ctx, ctx->avg[0], ctx->prec ? ctx->avh[0] : nullptr, 1)) != CGKS_OK) return s;
  if ((s = run_stage<DIM>(ctx, 1)) != CGKS_OK) return s;
  if ((s = run_stage<DIM>(ctx, 2)) != CGKS_OK) return s;
  k_time_advance<<<1, 1, 0, ctx->stream>>>(ctx->dts, ctx->st);
  CK(cudaGetLastError());
  swap_state(ctx);
  return CGKS_OK;
}

/* FP32 form: staging (public layout, U) <-> internal arrays of the current state */
static cgks_status split_in(cgks_ctx* ctx) {
  if (ctx->prec == 0) return CGKS_OK;
  const long navg = (long)ctx->nv * ctx->ncell, nder = (long)(ctx->nf - 1) * ctx->nv * ctx->ncell;
  k_split<float><<<cdiv(navg + nder, 256), 256, 0, ctx->stream>>>(ctx->U, ctx->avg[0], ctx->avh[0], ctx->avl[0],
                                                                  (float*)ctx->der[0], navg, nder);
  CK(cudaGetLastError());
  return CGKS_OK;
}
static cgks_status join_out(cgks_ctx* ctx) {
  if (ctx->prec == 0) return CGKS_OK;
  const long navg = (long)ctx->nv * ctx->ncell, nder = (long)(ctx->nf - 1) * ctx->nv * ctx->ncell;
  k_join<float><<<cdiv(navg + nder, 256), 256, 0, ctx->stream>>>(ctx->avg[0], (const float*)ctx->der[0], ctx->U, navg,
                                                                 nder);
  CK(cudaGetLastError());
  return CGKS_OK;
}

extern "C" {

/* The tensor map of a Gauss-point state array (gpL or gpR) for the flux
   kernel's TMA tiles: a 2-D array [row][cell] of N cells per row and
   dim * GPF * NV * (1 + dim) rows (row = (ax * GPF + k) * NQ + q), boxes of
   NQ rows x 128 cells.  The encoder comes from the driver through the
   runtime (no link against the driver library); false if it is not there
   or refuses the map. */
static bool encode_gp_map(const cgks_ctx* ctx, void* base, CUtensorMap* map) {
  static const PFN_cuTensorMapEncodeTiled_v12000 encode = []() -> PFN_cuTensorMapEncodeTiled_v12000 {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    return (PFN_cuTensorMapEncodeTiled_v12000)fn;
  }();
  if (!encode) return false;
  const int dim = ctx->dim, gpf = dim == 3 ? 4 : 2;
  const cuuint32_t nq = (cuuint32_t)(ctx->nv * (1 + dim));
  const size_t es = ctx->prec == 0 ? sizeof(double) : sizeof(float);
  const cuuint64_t gdim[2] = {(cuuint64_t)ctx->ncell, (cuuint64_t)dim * gpf * nq};
  const cuuint64_t gstride[1] = {(cuuint64_t)ctx->ncell * es};
  const cuuint32_t box[2] = {128, nq};
  const cuuint32_t estride[2] = {1, 1};
  return encode(map, es == sizeof(float) ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, base,
                gdim, gstride, box, estride, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

cgks_status cgks_create_mesh(const cgks_mesh_desc* d, cgks_ctx** out) {
  cgks_ctx* ctx = nullptr;
  if (!d || !out) return CGKS_EINVAL;
  if (d->dim != 2 && d->dim != 3) return CGKS_EINVAL;
  for (int a = 0; a < d->dim; ++a)
    if (d->n[a] < 3) return CGKS_EINVAL;
  if (d->precision < 0 || d->precision > 2) return CGKS_EUNSUPPORTED;
  for (int f = 0; f < 2 * d->dim; ++f) {
    if (d->bc[f] < CGKS_BC_PERIODIC || d->bc[f] > CGKS_BC_INFLOW) return CGKS_EINVAL;
    if ((d->bc[f] == CGKS_BC_PERIODIC) != (d->bc[f ^ 1] == CGKS_BC_PERIODIC)) return CGKS_EINVAL;
    if (d->bc[f] >= CGKS_BC_SLIP_WALL && d->nodes) return CGKS_EUNSUPPORTED;
  }
  if (!(d->gamma > 1.0) || d->mu < 0.0 || !(d->cfl > 0.0) || d->tau_mode < 0 || d->tau_mode > 2)
    return CGKS_EINVAL;
  ctx = new cgks_ctx();
  ctx->desc = *d;
  ctx->desc.nodes = nullptr;
  ctx->dim = d->dim;
  ctx->nv = d->dim + 2;
  ctx->nf = d->dim == 3 ? Sz<3>::NF : Sz<2>::NF;
  ctx->n[0] = d->n[0];
  ctx->n[1] = d->n[1];
  ctx->n[2] = d->dim == 3 ? d->n[2] : 1;
  ctx->ncell = (long)ctx->n[0] * ctx->n[1] * ctx->n[2];
  ctx->stream = (cudaStream_t)d->stream;
  ctx->prec = d->precision == 1 ? 1 : 0;
  ctx->pair_flux = d->precision == 2;
  ctx->ph.gamma = d->gamma;
  ctx->ph.mu = d->mu;
  ctx->ph.prandtl = d->prandtl > 0.0 ? d->prandtl : 1.0;
  ctx->ph.cfl = d->cfl;
  ctx->ph.c_chi = d->c_chi > 0.0 ? d->c_chi : 100.0;
  ctx->ph.tau_mode = d->tau_mode;
  ctx->ph.linear = d->linear;
  ctx->ph.gammaf = (float)ctx->ph.gamma;
  ctx->ph.muf = (float)ctx->ph.mu;
  ctx->ph.prandtlf = (float)ctx->ph.prandtl;
  ctx->ph.c_chif = (float)ctx->ph.c_chi;
  ctx->ph.prfix = (ctx->ph.mu > 0.0 && ctx->ph.prandtl > 0.0 && ctx->ph.prandtl != 1.0) ? 1 : 0;
  DevGeo& g = ctx->geo;
  for (int a = 0; a < 3; ++a) {
    g.n[a] = ctx->n[a];
    g.h[a] = a < d->dim ? (d->hi[a] - d->lo[a]) / d->n[a] : 1.0;
    g.ih[a] = 1.0 / g.h[a];
    g.hf[a] = (float)g.h[a];
    g.ihf[a] = (float)g.ih[a];
  }
  g.ncell = ctx->ncell;
  g.curvi = d->nodes ? 1 : 0;
  g.met = nullptr;
  g.rmet = nullptr;
  g.bcq = nullptr;
  g.nplane = 0;
  g.bcm = 0;
  ctx->walls = false;
  for (int f = 0; f < 2 * d->dim; ++f) {
    g.bcm |= d->bc[f] << (3 * f);
    if (d->bc[f] >= CGKS_BC_SLIP_WALL) ctx->walls = true;
    if (d->bc[f] != CGKS_BC_PERIODIC) g.nplane = std::max(g.nplane, ctx->ncell / ctx->n[f / 2]);
  }
  const long N = ctx->ncell;
  const int dim = ctx->dim, nv = ctx->nv, nf = ctx->nf;
  const int gpf = dim == 3 ? 4 : 2;
  const size_t st_sz = sizeof(double) * (size_t)nf * nv * N;
  const size_t rsz = ctx->prec == 0 ? sizeof(double) : sizeof(float);
  const size_t gp_sz = rsz * (size_t)dim * gpf * nv * (1 + dim) * N;
  const size_t fx_sz = rsz * (size_t)dim * gpf * 6 * nv * N;
  const size_t navg = (size_t)nv * N, nder = (size_t)(nf - 1) * nv * N;
#define ALLOC(p, sz)                                                                         \
  do {                                                                                       \
    if (cudaMalloc((void**)&(p), (sz)) != cudaSuccess) {                                     \
      cudaGetLastError();                                                                    \
      cgks_destroy(ctx);                                                                     \
      return CGKS_ENOMEM;                                                                    \
    }                                                                                        \
  } while (0)
  ALLOC(ctx->U, st_sz);
  if (ctx->prec == 0) {
    ALLOC(ctx->Us, st_sz);
    ALLOC(ctx->stash, st_sz);
    ctx->avg[0] = ctx->U;
    ctx->der[0] = ctx->U + navg;
    ctx->avg[1] = ctx->Us;
    ctx->der[1] = ctx->Us + navg;
    ctx->savg = ctx->stash;
    ctx->sder = ctx->stash + navg;
  } else {
    /* averages: three FP64 arrays in one allocation; derivatives: three FP32 */
    ALLOC(ctx->Us, sizeof(double) * navg * 3);
    ALLOC(ctx->f32, sizeof(float) * nder * 3);
    ctx->avg[0] = ctx->Us;
    ctx->avg[1] = ctx->Us + navg;
    ctx->savg = ctx->Us + 2 * navg;
    ctx->der[0] = (float*)ctx->f32;
    ctx->der[1] = (float*)ctx->f32 + nder;
    ctx->sder = (float*)ctx->f32 + 2 * nder;
    ALLOC(ctx->pairs, sizeof(float) * navg * 4);
    ctx->avh[0] = ctx->pairs;
    ctx->avl[0] = ctx->pairs + navg;
    ctx->avh[1] = ctx->pairs + 2 * navg;
    ctx->avl[1] = ctx->pairs + 3 * navg;
  }
  ALLOC(ctx->gpL, gp_sz);
  ALLOC(ctx->gpR, gp_sz);
  /* CGKS_FLUX_STAGING=cp.async in the environment keeps the per-thread
     staging (the tests compare the two) */
  const char* staging = getenv("CGKS_FLUX_STAGING");
  if (!d->nodes && N % 128 == 0 && !(staging && !strcmp(staging, "cp.async")))
    ctx->tma = encode_gp_map(ctx, ctx->gpL, &ctx->tmL) && encode_gp_map(ctx, ctx->gpR, &ctx->tmR);
  /* test hook of the bounded staging wait: CGKS_TEST_STAGING_STALL=1 makes
     every TMA barrier of this context wait for 16 bytes that never come */
  const char* stall = getenv("CGKS_TEST_STAGING_STALL");
  ctx->ph.stall_tx = (ctx->tma && stall && !strcmp(stall, "1")) ? 16 : 0;
  ALLOC(ctx->flux, fx_sz);
  if (g.nplane > 0) ALLOC(ctx->fxb, rsz * (size_t)dim * gpf * 6 * nv * g.nplane);
  g.bcq = nullptr;
  for (int f = 0; f < 2 * dim; ++f)
    if (d->bc[f] == CGKS_BC_INFLOW && !ctx->d_bcq) {
      double hq[cgks::BCQ_DOUBLES];
      cgks::pack_bcq(d->bc_state, hq);
      ALLOC(ctx->d_bcq, sizeof(hq));
      CK(cudaMemcpy(ctx->d_bcq, hq, sizeof(hq), cudaMemcpyHostToDevice));
      g.bcq = ctx->d_bcq;
    }
  ALLOC(ctx->chi, sizeof(double) * (size_t)nv * N);
  ALLOC(ctx->dts, sizeof(DtState));
  ALLOC(ctx->st, sizeof(int) * ST_N);
  ALLOC(ctx->d_lo, sizeof(double) * 3);
  CK(cudaMemsetAsync(ctx->st, 0, sizeof(int) * ST_N, ctx->stream));
  CK(cudaMemsetAsync(ctx->U, 0, st_sz, ctx->stream));
  CK(cudaMemsetAsync(ctx->chi, 0, sizeof(double) * (size_t)nv * N, ctx->stream));
  CK(cudaMemcpyAsync(ctx->d_lo, d->lo, sizeof(double) * 3, cudaMemcpyHostToDevice, ctx->stream));
  if (d->nodes) {
    long nn = (long)(ctx->n[0] + 1) * (ctx->n[1] + 1) * (dim == 3 ? ctx->n[2] + 1 : 1);
    int nmet = dim == 3 ? Met<3>::N : Met<2>::N;
    ALLOC(ctx->d_nodes, sizeof(double) * nn * dim);
    ALLOC(ctx->d_met, sizeof(double) * (size_t)nmet * N);
    CK(cudaMemcpyAsync(ctx->d_nodes, d->nodes, sizeof(double) * nn * dim, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (dim == 3) k_metrics<3><<<cdiv(N, 128), 128, 0, ctx->stream>>>(ctx->d_nodes, g, ctx->d_met);
    else k_metrics<2><<<cdiv(N, 128), 128, 0, ctx->stream>>>(ctx->d_nodes, g, ctx->d_met);
    CK(cudaGetLastError());
    g.met = ctx->d_met;
    int nrm = dim == 3 ? RateMet<3>::N : RateMet<2>::N;
    ALLOC(ctx->d_rmet, sizeof(float) * (size_t)nrm * N);
    if (dim == 3) k_rate_metrics<3><<<cdiv(N, 128), 128, 0, ctx->stream>>>(g, ctx->d_rmet);
    else k_rate_metrics<2><<<cdiv(N, 128), 128, 0, ctx->stream>>>(g, ctx->d_rmet);
    CK(cudaGetLastError());
    g.rmet = ctx->d_rmet;
  }
#undef ALLOC
  DtState init{};
  init.t = 0.0;
  init.dt_fixed = d->dt_fixed;
  CK(cudaMemcpyAsync(ctx->dts, &init, sizeof init, cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  *out = ctx;
  return CGKS_OK;
}

void cgks_destroy(cgks_ctx* ctx) {
  if (!ctx) return;
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  else cudaDeviceSynchronize();
  cudaFree(ctx->U);
  cudaFree(ctx->Us);
  cudaFree(ctx->stash);
  cudaFree(ctx->f32);
  cudaFree(ctx->pairs);
  cudaFree(ctx->gpL);
  cudaFree(ctx->gpR);
  cudaFree(ctx->flux);
  cudaFree(ctx->fxb);
  cudaFree(ctx->chi);
  cudaFree(ctx->dts);
  cudaFree(ctx->st);
  cudaFree(ctx->d_lo);
  cudaFree(ctx->d_nodes);
  cudaFree(ctx->d_met);
  cudaFree(ctx->d_rmet);
  cudaFree(ctx->d_bcq);
  cudaFree(ctx->sel_buf);
  for (auto e : ctx->prof.pool) cudaEventDestroy(e);
  delete ctx;
}

int cgks_num_vars(const cgks_ctx* ctx) { return ctx ? ctx->nv : -1; }
int cgks_num_fields(const cgks_ctx* ctx) { return ctx ? ctx->nf : -1; }
long cgks_num_cells(const cgks_ctx* ctx) { return ctx ? ctx->ncell : -1; }
int cgks_flux_staging(const cgks_ctx* ctx) { return ctx ? (ctx->tma ? 1 : 0) : -1; }

/* the copy in, the FP32 split and a fresh time-step record, enqueued on the
   context's stream without waiting */
static cgks_status enqueue_set(cgks_ctx* ctx, const double* src, int is_device, double t) {
  size_t sz = sizeof(double) * (size_t)ctx->nf * ctx->nv * ctx->ncell;
  CK(cudaMemcpyAsync(ctx->U, src, sz, is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, ctx->stream));
  cgks_status r0 = split_in(ctx);
  if (r0 != CGKS_OK) return r0;
  k_dt_init<<<1, 1, 0, ctx->stream>>>(ctx->dts, t, ctx->desc.dt_fixed);
  CK(cudaGetLastError());
  ctx->t = t;
  return CGKS_OK;
}
/* the FP32 join and the copy out, enqueued without waiting */
static cgks_status enqueue_get(cgks_ctx* ctx, double* dst, int is_device) {
  size_t sz = sizeof(double) * (size_t)ctx->nf * ctx->nv * ctx->ncell;
  cgks_status r0 = join_out(ctx);
  if (r0 != CGKS_OK) return r0;
  CK(cudaMemcpyAsync(dst, ctx->U, sz, is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, ctx->stream));
  return CGKS_OK;
}

cgks_status cgks_set_state(cgks_ctx* ctx, const double* src, int is_device, double t) {
  if (!ctx || !src) return CGKS_EINVAL;
  cgks_status r0 = enqueue_set(ctx, src, is_device, t);
  if (r0 != CGKS_OK) return r0;
  if (!is_device) CK(cudaStreamSynchronize(ctx->stream));
  return CGKS_OK;
}

cgks_status cgks_set_state_async(cgks_ctx* ctx, const double* src, int is_device, double t) {
  if (!ctx || !src) return CGKS_EINVAL;
  return enqueue_set(ctx, src, is_device, t);
}

cgks_status cgks_get_state_async(cgks_ctx* ctx, double* dst, int is_device) {
  if (!ctx || !dst) return CGKS_EINVAL;
  return enqueue_get(ctx, dst, is_device);
}

cgks_status cgks_sync(cgks_ctx* ctx) {
  if (!ctx) return CGKS_EINVAL;
  CK(cudaStreamSynchronize(ctx->stream));
  return CGKS_OK;
}

cgks_status cgks_get_state(cgks_ctx* ctx, double* dst, int is_device, double* t) {
  if (!ctx || !dst) return CGKS_EINVAL;
  cgks_status r0 = enqueue_get(ctx, dst, is_device);
  if (r0 != CGKS_OK) return r0;
  DtState h;
  CK(cudaMemcpyAsync(&h, ctx->dts, sizeof h, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->t = h.t;
  if (t) *t = h.t;
  return CGKS_OK;
}

static cgks_status check_status(cgks_ctx* ctx) {
  int st[ST_N];
  CK(cudaMemcpyAsync(st, ctx->st, sizeof st, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (st[ST_NONPHYS] || st[ST_FLUX] || st[ST_DT]) {
    int z[ST_N] = {0, st[ST_FALLBACK], 0, 0};
    CK(cudaMemcpyAsync(ctx->st, z, sizeof z, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (st[ST_FLUX] & 2) /* a flux block's TMA tile did not arrive within its bounded wait */
      return fail(ctx, CGKS_ETIMEOUT, "a staging wait of the interface flux gave up");
    return fail(ctx, CGKS_ENONPHYS, "non-physical state (recon %d, interface %d, cell %d)", st[ST_NONPHYS],
                st[ST_FLUX], st[ST_DT]);
  }
  return CGKS_OK;
}

cgks_status cgks_step(cgks_ctx* ctx, int nsteps, double t_end, double* t_out, double* dt_last) {
  if (!ctx || nsteps < 0) return CGKS_EINVAL;
  DtState h;
  CK(cudaMemcpyAsync(&h, ctx->dts, sizeof h, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  h.t_end = t_end > 0.0 ? t_end : 0.0;
  h.nok = 0;
  h.t_prev = h.t;
  CK(cudaMemcpyAsync(ctx->dts, &h, sizeof h, cudaMemcpyHostToDevice, ctx->stream));
  int nrun = 0;
  for (int s = 0; s < nsteps; ++s) {
    if (t_end > 0.0) {
      CK(cudaMemcpyAsync(&h, ctx->dts, sizeof h, cudaMemcpyDeviceToHost, ctx->stream));
      CK(cudaStreamSynchronize(ctx->stream));
      if (h.t >= t_end * (1.0 - 1e-14)) break;
    }
    cgks_status r = ctx->dim == 3 ? run_step<3>(ctx) : run_step<2>(ctx);
    if (r != CGKS_OK) return r;
    ++nrun;
  }
  if (ctx->prof.on) prof_fold(ctx);
  cgks_status r = check_status(ctx);
  CK(cudaMemcpyAsync(&h, ctx->dts, sizeof h, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  /* after a failure the last good state is the input of step nok of the
     call: no later step wrote into it, and each step swapped the two sets */
  if (r == CGKS_ENONPHYS && ((nrun - h.nok) & 1)) swap_state(ctx);
  ctx->t = h.t;
  if (t_out) *t_out = h.t;
  if (dt_last) *dt_last = h.dt;
  return r;
}

cgks_status cgks_compute_dt(cgks_ctx* ctx, double* dt) {
  if (!ctx || !dt) return CGKS_EINVAL;
  DtState h;
  CK(cudaMemcpyAsync(&h, ctx->dts, sizeof h, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  double keep_end = h.t_end;
  h.t_end = 0.0;
  CK(cudaMemcpyAsync(ctx->dts, &h, sizeof h, cudaMemcpyHostToDevice, ctx->stream));
  cgks_status r = ctx->dim == 3 ? run_dt<3>(ctx, ctx->avg[0], ctx->prec ? ctx->avh[0] : nullptr, 0)
                                 : run_dt<2>(ctx, ctx->avg[0], ctx->prec ? ctx->avh[0] : nullptr, 0);
  if (r != CGKS_OK) return r;
  CK(cudaMemcpyAsync(&h, ctx->dts, sizeof h, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  *dt = h.dt;
  h.t_end = keep_end;
  CK(cudaMemcpyAsync(ctx->dts, &h, sizeof h, cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return check_status(ctx);
}

int cgks_init_points_per_cell(const cgks_ctx* ctx) {
  if (!ctx) return -1;
  return ctx->dim == 3 ? npts_cell<3>() : npts_cell<2>();
}

cgks_status cgks_init_points(cgks_ctx* ctx, long cell0, long ncells, double* dev_pts) {
  if (!ctx || !dev_pts || cell0 < 0 || ncells < 0 || cell0 + ncells > ctx->ncell) return CGKS_EINVAL;
  long tot = ncells * cgks_init_points_per_cell(ctx);
  if (tot == 0) return CGKS_OK;
  if (ctx->dim == 3)
    k_init_points<3><<<cdiv(tot, 128), 128, 0, ctx->stream>>>(ctx->d_nodes, ctx->geo, ctx->d_lo, cell0, ncells,
                                                              dev_pts);
  else
    k_init_points<2><<<cdiv(tot, 128), 128, 0, ctx->stream>>>(ctx->d_nodes, ctx->geo, ctx->d_lo, cell0, ncells,
                                                              dev_pts);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(ctx->stream));
  return CGKS_OK;
}

cgks_status cgks_init_from_prims(cgks_ctx* ctx, long cell0, long ncells, const double* dev_prims) {
  if (!ctx || !dev_prims || cell0 < 0 || ncells < 0 || cell0 + ncells > ctx->ncell) return CGKS_EINVAL;
  if (ncells == 0) return CGKS_OK;
  if (ctx->dim == 3)
    k_init_from_prims<3><<<cdiv(ncells, 128), 128, 0, ctx->stream>>>(ctx->d_nodes, ctx->geo, ctx->ph, ctx->d_lo,
                                                                     cell0, ncells, dev_prims, ctx->U);
  else
    k_init_from_prims<2><<<cdiv(ncells, 128), 128, 0, ctx->stream>>>(ctx->d_nodes, ctx->geo, ctx->ph, ctx->d_lo,
                                                                     cell0, ncells, dev_prims, ctx->U);
  CK(cudaGetLastError());
  if (ctx->prec == 1) {
    const long tot = (long)ctx->nf * ctx->nv * ncells;
    k_split_cells<float><<<cdiv(tot, 256), 256, 0, ctx->stream>>>(ctx->U, ctx->avg[0], ctx->avh[0], ctx->avl[0],
                                                                  (float*)ctx->der[0], ctx->ncell, ctx->nv, ctx->nf,
                                                                  cell0, ncells);
    CK(cudaGetLastError());
  }
  DtState init{};
  init.t = 0.0;
  init.dt_fixed = ctx->desc.dt_fixed;
  CK(cudaMemcpyAsync(ctx->dts, &init, sizeof init, cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->t = 0.0;
  return CGKS_OK;
}

cgks_status cgks_get_chi(cgks_ctx* ctx, double* dst, int is_device) {
  if (!ctx || !dst) return CGKS_EINVAL;
  CK(cudaMemcpyAsync(dst, ctx->chi, sizeof(double) * (size_t)ctx->nv * ctx->ncell,
                     is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return CGKS_OK;
}

cgks_status cgks_profile_enable(cgks_ctx* ctx, int on) {
  if (!ctx) return CGKS_EINVAL;
  prof_fold(ctx);
  ctx->prof.on = on != 0;
  for (int k = 0; k < KID_N; ++k) {
    ctx->prof.launches[k] = 0;
    ctx->prof.ms[k] = 0.0;
  }
  return CGKS_OK;
}

int cgks_profile_read(cgks_ctx* ctx, const char** names, long* launches, double* total_ms, int cap) {
  if (!ctx) return -1;
  prof_fold(ctx);
  int n = 0;
  for (int k = 0; k < KID_N && n < cap; ++k, ++n) {
    if (names) names[n] = kKernelNames[k];
    if (launches) launches[n] = ctx->prof.launches[k];
    if (total_ms) total_ms[n] = ctx->prof.ms[k];
  }
  return n;
}

}  // extern "C"

/* ---- learned selector ---------------------------------------------------- */
/* float -> bfloat16, round to nearest, ties to even (finite values) */
static uint16_t to_bf16(float x) {
  uint32_t u;
  memcpy(&u, &x, 4);
  u += 0x7FFFu + ((u >> 16) & 1u);
  return (uint16_t)(u >> 16);
}

/* device copy of a selector: BF16 weights then FP32 biases then counters */
cgks_status selector_upload(void** buf, SelectorDev* sd, const float* params, float thr_skip, float thr_lo,
                            cudaStream_t stream) {
  const size_t wbytes = sizeof(uint16_t) * SEL_NW, bbytes = sizeof(float) * SEL_NB;
  const size_t off_b = (wbytes + 255) & ~size_t(255), off_c = (off_b + bbytes + 255) & ~size_t(255);
  if (!*buf && cudaMalloc(buf, off_c + 2 * SEL_SLOTS * sizeof(unsigned long long)) != cudaSuccess) {
    cudaGetLastError();
    return CGKS_ENOMEM;
  }
  std::vector<uint16_t> w(SEL_NW);
  std::vector<float> b(SEL_NB);
  const float* W1 = params;
  const float* b1 = W1 + SEL_H * SEL_NF;
  const float* W2 = b1 + SEL_H;
  const float* b2 = W2 + SEL_H * SEL_H;
  const float* W3 = b2 + SEL_H;
  const float* b3 = W3 + SEL_H * SEL_H;
  const float* w4 = b3 + SEL_H;
  int o = 0;
  for (int i = 0; i < SEL_H * SEL_NF; ++i) w[o++] = to_bf16(W1[i]);
  for (int i = 0; i < SEL_H * SEL_H; ++i) w[o++] = to_bf16(W2[i]);
  for (int i = 0; i < SEL_H * SEL_H; ++i) w[o++] = to_bf16(W3[i]);
  for (int i = 0; i < SEL_H; ++i) w[o++] = to_bf16(w4[i]);
  for (int i = 0; i < SEL_H; ++i) {
    b[i] = b1[i];
    b[SEL_H + i] = b2[i];
    b[2 * SEL_H + i] = b3[i];
  }
  b[3 * SEL_H] = w4[SEL_H];
  char* base = (char*)*buf;
  if (cudaMemcpyAsync(base, w.data(), wbytes, cudaMemcpyHostToDevice, stream) != cudaSuccess ||
      cudaMemcpyAsync(base + off_b, b.data(), bbytes, cudaMemcpyHostToDevice, stream) != cudaSuccess ||
      cudaMemsetAsync(base + off_c, 0, 2 * SEL_SLOTS * sizeof(unsigned long long), stream) != cudaSuccess ||
      cudaStreamSynchronize(stream) != cudaSuccess)
    return CGKS_ECUDA;
  sd->w = (const __nv_bfloat16*)base;
  sd->b = (const float*)(base + off_b);
  sd->counts = (unsigned long long*)(base + off_c);
  sd->thr_skip = thr_skip;
  sd->thr_lo = thr_lo;
  sd->on = 1;
  return CGKS_OK;
}

extern "C" {

cgks_status cgks_set_selector(cgks_ctx* ctx, const float* params, float thr_skip, float thr_lo) {
  if (!ctx) return CGKS_EINVAL;
  if (!params) {
    ctx->sel.on = 0;
    return CGKS_OK;
  }
  if (!(thr_lo <= thr_skip)) return CGKS_EINVAL;
  cgks_status s = selector_upload(&ctx->sel_buf, &ctx->sel, params, thr_skip, thr_lo, ctx->stream);
  if (s != CGKS_OK) return fail(ctx, s, "selector upload failed");
  return CGKS_OK;
}

cgks_status cgks_selector_stats(cgks_ctx* ctx, unsigned long long* skips, unsigned long long* unsure) {
  if (!ctx) return CGKS_EINVAL;
  unsigned long long h[2 * SEL_SLOTS] = {0};
  if (ctx->sel.counts) {
    CK(cudaMemcpyAsync(h, ctx->sel.counts, sizeof h, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
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

cgks_status cgks_selector_features(cgks_ctx* ctx, float* dev_out) {
  if (!ctx || !dev_out) return CGKS_EINVAL;
  const long N = ctx->ncell;
  const int nb = (int)cdiv(N, 128);
  const DevGeo& g = ctx->geo;
  const bool w = ctx->walls;
#define SELF(T, D)                                                                                        \
  do {                                                                                                    \
    if (w) k_selector_features<T, D, true><<<nb, 128, 0, ctx->stream>>>(ctx->avg[0], ctx->avh[0],         \
                                                                         (const T*)ctx->der[0], g, dev_out); \
    else k_selector_features<T, D, false><<<nb, 128, 0, ctx->stream>>>(ctx->avg[0], ctx->avh[0],          \
                                                                        (const T*)ctx->der[0], g, dev_out); \
  } while (0)
  if (ctx->prec == 0) {
    if (ctx->dim == 3) SELF(double, 3);
    else SELF(double, 2);
  } else {
    if (ctx->dim == 3) SELF(float, 3);
    else SELF(float, 2);
  }
#undef SELF
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(ctx->stream));
  return CGKS_OK;
}

cgks_status cgks_diagnostics(cgks_ctx* ctx, double* ek, double* enstrophy) {
  if (!ctx) return CGKS_EINVAL;
  const int nblk = 304;
  double* part = nullptr;
  if (cudaMallocAsync((void**)&part, sizeof(double) * 4 * nblk, ctx->stream) != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, CGKS_ENOMEM, "diagnostics work space");
  }
  const DevGeo& g = ctx->geo;
  const double mu = ctx->ph.mu;
  if (ctx->prec == 0) {
    if (ctx->dim == 3) k_diagnostics<double, 3><<<nblk, 256, 0, ctx->stream>>>(g, ctx->avg[0], (const double*)ctx->der[0], mu, part);
    else k_diagnostics<double, 2><<<nblk, 256, 0, ctx->stream>>>(g, ctx->avg[0], (const double*)ctx->der[0], mu, part);
  } else {
    if (ctx->dim == 3) k_diagnostics<float, 3><<<nblk, 256, 0, ctx->stream>>>(g, ctx->avg[0], (const float*)ctx->der[0], mu, part);
    else k_diagnostics<float, 2><<<nblk, 256, 0, ctx->stream>>>(g, ctx->avg[0], (const float*)ctx->der[0], mu, part);
  }
  std::vector<double> h(4 * nblk);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), part, sizeof(double) * 4 * nblk, cudaMemcpyDeviceToHost, ctx->stream);
  cudaFreeAsync(part, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return fail(ctx, CGKS_ECUDA, "diagnostics: %s", cudaGetErrorString(e));
  double s[4] = {0.0, 0.0, 0.0, 0.0};
  for (int b = 0; b < nblk; ++b)
    for (int q = 0; q < 4; ++q) s[q] += h[4 * b + q];
  const double rho0 = s[2] / s[3];
  if (ek) *ek = s[0] / (rho0 * s[3]);
  if (enstrophy) *enstrophy = s[1] / (rho0 * s[3]);
  return CGKS_OK;
}

cgks_status cgks_last_error(const cgks_ctx* ctx, char* msg, size_t cap) {
  if (!ctx || !msg || cap == 0) return CGKS_EINVAL;
  snprintf(msg, cap, "%s", ctx->err.c_str());
  return CGKS_OK;
}

}  // extern "C"
