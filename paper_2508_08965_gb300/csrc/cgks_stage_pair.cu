/* Interface flux of the paired form (precision 2) on Cartesian meshes
   (cgks_stage_pair_curvi.cu holds the other kind): FP64 Gauss-point states in, the
   GKS solve of every interior face Gauss point in paired-FP32 arithmetic
   (cgks_pair.cuh), FP64 fluxes out.  Boundary faces and the other kernels
   of the stage are the FP64 ones. */
#include "cgks_ctx.h"

using namespace cgks;
using namespace cgks_host;

template <int DIM, bool CURVI>
void launch_flux_pair(cgks_ctx* ctx, const double* gpL, const double* gpR, double* flux) {
  const long nf = (long)DIM * Sz<DIM>::GPF * ctx->ncell;
  if (ctx->tma)
    k_flux<double, DIM, CURVI, fpair, true><<<cdiv(nf, 128), 128, 0, ctx->stream>>>(
        ctx->geo, ctx->ph, ctx->dts, gpL, gpR, flux, ctx->st, ctx->tmL, ctx->tmR);
  else
    k_flux<double, DIM, CURVI, fpair><<<cdiv(nf, 128), 128, 0, ctx->stream>>>(ctx->geo, ctx->ph, ctx->dts, gpL,
                                                                                gpR, flux, ctx->st, ctx->tmL,
                                                                                ctx->tmR);
}

template void launch_flux_pair<2, false>(cgks_ctx*, const double*, const double*, double*);
template void launch_flux_pair<3, false>(cgks_ctx*, const double*, const double*, double*);
