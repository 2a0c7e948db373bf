/* Reconstruction of the paired form (precision 2) on Cartesian meshes: FP64
   averages and derivatives in, the reconstruction's linear maps (a = M d and
   the Gauss-point transform) in unnormalised paired FP32 (recon_var_pair),
   FP64 Gauss-point states out.  Curvilinear meshes keep the FP64 kernel. */
#include "cgks_ctx.h"

using namespace cgks;
using namespace cgks_host;

template <int DIM, bool WALL>
void launch_recon_pair(cgks_ctx* ctx, int in, int record_chi) {
  const long N = ctx->ncell;
  k_recon<double, DIM, false, WALL, true><<<cdiv(N, 128), 128, 0, ctx->stream>>>(
      ctx->avg[in], ctx->avh[in], ctx->avl[in], (const double*)ctx->der[in], ctx->geo, ctx->ph, (double*)ctx->gpL,
      (double*)ctx->gpR, ctx->chi, record_chi, ctx->st, ctx->sel);
}

template void launch_recon_pair<2, false>(cgks_ctx*, int, int);
template void launch_recon_pair<2, true>(cgks_ctx*, int, int);
template void launch_recon_pair<3, false>(cgks_ctx*, int, int);
template void launch_recon_pair<3, true>(cgks_ctx*, int, int);
