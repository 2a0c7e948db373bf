/*
 * Training arithmetic of the learned selector's network (include/cgks.h,
 * cgks_mlp_*), FP32 on device buffers: the forward pass, the weighted binary
 * cross-entropy of the logits and its gradient by back-propagation, and an
 * Adam step.  Reductions over samples are blocked and summed in a fixed
 * order, so results are deterministic.
 *
 * Network: x (16) -> 32 -> 32 -> 32 -> logit, ReLU after each hidden layer;
 * parameters packed W1[32][16] b1[32] W2[32][32] b2 W3[32][32] b3 w4[32] b4.
 * Loss: L = sum_s w_s (softplus(z_s) - y_s z_s) / sum_s w_s.
 */
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "../../include/cgks.h"

namespace {

constexpr int NF = 16, H = 32;
constexpr int O_W1 = 0, O_B1 = O_W1 + H * NF, O_W2 = O_B1 + H, O_B2 = O_W2 + H * H, O_W3 = O_B2 + H,
              O_B3 = O_W3 + H * H, O_W4 = O_B3 + H, O_B4 = O_W4 + H, NPARAM = O_B4 + 1;
static_assert(NPARAM == CGKS_SEL_NPARAM, "parameter count");
constexpr int TPB = 128;   /* samples per block of the per-sample kernels */
constexpr int CHUNK = 32;  /* samples staged per step of the gradient reduction */
constexpr int RTPB = 256;  /* threads of the gradient reduction */
constexpr int PPT = (NPARAM + RTPB - 1) / RTPB;

__device__ __forceinline__ float softplusf(float z) { return fmaxf(z, 0.f) + log1pf(expf(-fabsf(z))); }

/* per-sample forward and backward.  Writes the hidden activations h1..h3 and
   the pre-activation gradients d1..d3 ([n][32] each, unscaled: the factor
   1/sum(w) is applied in the reduction), d4 = w (sigmoid(z) - y), and the
   sample's loss term w (softplus(z) - y z). */
__global__ void __launch_bounds__(TPB) k_mlp_fb(const float* __restrict__ P, const float* __restrict__ X,
                                                const float* __restrict__ y, const float* __restrict__ w, long n,
                                                float* __restrict__ act, float* __restrict__ dlt,
                                                float* __restrict__ d4, float* __restrict__ lterm) {
  __shared__ float sp[NPARAM];
  for (int i = threadIdx.x; i < NPARAM; i += blockDim.x) sp[i] = P[i];
  __syncthreads();
  const long s = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (s >= n) return;
  float x[NF], h1[H], h2[H], h3[H];
  for (int k = 0; k < NF; ++k) x[k] = X[s * NF + k];
  for (int o = 0; o < H; ++o) {
    float z = sp[O_B1 + o];
    for (int k = 0; k < NF; ++k) z = fmaf(sp[O_W1 + o * NF + k], x[k], z);
    h1[o] = fmaxf(z, 0.f);
  }
  for (int o = 0; o < H; ++o) {
    float z = sp[O_B2 + o];
    for (int k = 0; k < H; ++k) z = fmaf(sp[O_W2 + o * H + k], h1[k], z);
    h2[o] = fmaxf(z, 0.f);
  }
  float z4 = sp[O_B4];
  for (int o = 0; o < H; ++o) {
    float z = sp[O_B3 + o];
    for (int k = 0; k < H; ++k) z = fmaf(sp[O_W3 + o * H + k], h2[k], z);
    h3[o] = fmaxf(z, 0.f);
    z4 = fmaf(sp[O_W4 + o], h3[o], z4);
  }
  const float ws = w[s], ys = y[s];
  lterm[s] = ws * (softplusf(z4) - ys * z4);
  const float g4 = ws * (1.f / (1.f + expf(-z4)) - ys);
  d4[s] = g4;
  float* A = act + s * 3 * H;
  float* D = dlt + s * 3 * H;
  for (int o = 0; o < H; ++o) {
    A[o] = h1[o];
    A[H + o] = h2[o];
    A[2 * H + o] = h3[o];
  }
  /* back-propagation: d3 = g4 w4 [z3 > 0]; d2 = W3^T d3 [z2 > 0]; d1 = W2^T d2 [z1 > 0] */
  float d3[H];
  for (int o = 0; o < H; ++o) d3[o] = h3[o] > 0.f ? g4 * sp[O_W4 + o] : 0.f;
  for (int i = 0; i < H; ++i) {
    float a = 0.f;
    for (int o = 0; o < H; ++o) a = fmaf(sp[O_W3 + o * H + i], d3[o], a);
    h3[i] = h2[i] > 0.f ? a : 0.f; /* h3 now holds d2 */
  }
  for (int i = 0; i < H; ++i) {
    float a = 0.f;
    for (int o = 0; o < H; ++o) a = fmaf(sp[O_W2 + o * H + i], h3[o], a);
    D[i] = h1[i] > 0.f ? a : 0.f; /* d1 */
  }
  for (int o = 0; o < H; ++o) {
    D[H + o] = h3[o];     /* d2 */
    D[2 * H + o] = d3[o]; /* d3 */
  }
}

/* gradient partial sums: block b accumulates, over its chunks of CHUNK
   samples (chunks b, b + gridDim.x, ...), every parameter's sum of
   (delta of its output) x (its input), into part[b][NPARAM] */
__global__ void __launch_bounds__(RTPB) k_mlp_gred(const float* __restrict__ X, const float* __restrict__ act,
                                                   const float* __restrict__ dlt, const float* __restrict__ d4,
                                                   long n, float* __restrict__ part) {
  __shared__ float sx[CHUNK][NF], sa[CHUNK][3 * H], sd[CHUNK][3 * H], s4[CHUNK];
  float acc[PPT];
  for (int q = 0; q < PPT; ++q) acc[q] = 0.f;
  const long nch = (n + CHUNK - 1) / CHUNK;
  for (long ch = blockIdx.x; ch < nch; ch += gridDim.x) {
    const long s0 = ch * CHUNK;
    const int m = (int)(n - s0 < CHUNK ? n - s0 : CHUNK);
    __syncthreads();
    for (int i = threadIdx.x; i < CHUNK * NF; i += blockDim.x) {
      const int r = i / NF, k = i % NF;
      sx[r][k] = r < m ? X[(s0 + r) * NF + k] : 0.f;
    }
    for (int i = threadIdx.x; i < CHUNK * 3 * H; i += blockDim.x) {
      const int r = i / (3 * H), k = i % (3 * H);
      sa[r][k] = r < m ? act[(s0 + r) * 3 * H + k] : 0.f;
      sd[r][k] = r < m ? dlt[(s0 + r) * 3 * H + k] : 0.f;
    }
    for (int r = threadIdx.x; r < CHUNK; r += blockDim.x) s4[r] = r < m ? d4[s0 + r] : 0.f;
    __syncthreads();
    for (int q = 0; q < PPT; ++q) {
      const int p = threadIdx.x + q * RTPB;
      if (p >= NPARAM) break;
      float a = acc[q];
      if (p < O_B1) { /* W1[o][k]: d1[o] x[k] */
        const int o = p / NF, k = p % NF;
        for (int r = 0; r < CHUNK; ++r) a = fmaf(sd[r][o], sx[r][k], a);
      } else if (p < O_W2) {
        const int o = p - O_B1;
        for (int r = 0; r < CHUNK; ++r) a += sd[r][o];
      } else if (p < O_B2) { /* W2[o][k]: d2[o] h1[k] */
        const int o = (p - O_W2) / H, k = (p - O_W2) % H;
        for (int r = 0; r < CHUNK; ++r) a = fmaf(sd[r][H + o], sa[r][k], a);
      } else if (p < O_W3) {
        const int o = p - O_B2;
        for (int r = 0; r < CHUNK; ++r) a += sd[r][H + o];
      } else if (p < O_B3) { /* W3[o][k]: d3[o] h2[k] */
        const int o = (p - O_W3) / H, k = (p - O_W3) % H;
        for (int r = 0; r < CHUNK; ++r) a = fmaf(sd[r][2 * H + o], sa[r][H + k], a);
      } else if (p < O_W4) {
        const int o = p - O_B3;
        for (int r = 0; r < CHUNK; ++r) a += sd[r][2 * H + o];
      } else if (p < O_B4) { /* w4[k]: d4 h3[k] */
        const int k = p - O_W4;
        for (int r = 0; r < CHUNK; ++r) a = fmaf(s4[r], sa[r][2 * H + k], a);
      } else {
        for (int r = 0; r < CHUNK; ++r) a += s4[r];
      }
      acc[q] = a;
    }
  }
  for (int q = 0; q < PPT; ++q) {
    const int p = threadIdx.x + q * RTPB;
    if (p < NPARAM) part[(long)blockIdx.x * NPARAM + p] = acc[q];
  }
}

/* sum of x[0..n) in a fixed order: block partials, then one block */
__global__ void __launch_bounds__(256) k_sum_partial(const float* __restrict__ x, long n, float* __restrict__ out) {
  __shared__ float sh[256];
  float a = 0.f;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) a += x[i];
  sh[threadIdx.x] = a;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[blockIdx.x] = sh[0];
}

/* grad[p] = sum_b part[b][p] / wsum;  out2 = {loss, wsum} from the two sums */
__global__ void k_mlp_finish(const float* __restrict__ part, int nblk, const float* __restrict__ wsum_part,
                             const float* __restrict__ loss_part, int nsum, float* __restrict__ grad,
                             float* __restrict__ out2) {
  __shared__ float ws;
  if (threadIdx.x == 0) {
    float a = 0.f, l = 0.f;
    for (int b = 0; b < nsum; ++b) {
      a += wsum_part[b];
      l += loss_part[b];
    }
    ws = a;
    if (blockIdx.x == 0) {
      out2[0] = l / a;
      out2[1] = a;
    }
  }
  __syncthreads();
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= NPARAM) return;
  float g = 0.f;
  for (int b = 0; b < nblk; ++b) g += part[(long)b * NPARAM + p];
  grad[p] = g / ws;
}

__global__ void __launch_bounds__(TPB) k_mlp_logits(const float* __restrict__ P, const float* __restrict__ X, long n,
                                                    float* __restrict__ out) {
  __shared__ float sp[NPARAM];
  for (int i = threadIdx.x; i < NPARAM; i += blockDim.x) sp[i] = P[i];
  __syncthreads();
  const long s = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (s >= n) return;
  float x[NF], h1[H], h2[H];
  for (int k = 0; k < NF; ++k) x[k] = X[s * NF + k];
  for (int o = 0; o < H; ++o) {
    float z = sp[O_B1 + o];
    for (int k = 0; k < NF; ++k) z = fmaf(sp[O_W1 + o * NF + k], x[k], z);
    h1[o] = fmaxf(z, 0.f);
  }
  for (int o = 0; o < H; ++o) {
    float z = sp[O_B2 + o];
    for (int k = 0; k < H; ++k) z = fmaf(sp[O_W2 + o * H + k], h1[k], z);
    h2[o] = fmaxf(z, 0.f);
  }
  float z4 = sp[O_B4];
  for (int o = 0; o < H; ++o) {
    float z = sp[O_B3 + o];
    for (int k = 0; k < H; ++k) z = fmaf(sp[O_W3 + o * H + k], h2[k], z);
    z4 = fmaf(sp[O_W4 + o], fmaxf(z, 0.f), z4);
  }
  out[s] = z4;
}

__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       long n, float lr, float b1, float b2, float eps, float c1, float c2) {
  const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

}  // namespace

extern "C" {

cgks_status cgks_mlp_loss_grad(const float* dev_params, const float* dev_X, const float* dev_y, const float* dev_w,
                               long n, float* dev_grad, float* loss_out, void* stream) {
  if (!dev_params || !dev_X || !dev_y || !dev_w || !dev_grad || n < 1) return CGKS_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const int nblk = (int)std::min<long>((n + CHUNK - 1) / CHUNK, 608);
  const int nsum = (int)std::min<long>((n + 255) / 256, 256);
  float* ws = nullptr;
  const size_t need = (size_t)n * (3 * H * 2 + 2) + (size_t)nblk * NPARAM + 2 * nsum + 2;
  if (cudaMallocAsync((void**)&ws, sizeof(float) * need, st) != cudaSuccess) {
    cudaGetLastError();
    return CGKS_ENOMEM;
  }
  float* act = ws;
  float* dlt = act + (size_t)n * 3 * H;
  float* d4 = dlt + (size_t)n * 3 * H;
  float* lterm = d4 + n;
  float* part = lterm + n;
  float* wsp = part + (size_t)nblk * NPARAM;
  float* lsp = wsp + nsum;
  float* out2 = lsp + nsum;
  k_mlp_fb<<<(int)((n + TPB - 1) / TPB), TPB, 0, st>>>(dev_params, dev_X, dev_y, dev_w, n, act, dlt, d4, lterm);
  k_mlp_gred<<<nblk, RTPB, 0, st>>>(dev_X, act, dlt, d4, n, part);
  k_sum_partial<<<nsum, 256, 0, st>>>(dev_w, n, wsp);
  k_sum_partial<<<nsum, 256, 0, st>>>(lterm, n, lsp);
  k_mlp_finish<<<(NPARAM + 255) / 256, 256, 0, st>>>(part, nblk, wsp, lsp, nsum, dev_grad, out2);
  float h2[2] = {0.f, 0.f};
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(h2, out2, sizeof h2, cudaMemcpyDeviceToHost, st);
  cudaFreeAsync(ws, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return CGKS_ECUDA;
  if (loss_out) *loss_out = h2[0];
  return CGKS_OK;
}

cgks_status cgks_mlp_logits(const float* dev_params, const float* dev_X, long n, float* dev_out, void* stream) {
  if (!dev_params || !dev_X || !dev_out || n < 0) return CGKS_EINVAL;
  if (n == 0) return CGKS_OK;
  k_mlp_logits<<<(int)((n + TPB - 1) / TPB), TPB, 0, (cudaStream_t)stream>>>(dev_params, dev_X, n, dev_out);
  return cudaGetLastError() == cudaSuccess ? CGKS_OK : CGKS_ECUDA;
}

cgks_status cgks_mlp_adam(float* dev_params, const float* dev_grad, float* dev_m, float* dev_v, int step, float lr,
                          float beta1, float beta2, float eps, void* stream) {
  if (!dev_params || !dev_grad || !dev_m || !dev_v || step < 1) return CGKS_EINVAL;
  const float c1 = 1.f - powf(beta1, (float)step), c2 = 1.f - powf(beta2, (float)step);
  k_adam<<<(NPARAM + 255) / 256, 256, 0, (cudaStream_t)stream>>>(dev_params, dev_grad, dev_m, dev_v, NPARAM, lr, beta1,
                                                                 beta2, eps, c1, c2);
  return cudaGetLastError() == cudaSuccess ? CGKS_OK : CGKS_ECUDA;
}

}  // extern "C"
