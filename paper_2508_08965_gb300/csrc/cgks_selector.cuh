/*
 * Learned troubled-cell selector (not in the paper): a small network that
 * predicts, from normalised stencil jumps, which cells can skip the GENO
 * adaptive weights (Sec. 3.3) and take the fifth-order polynomial directly
 * (chi = 1).  Inference runs inside the reconstruction kernel: one warp
 * evaluates its 32 cells' 16-32-32-32-1 ReLU network with BF16 tensor-core
 * MMAs (mma.sync m16n8k16, FP32 accumulation), staging each layer's 32 x K
 * activations in shared memory.
 *
 * Features (per cell, float, every operation rounded as written so that an
 * independent implementation reproduces them): for each variable v and axis
 * a, with face-neighbour differences dm = Q0 - Q(-a), dp = Q(+a) - Q0 and
 * scale = |Q0| (+ sqrt(|rho| |rho E|) for momentum):
 *   J = max(|dm|, |dp|) / scale,
 *   E = |Q(edge neighbour) - Q0| / scale over the edge (corner) neighbours,
 *   R = |dp - dm| / (|dm| + |dp| + 1e-7 scale),
 *   S = (max - min of the line differences along a) / scale,
 *   C = |mean line difference - (dp + dm)/2| / (|dm| + |dp| + 1e-7 scale),
 *   G = |grad_k Q(face neighbour) - grad_k Q0| h_k / scale;
 * J, E, R, S, C pooled (max) over the variables of each class (density,
 * momentum, energy) and the axes, G over everything; J, E, S, C, G mapped by
 * x/(1+x).  16 features.
 */
#ifndef CGKS_SELECTOR_CUH
#define CGKS_SELECTOR_CUH

#include <cuda_bf16.h>

#include "cgks_device.cuh"

namespace cgks {

constexpr int SEL_NF = 16, SEL_H = 32;
/* parameters, packed: W1[32][16] b1[32] W2[32][32] b2 W3[32][32] b3 w4[32] b4 */
constexpr int SEL_NPARAM = SEL_H * SEL_NF + SEL_H + 2 * (SEL_H * SEL_H + SEL_H) + SEL_H + 1;
/* the same in the device copy: BF16 weights (W1, W2, W3, w4 in this order,
   row-major [out][in]) and FP32 biases (b1, b2, b3, b4) */
constexpr int SEL_NW = SEL_H * SEL_NF + 2 * SEL_H * SEL_H + SEL_H;
constexpr int SEL_NB = 3 * SEL_H + 1;
constexpr int SEL_PITCH = 20; /* 32-bit words per staged row (40 bf16): conflict-free fragment loads */
constexpr int SEL_SLOTS = 64; /* counter slot pairs (skips, unsure), summed when read */

struct SelectorDev {
  const __nv_bfloat16* w; /* SEL_NW */
  const float* b;         /* SEL_NB */
  float thr_skip, thr_lo; /* skip when logit >= thr_skip; unsure when thr_lo < logit < thr_skip */
  int on;
  unsigned long long* counts; /* SEL_SLOTS pairs: skips, unsure (low confidence: full GENO) */
};

enum { SEL_GENO = 0, SEL_SKIP = 1 };

/* an average (index i of avg) or an inflow state (index i of the face
   states, in the averages' type: FP64, or the FP32 form's hi parts) */
__device__ __forceinline__ double sel_avg(const double* avg, const DevGeo& g, bool inflow, long i) {
  return (inflow ? g.bcq : avg)[i];
}
__device__ __forceinline__ float sel_avg(const float* avg, const DevGeo& g, bool inflow, long i) {
  return (inflow ? bcq_hi(g) : avg)[i];
}

/* features of cell c; S: the averages' type (double or the FP32 form's hi
   parts), D: the derivative fields' type */
/* per-variable maxima over the axes (J, E, R, S, C) and the running G */
template <int DIM, bool WALL, typename S, typename D>
__device__ __forceinline__ void selector_var(const S* __restrict__ avg, const D* __restrict__ der, const DevGeo& g,
                                             const NbrOff<DIM>& nb, long c, int v, float q0v, float scale, float* o5,
                                             float& fg) {
  constexpr int NV = DIM + 2, GPF = Sz<DIM>::GPF;
  const long N = g.ncell;
  const float inv = __frcp_rn(scale);
  float fj = 0.f, fe = 0.f, fr = 0.f, fs = 0.f, fc = 0.f;
#pragma unroll
  for (int a = 0; a < DIM; ++a) {
    float qn[2];
#pragma unroll
    for (int sd = 0; sd < 2; ++sd) {
      int o[3] = {0, 0, 0};
      o[a] = sd ? 1 : -1;
      int mm;
      const long i = nb.template at<WALL>(c, o[0], o[1], o[2], &mm);
      /* branch-free loads: an inflow neighbour switches the load's base and
         index to the face's state (FP32 form: its hi part, = its float) */
      const bool inflow = WALL && (mm & MM_INFLOW);
      const int odd = WALL ? mirror_odd<DIM>(v, mm) : 0;
      float q = (float)sel_avg(avg, g, inflow, inflow ? NbrOff<DIM>::inflow_face(mm, o[0], o[1], o[2]) * 5 + v
                                                      : (long)v * N + i);
      if (odd && !inflow) q = -q;
      qn[sd] = q;
#pragma unroll
      for (int k = 0; k < DIM; ++k) {
        float gm = (float)der[((long)k * NV + v) * N + i];
        if (WALL && (odd ^ ((mm >> k) & 1))) gm = -gm;
        if (inflow) gm = 0.f;
        const float g0 = (float)der[((long)k * NV + v) * N + c];
        const float len = g.curvi ? (float)met_len<DIM>(g, c, k * GPF) : g.hf[k];
        fg = fmaxf(fg, __fmul_rn(__fmul_rn(fabsf(__fsub_rn(gm, g0)), len), inv));
      }
    }
    const float dm = __fsub_rn(q0v, qn[0]), dp = __fsub_rn(qn[1], q0v);
    const float adm = fabsf(dm), adp = fabsf(dp);
    const float J = __fmul_rn(fmaxf(adm, adp), inv);
    const float den = __fadd_rn(__fadd_rn(adm, adp), __fmul_rn(1e-7f, scale));
    const float R = __fdiv_rn(fabsf(__fsub_rn(dp, dm)), den);
    float lsum = 0.f, lmin = 0.f, lmax = 0.f;
#pragma unroll
    for (int k = 0; k < GPF; ++k) {
      const int s = a * GPF + k;
      const float len = g.curvi ? (float)met_len<DIM>(g, c, s) : g.hf[a];
      const float lh = __fmul_rn((float)der[((long)(DIM + s) * NV + v) * N + c], len);
      lsum = __fadd_rn(lsum, lh);
      if (k == 0 || lh < lmin) lmin = lh;
      if (k == 0 || lh > lmax) lmax = lh;
    }
    const float lhm = __fmul_rn(lsum, 1.0f / (float)GPF);
    const float sp = __fmul_rn(__fsub_rn(lmax, lmin), inv);
    const float cd = __fmul_rn(__fadd_rn(dp, dm), 0.5f);
    const float cm = __fdiv_rn(fabsf(__fsub_rn(lhm, cd)), den);
    fj = fmaxf(fj, J);
    fr = fmaxf(fr, R);
    fs = fmaxf(fs, sp);
    fc = fmaxf(fc, cm);
#pragma unroll
    for (int b = a + 1; b < DIM; ++b)
#pragma unroll
      for (int sg = 0; sg < 4; ++sg) {
        int o[3] = {0, 0, 0};
        o[a] = (sg & 1) ? 1 : -1;
        o[b] = (sg & 2) ? 1 : -1;
        int mm;
        const long i = nb.template at<WALL>(c, o[0], o[1], o[2], &mm);
        const bool inflow = WALL && (mm & MM_INFLOW);
        float q = (float)sel_avg(avg, g, inflow, inflow ? NbrOff<DIM>::inflow_face(mm, o[0], o[1], o[2]) * 5 + v
                                                        : (long)v * N + i);
        if (WALL && !inflow && mirror_odd<DIM>(v, mm)) q = -q;
        fe = fmaxf(fe, __fmul_rn(fabsf(__fsub_rn(q, q0v)), inv));
      }
  }
  o5[0] = fmaxf(o5[0], fj);
  o5[1] = fmaxf(o5[1], fe);
  o5[2] = fmaxf(o5[2], fr);
  o5[3] = fmaxf(o5[3], fs);
  o5[4] = fmaxf(o5[4], fc);
}

template <int DIM, bool WALL, typename S, typename D>
__device__ __forceinline__ void selector_features(const S* __restrict__ avg, const D* __restrict__ der,
                                                  const DevGeo& g, long c, int ci, int cj, int ck, float* f) {
  constexpr int NV = DIM + 2;
  const long N = g.ncell;
  NbrOff<DIM> nb;
  nb.setup(g, ci, cj, ck);
  const float rho = (float)avg[c], rhoe = (float)avg[(long)(NV - 1) * N + c];
  const float mscale = __fsqrt_rn(__fmul_rn(fabsf(rho), fabsf(rhoe)));
  float p0[5] = {0.f, 0.f, 0.f, 0.f, 0.f}, p1[5] = {0.f, 0.f, 0.f, 0.f, 0.f}, p2[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
  float fg = 0.f;
  selector_var<DIM, WALL>(avg, der, g, nb, c, 0, rho, fabsf(rho), p0, fg);
#pragma unroll 1
  for (int v = 1; v <= DIM; ++v) {
    const float q = (float)avg[(long)v * N + c];
    selector_var<DIM, WALL>(avg, der, g, nb, c, v, q, __fadd_rn(fabsf(q), mscale), p1, fg);
  }
  selector_var<DIM, WALL>(avg, der, g, nb, c, NV - 1, rhoe, fabsf(rhoe), p2, fg);
  const float* pc[3] = {p0, p1, p2};
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    f[5 * k + 0] = __fdiv_rn(pc[k][0], __fadd_rn(1.0f, pc[k][0]));
    f[5 * k + 1] = __fdiv_rn(pc[k][1], __fadd_rn(1.0f, pc[k][1]));
    f[5 * k + 2] = pc[k][2];
    f[5 * k + 3] = __fdiv_rn(pc[k][3], __fadd_rn(1.0f, pc[k][3]));
    f[5 * k + 4] = __fdiv_rn(pc[k][4], __fadd_rn(1.0f, pc[k][4]));
  }
  f[15] = __fdiv_rn(fg, __fadd_rn(1.0f, fg));
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  __nv_bfloat162 p = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&p);
}

__device__ __forceinline__ void mma_bf16_16816(float* d, const uint32_t* a, const uint32_t* b) {
#if defined(__CUDA_ARCH__)
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
#endif
}

/* One dense layer of the warp's 32 rows: stage (32 x K bf16, SEL_PITCH words
   per row) times W (32 x K, row-major [out][in]) plus bias, ReLU, back to
   stage as bf16.  Fragment layouts of m16n8k16 (PTX ISA): lane = 4 g + t;
   A holds rows g, g + 8 and columns 2t, 2t + 1 (+ 8); B holds rows (k) 2t,
   2t + 1 (+ 8) of column (n) g; C holds rows g, g + 8 and columns 2t, 2t + 1. */
template <int K>
__device__ __forceinline__ void sel_layer(uint32_t* stage, const __nv_bfloat16* __restrict__ W,
                                          const float* __restrict__ bias) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  float acc[2][4][4];
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int nt = 0; nt < 4; ++nt)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[mt][nt][q] = 0.f;
#pragma unroll
  for (int ks = 0; ks < K / 16; ++ks) {
    uint32_t a[2][4];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
      const int r0 = (mt * 16 + g) * SEL_PITCH, r1 = (mt * 16 + g + 8) * SEL_PITCH;
      const int c0 = ks * 8 + t; /* in 32-bit words: column 2 (ks*8 + t) */
      a[mt][0] = stage[r0 + c0];
      a[mt][1] = stage[r1 + c0];
      a[mt][2] = stage[r0 + c0 + 4];
      a[mt][3] = stage[r1 + c0 + 4];
    }
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
      const uint32_t* wr = reinterpret_cast<const uint32_t*>(W + (nt * 8 + g) * K + ks * 16);
      uint32_t b[2] = {__ldg(wr + t), __ldg(wr + t + 4)};
#pragma unroll
      for (int mt = 0; mt < 2; ++mt) mma_bf16_16816(acc[mt][nt], a[mt], b);
    }
  }
  __syncwarp();
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
      const int col = nt * 8 + 2 * t;
      const float b0 = __ldg(bias + col), b1 = __ldg(bias + col + 1);
      const float z0 = __fadd_rn(acc[mt][nt][0], b0), z1 = __fadd_rn(acc[mt][nt][1], b1);
      const float z2 = __fadd_rn(acc[mt][nt][2], b0), z3 = __fadd_rn(acc[mt][nt][3], b1);
      stage[(mt * 16 + g) * SEL_PITCH + col / 2] = pack_bf16x2(fmaxf(z0, 0.f), fmaxf(z1, 0.f));
      stage[(mt * 16 + g + 8) * SEL_PITCH + col / 2] = pack_bf16x2(fmaxf(z2, 0.f), fmaxf(z3, 0.f));
    }
  __syncwarp();
}

/* Block-collective: every thread of the block must call it (inactive lanes
   with active = false).  Returns SEL_SKIP or SEL_GENO for the lane's cell and
   counts skips and low-confidence cells. */
__device__ __forceinline__ int selector_decide(const SelectorDev& s, const float* feat, bool active,
                                               uint32_t* stage) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int j = 0; j < SEL_NF / 2; ++j)
    stage[lane * SEL_PITCH + j] = active ? pack_bf16x2(feat[2 * j], feat[2 * j + 1]) : 0u;
  __syncwarp();
  sel_layer<SEL_NF>(stage, s.w, s.b);
  sel_layer<SEL_H>(stage, s.w + SEL_H * SEL_NF, s.b + SEL_H);
  sel_layer<SEL_H>(stage, s.w + SEL_H * SEL_NF + SEL_H * SEL_H, s.b + 2 * SEL_H);
  /* output layer: the lane's own row, sequential FP32 sum of exact products */
  const __nv_bfloat16* w4 = s.w + SEL_H * SEL_NF + 2 * SEL_H * SEL_H;
  float acc = 0.f;
#pragma unroll
  for (int j = 0; j < SEL_H / 2; ++j) {
    const uint32_t hv = stage[lane * SEL_PITCH + j];
    const float h0 = __uint_as_float(hv << 16), h1 = __uint_as_float(hv & 0xFFFF0000u);
    acc = __fadd_rn(acc, __fmul_rn(__bfloat162float(w4[2 * j]), h0));
    acc = __fadd_rn(acc, __fmul_rn(__bfloat162float(w4[2 * j + 1]), h1));
  }
  __syncwarp();
  const float logit = __fadd_rn(acc, __ldg(s.b + 3 * SEL_H));
  const bool skip = active && logit >= s.thr_skip;
  const bool unsure = active && !skip && logit > s.thr_lo;
  const unsigned ms = __ballot_sync(0xffffffffu, skip), mu = __ballot_sync(0xffffffffu, unsure);
  /* counters: per block in shared memory, then one global atomic per block
     into one of SEL_SLOTS slot pairs (same-address atomics from every warp
     would serialise) */
  __shared__ unsigned int bc[2];
  if (threadIdx.x == 0) bc[0] = bc[1] = 0u;
  __syncthreads();
  if (lane == 0) {
    if (ms) atomicAdd(&bc[0], (unsigned)__popc(ms));
    if (mu) atomicAdd(&bc[1], (unsigned)__popc(mu));
  }
  __syncthreads();
  if (threadIdx.x == 0 && s.counts && (bc[0] | bc[1])) {
    unsigned long long* slot = s.counts + 2 * (blockIdx.x % SEL_SLOTS);
    if (bc[0]) atomicAdd(&slot[0], (unsigned long long)bc[0]);
    if (bc[1]) atomicAdd(&slot[1], (unsigned long long)bc[1]);
  }
  return skip ? SEL_SKIP : SEL_GENO;
}

}  // namespace cgks

#endif
