// Algorithmic operation count of the library's arithmetic, per unit of
// work, without a GPU and without a profiler.
//
// The device routines are compiled for the host (as in host_kernels.cpp)
// with a compute type that records, for each work item (a cell of the
// reconstruction, a face Gauss point of the flux, a cell variable of the
// update), the graph of the operations applied to its values.  The graph is
// value-numbered: an operation that repeats one already made on the same
// operands is not new (common subexpressions), a product with an exact 0 or
// +-1 and a sum with an exact 0 are no operations (constants of the
// source), and only operations on which a stored result depends are
// counted (dead code).  So the count is that of the algorithm as written,
// independent of how a compiler schedules it: every +, - and * one flop, a
// fused multiply-add two, a division one (also reported apart), and each
// call of exp, erfc, expm1, tanh, sqrt or 1/sqrt one special-function
// evaluation (reported apart).  What a GPU executes for a division or a
// special function (a sequence of FMAs) is not in it; the executed count
// of a profiler is.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <unordered_map>
#include <vector>

namespace fc {
enum Op : uint8_t { LEAF, ADD, SUB, MUL, DIV, FMA, NEG, SFU };
struct Node {
  Op op;
  uint8_t fn;
  int a, b, c;
};
struct Key {
  uint64_t a, b;
  bool operator==(const Key& o) const { return a == o.a && b == o.b; }
};
struct KeyHash {
  size_t operator()(const Key& k) const { return (size_t)(k.a * 0x9E3779B97F4A7C15ull ^ (k.b + (k.a >> 29))); }
};
struct Graph {
  std::vector<Node> nodes;
  std::unordered_map<uint64_t, int> leaves; /* by the bits of the value */
  std::unordered_map<Key, int, KeyHash> ops; /* by (op, fn, operands) */
  std::vector<int> escapes;                  /* values converted out of the type: results stored as double */
  void clear() {
    nodes.clear();
    leaves.clear();
    ops.clear();
    escapes.clear();
  }
  int leaf(double v) {
    uint64_t k;
    memcpy(&k, &v, 8);
    auto it = leaves.find(k);
    if (it != leaves.end()) return it->second;
    nodes.push_back({LEAF, 0, -1, -1, -1});
    return leaves[k] = (int)nodes.size() - 1;
  }
  int op(Op o, uint8_t fn, int a, int b, int c) {
    if ((o == ADD || o == MUL || o == FMA) && b >= 0 && a > b) std::swap(a, b); /* commutative */
    const Key k{((uint64_t)o << 56) | ((uint64_t)fn << 48) | (uint64_t)(uint32_t)(a + 1),
                ((uint64_t)(uint32_t)(b + 1) << 32) | (uint32_t)(c + 1)};
    auto it = ops.find(k);
    if (it != ops.end()) return it->second;
    nodes.push_back({o, fn, a, b, c});
    return ops[k] = (int)nodes.size() - 1;
  }
};
Graph G;
}  // namespace fc

struct fcount {
  double v;
  int id;
  fcount() : v(0.0), id(fc::G.leaf(0.0)) {}
  fcount(double x) : v(x), id(fc::G.leaf(x)) {}
  fcount(float x) : v(x), id(fc::G.leaf((double)x)) {}
  fcount(int x) : v(x), id(fc::G.leaf((double)x)) {}
  fcount(long x) : v((double)x), id(fc::G.leaf((double)x)) {}
  fcount(double x, int i) : v(x), id(i) {}
  explicit operator double() const {
    fc::G.escapes.push_back(id);
    return v;
  }
  explicit operator float() const {
    fc::G.escapes.push_back(id);
    return (float)v;
  }
};
static inline bool is0(const fcount& a) { return a.v == 0.0 && fc::G.nodes[a.id].op == fc::LEAF; }
static inline bool is1(const fcount& a) { return a.v == 1.0 && fc::G.nodes[a.id].op == fc::LEAF; }
static inline bool ism1(const fcount& a) { return a.v == -1.0 && fc::G.nodes[a.id].op == fc::LEAF; }
inline fcount operator-(fcount a) { return fcount(-a.v, fc::G.op(fc::NEG, 0, a.id, -1, -1)); }
inline fcount operator+(fcount a, fcount b) {
  if (is0(a)) return b;
  if (is0(b)) return a;
  return fcount(a.v + b.v, fc::G.op(fc::ADD, 0, a.id, b.id, -1));
}
inline fcount operator-(fcount a, fcount b) {
  if (is0(b)) return a;
  if (is0(a)) return -b;
  return fcount(a.v - b.v, fc::G.op(fc::SUB, 0, a.id, b.id, -1));
}
inline fcount operator*(fcount a, fcount b) {
  if (is0(a) || is0(b)) return fcount(0.0);
  if (is1(a)) return b;
  if (is1(b)) return a;
  if (ism1(a)) return -b;
  if (ism1(b)) return -a;
  return fcount(a.v * b.v, fc::G.op(fc::MUL, 0, a.id, b.id, -1));
}
inline fcount operator/(fcount a, fcount b) {
  if (is1(b)) return a;
  return fcount(a.v / b.v, fc::G.op(fc::DIV, 0, a.id, b.id, -1));
}
inline fcount& operator+=(fcount& a, fcount b) { return a = a + b; }
inline fcount& operator-=(fcount& a, fcount b) { return a = a - b; }
inline fcount& operator*=(fcount& a, fcount b) { return a = a * b; }
inline fcount& operator/=(fcount& a, fcount b) { return a = a / b; }
inline bool operator<(fcount a, fcount b) { return a.v < b.v; }
inline bool operator>(fcount a, fcount b) { return a.v > b.v; }
inline bool operator<=(fcount a, fcount b) { return a.v <= b.v; }
inline bool operator>=(fcount a, fcount b) { return a.v >= b.v; }
inline bool operator==(fcount a, fcount b) { return a.v == b.v; }
inline bool operator!=(fcount a, fcount b) { return a.v != b.v; }
static inline fcount sfu(int fn, fcount x, double y) { return fcount(y, fc::G.op(fc::SFU, (uint8_t)fn, x.id, -1, -1)); }
inline fcount cg_exp(fcount x) { return sfu(1, x, std::exp(x.v)); }
inline fcount cg_erfc(fcount x) { return sfu(2, x, std::erfc(x.v)); }
inline fcount cg_expm1(fcount x) { return sfu(3, x, std::expm1(x.v)); }
inline fcount cg_tanh(fcount x) { return sfu(4, x, std::tanh(x.v)); }
inline fcount cg_sqrt(fcount x) { return sfu(5, x, std::sqrt(x.v)); }
inline fcount cg_rsqrt(fcount x) { return sfu(6, x, 1.0 / std::sqrt(x.v)); }
inline fcount cg_fabs(fcount x) { return x.v < 0 ? -x : x; }
inline fcount cg_fma(fcount a, fcount b, fcount c) {
  if (is0(a) || is0(b) || is1(a) || is1(b) || ism1(a) || ism1(b) || is0(c)) return a * b + c;
  return fcount(std::fma(a.v, b.v, c.v), fc::G.op(fc::FMA, 0, a.id, b.id, c.id));
}

inline fcount cg_dot2(fcount a, fcount b, fcount c, fcount d) { return a * b + c * d; }
inline fcount cg_madd(fcount a, fcount b, fcount c) { return a * b + c; }
inline fcount cg_norm(fcount x) { return x; }
inline fcount cg_dot3(fcount a, fcount b, fcount c, fcount d, fcount e, fcount f) { return a * b + c * d + e * f; }

#include "host_kernels.cpp"

namespace {

/* counts of the operations reachable from the given results */
struct Counts {
  double add = 0, mul = 0, fma = 0, div = 0, sfu = 0;
};
void count_live(const std::vector<int>& roots, Counts& c) {
  std::vector<char> seen(fc::G.nodes.size(), 0);
  std::vector<int> stack(roots.begin(), roots.end());
  while (!stack.empty()) {
    const int i = stack.back();
    stack.pop_back();
    if (i < 0 || seen[i]) continue;
    seen[i] = 1;
    const fc::Node& n = fc::G.nodes[i];
    switch (n.op) {
      case fc::ADD: case fc::SUB: c.add += 1; break;
      case fc::MUL: c.mul += 1; break;
      case fc::DIV: c.div += 1; break;
      case fc::FMA: c.fma += 1; break;
      case fc::SFU: c.sfu += 1; break;
      default: break;
    }
    stack.push_back(n.a);
    stack.push_back(n.b);
    stack.push_back(n.c);
  }
}

/* every value an item left in `v` (all entries whose id belongs to the
   item's graph: each array is filled with fresh leaves before the item),
   and every value it converted to double or float (its results stored in
   those types) */
void roots_of(const std::vector<fcount>& v, size_t nodes_before, std::vector<int>& roots) {
  for (const auto& x : v)
    if ((size_t)x.id >= nodes_before) roots.push_back(x.id);
  for (int e : fc::G.escapes) roots.push_back(e);
}

template <int DIM>
int count_stage(const int* n, const double* lo, const double* hi, const double* phys, const double* U, double dt,
                long stride, double* out /* 3 kernels x 5 counts + 3 item counts */) {
  typedef fcount T;
  DevGeo g{};
  geometry<DIM>(g, n, lo, hi);
  const double gamma = phys[0], mu = phys[1], pr = phys[2], cfl = phys[3], cchi = phys[4];
  Phys ph{gamma, mu, pr, cfl, cchi, (int)phys[5], (int)phys[6], (float)gamma, (float)mu, (float)pr, (float)cchi,
          (mu > 0 && pr > 0 && pr != 1.0) ? 1 : 0};
  const long N = g.ncell;
  const int NV = Sz<DIM>::NV, NF = Sz<DIM>::NF, GPF = Sz<DIM>::GPF;
  const size_t navg = (size_t)NV * N, nder = (size_t)(NF - 1) * NV * N;
  std::vector<double> A0(U, U + navg), A1(navg), SA(navg);
  std::vector<double> D0d(U + navg, U + navg + nder);
  std::vector<float> H0(navg), L0(navg), H1(navg), L1(navg);
  for (size_t i = 0; i < navg; ++i) {
    H0[i] = float(A0[i]);
    L0[i] = float(A0[i] - double(H0[i]));
  }
  int st[ST_N] = {0};
  std::vector<double> chi(navg);
  DtState dts{};
  set_dt(dts, dt);
  blockDim.x = 1;
  threadIdx.x = 0;
  Counts c[3];
  /* the arrays hold values of the graph being built, so each item starts a
     new graph over fresh leaves of the stored values */
  std::vector<T> D0(nder), D1(nder), SD(nder);
  std::vector<T> gpL((size_t)DIM * GPF * NV * (1 + DIM) * N), gpR(gpL.size()), fx((size_t)DIM * GPF * 6 * NV * N);
  std::vector<T> fxb(1);
  std::vector<double> gpLd(gpL.size()), gpRd(gpL.size()), fxd(fx.size());
  std::vector<int> roots;
  auto fresh = [&](std::vector<T>& a, const std::vector<double>* vals) {
    for (size_t i = 0; i < a.size(); ++i) a[i] = T(vals ? (*vals)[i] : 0.0);
  };
  long items[3] = {0, 0, 0};
  /* every cell is reconstructed (the flux needs all Gauss-point states); only
     every stride-th item of each kernel is counted */
  for (long t = 0; t < N; ++t) {
    fc::G.clear();
    fresh(D0, &D0d);
    fresh(gpL, &gpLd);
    fresh(gpR, &gpRd);
    const size_t before = fc::G.nodes.size();
    blockIdx.x = (unsigned)t;
    k_recon<T, DIM, false, false>(A0.data(), H0.data(), L0.data(), D0.data(), g, ph, gpL.data(), gpR.data(),
                                  chi.data(), 1, st, SelectorDev{});
    if (t % stride == 0) {
      roots.clear();
      roots_of(gpL, before, roots);
      roots_of(gpR, before, roots);
      count_live(roots, c[0]);
      ++items[0];
    }
    for (size_t i = 0; i < gpL.size(); ++i) {
      gpLd[i] = gpL[i].v;
      gpRd[i] = gpR[i].v;
    }
  }
  for (long t = 0; t < (long)DIM * GPF * N; t += stride) {
    fc::G.clear();
    fresh(gpL, &gpLd);
    fresh(gpR, &gpRd);
    fresh(fx, &fxd);
    const size_t before = fc::G.nodes.size();
    blockIdx.x = (unsigned)t;
    k_flux<T, DIM, false, T>(g, ph, &dts, gpL.data(), gpR.data(), fx.data(), st, CUtensorMap{}, CUtensorMap{});
    roots.clear();
    roots_of(fx, before, roots);
    count_live(roots, c[1]);
    ++items[1];
    for (size_t i = 0; i < fx.size(); ++i) fxd[i] = fx[i].v;
  }
  std::vector<double> SDd(nder), D1d(nder);
  for (long t = 0; t < (long)NV * N; t += stride) {
    fc::G.clear();
    fresh(fx, &fxd);
    fresh(SD, &SDd);
    fresh(D1, &D1d);
    const size_t before = fc::G.nodes.size();
    blockIdx.x = (unsigned)t;
    k_update<T, DIM, false>(g, &dts, 1, A0.data(), fx.data(), fxb.data(), SA.data(), SD.data(), A1.data(),
                            D1.data(), H1.data(), L1.data());
    roots.clear();
    roots_of(SD, before, roots);
    roots_of(D1, before, roots);
    count_live(roots, c[2]);
    ++items[2];
    for (size_t i = 0; i < nder; ++i) {
      SDd[i] = SD[i].v;
      D1d[i] = D1[i].v;
    }
  }
  for (int k = 0; k < 3; ++k) {
    out[5 * k + 0] = c[k].add;
    out[5 * k + 1] = c[k].mul;
    out[5 * k + 2] = c[k].fma;
    out[5 * k + 3] = c[k].div;
    out[5 * k + 4] = c[k].sfu;
    out[15 + k] = (double)items[k];
  }
  return (st[ST_FLUX] || st[ST_NONPHYS]) ? 1 : 0;
}

}  // namespace

extern "C" {
/* counts of one stage-1 pass over a periodic uniform box with state U
   (public layout), over every stride-th work item of each kernel:
   out[kernel][count] for the kernels reconstruction, interface flux and
   update and the counts additions (and subtractions), multiplications,
   FMAs, divisions and special functions, then out[15 + kernel] the items
   counted.  Returns 0, or 1 on a non-physical state. */
int count_stage_ops(int dim, const int* n, const double* lo, const double* hi, const double* phys, const double* U,
                    double dt, long stride, double* out) {
  for (int f = 0; f < 6; ++f) g_bc[f] = 0;
  if (stride < 1) stride = 1;
  if (dim == 3) return count_stage<3>(n, lo, hi, phys, U, dt, stride, out);
  return count_stage<2>(n, lo, hi, phys, U, dt, stride, out);
}
}
