// Host build of the paired-FP32 type (paper_2508_08965_gb300/csrc/cgks_pair.cuh)
// for its arithmetic tests: error-free sums, and the relative errors of
// sums, products, quotients and conversions on random operands.
#define CGKS_HD inline
#include <cmath>
#include <cstdint>
#include <cstring>
#include <random>
#include <cmath>
namespace cgks {
inline double cg_erfc(double x) { return erfc(x); }
inline double cg_exp(double x) { return exp(x); }
inline double cg_expm1(double x) { return expm1(x); }
inline double cg_sqrt(double x) { return sqrt(x); }
inline double cg_rsqrt(double x) { return 1.0 / sqrt(x); }
#include "../paper_2508_08965_gb300/csrc/cgks_pair.cuh"
}  // namespace cgks
using cgks::fpair;

extern "C" {
/* out: [0] two-sum failures, [1] fast-two-sum failures, [2] max rel error of
   sums, [3] of differences of nearby values (relative to the operands), [4]
   of products, [5] of quotients, [6] of conversions from double */
void pair_stats(int n, unsigned seed, double* out) {
  std::mt19937_64 rng(seed);
  std::uniform_real_distribution<double> u(-1.0, 1.0), ex(-20.0, 20.0);
  auto rnd = [&]() { return u(rng) * std::ldexp(1.0, (int)ex(rng)); };
  for (int i = 0; i < 7; ++i) out[i] = 0;
  for (int it = 0; it < n; ++it) {
    const float a = (float)rnd(), b = (float)rnd();
    float s, e;
    cgks::fp_two_sum(a, b, s, e);
    if ((long double)s + e != (long double)a + b) out[0] += 1;
    const float big = std::fabs(a) >= std::fabs(b) ? a : b, small = big == a ? b : a;
    cgks::fp_fast_two_sum(big, small, s, e);
    if ((long double)s + e != (long double)big + small) out[1] += 1;
    const double x = rnd(), y = rnd();
    const fpair px(x), py(y);
    const long double X = (long double)px.hi + px.lo, Y = (long double)py.hi + py.lo;
    out[6] = std::fmax(out[6], (double)(fabsl(X - x) / fabsl((long double)x)));
    const fpair ps = px + py, pm = px * py, pq = px / py;
    const long double S = X + Y, M = X * Y, Q = X / Y;
    out[2] = std::fmax(out[2], (double)(fabsl((long double)ps.hi + ps.lo - S) / (fabsl(X) + fabsl(Y))));
    out[4] = std::fmax(out[4], (double)(fabsl((long double)pm.hi + pm.lo - M) / fabsl(M)));
    out[5] = std::fmax(out[5], (double)(fabsl((long double)pq.hi + pq.lo - Q) / fabsl(Q)));
    const fpair pz(x * (1.0 + 1e-9 * u(rng)));
    const fpair pd = px - pz;
    const long double Z = (long double)pz.hi + pz.lo;
    out[3] = std::fmax(out[3], (double)(fabsl((long double)pd.hi + pd.lo - (X - Z)) / fabsl(X)));
  }
}
}

extern "C" {
/* largest relative errors of the pair special functions against long double
   references on random arguments: out[0] exp on [-40, 2], [1] expm1 on
   [-2, 2], [2] erfc on [-3, 3] (the series below |x| = 3/4), [3] 1/sqrt on
   [1e-8, 1e8]; out[4] exp on [-1, 1] relative to the result */
void pair_func_stats(int n, unsigned seed, double* out) {
  std::mt19937_64 rng(seed);
  std::uniform_real_distribution<double> u(0.0, 1.0);
  for (int i = 0; i < 5; ++i) out[i] = 0;
  auto val = [](const fpair& p) { return (long double)p.hi + p.lo; };
  for (int it = 0; it < n; ++it) {
    const double a = -40.0 + 42.0 * u(rng);
    const fpair pa(a);
    const long double A = val(pa);
    out[0] = std::fmax(out[0], (double)fabsl(val(cgks::cg_exp(pa)) / expl(A) - 1.0L));
    const double b = -2.0 + 4.0 * u(rng);
    const fpair pb(b);
    const long double B = val(pb);
    out[1] = std::fmax(out[1], (double)fabsl(val(cgks::cg_expm1(pb)) / expm1l(B) - 1.0L));
    const double c = -3.0 + 6.0 * u(rng);
    const fpair pc(c);
    const long double Cc = val(pc);
    out[2] = std::fmax(out[2], (double)fabsl(val(cgks::cg_erfc(pc)) / erfcl(Cc) - 1.0L));
    const double d = std::pow(10.0, -8.0 + 16.0 * u(rng));
    const fpair pd(d);
    const long double D = val(pd);
    out[3] = std::fmax(out[3], (double)fabsl(val(cgks::cg_rsqrt(pd)) * sqrtl(D) - 1.0L));
    const double e = -1.0 + 2.0 * u(rng);
    const fpair pe(e);
    out[4] = std::fmax(out[4], (double)fabsl(val(cgks::cg_exp(pe)) / expl(val(pe)) - 1.0L));
  }
}
}

extern "C" {
/* the integer-pipe conversions and unnormalised sums of the paired
   reconstruction (fpacc).  out: [0] max relative error of double -> fpacc
   on [2^-100, 2^100] (either sign), [1] conversions of x whose exact value
   hi exceeds |x| in magnitude (hi is a truncation of x),
   [2] float -> double mismatches against the plain conversion (subnormal
   floats: signed 0) and hi + lo -> double mismatches against the exact sum
   for |x| >= 2^-80, [3] special-value failures (zeros, values below 2^-103, beyond the
   float range, inf, NaN), [4] max error of 80-term sums of products
   (cg_fma chains with rounded-double constants) relative to the sum of the
   products' magnitudes */
void pair_conv_stats(int n, unsigned seed, double* out) {
  using cgks::fpacc;
  std::mt19937_64 rng(seed);
  std::uniform_real_distribution<double> u(-1.0, 1.0), ex(-100.0, 100.0);
  for (int i = 0; i < 5; ++i) out[i] = 0;
  auto val = [](const fpacc& p) { return (long double)p.hi + p.lo; };
  for (int it = 0; it < n; ++it) {
    const double x = u(rng) * std::ldexp(1.0, (int)ex(rng));
    if (std::fabs(x) < std::ldexp(1.0, -100)) continue; /* the flushed range is checked below */
    const fpacc p = cgks::fpacc_from_double(x);
    out[0] = std::fmax(out[0], (double)(fabsl(val(p) - x) / fabsl((long double)x)));
    if (fabsl((long double)p.hi) > fabsl((long double)x)) out[1] += 1;
    const float f = (float)(u(rng) * std::ldexp(1.0, (int)(ex(rng) * 1.2)));
    if (cgks::fp_f2d_bits(f) != (std::fpclassify(f) == FP_SUBNORMAL ? std::copysign(0.0, f) : (double)f)) out[2] += 1;
    if (std::fabs(x) >= std::ldexp(1.0, -80) && cgks::fpacc_to_double(p) != (double)((long double)p.hi + p.lo))
      out[2] += 1;
  }
  const double specials[] = {0.0, -0.0, 1e-32, -3e-40, 1e300, -1e300, INFINITY, -INFINITY};
  for (double x : specials) {
    const fpacc p = cgks::fpacc_from_double(x);
    const bool tiny = std::fabs(x) < std::ldexp(1.0, -103);
    if (tiny && !(p.hi == 0.f && p.lo == 0.f && std::signbit(p.hi) == std::signbit(x))) out[3] += 1;
    if (!tiny && std::fabs(x) > 1e200 && !(std::isinf(p.hi) && std::signbit(p.hi) == std::signbit(x))) out[3] += 1;
  }
  if (!std::isnan(cgks::fpacc_from_double(NAN).hi)) out[3] += 1;
  if (!std::isnan(cgks::fp_f2d_bits(NAN)) || !std::isinf(cgks::fp_f2d_bits(INFINITY))) out[3] += 1;
  if (cgks::fp_f2d_bits(1e-40f) != 0.0 || !std::signbit(cgks::fp_f2d_bits(-1e-40f)) ||
      !std::signbit(cgks::fp_f2d_bits(-0.0f)))
    out[3] += 1;
  std::uniform_real_distribution<double> uc(-1.0, 1.0);
  for (int it = 0; it < n / 100; ++it) {
    fpacc acc(0.0f);
    long double ref = 0.0L, mag = 0.0L;
    for (int q = 0; q < 80; ++q) {
      const double c = uc(rng), d = uc(rng) * std::ldexp(1.0, (int)(ex(rng) / 20));
      const fpacc pc(c), pd = cgks::fpacc_from_double(d);
      acc = cgks::cg_fma(pc, pd, acc);
      ref += val(pc) * val(pd);
      mag += fabsl(val(pc) * val(pd));
    }
    const fpacc nrm = cgks::fpacc_norm(acc);
    out[4] = std::fmax(out[4], (double)(fabsl(val(nrm) - ref) / mag));
  }
}
}

extern "C" {
/* fp_f2d_exact (float -> double on the integer pipe, used by the FP32
   form's update) against the compiler's conversion, bit for bit: every
   37th subnormal pattern of either sign, n random bit patterns (normal,
   inf, NaN), and zeros, the extremes and the boundary of the normal
   range.  Returns the mismatches (NaN: any NaN matches). */
long f2d_exact_mismatches(int n, unsigned seed) {
  long bad = 0;
  auto chk = [&](float f) {
    const double a = cgks::fp_f2d_exact(f), b = (double)f;
    if (std::isnan(a) && std::isnan(b)) return;
    if (std::memcmp(&a, &b, sizeof a) != 0) ++bad;
  };
  for (unsigned u = 0; u < 0x00800000u; u += 37) {
    float f;
    std::memcpy(&f, &u, 4);
    chk(f);
    chk(-f);
  }
  std::mt19937 rng(seed);
  for (int i = 0; i < n; ++i) {
    const unsigned u = rng();
    float f;
    std::memcpy(&f, &u, 4);
    chk(f);
  }
  const float sp[] = {0.f, -0.f, INFINITY, -INFINITY, 1.f, -1.f, 1e-45f, -1e-45f, 3.4028235e38f, 1.17549435e-38f,
                      1.1754942e-38f};
  for (float f : sp) chk(f);
  return bad;
}
}
