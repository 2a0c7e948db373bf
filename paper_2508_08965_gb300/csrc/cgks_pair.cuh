/*
 * Paired-FP32 arithmetic: the compute type of the interface flux in the
 * paired form (precision 2).  A value is the unevaluated sum hi + lo of two
 * floats: about 48 significant bits, on the FP32 pipe.
 *
 *   sum      Knuth's error-free two-sum of the high parts, plus the sum of
 *            the low parts (8 operations);
 *   product  hi*hi, and its FMA residual plus the two cross terms (4);
 *   a b + c d, a b + c d + e f, a b + c: compensated dot products (Dot2);
 *   quotient operands renormalised, a reciprocal estimate and two
 *            remainder corrections.
 * None of these renormalises its result (|lo| <= ulp(hi)/2 is not kept):
 * the instruction fetch of the flux kernel is its bound, and the three
 * operations of a final fast two-sum on every result cost 13% of the
 * kernel's time (TGV 128^3), while whole steps stay within the FP64 parity
 * bars with a margin of 4x or more.  Where a sign or a float of the value is
 * read (the quotient, square roots, special functions, the pressure's
 * positivity test), the value is renormalised first (fp_norm); the
 * renormalised sum and product (fp_addn, fp_muln) serve those steps.
 *
 * exp, expm1, erfc (|x| < 3/4) and 1/sqrt are series and Newton steps in
 * pair arithmetic (below); erfc beyond 3/4 is the FP64 function rounded to
 * a pair.
 *
 * Every operation goes through the round-to-nearest intrinsics (fp_add
 * ...), which the compiler never contracts into multiply-adds, so the
 * error-free steps stay exact.  Conversions from double round twice
 * (hi, then the remainder), exactly for constants, which fold at compile
 * time.  Included by cgks_device.cuh after its math wrappers.
 */
#ifndef CGKS_PAIR_CUH
#define CGKS_PAIR_CUH

struct fpair {
  float hi, lo;
  CGKS_HD fpair() : hi(0.f), lo(0.f) {}
  CGKS_HD fpair(double x) : hi((float)x), lo((float)(x - (double)(float)x)) {}
  CGKS_HD fpair(float x) : hi(x), lo(0.f) {}
  CGKS_HD fpair(int x) : fpair((double)x) {}
  CGKS_HD explicit operator double() const { return (double)hi + (double)lo; }
};

/* single operations rounded to nearest and never contracted (on the host:
   plain IEEE single arithmetic, built without contraction) */
CGKS_HD float fp_add(float a, float b) {
#if defined(__CUDA_ARCH__)
  return __fadd_rn(a, b);
#else
  return a + b;
#endif
}
CGKS_HD float fp_sub(float a, float b) {
#if defined(__CUDA_ARCH__)
  return __fsub_rn(a, b);
#else
  return a - b;
#endif
}
CGKS_HD float fp_mul(float a, float b) {
#if defined(__CUDA_ARCH__)
  return __fmul_rn(a, b);
#else
  return a * b;
#endif
}
CGKS_HD float fp_fma(float a, float b, float c) {
#if defined(__CUDA_ARCH__)
  return __fmaf_rn(a, b, c);
#else
  return fmaf(a, b, c);
#endif
}
CGKS_HD float fp_rcp(float a) {
#if defined(__CUDA_ARCH__)
  return __frcp_rn(a);
#else
  return 1.0f / a;
#endif
}

CGKS_HD fpair fp_make(float h, float l) {
  fpair r;
  r.hi = h;
  r.lo = l;
  return r;
}
/* s + e = a + b exactly */
CGKS_HD void fp_two_sum(float a, float b, float& s, float& e) {
  s = fp_add(a, b);
  const float bb = fp_sub(s, a);
  e = fp_add(fp_sub(a, fp_sub(s, bb)), fp_sub(b, bb));
}
/* s + e = a + b exactly, for |a| >= |b| (or a = 0) */
CGKS_HD void fp_fast_two_sum(float a, float b, float& s, float& e) {
  s = fp_add(a, b);
  e = fp_sub(b, fp_sub(s, a));
}

/* renormalised forms: hi the rounded value, |lo| <= ulp(hi)/2 */
CGKS_HD fpair fp_norm(fpair a) { /* two-sum: after a cancellation |lo| may exceed |hi| */
  float s, e;
  fp_two_sum(a.hi, a.lo, s, e);
  return fp_make(s, e);
}
CGKS_HD fpair fp_addn(fpair a, fpair b) {
  float s, e;
  fp_two_sum(a.hi, b.hi, s, e);
  e = fp_add(e, fp_add(a.lo, b.lo));
  fp_fast_two_sum(s, e, s, e);
  return fp_make(s, e);
}
CGKS_HD fpair fp_muln(fpair a, fpair b) {
  const float p = fp_mul(a.hi, b.hi);
  float e = fp_fma(a.hi, b.hi, -p);
  e = fp_fma(a.hi, b.lo, e);
  e = fp_fma(a.lo, b.hi, e);
  float s;
  fp_fast_two_sum(p, e, s, e);
  return fp_make(s, e);
}
/* the operators leave the last renormalisation out (the sum keeps the
   two-sum of the high parts and gathers the errors in lo, the product is
   its exact high product and the error terms): compensated arithmetic in
   the manner of Sum2/Dot2, as accurate as the renormalised forms except
   that after a cancellation lo may hold more than half an ulp of hi, or
   the whole value.  Quotients, square roots, the special functions and
   sign tests renormalise their operands first (fp_norm). */
CGKS_HD fpair operator+(fpair a, fpair b) {
  float s, e;
  fp_two_sum(a.hi, b.hi, s, e);
  return fp_make(s, fp_add(e, fp_add(a.lo, b.lo)));
}
CGKS_HD fpair operator-(fpair a) { return fp_make(-a.hi, -a.lo); }
CGKS_HD fpair operator-(fpair a, fpair b) { return a + (-b); }
CGKS_HD fpair operator*(fpair a, fpair b) {
  const float p = fp_mul(a.hi, b.hi);
  float e = fp_fma(a.hi, b.hi, -p);
  e = fp_fma(a.hi, b.lo, e);
  e = fp_fma(a.lo, b.hi, e);
  return fp_make(p, e);
}
CGKS_HD fpair operator/(fpair a, fpair b) {
  a = fp_norm(a);
  b = fp_norm(b);
  const float r = fp_rcp(b.hi);
  const float q1 = fp_mul(a.hi, r);
  fpair rem = fp_addn(a, -fp_muln(b, fpair(q1)));
  const float q2 = fp_mul(rem.hi, r);
  rem = fp_addn(rem, -fp_muln(b, fpair(q2)));
  const float q3 = fp_mul(rem.hi, r);
  float s, e;
  fp_fast_two_sum(q1, q2, s, e);
  return fp_addn(fp_make(s, e), fpair(q3));
}
CGKS_HD fpair& operator+=(fpair& a, fpair b) { return a = a + b; }
CGKS_HD fpair& operator-=(fpair& a, fpair b) { return a = a - b; }
CGKS_HD fpair& operator*=(fpair& a, fpair b) { return a = a * b; }
CGKS_HD fpair& operator/=(fpair& a, fpair b) { return a = a / b; }
CGKS_HD bool operator<(fpair a, fpair b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
CGKS_HD bool operator>(fpair a, fpair b) { return b < a; }
CGKS_HD bool operator<=(fpair a, fpair b) { return !(b < a); }
CGKS_HD bool operator>=(fpair a, fpair b) { return !(a < b); }
CGKS_HD bool operator==(fpair a, fpair b) { return a.hi == b.hi && a.lo == b.lo; }
CGKS_HD bool operator!=(fpair a, fpair b) { return !(a == b); }

/* a b + c d and a b + c d + e f: the high-part products and their FMA
   residuals, Knuth's two-sum of the products, the residuals and sum errors
   gathered in the low part (a compensated dot product in the manner of
   Ogita, Rump and Oishi's Dot2, on pairs), left unrenormalised like the
   operators */
CGKS_HD void fp_prod_parts(fpair a, fpair b, float& p, float& e) {
  p = fp_mul(a.hi, b.hi);
  e = fp_fma(a.hi, b.hi, -p);
  e = fp_fma(a.hi, b.lo, e);
  e = fp_fma(a.lo, b.hi, e);
}
CGKS_HD fpair fp_dot2(fpair a, fpair b, fpair c, fpair d) {
  float p1, e1, p2, e2, s, t;
  fp_prod_parts(a, b, p1, e1);
  fp_prod_parts(c, d, p2, e2);
  fp_two_sum(p1, p2, s, t);
  t = fp_add(t, fp_add(e1, e2));
  return fp_make(s, t);
}
CGKS_HD fpair fp_dot3(fpair a, fpair b, fpair c, fpair d, fpair e, fpair f) {
  float p1, e1, p2, e2, p3, e3, s, t, u;
  fp_prod_parts(a, b, p1, e1);
  fp_prod_parts(c, d, p2, e2);
  fp_prod_parts(e, f, p3, e3);
  fp_two_sum(p1, p2, s, t);
  fp_two_sum(s, p3, s, u);
  t = fp_add(fp_add(t, u), fp_add(fp_add(e1, e2), e3));
  return fp_make(s, t);
}
/* a b + c (unrenormalised) */
CGKS_HD fpair fp_madd(fpair a, fpair b, fpair c) {
  float p, e, s, t;
  fp_prod_parts(a, b, p, e);
  fp_two_sum(p, c.hi, s, t);
  t = fp_add(t, fp_add(e, c.lo));
  return fp_make(s, t);
}
CGKS_HD fpair cg_madd(fpair a, fpair b, fpair c) { return fp_madd(a, b, c); }
CGKS_HD fpair cg_dot2(fpair a, fpair b, fpair c, fpair d) { return fp_dot2(a, b, c, d); }
CGKS_HD fpair cg_dot3(fpair a, fpair b, fpair c, fpair d, fpair e, fpair f) { return fp_dot3(a, b, c, d, e, f); }

/* ---- special functions in pair arithmetic, on the FP32 pipe ----
   (GB300's FP64 pipe runs at 1/64 of the FP32 rate, so the FP64 library
   functions cost more than these series.) */

/* 2^k as a float, -126 <= k <= 127 */
CGKS_HD float fp_pow2(int k) {
#if defined(__CUDA_ARCH__)
  return __int_as_float((k + 127) << 23);
#else
  return std::ldexp(1.0f, k);
#endif
}
CGKS_HD float fp_rint(float a) {
#if defined(__CUDA_ARCH__)
  return rintf(a);
#else
  return std::rint(a);
#endif
}
CGKS_HD float fp_rsqrt_est(float a) {
#if defined(__CUDA_ARCH__)
  return rsqrtf(a);
#else
  return 1.0f / std::sqrt(a);
#endif
}
/* a * s for s a power of two: exact unless it underflows */
CGKS_HD fpair fp_scale(fpair a, float s) { return fp_make(fp_mul(a.hi, s), fp_mul(a.lo, s)); }

/* exp(r) - 1 = sum_{n=1..13} r^n / n! for |r| <= ln2/2 (truncation below
   2e-16 of exp(r)), Horner's rule in renormalised pairs (r renormalised) */
CGKS_HD fpair fp_horner_step(fpair p, fpair r, double c) { return fp_addn(fp_muln(p, r), fpair(c)); }
CGKS_HD fpair fp_expm1_small(fpair r) {
  fpair p(1.0 / 6227020800.0);
  p = fp_horner_step(p, r, 1.0 / 479001600.0);
  p = fp_horner_step(p, r, 1.0 / 39916800.0);
  p = fp_horner_step(p, r, 1.0 / 3628800.0);
  p = fp_horner_step(p, r, 1.0 / 362880.0);
  p = fp_horner_step(p, r, 1.0 / 40320.0);
  p = fp_horner_step(p, r, 1.0 / 5040.0);
  p = fp_horner_step(p, r, 1.0 / 720.0);
  p = fp_horner_step(p, r, 1.0 / 120.0);
  p = fp_horner_step(p, r, 1.0 / 24.0);
  p = fp_horner_step(p, r, 1.0 / 6.0);
  p = fp_horner_step(p, r, 0.5);
  p = fp_horner_step(p, r, 1.0);
  return fp_muln(p, r);
}

/* exp(x) = 2^k exp(r), x = k ln2 + r, |r| <= ln2/2.  ln2 is split Cody-Waite
   style into a 16-bit float (k * its part is exact for |k| < 256), a float
   and a float remainder.  Below -87 the result is under the float range and
   is returned as 0 (the flux only adds such values to O(1) ones). */
CGKS_HD fpair cg_exp(fpair x) {
  x = fp_norm(x);
  if (x.hi < -87.0f) return fpair(0.0f);
  const float kf = fp_rint(fp_mul(x.hi, 1.44269504088896341f));
  const float L1 = 0.693145751953125f;        /* 16 significant bits */
  const float L2 = 1.42860676533018705e-06f; /* ln2 - L1 rounded to a float */
  const float L3 = 5.49792314810410715e-14f; /* ln2 - L1 - L2 rounded (residual 1.3e-21) */
  fpair r = fp_addn(x, -fpair(fp_mul(kf, L1)));
  float p2 = fp_mul(kf, L2);
  r = fp_addn(r, -fp_make(p2, fp_fma(kf, L2, -p2)));
  r = fp_addn(r, -fpair(fp_mul(kf, L3)));
  return fp_scale(fp_addn(fp_expm1_small(r), fpair(1.0f)), fp_pow2((int)kf));
}

CGKS_HD fpair cg_expm1(fpair x) {
  x = fp_norm(x);
  if (x.hi > -0.34657359f && x.hi < 0.34657359f) return fp_expm1_small(x);
  return fp_addn(cg_exp(x), fpair(-1.0f));
}

/* erfc(x) = 1 - (2/sqrt(pi)) x sum_{n>=0} (-x^2)^n / (n! (2n+1)) for |x| < 3/4
   (terms n <= 15; truncation below 5e-18); beyond, the FP64 library
   function rounded to a pair */
CGKS_HD fpair cg_erfc(fpair x) {
  x = fp_norm(x);
  if (!(x.hi > -0.75f && x.hi < 0.75f)) return fpair(cg_erfc((double)x));
  const fpair t = fp_muln(x, x);
  fpair p(-1.0 / (1307674368000.0 * 31.0));
  p = fp_horner_step(p, t, 1.0 / (87178291200.0 * 29.0));
  p = fp_horner_step(p, t, -1.0 / (6227020800.0 * 27.0));
  p = fp_horner_step(p, t, 1.0 / (479001600.0 * 25.0));
  p = fp_horner_step(p, t, -1.0 / (39916800.0 * 23.0));
  p = fp_horner_step(p, t, 1.0 / (3628800.0 * 21.0));
  p = fp_horner_step(p, t, -1.0 / (362880.0 * 19.0));
  p = fp_horner_step(p, t, 1.0 / (40320.0 * 17.0));
  p = fp_horner_step(p, t, -1.0 / (5040.0 * 15.0));
  p = fp_horner_step(p, t, 1.0 / (720.0 * 13.0));
  p = fp_horner_step(p, t, -1.0 / (120.0 * 11.0));
  p = fp_horner_step(p, t, 1.0 / (24.0 * 9.0));
  p = fp_horner_step(p, t, -1.0 / (6.0 * 7.0));
  p = fp_horner_step(p, t, 1.0 / (2.0 * 5.0));
  p = fp_horner_step(p, t, -1.0 / 3.0);
  p = fp_horner_step(p, t, 1.0);
  return fp_addn(fpair(1.0f), -fp_muln(fpair(1.12837916709551257390), fp_muln(x, p))); /* 2/sqrt(pi) */
}

/* 1/sqrt(x), x > 0: the FP32 estimate and two Newton steps
   y <- y + y (1 - x y^2) / 2 in renormalised pairs */
CGKS_HD fpair cg_rsqrt(fpair x) {
  x = fp_norm(x);
  fpair y(fp_rsqrt_est(x.hi));
  y = fp_addn(y, fp_scale(fp_muln(y, fp_addn(fpair(1.0f), -fp_muln(x, fp_muln(y, y)))), 0.5f));
  y = fp_addn(y, fp_scale(fp_muln(y, fp_addn(fpair(1.0f), -fp_muln(x, fp_muln(y, y)))), 0.5f));
  return y;
}
CGKS_HD fpair cg_sqrt(fpair x) {
  x = fp_norm(x);
  return x.hi > 0.f ? fp_muln(x, cg_rsqrt(x)) : fpair(0.0f);
}
CGKS_HD fpair cg_fabs(fpair x) {
  x = fp_norm(x);
  return x.hi < 0.f ? -x : x;
}
CGKS_HD fpair cg_norm(fpair x) { return fp_norm(x); }
CGKS_HD fpair cg_fma(fpair a, fpair b, fpair c) { return a * b + c; }

/* ---- unnormalised pairs for the reconstruction's linear maps ----
   fpacc holds hi + lo without the renormalisation after every operation: a
   sum is Knuth's two-sum of the high parts with the low parts and the sum
   error added into lo (8 operations), a multiply-add the exact product parts
   two-summed into the accumulator (12), a product the product parts (4).
   This is compensated summation in the manner of Ogita, Rump and Oishi's
   Sum2 / Dot2: the result is as accurate as if the sums of products were
   formed with about 48 bits and rounded once, which is what the
   reconstruction's maps (sums of at most ~100 products of the data with
   fixed rational coefficients) need.  Values are normalised only where a
   float of them is read (fpacc_norm). */
struct fpacc {
  float hi, lo;
  CGKS_HD fpacc() : hi(0.f), lo(0.f) {}
  CGKS_HD fpacc(double x) : hi((float)x), lo((float)(x - (double)(float)x)) {}
  CGKS_HD fpacc(float x) : hi(x), lo(0.f) {}
  CGKS_HD fpacc(int x) : fpacc((double)x) {}
};
CGKS_HD fpacc fpacc_make(float h, float l) {
  fpacc r;
  r.hi = h;
  r.lo = l;
  return r;
}
CGKS_HD fpacc operator+(fpacc a, fpacc b) {
  float s, e;
  fp_two_sum(a.hi, b.hi, s, e);
  return fpacc_make(s, fp_add(fp_add(a.lo, b.lo), e));
}
CGKS_HD fpacc operator-(fpacc a) { return fpacc_make(-a.hi, -a.lo); }
CGKS_HD fpacc operator-(fpacc a, fpacc b) { return a + (-b); }
CGKS_HD fpacc operator*(fpacc a, fpacc b) {
  const float p = fp_mul(a.hi, b.hi);
  float e = fp_fma(a.hi, b.hi, -p);
  e = fp_fma(a.hi, b.lo, e);
  e = fp_fma(a.lo, b.hi, e);
  return fpacc_make(p, e);
}
/* a b + c */
CGKS_HD fpacc cg_fma(fpacc a, fpacc b, fpacc c) {
  const float p = fp_mul(a.hi, b.hi);
  float e = fp_fma(a.hi, b.hi, -p);
  e = fp_fma(a.hi, b.lo, e);
  e = fp_fma(a.lo, b.hi, e);
  float s, t;
  fp_two_sum(c.hi, p, s, t);
  return fpacc_make(s, fp_add(c.lo, fp_add(e, t)));
}
/* hi + lo renormalised (two-sum: |lo| may exceed |hi| after cancellation) */
CGKS_HD fpacc fpacc_norm(fpacc a) {
  float s, e;
  fp_two_sum(a.hi, a.lo, s, e);
  return fpacc_make(s, e);
}

/* bit casts (host: the same bit logic through memcpy) */
CGKS_HD unsigned fp_fbits(float f) {
#if defined(__CUDA_ARCH__)
  return __float_as_uint(f);
#else
  unsigned u;
  __builtin_memcpy(&u, &f, sizeof u);
  return u;
#endif
}
CGKS_HD float fp_bitsf(unsigned u) {
#if defined(__CUDA_ARCH__)
  return __uint_as_float(u);
#else
  float f;
  __builtin_memcpy(&f, &u, sizeof f);
  return f;
#endif
}
CGKS_HD unsigned long long fp_dbits(double d) {
#if defined(__CUDA_ARCH__)
  return (unsigned long long)__double_as_longlong(d);
#else
  unsigned long long u;
  __builtin_memcpy(&u, &d, sizeof u);
  return u;
#endif
}
CGKS_HD double fp_bitsd(unsigned hi32, unsigned lo32) {
#if defined(__CUDA_ARCH__)
  return __hiloint2double((int)hi32, (int)lo32);
#else
  const unsigned long long u = ((unsigned long long)hi32 << 32) | lo32;
  double d;
  __builtin_memcpy(&d, &u, sizeof d);
  return d;
#endif
}

/* conversions on the integer pipe (GB300's FP64 pipe, which also converts
   between double and float, runs at 1/64 of the FP32 rate).
   double -> fpacc: hi = x truncated to its leading 24 bits, lo = the other
   29 bits of the significand rounded to 23 (relative error at most 2^-47).
   Magnitudes below 2^-103 are taken as (signed) 0; beyond the float range
   (and inf, NaN) the conversion is the rounded one, so inf and NaN carry
   through. */
CGKS_HD fpacc fpacc_from_double(double x) {
  const unsigned long long b = fp_dbits(x);
  const unsigned h32 = (unsigned)(b >> 32), l32 = (unsigned)b;
  const int ef = (int)((h32 >> 20) & 0x7ffu) - 896; /* biased float exponent of hi */
  if (ef > 254) return fpacc(x);
  const unsigned sgn = h32 & 0x80000000u;
  if (ef < 24) return fpacc_make(fp_bitsf(sgn), fp_bitsf(sgn));
  const float hi = fp_bitsf(sgn | ((unsigned)ef << 23) | ((h32 & 0xfffffu) << 3) | (l32 >> 29));
  const unsigned el = (unsigned)(ef - 23) << 23;          /* 2^(E-23), E the exponent of x */
  const unsigned r = ((l32 & 0x1fffffffu) + 32u) >> 6;   /* low 29 bits rounded to 23 (r <= 2^23) */
  const float lo = fp_sub(fp_bitsf(el + r), fp_bitsf(el)); /* 2^(E-46) r, exact */
  return fpacc_make(hi, fp_bitsf(fp_fbits(lo) | sgn));
}
/* float -> double, exact for normal floats; subnormal ones (below 2^-126,
   which the reconstruction meets only in the low part of values below
   about 2^-100) give a signed 0.  A branch to the rounded conversion for
   them would cost a conversion on the FP64 pipe at every call (measured
   +1.8 ms per TGV 128^3 reconstruction) */
CGKS_HD double fp_f2d_bits(float f) {
  const unsigned u = fp_fbits(f);
  const unsigned e = (u >> 23) & 0xffu;
  const unsigned e2 = e == 0u ? 0u : (e == 255u ? 2047u : e + 896u);
  const unsigned m = e == 0u ? 0u : (u & 0x7fffffu);
  return fp_bitsd((u & 0x80000000u) | (e2 << 20) | (m >> 3), m << 29);
}
/* hi + lo rounded once to double */
CGKS_HD double fpacc_to_double(fpacc a) { return fp_f2d_bits(a.hi) + fp_f2d_bits(a.lo); }

/* float -> double on the integer pipe, exact for every float: subnormals
   normalised by a count of leading zeros (a rare branch), infinities and
   NaNs carried through; the same value as the hardware conversion, which
   GB300 runs on its FP64 pipe */
CGKS_HD double fp_f2d_exact(float f) {
  const unsigned u = fp_fbits(f);
  const unsigned sgn = u & 0x80000000u;
  int e = (int)((u >> 23) & 0xffu);
  unsigned m = u & 0x7fffffu;
  if (e == 0) {
    if (m == 0u) return fp_bitsd(sgn, 0u);
#if defined(__CUDA_ARCH__)
    const int sh = __clz(m) - 8;
#else
    const int sh = __builtin_clz(m) - 8;
#endif
    m = (m << sh) & 0x7fffffu; /* the leading one becomes the implicit bit */
    e = 1 - sh;
  }
  const unsigned e2 = e == 255 ? 2047u : (unsigned)(e + 896);
  return fp_bitsd(sgn | (e2 << 20) | (m >> 3), m << 29);
}

template <class A, class B> struct cg_same { static constexpr bool value = false; };
template <class A> struct cg_same<A, A> { static constexpr bool value = true; };

/* storage <- compute type */
template <typename T> CGKS_HD T to_storage(const T& x) { return x; }
template <typename T> CGKS_HD T to_storage(const fpair& x) { return T((double)x); }

#endif
