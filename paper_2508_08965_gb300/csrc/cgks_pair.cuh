/*
 * Paired-FP32 arithmetic: the compute type of the interface flux in the
 * paired form (precision 2).  A value is the unevaluated sum hi + lo of two
 * floats, |lo| <= ulp(hi)/2: about 48 significant bits, on the FP32 pipe.
 *
 *   sum      Knuth's error-free two-sum of the high parts, plus the sum of
 *            the low parts, one renormalisation (11 operations; the form
 *            with a second two-sum for the low parts, 20 operations, is
 *            tighter when the sum cancels but measured no more accurate on
 *            whole steps of the flux against the FP64 oracle);
 *   product  the FMA residual of hi*hi plus the two cross terms;
 *   quotient a reciprocal estimate and two remainder corrections.
 *
 * Every operation goes through the round-to-nearest intrinsics (fp_add
 * ...), which the compiler never contracts into multiply-adds, so the
 * error-free steps stay exact.  exp, erfc, expm1, sqrt and 1/sqrt are taken in FP64 and rounded to
 * a pair (a few per Gauss point).  Conversions from double round twice
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

CGKS_HD fpair operator+(fpair a, fpair b) {
  float s, e;
  fp_two_sum(a.hi, b.hi, s, e);
  e = fp_add(e, fp_add(a.lo, b.lo));
  fp_fast_two_sum(s, e, s, e);
  return fp_make(s, e);
}
CGKS_HD fpair operator-(fpair a) { return fp_make(-a.hi, -a.lo); }
CGKS_HD fpair operator-(fpair a, fpair b) { return a + (-b); }
CGKS_HD fpair operator*(fpair a, fpair b) {
  const float p = fp_mul(a.hi, b.hi);
  float e = fp_fma(a.hi, b.hi, -p);
  e = fp_fma(a.hi, b.lo, e);
  e = fp_fma(a.lo, b.hi, e);
  float s;
  fp_fast_two_sum(p, e, s, e);
  return fp_make(s, e);
}
CGKS_HD fpair operator/(fpair a, fpair b) {
  const float r = fp_rcp(b.hi);
  const float q1 = fp_mul(a.hi, r);
  fpair rem = a - b * fpair(q1);
  const float q2 = fp_mul(rem.hi, r);
  rem = rem - b * fpair(q2);
  const float q3 = fp_mul(rem.hi, r);
  float s, e;
  fp_fast_two_sum(q1, q2, s, e);
  return fp_make(s, e) + fpair(q3);
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

CGKS_HD fpair cg_erfc(fpair x) { return fpair(cg_erfc((double)x)); }
CGKS_HD fpair cg_exp(fpair x) { return fpair(cg_exp((double)x)); }
CGKS_HD fpair cg_expm1(fpair x) { return fpair(cg_expm1((double)x)); }
CGKS_HD fpair cg_sqrt(fpair x) { return fpair(cg_sqrt((double)x)); }
CGKS_HD fpair cg_rsqrt(fpair x) { return fpair(cg_rsqrt((double)x)); }
CGKS_HD fpair cg_fabs(fpair x) { return x.hi < 0.f ? -x : x; }
CGKS_HD fpair cg_fma(fpair a, fpair b, fpair c) { return a * b + c; }

template <class A, class B> struct cg_same { static constexpr bool value = false; };
template <class A> struct cg_same<A, A> { static constexpr bool value = true; };

/* storage <- compute type */
template <typename T> CGKS_HD T to_storage(const T& x) { return x; }
template <typename T> CGKS_HD T to_storage(const fpair& x) { return T((double)x); }

#endif
