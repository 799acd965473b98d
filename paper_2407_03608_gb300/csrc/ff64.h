// Float-float ("double-float") arithmetic for the GP_DF64 plans: a value is the
// unevaluated sum hi + lo of two FP32 numbers, normalised so that |lo| <= ulp(hi) / 2,
// which carries about 48 significant bits.  On GB300 the FP64 pipe issues about one
// sixtieth of the FP32 rate, so the transforms, spreading and interpolation of the
// FP64-grade plans run their sums in this type on the FP32 pipe instead.
//
// Building blocks (error-free transformations):
//   TwoSum (Knuth): s = fl(a + b) and the exact rounding error e, a + b = s + e, in six
//     additions and no branch (any order of magnitudes);
//   FastTwoSum (Dekker): the same in three additions when |a| >= |b|;
//   TwoProd by fused multiply-add: p = fl(a b), e = fma(a, b, -p), a b = p + e exactly.
// Addition is the "sloppy" form (TwoSum of the high words, the low words added with the
// error, renormalised by FastTwoSum): its error is within a few u^2 (|a| + |b|), u = 2^-24,
// the normwise bound an FFT's error analysis asks for.  Multiplication takes the TwoProd
// of the high words plus the two cross products.  Every FP32 operation uses the
// round-to-nearest intrinsics, which the compiler never contracts into a fused
// multiply-add (a contraction would break the error-free steps).
//
// Host versions (for the CPU checks of the FFT building blocks) use plain float
// arithmetic; compile them without floating-point contraction.
#pragma once

#include <cmath>

#ifdef __CUDACC__
#define FF_HD __host__ __device__ __forceinline__
#else
#define FF_HD inline
#endif

namespace gpn {

namespace ffops {
#ifdef __CUDA_ARCH__
FF_HD float add(float a, float b) { return __fadd_rn(a, b); }
FF_HD float sub(float a, float b) { return __fsub_rn(a, b); }
FF_HD float mul(float a, float b) { return __fmul_rn(a, b); }
FF_HD float fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
#else
FF_HD float add(float a, float b) { return a + b; }
FF_HD float sub(float a, float b) { return a - b; }
FF_HD float mul(float a, float b) { return a * b; }
FF_HD float fma(float a, float b, float c) { return __builtin_fmaf(a, b, c); }
#endif
}  // namespace ffops

struct alignas(8) dd {
  float hi, lo;

  dd() = default;
  FF_HD constexpr dd(float h, float l) : hi(h), lo(l) {}
  // the nearest float and the float nearest to the remainder (exact for |x| in the
  // normal float range, to about 2^-48 relative)
  FF_HD dd(double x) : hi((float)x), lo((float)(x - (double)(float)x)) {}
  FF_HD dd(int x) : dd((double)x) {}
  FF_HD explicit operator double() const { return (double)hi + (double)lo; }
};

// s + e = a + b exactly (Knuth's TwoSum)
FF_HD dd two_sum(float a, float b) {
  using namespace ffops;
  const float s = add(a, b);
  const float bb = sub(s, a);
  const float e = add(sub(a, sub(s, bb)), sub(b, bb));
  return {s, e};
}

// s + e = a + b exactly when |a| >= |b| (Dekker's FastTwoSum)
FF_HD dd fast_two_sum(float a, float b) {
  using namespace ffops;
  const float s = add(a, b);
  return {s, sub(b, sub(s, a))};
}

FF_HD dd operator+(dd a, dd b) {
  using namespace ffops;
  const dd s = two_sum(a.hi, b.hi);
  return fast_two_sum(s.hi, add(s.lo, add(a.lo, b.lo)));
}

FF_HD dd operator-(dd a) { return {-a.hi, -a.lo}; }

FF_HD dd operator-(dd a, dd b) { return a + (-b); }

FF_HD dd operator*(dd a, dd b) {
  using namespace ffops;
  const float p = mul(a.hi, b.hi);
  float e = fma(a.hi, b.hi, -p);
  e = fma(a.hi, b.lo, e);
  e = fma(a.lo, b.hi, e);
  return fast_two_sum(p, e);
}

// a / b: the float quotient q = a.hi / b.hi refined by one correction, q + (a - q b) / b.hi,
// with q b formed exactly (TwoProd); relative error a few u^2
FF_HD dd operator/(dd a, dd b) {
  using namespace ffops;
  const float q = a.hi / b.hi;
  const float p = mul(q, b.hi);
  const float e = fma(q, b.hi, -p);                    // q b.hi = p + e exactly
  const float r = sub(add(sub(sub(a.hi, p), e), a.lo), mul(q, b.lo));
  return fast_two_sum(q, r / b.hi);
}

// The same sum and product without the closing FastTwoSum: the two words still add up to
// the result, but the low word may exceed half an ulp of the high one.  The FFT passes
// chain these inside a butterfly and renormalise each output once (renorm), which saves
// three operations per step; a few unnormalised steps in a row cost a few u^2 of
// accuracy, as the normalised forms do.
FF_HD dd add_lazy(dd a, dd b) {
  using namespace ffops;
  const dd s = two_sum(a.hi, b.hi);
  return {s.hi, add(s.lo, add(a.lo, b.lo))};
}
FF_HD dd sub_lazy(dd a, dd b) { return add_lazy(a, dd(-b.hi, -b.lo)); }
FF_HD dd renorm(dd a) { return fast_two_sum(a.hi, a.lo); }

FF_HD dd& operator+=(dd& a, dd b) { return a = a + b; }
FF_HD dd& operator-=(dd& a, dd b) { return a = a - b; }
FF_HD dd& operator*=(dd& a, dd b) { return a = a * b; }

// a * b + c in one step (TwoProd of the high words, cross products and c.lo folded into
// the error word before one TwoSum with c.hi)
FF_HD dd fma_dd(dd a, dd b, dd c) {
  using namespace ffops;
  const float p = mul(a.hi, b.hi);
  float e = fma(a.hi, b.hi, -p);
  e = fma(a.hi, b.lo, e);
  e = fma(a.lo, b.hi, e);
  const dd s = two_sum(p, c.hi);
  return fast_two_sum(s.hi, add(s.lo, add(e, c.lo)));
}

// a * b + c without the closing FastTwoSum (12 operations instead of 15): for sums of a
// bounded number of terms, renormalised (renorm) before the low word grows past a few
// ulps of the high one
FF_HD dd fma_dd_lazy(dd a, dd b, dd c) {
  using namespace ffops;
  const float p = mul(a.hi, b.hi);
  float e = fma(a.hi, b.hi, -p);
  e = fma(a.hi, b.lo, e);
  e = fma(a.lo, b.hi, e);
  const dd s = two_sum(p, c.hi);
  return {s.hi, add(s.lo, add(e, c.lo))};
}

// A float-float constant from a double (folded at compile time)
FF_HD constexpr dd ddc(double x) { return dd((float)x, (float)(x - (double)(float)x)); }

// Square root of a non-negative float-float value: the float square root refined by one
// Newton step, s + (a - s^2) / (2 s), with s^2 formed exactly by TwoProd (relative error
// a few u^2).  Zero or negative inputs give zero.
FF_HD dd sqrt_dd(dd a) {
  using namespace ffops;
  if (!(a.hi > 0.0f)) return dd(0.0f, 0.0f);
  const float s = sqrtf(a.hi);
  const float p = mul(s, s);
  const float e = fma(s, s, -p);                       // s^2 = p + e exactly
  const float r = add(sub(sub(a.hi, p), e), a.lo);     // a - s^2 (a.hi - p is exact: p ~ a.hi)
  return fast_two_sum(s, r / add(s, s));
}

// e^u of a float-float value by range reduction: u = k ln 2 + r with k = round(u / ln 2),
// r = u - k ln 2 in float-float (|r| <= ln(2)/2), then e^r = (e^(r/8))^8 with e^(r/8) from
// its Taylor series to degree 9 (|r/8| < 0.044: the remainder is below 1e-20), three
// squarings, and the exact scaling by 2^k.  Relative error about 1e-14 (the squarings
// multiply the rounding of e^(r/8) by eight).  For the arguments used here, -60 < u <= 0.
FF_HD dd exp_dd(dd u) {
  using namespace ffops;
  const float k = rintf(mul(u.hi, 1.44269504088896340736f));
  const dd r0 = u - dd(k, 0.0f) * ddc(0.69314718055994530942);
  const dd r = dd(ldexpf(r0.hi, -3), ldexpf(r0.lo, -3));
  dd p = ddc(1.0 / 362880.0);                          // 1/9!
  p = fma_dd(p, r, ddc(1.0 / 40320.0));
  p = fma_dd(p, r, ddc(1.0 / 5040.0));
  p = fma_dd(p, r, ddc(1.0 / 720.0));
  p = fma_dd(p, r, ddc(1.0 / 120.0));
  p = fma_dd(p, r, ddc(1.0 / 24.0));
  p = fma_dd(p, r, ddc(1.0 / 6.0));
  p = fma_dd(p, r, dd(0.5f, 0.0f));
  p = fma_dd(p, r, dd(1.0f, 0.0f));
  p = fma_dd(p, r, dd(1.0f, 0.0f));
  p = p * p;
  p = p * p;
  p = p * p;
  const int ki = (int)k;
  return dd(ldexpf(p.hi, ki), ldexpf(p.lo, ki));
}

// The exponential-of-semicircle spreading kernel psi(s) = exp(beta (sqrt(1 - z^2) - 1)),
// z = s inv_halfw, at s = j - xi (integer cell offset j), in float-float.  The exponent is
// formed as -beta z^2 / (1 + sqrt(1 - z^2)), which avoids the cancellation of
// sqrt(1 - z^2) - 1 near z = 0.  Zero outside |z| < 1.
FF_HD dd es_psi_dd(int j, dd xi, dd beta, dd inv_halfw) {
  const dd z = (dd((float)j, 0.0f) - xi) * inv_halfw;
  const dd z2 = z * z;
  const dd q = dd(1.0f, 0.0f) - z2;
  if (!(q.hi > 0.0f)) return dd(0.0f, 0.0f);
  return exp_dd(-(beta * z2) / (sqrt_dd(q) + dd(1.0f, 0.0f)));
}

}  // namespace gpn
