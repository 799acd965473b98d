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

}  // namespace gpn
