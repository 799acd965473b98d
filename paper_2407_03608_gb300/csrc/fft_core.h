// Building blocks of the shared-memory row FFTs (App. D's uniform FFT stage, computed
// row by row): small DFTs held in registers and one Stockham pass of a power-of-two
// complex FFT.  Everything here is __host__ __device__ so that the same code can be
// checked on the CPU.
//
// Conventions: forward transforms use e^{-2 pi i jk/N}, inverse ones e^{+2 pi i jk/N};
// nothing is normalised (the same as cuFFT).
#pragma once

#include <cmath>
#include <vector>

#include "ff64.h"

namespace gpn {
namespace fft {

#ifdef __CUDACC__
#define GPN_HD __host__ __device__ __forceinline__
#define GPN_HDC __host__ __device__ constexpr
#else
#define GPN_HD inline
#define GPN_HDC constexpr
#endif

template <typename T>
struct cpx {
  T x, y;
};
// a float-float complex value is 16 bytes: aligned so that it moves in one vector access
template <>
struct alignas(16) cpx<dd> {
  dd x, y;
};

template <typename T>
GPN_HD cpx<T> operator+(cpx<T> a, cpx<T> b) { return {a.x + b.x, a.y + b.y}; }
template <typename T>
GPN_HD cpx<T> operator-(cpx<T> a, cpx<T> b) { return {a.x - b.x, a.y - b.y}; }
template <typename T>
GPN_HD cpx<T> cmul(cpx<T> a, cpx<T> b) { return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }

// Float-float complex values inside the passes: sums without the closing renormalisation
// (add_lazy), and a product that forms each component as TwoProd(hi, hi) - TwoProd(hi, hi)
// with one TwoSum and the cross terms in the low word (16 operations a component instead
// of 25 for two products and a sum).  Pass::compute renormalises its outputs once.
GPN_HD cpx<dd> operator+(cpx<dd> a, cpx<dd> b) { return {add_lazy(a.x, b.x), add_lazy(a.y, b.y)}; }
GPN_HD cpx<dd> operator-(cpx<dd> a, cpx<dd> b) { return {sub_lazy(a.x, b.x), sub_lazy(a.y, b.y)}; }
// p.hi + p.lo = a b - c d (float-float, unnormalised)
GPN_HD dd dd_dot2(dd a, dd b, dd c, dd d, float sign) {
  using namespace ffops;
  const float p1 = mul(a.hi, b.hi);
  float e1 = fma(a.hi, b.hi, -p1);
  e1 = fma(a.hi, b.lo, e1);
  e1 = fma(a.lo, b.hi, e1);
  const float p2 = mul(c.hi, d.hi);
  float e2 = fma(c.hi, d.hi, -p2);
  e2 = fma(c.hi, d.lo, e2);
  e2 = fma(c.lo, d.hi, e2);
  const dd s = two_sum(p1, sign * p2);
  return {s.hi, add(s.lo, fma(sign, e2, e1))};
}
GPN_HD cpx<dd> cmul(cpx<dd> a, cpx<dd> b) {
  return {dd_dot2(a.x, b.x, a.y, b.y, -1.0f), dd_dot2(a.x, b.y, a.y, b.x, 1.0f)};
}
template <typename T>
GPN_HD cpx<T> renorm_c(cpx<T> a) { return a; }
GPN_HD cpx<dd> renorm_c(cpx<dd> a) { return {renorm(a.x), renorm(a.y)}; }
template <typename T>
GPN_HD cpx<T> conj(cpx<T> a) { return {a.x, -a.y}; }
// multiply by -i (forward) or +i (inverse)
template <bool INV, typename T>
GPN_HD cpx<T> rot90(cpx<T> a) { return INV ? cpx<T>{-a.y, a.x} : cpx<T>{a.y, -a.x}; }

// sqrt(1/2) and cos/sin(pi/8) to double precision (values of the constants, not of any
// library routine)
constexpr double kS45 = 0.70710678118654752440084436210485;
constexpr double kC22 = 0.92387953251128675612818318939679;
constexpr double kS22 = 0.38268343236508977172845998403040;

// in-place DFTs of v[0..R) with stride S in the register array (so that a DFT-16 can
// run its sub-transforms in place)
template <bool INV, typename T, int S = 1>
GPN_HD void dft2(cpx<T>* v) {
  const cpx<T> a = v[0], b = v[S];
  v[0] = a + b;
  v[S] = a - b;
}

template <bool INV, typename T, int S = 1>
GPN_HD void dft4(cpx<T>* v) {
  const cpx<T> a0 = v[0] + v[2 * S], a1 = v[0] - v[2 * S];
  const cpx<T> b0 = v[S] + v[3 * S], b1 = rot90<INV>(v[S] - v[3 * S]);
  v[0] = a0 + b0;
  v[2 * S] = a0 - b0;
  v[S] = a1 + b1;
  v[3 * S] = a1 - b1;
}

// multiply by e^{-+ 2 pi i k / 8}
template <bool INV, int K, typename T>
GPN_HD cpx<T> w8(cpx<T> a) {
  const T s = (T)kS45;
  if constexpr (K == 0) return a;
  if constexpr (K == 1) return INV ? cpx<T>{s * (a.x - a.y), s * (a.x + a.y)} : cpx<T>{s * (a.x + a.y), s * (a.y - a.x)};
  if constexpr (K == 2) return rot90<INV>(a);
  if constexpr (K == 3) return INV ? cpx<T>{-s * (a.x + a.y), s * (a.x - a.y)} : cpx<T>{s * (a.y - a.x), -s * (a.x + a.y)};
  return a;
}

// radix-8 = 2 x 4: even/odd split, DFT-4 of each, twiddles W8^k on the odd half
template <bool INV, typename T, int S = 1>
GPN_HD void dft8(cpx<T>* v) {
  dft4<INV, T, 2 * S>(v);      // v[0], v[2S], v[4S], v[6S]: even samples
  dft4<INV, T, 2 * S>(v + S);  // odd samples
  const cpx<T> o0 = v[S], o1 = w8<INV, 1>(v[3 * S]), o2 = w8<INV, 2>(v[5 * S]), o3 = w8<INV, 3>(v[7 * S]);
  const cpx<T> e0 = v[0], e1 = v[2 * S], e2 = v[4 * S], e3 = v[6 * S];
  v[0] = e0 + o0;
  v[4 * S] = e0 - o0;
  v[S] = e1 + o1;
  v[5 * S] = e1 - o1;
  v[2 * S] = e2 + o2;
  v[6 * S] = e2 - o2;
  v[3 * S] = e3 + o3;
  v[7 * S] = e3 - o3;
}

// multiply by e^{-+ 2 pi i k / 16} for k = 0..7 (exact constants)
template <bool INV, int K, typename T>
GPN_HD cpx<T> w16(cpx<T> a) {
  if constexpr (K % 2 == 0) {
    return w8<INV, K / 2>(a);
  } else {
    // theta = 2 pi K / 16: (cos, sin) = (C22, S22), (S22, C22), (-S22, C22), (-C22, S22)
    const T cr = K == 1 ? (T)kC22 : K == 3 ? (T)kS22 : K == 5 ? -(T)kS22 : -(T)kC22;
    const T si = K == 1 ? (T)kS22 : K == 3 ? (T)kC22 : K == 5 ? (T)kC22 : (T)kS22;
    const T sn = INV ? si : -si;
    return cmul(a, cpx<T>{cr, sn});   // {a.x cr - a.y sn, a.x sn + a.y cr}
  }
}

// radix-16 = 2 x 8
template <bool INV, typename T>
GPN_HD void dft16(cpx<T>* v) {
  dft8<INV, T, 2>(v);
  dft8<INV, T, 2>(v + 1);
  cpx<T> e[8], o[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    e[k] = v[2 * k];
    o[k] = v[2 * k + 1];
  }
  o[1] = w16<INV, 1>(o[1]);
  o[2] = w16<INV, 2>(o[2]);
  o[3] = w16<INV, 3>(o[3]);
  o[4] = w16<INV, 4>(o[4]);
  o[5] = w16<INV, 5>(o[5]);
  o[6] = w16<INV, 6>(o[6]);
  o[7] = w16<INV, 7>(o[7]);
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    v[k] = e[k] + o[k];
    v[k + 8] = e[k] - o[k];
  }
}

template <bool INV, int R, typename T>
GPN_HD void dft(cpx<T>* v) {
  if constexpr (R == 2) dft2<INV, T>(v);
  if constexpr (R == 4) dft4<INV, T>(v);
  if constexpr (R == 8) dft8<INV, T>(v);
  if constexpr (R == 16) dft16<INV, T>(v);
}

// Padded shared-memory index: one spare element per 16 spreads the stride-16 accesses
// of the first pass over the banks.
GPN_HD int pad(int i) { return i + (i >> 4); }

// One Stockham (autosort) pass of a length-N complex FFT, radix R, span Ns (the
// product of the radices of the earlier passes).  Butterfly j (0 <= j < N/R) reads
// the R inputs j + r N/R, multiplies input r by W_{Ns R}^{r (j mod Ns)}, takes a
// DFT-R and writes output r to ((j - j mod Ns) R + j mod Ns) + r Ns.  After the
// passes with spans 1, R1, R1 R2, ... the buffer holds the transform in natural
// order.  A thread handles NB butterflies j = t + b * nthreads.  The pass is split
// in a load and a store half because the transform is done in place: all loads of a
// pass must precede its stores (a block barrier in between on the device).
// tw(r, k, i) returns the twiddle of input r of a butterfly with k = j mod Ns, which is
// W_N^i with i = r k N / (Ns R) (0 <= i < N).
template <int R, int NB, typename T>
struct Pass {
  cpx<T> v[NB][R];

  GPN_HD void load(const cpx<T>* buf, int N, int t, int nthreads) {
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      const int j = t + b * nthreads;
#pragma unroll
      for (int r = 0; r < R; ++r) v[b][r] = buf[pad(j + r * (N / R))];
    }
  }

  // twiddles and the DFT-R of every butterfly, in registers
  template <bool INV, typename TW>
  GPN_HD void compute(const TW& tw, int N, int Ns, int t, int nthreads) {
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      const int j = t + b * nthreads;
      const int k = j & (Ns - 1);
      if (Ns > 1) {
        const int step = k * (N / (Ns * R));
#pragma unroll
        for (int r = 1; r < R; ++r) {
          cpx<T> w = tw(r, k, r * step);
          if (INV) w.y = -w.y;
          v[b][r] = cmul(v[b][r], w);
        }
      }
      dft<INV, R>(v[b]);
#pragma unroll
      for (int r = 0; r < R; ++r) v[b][r] = renorm_c(v[b][r]);
    }
  }

  // the outputs to their Stockham positions
  GPN_HD void write(cpx<T>* buf, int Ns, int t, int nthreads) const {
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      const int j = t + b * nthreads;
      const int k = j & (Ns - 1);
      const int base = (j - k) * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) buf[pad(base + r * Ns)] = v[b][r];
    }
  }

  template <bool INV, typename TW>
  GPN_HD void store(cpx<T>* buf, const TW& tw, int N, int Ns, int t, int nthreads) {
    compute<INV>(tw, N, Ns, t, nthreads);
    write(buf, Ns, t, nthreads);
  }
};

// Register view of the first pass: with nthreads = N / 16, the elements
// t + u * nthreads (u = 0..15) that a thread holds are exactly the inputs of its
// butterflies in the first pass (radix R at span 1): butterfly b, input r is u = b + r 16/R.
template <int R, int NB, typename T>
GPN_HD void first_pass_inputs(Pass<R, NB, T>& p, const cpx<T> (&x)[16]) {
#pragma unroll
  for (int b = 0; b < NB; ++b)
#pragma unroll
    for (int r = 0; r < R; ++r) p.v[b][r] = x[b + r * (16 / R)];
}

// W_N^i from two short tables, W_N^i = W_N^{64 (i / 64)} W_N^{i mod 64}: hi[q] = W_N^{64 q}
// (q < N / 64, at least one entry), lo[j] = W_N^j (j < 64).  One complex product per
// twiddle; the tables fit in shared memory for any N used here.
template <typename T>
struct Twiddle2 {
  const cpx<T>* hi;
  const cpx<T>* lo;
  GPN_HD cpx<T> operator()(int i) const { return cmul(hi[i >> 6], lo[i & 63]); }
  GPN_HD cpx<T> operator()(int, int, int i) const { return (*this)(i); }
};

// The radix-16 passes of a length-N FFT in the device kernels' order: one pass of radix
// 2^(L mod 4) at span 1 when L = log2 N is not a multiple of 4, then radix-16 passes at
// spans s0, 16 s0, ... (s0 = 2^(L mod 4)).  A radix-16 pass at span Ns > 1 needs the
// 15 Ns twiddles W_{16 Ns}^{r k} (r = 1..15, k < Ns); pass_table lays them out as
// [r - 1][k] (consecutive k for consecutive threads) and concatenates the passes.
GPN_HDC int first_span(int L) { return 1 << (L % 4); }
// offset of the table of the radix-16 pass at span Ns (a power of two >= first_span)
GPN_HDC int pass_table_offset(int L, int Ns) {
  int off = 0;
  for (int s = first_span(L); s < Ns; s *= 16)
    if (s > 1) off += 15 * s;
  return off;
}
GPN_HDC int pass_table_size(int L) { return pass_table_offset(L, 1 << L); }

// Host: the concatenated pass tables of a length-2^L FFT as interleaved (re, im)
// float64 values, computed from the angle 2 pi r k / (16 Ns) directly.
inline std::vector<double> pass_tables(int L) {
  std::vector<double> t(2 * (size_t)pass_table_size(L));
  for (int s = first_span(L); s < (1 << L); s *= 16) {
    if (s == 1) continue;
    const int off = pass_table_offset(L, s);
    for (int r = 1; r < 16; ++r)
      for (int k = 0; k < s; ++k) {
        const double th = 2.0 * 3.14159265358979323846264338327950288 * (double)(r * k) / (16.0 * s);
        t[2 * ((size_t)off + (r - 1) * s + k)] = std::cos(th);
        t[2 * ((size_t)off + (r - 1) * s + k) + 1] = -std::sin(th);
      }
  }
  return t;
}

// twiddle functor of one radix-16 pass over its table in consumption order
template <typename T>
struct PassTwiddle {
  const cpx<T>* tab;  // [15][Ns]
  int Ns;
  GPN_HD cpx<T> operator()(int r, int k, int) const { return tab[(r - 1) * Ns + k]; }
};

// Real-input split (forward): z[n] = x[2n] + i x[2n+1] with Z = FFT_{N2}(z).  The
// spectrum of x (length nf = 2 N2) at k, 0 <= k <= N2, is
//   X[k] = (Z[k] + conj(Z[N2-k])) / 2 - (i/2) W_nf^k (Z[k] - conj(Z[N2-k])),
// with Z[N2] = Z[0] and W_nf^k = e^{-2 pi i k / nf} given as wk.
template <typename T>
GPN_HD cpx<T> r2c_split(cpx<T> zk, cpx<T> znk, cpx<T> wk) {
  const cpx<T> c = conj(znk);
  const cpx<T> e = zk + c, o = zk - c;  // 2 Fe, 2 i Fo
  const cpx<T> wo = cmul(wk, o);
  // X = e/2 - (i/2) wo
  return {(T)0.5 * (e.x + wo.y), (T)0.5 * (e.y - wo.x)};
}

// Inverse split: given the half spectrum X[0..N2] of a real x of length nf, with
// X[N2 - k] passed as xnk, the length-N2 input of the inverse complex FFT whose
// result is z[n] = x[2n] + i x[2n+1] (unnormalised, as a C2R transform) is
//   Z'[k] = (X[k] + conj(X[N2-k])) + i conj(W_nf^k) (X[k] - conj(X[N2-k])).
template <typename T>
GPN_HD cpx<T> c2r_merge(cpx<T> xk, cpx<T> xnk, cpx<T> wk) {
  const cpx<T> c = conj(xnk);
  const cpx<T> e = xk + c, o = xk - c;
  const cpx<T> wo = cmul(conj(wk), o);
  return {e.x - wo.y, e.y + wo.x};
}

}  // namespace fft
}  // namespace gpn
