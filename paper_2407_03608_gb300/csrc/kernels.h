// Device helpers shared by the hot-path kernels (spread, diag, interp).
#pragma once

#include <cuda_runtime.h>

#include "ff64.h"
#include "plan.h"

namespace gpn {

template <typename T>
struct Cplx;
template <>
struct Cplx<float> {
  using type = float2;
};
template <>
struct Cplx<double> {
  using type = double2;
};

// Storage type of a plan precision: GP_FP32 float, GP_FP64 double, GP_DF64 dd (float-float).
template <typename T>
struct is_dd {
  static constexpr bool value = false;
};
template <>
struct is_dd<dd> {
  static constexpr bool value = true;
};

// Exponential-of-semicircle spreading kernel psi(s) = exp(beta (sqrt(1 - (2s/w)^2) - 1))
// for |s| < w/2 (Barnett, Magland & af Klinteberg's ES kernel), s in fine-grid cells.
// The float version takes beta2 = beta * log2(e) (folded on the host) and uses the
// hardware base-2 exponential; the double version takes beta itself.
template <typename T>
__device__ __forceinline__ T es_psi(T s, T beta, T inv_halfw);

template <>
__device__ __forceinline__ float es_psi<float>(float s, float beta2, float inv_halfw) {
  const float z = s * inv_halfw;
  const float q = 1.0f - z * z;
  return q > 0.0f ? exp2f(beta2 * (sqrtf(q) - 1.0f)) : 0.0f;
}

template <>
__device__ __forceinline__ double es_psi<double>(double s, double beta, double inv_halfw) {
  const double z = s * inv_halfw;
  const double q = 1.0 - z * z;
  return q > 0.0 ? exp(beta * (sqrt(q) - 1.0)) : 0.0;
}

// Kernel shape parameter as the device code expects it (see es_psi).
template <typename T>
inline T es_beta_arg(double beta) {
  return sizeof(T) == 4 ? (T)(beta * 1.4426950408889634074) : (T)beta;
}

// psi(j - xi) at the integer cell offset j.  Float-float plans evaluate the kernel in
// float-float on the FP32 pipe (es_psi_dd of ff64.h: within about 5e-14 of psi(0) = 1),
// not with the float64 exp, which on GB300 made the kernel values the largest cost of the
// spread and the interpolation.
template <typename T>
__device__ __forceinline__ T psi_at(int j, T xi, T beta, T inv_halfw) {
  return es_psi<T>((T)j - xi, beta, inv_halfw);
}
template <>
__device__ __forceinline__ dd psi_at<dd>(int j, dd xi, dd beta, dd inv_halfw) {
  return es_psi_dd(j, xi, beta, inv_halfw);
}

// Warp shuffles of plan values (a float-float value moves as its two words).
template <typename T>
__device__ __forceinline__ T shfl_val(T v, int src) {
  return __shfl_sync(0xffffffffu, v, src);
}
template <>
__device__ __forceinline__ dd shfl_val<dd>(dd v, int src) {
  return {__shfl_sync(0xffffffffu, v.hi, src), __shfl_sync(0xffffffffu, v.lo, src)};
}
template <typename T>
__device__ __forceinline__ T shfl_down_val(T v, int o) {
  return __shfl_down_sync(0xffffffffu, v, o);
}
template <>
__device__ __forceinline__ dd shfl_down_val<dd>(dd v, int o) {
  return {__shfl_down_sync(0xffffffffu, v.hi, o), __shfl_down_sync(0xffffffffu, v.lo, o)};
}
template <typename T>
__device__ __forceinline__ T shfl_xor_val(T v, int o) {
  return __shfl_xor_sync(0xffffffffu, v, o);
}
template <>
__device__ __forceinline__ dd shfl_xor_val<dd>(dd v, int o) {
  return {__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
}

// acc += a b (one fused step for float-float)
template <typename T>
__device__ __forceinline__ void madd(T& acc, T a, T b) {
  acc += a * b;
}
template <>
__device__ __forceinline__ void madd<dd>(dd& acc, dd a, dd b) {
  acc = fma_dd(a, b, acc);
}

// Read-only load of a plan value
template <typename T>
__device__ __forceinline__ T ldg_val(const T* p) {
  return __ldg(p);
}
template <>
__device__ __forceinline__ dd ldg_val<dd>(const dd* p) {
  const float2 u = __ldg(reinterpret_cast<const float2*>(p));
  return {u.x, u.y};
}

// acc += a b without renormalising float-float sums; renorm_val() closes them (identity for
// float and double)
template <typename T>
__device__ __forceinline__ void madd_lazy(T& acc, T a, T b) {
  acc += a * b;
}
template <>
__device__ __forceinline__ void madd_lazy<dd>(dd& acc, dd a, dd b) {
  acc = fma_dd_lazy(a, b, acc);
}
template <typename T>
__device__ __forceinline__ T renorm_val(T v) {
  return v;
}
template <>
__device__ __forceinline__ dd renorm_val<dd>(dd v) {
  return renorm(v);
}

// A plan value to float64
template <typename T>
__device__ __forceinline__ double to_f64(T v) {
  return (double)v;
}

// Chebyshev weights of Eq. (Wk) from the paper-native fields of one point:
// w_k(x) = w (2 pi sigma^2)^(-d/2) P_k(sigma), P_k by the barycentric formula on the
// Chebyshev-Lobatto nodes (weights (-1)^k, halved at both ends); exact at a node.
struct ChebArgs {
  double nodes[kMaxChannels];
  double bary[kMaxChannels];
  int C;
  int d;
};
__device__ __forceinline__ void cheb_weights(double w, double s, const ChebArgs& cb, double* out) {
  const double pre = w * pow(6.283185307179586476925286766559 * s * s, -0.5 * cb.d);
  int hit = -1;
  for (int k = 0; k < cb.C; ++k)
    if (s == cb.nodes[k]) hit = k;
  if (hit >= 0 || cb.C == 1) {
    for (int k = 0; k < cb.C; ++k) out[k] = (k == hit || cb.C == 1) ? pre : 0.0;
    return;
  }
  double den = 0.0;
  for (int k = 0; k < cb.C; ++k) den += cb.bary[k] / (s - cb.nodes[k]);
  for (int k = 0; k < cb.C; ++k) out[k] = pre * (cb.bary[k] / (s - cb.nodes[k])) / den;
}

// Channel-count buckets: kernels keep per-channel values in registers sized by a
// compile-time bound CMAX >= C.
inline int cmax_bucket(int C) { return C <= 8 ? 8 : (C <= 12 ? 12 : (C <= 16 ? 16 : 32)); }

inline int blocks_for(long long n, int t) { return (int)((n + t - 1) / t); }

// ---- mbarrier + TMA (cp.async.bulk.tensor) helpers, sm_90+ PTX -------------------

__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
  // make the initialised barrier visible to the async (TMA) proxy
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for the phase with the given parity: returns false after
// max_polls failed polls (each poll itself blocks for a short hardware interval).
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, unsigned parity, long long max_polls) {
  for (long long i = 0; i < max_polls; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// TMA tile loads into shared memory, completing on the mbarrier (coordinates in
// elements, innermost first).
__device__ __forceinline__ void tma_load_3d(void* dst, const void* tmap, int c0, int c1, int c2,
                                            unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
      ::"r"(smem_addr(dst)), "l"(tmap), "r"(c0), "r"(c1), "r"(c2), "r"(smem_addr(bar))
      : "memory");
}

__device__ __forceinline__ void tma_load_4d(void* dst, const void* tmap, int c0, int c1, int c2, int c3,
                                            unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];"
      ::"r"(smem_addr(dst)), "l"(tmap), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_addr(bar))
      : "memory");
}

// Device status codes written by kernels whose bounded waits ran out.
constexpr int kStatusTimeout = 1;

}  // namespace gpn
