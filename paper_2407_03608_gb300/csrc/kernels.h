// Device helpers shared by the hot-path kernels (spread, diag, interp).
#pragma once

#include <cuda_runtime.h>

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
