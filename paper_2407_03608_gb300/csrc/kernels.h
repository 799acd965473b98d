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
template <typename T>
__device__ __forceinline__ T es_psi(T s, T beta, T inv_halfw) {
  T z = s * inv_halfw;
  T q = T(1) - z * z;
  return q > T(0) ? exp(beta * (sqrt(q) - T(1))) : T(0);
}

// Channel-count buckets: kernels keep per-channel values in registers sized by a
// compile-time bound CMAX >= C.
inline int cmax_bucket(int C) { return C <= 8 ? 8 : (C <= 12 ? 12 : (C <= 16 ? 16 : 32)); }

inline int blocks_for(long long n, int t) { return (int)((n + t - 1) / t); }

}  // namespace gpn
