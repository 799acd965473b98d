// Steps (2b) + (3) + (4a) of Sec. 4.2 on the R2C half spectrum of the fine grids.
//
// Inside the mode box |n_a| <= M:   a_k'[n] = sum_k A'_k'k[n] b_k[n],
// with A' = A / psihat(n)^2 the tensor of Remark rem:step3 with both NUFFT
// deconvolutions folded in; outside the box the spectrum is set to zero (the
// restriction Pi of Sec. 3.4), which is the input the inverse FFT of step (4)
// needs.  A' is real symmetric and stored as its packed upper triangle,
// A'[p][f] with p running over (k1 <= k2) pairs and f over the half box, so
// consecutive threads read consecutive frequencies.  The C inputs b_k[n] stay in
// registers; each output channel is one row of A' applied to them (the second
// read of each off-diagonal entry is served by L1).
//
// Launch: blockIdx.y = row of the spectrum (all coordinates but the last),
// threads over the last (halved) coordinate.
#include <algorithm>

#include "kernels.h"

namespace gpn {

namespace {

template <typename T>
struct DiagArgs {
  typename Cplx<T>::type* spec;   // (R*C) x S
  const T* A;                     // packed upper triangle [p][f]
  long long S;                    // half-spectrum elements per channel
  long long half;                 // nf/2 + 1
  long long nf;
  long long M;
  long long n_freq;
  long long row0;                 // first spectrum row of this launch
  int d;
  int C;
  int R;
};

// EXACT: C == CMAX (<= 12); the C(C+1)/2 entries of A' at the frequency are loaded into
// registers at once, before the right-hand sides.
template <typename T, int D, int CMAX, bool EXACT>
__global__ void __launch_bounds__(128) k_diag(DiagArgs<T> a) {
  using C2 = typename Cplx<T>::type;
  const long long il = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (il >= a.half) return;
  const long long row = a.row0 + blockIdx.y;
  // leading coordinates of this row, as signed frequencies
  bool inbox = il <= a.M;
  long long lead = 0;
  {
    long long rest = row;
    long long mq[kMaxDim];
#pragma unroll
    for (int q = D - 2; q >= 0; --q) {
      long long i = rest % a.nf;
      rest /= a.nf;
      mq[q] = (i <= a.nf / 2) ? i : i - a.nf;
    }
#pragma unroll
    for (int q = 0; q < D - 1; ++q) {
      inbox = inbox && mq[q] >= -a.M && mq[q] <= a.M;
      lead = lead * (2 * a.M + 1) + (mq[q] + a.M);
    }
  }
  const long long s = row * a.half + il;
  const int C = a.C;
  if (!inbox) {
    for (int r = 0; r < a.R; ++r) {
      C2* base = a.spec + (size_t)r * C * a.S + s;
#pragma unroll
      for (int k = 0; k < CMAX; ++k)
        if (k < C) base[(size_t)k * a.S] = C2{T(0), T(0)};
    }
    return;
  }
  const long long f = lead * (a.M + 1) + il;
  if constexpr (EXACT) {
    constexpr int NP = CMAX * (CMAX + 1) / 2;
    T av[NP];
#pragma unroll
    for (int p = 0; p < NP; ++p) av[p] = __ldg(a.A + (size_t)p * a.n_freq + f);
    for (int r = 0; r < a.R; ++r) {
      C2* base = a.spec + (size_t)r * CMAX * a.S + s;
      C2 b[CMAX];
#pragma unroll
      for (int k = 0; k < CMAX; ++k) b[k] = base[(size_t)k * a.S];
#pragma unroll
      for (int k1 = 0; k1 < CMAX; ++k1) {
        T re = T(0), im = T(0);
#pragma unroll
        for (int k2 = 0; k2 < CMAX; ++k2) {
          const int lo = k1 < k2 ? k1 : k2, hi = k1 < k2 ? k2 : k1;
          const T av_ = av[lo * CMAX - lo * (lo - 1) / 2 + (hi - lo)];
          re += av_ * b[k2].x;
          im += av_ * b[k2].y;
        }
        base[(size_t)k1 * a.S] = C2{re, im};
      }
    }
    return;
  }
  for (int r = 0; r < a.R; ++r) {
    C2* base = a.spec + (size_t)r * C * a.S + s;
    C2 b[CMAX];
#pragma unroll
    for (int k = 0; k < CMAX; ++k) b[k] = k < C ? base[(size_t)k * a.S] : C2{T(0), T(0)};
#pragma unroll 1
    for (int k1 = 0; k1 < C; ++k1) {
      T re = T(0), im = T(0);
      const int rowp = k1 * C - (k1 * (k1 - 1)) / 2;   // packed index of (k1, k1)
#pragma unroll
      for (int k2 = 0; k2 < CMAX; ++k2) {
        if (k2 < C) {
          // (min, max) of (k1, k2) in the packed upper triangle
          const int p = k2 >= k1 ? rowp + (k2 - k1) : k2 * C - (k2 * (k2 - 1)) / 2 + (k1 - k2);
          const T av = __ldg(a.A + (size_t)p * a.n_freq + f);
          re += av * b[k2].x;
          im += av * b[k2].y;
        }
      }
      base[(size_t)k1 * a.S] = C2{re, im};
    }
  }
}

// Short spectra with more than 12 channels (1-D plans): one thread per (frequency,
// output channel), blockDim = (32 frequencies, C channels).  The block stages the C
// inputs of its frequencies in shared memory before any output is written (step 3 runs
// in place), so C times more threads share the work than in k_diag.
template <typename T>
__global__ void __launch_bounds__(1024) k_diag_small(DiagArgs<T> a) {
  using C2 = typename Cplx<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C2* s_b = reinterpret_cast<C2*>(smem_raw);   // [C][32]
  const int tx = threadIdx.x, k1 = threadIdx.y, C = a.C;
  const long long il = blockIdx.x * 32ll + tx;
  const long long row = a.row0 + blockIdx.y;
  bool inbox = il <= a.M;
  long long lead = 0;
  {
    long long rest = row;
    long long mq[kMaxDim];
    for (int q = a.d - 2; q >= 0; --q) {
      const long long i = rest % a.nf;
      rest /= a.nf;
      mq[q] = (i <= a.nf / 2) ? i : i - a.nf;
    }
    for (int q = 0; q < a.d - 1; ++q) {
      inbox = inbox && mq[q] >= -a.M && mq[q] <= a.M;
      lead = lead * (2 * a.M + 1) + (mq[q] + a.M);
    }
  }
  const bool valid = il < a.half;
  const long long s = row * a.half + il;
  const long long f = lead * (a.M + 1) + il;
  const int rowp = k1 * C - (k1 * (k1 - 1)) / 2;   // packed index of (k1, k1)
  for (int r = 0; r < a.R; ++r) {
    C2* base = a.spec + (size_t)r * C * a.S + s;
    s_b[k1 * 32 + tx] = valid ? base[(size_t)k1 * a.S] : C2{T(0), T(0)};
    __syncthreads();
    if (valid) {
      C2 out{T(0), T(0)};
      if (inbox) {
        for (int k2 = 0; k2 < C; ++k2) {
          const int p = k2 >= k1 ? rowp + (k2 - k1) : k2 * C - (k2 * (k2 - 1)) / 2 + (k1 - k2);
          const T av = __ldg(a.A + (size_t)p * a.n_freq + f);
          const C2 b = s_b[k2 * 32 + tx];
          out.x += av * b.x;
          out.y += av * b.y;
        }
      }
      base[(size_t)k1 * a.S] = out;
    }
    __syncthreads();   // s_b is refilled for the next rhs
  }
}

template <typename T, int D, int NC>
void launch_exact(const DiagArgs<T>& a, dim3 grid, cudaStream_t st) {
  if constexpr (NC <= 12) {
    if (a.C == NC) {
      k_diag<T, D, NC, true><<<grid, 128, 0, st>>>(a);
      return;
    }
    launch_exact<T, D, NC + 1>(a, grid, st);
  }
}

template <typename T, int D>
void launch_c(const DiagArgs<T>& a, dim3 grid, cudaStream_t st) {
  if (a.C <= 12) return launch_exact<T, D, 1>(a, grid, st);
  switch (cmax_bucket(a.C)) {
    case 16: k_diag<T, D, 16, false><<<grid, 128, 0, st>>>(a); break;
    default: k_diag<T, D, 32, false><<<grid, 128, 0, st>>>(a);
  }
}

template <typename T>
void diag_impl(Plan& plan, int R, cudaStream_t st) {
  const GridGeom& g = plan.geom;
  DiagArgs<T> a{};
  a.spec = (typename Cplx<T>::type*)plan.spec;
  a.A = (const T*)plan.a_tensor;
  a.S = plan.spec_elems;
  a.half = g.nf / 2 + 1;
  a.nf = g.nf;
  a.M = g.M;
  a.n_freq = plan.n_freq;
  a.C = g.C;
  a.R = R;
  a.d = g.d;
  const long long rows = a.S / a.half;
  if (g.C > 12 && a.S * g.C <= 152ll * 2048) {
    // short spectrum, many channels: thread per (frequency, output channel)
    const size_t smem = sizeof(typename Cplx<T>::type) * 32 * g.C;
    for (long long r0 = 0; r0 < rows; r0 += 65535) {
      a.row0 = r0;
      dim3 grid((unsigned)((a.half + 31) / 32), (unsigned)std::min<long long>(65535, rows - r0));
      k_diag_small<T><<<grid, dim3(32, g.C), smem, st>>>(a);
    }
    GPN_CUDA(cudaGetLastError());
    return;
  }
  // gridDim.y is limited to 65535: launch the rows in chunks
  for (long long r0 = 0; r0 < rows; r0 += 65535) {
    a.row0 = r0;
    dim3 grid((unsigned)blocks_for(a.half, 128), (unsigned)std::min<long long>(65535, rows - r0));
    switch (g.d) {
      case 1: launch_c<T, 1>(a, grid, st); break;
      case 2: launch_c<T, 2>(a, grid, st); break;
      default: launch_c<T, 3>(a, grid, st);
    }
  }
  GPN_CUDA(cudaGetLastError());
}

}  // namespace

void launch_diag(Plan& plan, int R, cudaStream_t st) {
  if (plan.lean) return launch_step3_lean(plan, R, st);
  if (plan.tr3) return tr3_diag(plan, R, st);
  if (plan.rowfft) return rowfft_diag(plan, R, st);
  if (plan.precision == GP_FP32)
    diag_impl<float>(plan, R, st);
  else
    diag_impl<double>(plan, R, st);
}

}  // namespace gpn
