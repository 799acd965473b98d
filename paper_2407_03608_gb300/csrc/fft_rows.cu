// Pruned fine-grid transforms for d <= 2 (App. D type-1/type-2 NUFFT stages, with
// step (3) of Sec. 4.2 between them).
//
// Only the modes |n_a| <= M are ever used (the grid restriction Pi of Sec. 3.4), and
// only the rows and columns of the fine grid that hold spread data (or that the
// interpolation reads) are non-zero or needed.  The 2-D transform is therefore
// split by axis:
//   1. row R2C (last axis, this file): each CTA transforms one grid row of length nf
//      in shared memory (a complex Stockham FFT of length nf/2 on even/odd pairs,
//      radix 4 with one radix-2 stage when needed, then the real-to-complex split)
//      and writes only the half-spectrum entries 0..M, into the compact layout
//      X[row][channel][0..M].  Rows without data are never touched and stay zero.
//   2. C2C along the first axis: cuFFT, one batched strided plan over every
//      (channel, column) pair of the compact layout.
//   3. step 3 on the compact layout (k_diag_compact): a' = A' b for |m_0| <= M; the
//      output buffer's other rows stay zero from plan creation on.
//   4. inverse C2C along the first axis: cuFFT.
//   5. row C2R (this file): each CTA rebuilds one grid row from its entries 0..M
//      (the others are zero) and writes only the columns the interpolation reads.
// The transforms are unnormalised with cuFFT's sign conventions (forward e^{-2 pi i},
// inverse e^{+2 pi i}), so the rest of the pipeline is unchanged.
#include <cufft.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "kernels.h"

namespace gpn {

namespace {

template <typename T2>
__device__ __forceinline__ T2 cmul(T2 a, T2 b) {
  return T2{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename T2>
__device__ __forceinline__ T2 cadd(T2 a, T2 b) {
  return T2{a.x + b.x, a.y + b.y};
}
template <typename T2>
__device__ __forceinline__ T2 csub(T2 a, T2 b) {
  return T2{a.x - b.x, a.y - b.y};
}
template <typename T2>
__device__ __forceinline__ T2 cconj(T2 a) {
  return T2{a.x, -a.y};
}

// Each thread does 4 radix-4 butterflies (8 radix-2 ones) per stage: a transform
// of length h runs on h/16 threads (at least one warp).
constexpr int kB4 = 4;
constexpr int kB2 = 8;
constexpr int kMaxFftThreads = 512;
inline int fft_threads(int L) { return std::max(32, (1 << L) / 16); }

// In-place complex FFT of length h = 2^L in shared memory, Stockham order
// (natural in, natural out).  stw holds the radix-4 stage twiddles in the order they
// are used: for the stage with span Ns (the radix-2 stage, when L is odd, comes
// first and needs none), the 3*Ns values exp(-2 pi i t k / (4 Ns)), t = 1..3,
// k < Ns, stored t-major, so consecutive threads read consecutive entries.
// Every thread of the block must call it.
template <typename T2, bool INV>
__device__ void fft_smem(T2* buf, int L, const T2* __restrict__ stw) {
  const int h = 1 << L;
  int Ns = 1;
  if (L & 1) {
    // radix-2 stage (Ns = 1: no twiddle)
    const int nb = h / 2;
    T2 v0[kB2], v1[kB2];
#pragma unroll
    for (int c = 0; c < kB2; ++c) {
      const int j = threadIdx.x + c * blockDim.x;
      if (j < nb) {
        v0[c] = buf[j];
        v1[c] = buf[j + nb];
      }
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < kB2; ++c) {
      const int j = threadIdx.x + c * blockDim.x;
      if (j < nb) {
        buf[2 * j] = cadd(v0[c], v1[c]);
        buf[2 * j + 1] = csub(v0[c], v1[c]);
      }
    }
    __syncthreads();
    Ns = 2;
  }
  const T2* tws = stw;  // this stage's block of 3*Ns twiddles
  while (Ns < h) {
    const int nb = h / 4;
    T2 v[kB4][4];
#pragma unroll
    for (int c = 0; c < kB4; ++c) {
      const int j = threadIdx.x + c * blockDim.x;
      if (j < nb) {
        const int k = j & (Ns - 1);
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          T2 x = buf[j + t * nb];
          if (t > 0) {
            T2 w = __ldg(&tws[(t - 1) * Ns + k]);
            if (INV) w = cconj(w);
            x = cmul(x, w);
          }
          v[c][t] = x;
        }
      }
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < kB4; ++c) {
      const int j = threadIdx.x + c * blockDim.x;
      if (j < nb) {
        const int k = j & (Ns - 1);
        const T2 a = cadd(v[c][0], v[c][2]);
        const T2 b = csub(v[c][0], v[c][2]);
        const T2 cc = cadd(v[c][1], v[c][3]);
        const T2 e = csub(v[c][1], v[c][3]);
        // forward: multiply e by -i ; inverse: by +i
        const T2 dd = INV ? T2{-e.y, e.x} : T2{e.y, -e.x};
        const int o = (j - k) * 4 + k;
        buf[o] = cadd(a, cc);
        buf[o + Ns] = cadd(b, dd);
        buf[o + 2 * Ns] = csub(a, cc);
        buf[o + 3 * Ns] = csub(b, dd);
      }
    }
    __syncthreads();
    tws += 3 * Ns;
    Ns *= 4;
  }
}

template <typename T>
struct RowArgs {
  const T* grid;                 // [CR][nf][nf] (d = 2) or [CR][nf] (d = 1)
  typename Cplx<T>::type* X;     // [rows][CR][M+1]
  const typename Cplx<T>::type* tw;    // exp(-2 pi i k / nf), k < nf
  const typename Cplx<T>::type* stw;   // stage twiddles of the length-nf/2 FFT
  long long nf;
  long long M;
  int L;                         // log2(nf / 2)
  int CR;                        // channels in use (C * R)
  int CP;                        // channel pitch of the compact layout (C * grid_rhs)
  int row_lo;                    // first grid row handled (d = 2); 0 for d = 1
  int col_lo, col_hi;            // columns that may hold data / that interp reads
  int d;
};

// One CTA per (grid row, channel): forward real FFT of the row, entries 0..M kept.
template <typename T>
__global__ void __launch_bounds__(kMaxFftThreads) k_row_r2c(RowArgs<T> a) {
  using T2 = typename Cplx<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T2* z = reinterpret_cast<T2*>(smem_raw);
  const int h = 1 << a.L;
  const long long row = (a.d == 2) ? a.row_lo + blockIdx.x : 0;
  const int ch = blockIdx.y;
  const T* src = a.grid + ((size_t)ch * (a.d == 2 ? a.nf : 1) + (size_t)row) * a.nf;
  const T2* src2 = reinterpret_cast<const T2*>(src);
  // z[j] = x[2j] + i x[2j+1]; columns outside [col_lo, col_hi) are zero
  for (int j = threadIdx.x; j < h; j += blockDim.x) {
    const int c = 2 * j;
    z[j] = (c + 1 >= a.col_lo && c < a.col_hi) ? src2[j] : T2{T(0), T(0)};
  }
  __syncthreads();
  fft_smem<T2, false>(z, a.L, a.stw);
  // X[k] = E + e^{-2 pi i k/nf} O,  E = (Z_k + conj Z_{h-k})/2,  O = (Z_k - conj Z_{h-k})/(2i)
  T2* dst = a.X + ((size_t)(a.d == 2 ? row : 0) * a.CP + ch) * (a.M + 1);
  for (int k = threadIdx.x; k <= a.M; k += blockDim.x) {
    const T2 zk = z[k];
    const T2 zc = cconj(z[(h - k) & (h - 1)]);
    const T2 e = T2{T(0.5) * (zk.x + zc.x), T(0.5) * (zk.y + zc.y)};
    const T2 dz = csub(zk, zc);
    const T2 o = T2{T(0.5) * dz.y, T(-0.5) * dz.x};  // dz / (2i)
    dst[k] = cadd(e, cmul(__ldg(&a.tw[k]), o));
  }
}

// One CTA per (grid row, channel): inverse real FFT from entries 0..M (others zero).
template <typename T>
__global__ void __launch_bounds__(kMaxFftThreads) k_row_c2r(RowArgs<T> a, const typename Cplx<T>::type* W, T* out) {
  using T2 = typename Cplx<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T2* z = reinterpret_cast<T2*>(smem_raw);
  const int h = 1 << a.L;
  const long long row = (a.d == 2) ? a.row_lo + blockIdx.x : 0;
  const int ch = blockIdx.y;
  const T2* srcX = W + ((size_t)(a.d == 2 ? row : 0) * a.CP + ch) * (a.M + 1);
  // Zin[k] = (X_k + conj X_{h-k}) + i e^{+2 pi i k/nf} (X_k - conj X_{h-k})
  for (int k = threadIdx.x; k < h; k += blockDim.x) {
    const T2 xk = k <= a.M ? srcX[k] : T2{T(0), T(0)};
    const int kc = h - k;  // k = 0 pairs with the Nyquist entry, which is zero
    const T2 xc = (k > 0 && kc <= a.M) ? cconj(srcX[kc]) : T2{T(0), T(0)};
    const T2 e = cadd(xk, xc);
    const T2 o = cmul(cconj(__ldg(&a.tw[k])), csub(xk, xc));
    z[k] = T2{e.x - o.y, e.y + o.x};  // e + i o
  }
  __syncthreads();
  fft_smem<T2, true>(z, a.L, a.stw);
  T* dst = out + ((size_t)ch * (a.d == 2 ? a.nf : 1) + (size_t)row) * a.nf;
  T2* dst2 = reinterpret_cast<T2*>(dst);
  for (int j = threadIdx.x; j < h; j += blockDim.x) {
    const int c = 2 * j;
    if (c + 1 >= a.col_lo && c < a.col_hi) dst2[j] = z[j];
  }
}

template <typename T>
struct DiagCArgs {
  const typename Cplx<T>::type* Y;   // [nf or 1][CR][M+1]
  typename Cplx<T>::type* Z;         // same layout
  const T* A;                        // packed upper triangle [p][f]
  long long nf;
  long long M;
  long long n_freq;
  int C;
  int R;
  int CP;                            // channel pitch (C * grid_rhs)
  int d;
};

// Step 3 on the compact layout: thread per (m_1, box row m_0).
template <typename T, int CMAX>
__global__ void __launch_bounds__(128) k_diag_compact(DiagCArgs<T> a) {
  using C2 = typename Cplx<T>::type;
  const long long m1 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (m1 > a.M) return;
  long long row = 0, f = m1;
  if (a.d == 2) {
    const long long m0 = (long long)blockIdx.y - a.M;  // -M..M
    row = m0 < 0 ? m0 + a.nf : m0;
    f = (long long)blockIdx.y * (a.M + 1) + m1;
  }
  const int C = a.C;
  for (int r = 0; r < a.R; ++r) {
    const size_t base = ((size_t)row * a.CP + (size_t)r * C) * (a.M + 1) + m1;
    C2 b[CMAX];
#pragma unroll
    for (int k = 0; k < CMAX; ++k) b[k] = k < C ? a.Y[base + (size_t)k * (a.M + 1)] : C2{T(0), T(0)};
#pragma unroll 1
    for (int k1 = 0; k1 < C; ++k1) {
      T re = T(0), im = T(0);
      const int rowp = k1 * C - (k1 * (k1 - 1)) / 2;
#pragma unroll
      for (int k2 = 0; k2 < CMAX; ++k2) {
        if (k2 < C) {
          const int p = k2 >= k1 ? rowp + (k2 - k1) : k2 * C - (k2 * (k2 - 1)) / 2 + (k1 - k2);
          const T av = __ldg(a.A + (size_t)p * a.n_freq + f);
          re += av * b[k2].x;
          im += av * b[k2].y;
        }
      }
      a.Z[base + (size_t)k1 * (a.M + 1)] = C2{re, im};
    }
  }
}

template <typename T>
RowArgs<T> row_args(Plan& plan, int R) {
  RowArgs<T> a{};
  a.grid = (const T*)plan.grid;
  a.X = (typename Cplx<T>::type*)plan.fx;
  a.tw = (const typename Cplx<T>::type*)plan.twiddle;
  a.stw = (const typename Cplx<T>::type*)plan.stage_twiddle;
  a.nf = plan.geom.nf;
  a.M = plan.geom.M;
  a.L = plan.fft_log2h;
  a.CR = plan.geom.C * R;
  a.CP = plan.geom.C * plan.grid_rhs;
  a.row_lo = plan.row_lo;
  a.col_lo = plan.col_lo;
  a.col_hi = plan.col_hi;
  a.d = plan.geom.d;
  return a;
}

#define GPN_CUFFT2(call)                                                                                \
  do {                                                                                                  \
    cufftResult r_ = (call);                                                                            \
    if (r_ != CUFFT_SUCCESS) ::gpn::fail(GP_ECUFFT, std::string(#call " failed: code ") + std::to_string((int)r_)); \
  } while (0)

template <typename T>
void forward_impl(Plan& plan, int R, cudaStream_t st) {
  RowArgs<T> a = row_args<T>(plan, R);
  const int h = 1 << a.L;
  const size_t smem = sizeof(typename Cplx<T>::type) * h;
  GPN_CUDA(cudaFuncSetAttribute(k_row_r2c<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int rows = plan.geom.d == 2 ? plan.row_hi - plan.row_lo : 1;
  k_row_r2c<T><<<dim3(rows, a.CR), fft_threads(a.L), smem, st>>>(a);
  GPN_CUDA(cudaGetLastError());
  prof_mark(plan, 0, st);
  if (plan.geom.d == 2) {
    cufftHandle hdl = plan.col_plan(R);
    GPN_CUFFT2(cufftSetStream(hdl, st));
    if (sizeof(T) == 4)
      GPN_CUFFT2(cufftExecC2C(hdl, (cufftComplex*)plan.fx, (cufftComplex*)plan.fy, CUFFT_FORWARD));
    else
      GPN_CUFFT2(cufftExecZ2Z(hdl, (cufftDoubleComplex*)plan.fx, (cufftDoubleComplex*)plan.fy, CUFFT_FORWARD));
  }
}

template <typename T>
void diag_impl(Plan& plan, int R, cudaStream_t st) {
  DiagCArgs<T> a{};
  const bool two = plan.geom.d == 2;
  a.Y = (const typename Cplx<T>::type*)(two ? plan.fy : plan.fx);
  a.Z = (typename Cplx<T>::type*)plan.fz;
  a.A = (const T*)plan.a_tensor;
  a.nf = plan.geom.nf;
  a.M = plan.geom.M;
  a.n_freq = plan.n_freq;
  a.C = plan.geom.C;
  a.R = R;
  a.CP = plan.geom.C * plan.grid_rhs;
  a.d = plan.geom.d;
  dim3 grid((unsigned)blocks_for(a.M + 1, 128), (unsigned)(two ? 2 * a.M + 1 : 1));
  switch (cmax_bucket(a.C)) {
    case 8: k_diag_compact<T, 8><<<grid, 128, 0, st>>>(a); break;
    case 12: k_diag_compact<T, 12><<<grid, 128, 0, st>>>(a); break;
    case 16: k_diag_compact<T, 16><<<grid, 128, 0, st>>>(a); break;
    default: k_diag_compact<T, 32><<<grid, 128, 0, st>>>(a);
  }
  GPN_CUDA(cudaGetLastError());
}

template <typename T>
void inverse_impl(Plan& plan, int R, cudaStream_t st) {
  RowArgs<T> a = row_args<T>(plan, R);
  const typename Cplx<T>::type* W = (const typename Cplx<T>::type*)plan.fz;
  if (plan.geom.d == 2) {
    cufftHandle hdl = plan.col_plan(R);
    GPN_CUFFT2(cufftSetStream(hdl, st));
    if (sizeof(T) == 4)
      GPN_CUFFT2(cufftExecC2C(hdl, (cufftComplex*)plan.fz, (cufftComplex*)plan.fy, CUFFT_INVERSE));
    else
      GPN_CUFFT2(cufftExecZ2Z(hdl, (cufftDoubleComplex*)plan.fz, (cufftDoubleComplex*)plan.fy, CUFFT_INVERSE));
    W = (const typename Cplx<T>::type*)plan.fy;
  }
  prof_mark(plan, 1, st);
  const int h = 1 << a.L;
  const size_t smem = sizeof(typename Cplx<T>::type) * h;
  GPN_CUDA(cudaFuncSetAttribute(k_row_c2r<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int rows = plan.geom.d == 2 ? plan.row_hi - plan.row_lo : 1;
  k_row_c2r<T><<<dim3(rows, a.CR), fft_threads(a.L), smem, st>>>(a, W, (T*)plan.grid_out);
  GPN_CUDA(cudaGetLastError());
}

}  // namespace

bool rowfft_supported(int d, long long nf, size_t rs) {
  if (d > 2) return false;
  if (nf < 8 || (nf & (nf - 1)) != 0) return false;
  const long long h = nf / 2;
  if (h * 2 * (long long)rs > (128ll << 10)) return false;       // one row in shared memory
  return h / 16 <= kMaxFftThreads;
}

// Twiddle tables, computed in float64 and rounded once to the plan's precision:
//   twiddle[k]      = exp(-2 pi i k / nf), k < nf (real/complex split of the rows)
//   stage_twiddle   = for each radix-4 stage of the length-nf/2 FFT (span Ns),
//                     exp(-2 pi i t k / (4 Ns)) for t = 1..3, k < Ns, t-major.
void build_twiddles(Plan& plan) {
  const long long n = plan.geom.nf;
  const double tau = 6.283185307179586476925286766559;
  int L = 0;
  while ((1ll << L) < n / 2) ++L;
  plan.fft_log2h = L;
  std::vector<double> re, im;
  for (long long k = 0; k < n; ++k) {
    re.push_back(std::cos(tau * k / n));
    im.push_back(-std::sin(tau * k / n));
  }
  std::vector<double> sre, sim;
  const long long h = n / 2;
  for (long long Ns = (L & 1) ? 2 : 1; Ns < h; Ns *= 4)
    for (int t = 1; t <= 3; ++t)
      for (long long k = 0; k < Ns; ++k) {
        sre.push_back(std::cos(tau * t * k / (4.0 * Ns)));
        sim.push_back(-std::sin(tau * t * k / (4.0 * Ns)));
      }
  if (sre.empty()) {
    sre.push_back(1.0);
    sim.push_back(0.0);
  }
  auto upload = [&](const std::vector<double>& a, const std::vector<double>& b) -> void* {
    const size_t m = a.size();
    void* dst;
    if (plan.real_size == 4) {
      std::vector<float2> t(m);
      for (size_t i = 0; i < m; ++i) t[i] = float2{(float)a[i], (float)b[i]};
      dst = plan.alloc(sizeof(float2) * m);
      GPN_CUDA(cudaMemcpy(dst, t.data(), sizeof(float2) * m, cudaMemcpyHostToDevice));
    } else {
      std::vector<double2> t(m);
      for (size_t i = 0; i < m; ++i) t[i] = double2{a[i], b[i]};
      dst = plan.alloc(sizeof(double2) * m);
      GPN_CUDA(cudaMemcpy(dst, t.data(), sizeof(double2) * m, cudaMemcpyHostToDevice));
    }
    return dst;
  };
  plan.twiddle = upload(re, im);
  plan.stage_twiddle = upload(sre, sim);
}

cufftHandle Plan::col_plan(int R) {
  auto it = fft_col.find(R);
  if (it != fft_col.end()) return it->second;
  // columns of all used channels are adjacent (idist 1); rows are C*grid_rhs*(M+1) apart
  int n[1] = {(int)geom.nf};
  const int pitch = geom.C * grid_rhs * (int)(geom.M + 1);
  const int cols = geom.C * R * (int)(geom.M + 1);
  cufftHandle hdl;
  GPN_CUFFT2(cufftPlanMany(&hdl, 1, n, n, pitch, 1, n, pitch, 1, precision == GP_FP32 ? CUFFT_C2C : CUFFT_Z2Z, cols));
  fft_col[R] = hdl;
  return hdl;
}

void rowfft_forward(Plan& plan, int R, cudaStream_t st) {
  if (plan.precision == GP_FP32)
    forward_impl<float>(plan, R, st);
  else
    forward_impl<double>(plan, R, st);
}

void rowfft_diag(Plan& plan, int R, cudaStream_t st) {
  if (plan.precision == GP_FP32)
    diag_impl<float>(plan, R, st);
  else
    diag_impl<double>(plan, R, st);
}

void rowfft_inverse(Plan& plan, int R, cudaStream_t st) {
  if (plan.precision == GP_FP32)
    inverse_impl<float>(plan, R, st);
  else
    inverse_impl<double>(plan, R, st);
}

}  // namespace gpn
