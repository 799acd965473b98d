// Hot path of the K~ matvec (Sec. 4.2 steps (1)-(5)) on sm_103a.
//
//  spread  (steps 1+2a): output-stationary.  One CTA owns one fine-grid tile of
//          tile^d cells for one right-hand side; it accumulates, in shared
//          memory, every point whose spreading support meets the tile (the points
//          of the 2^d bins at offsets {0,-1}^d), then writes the tile once with
//          coalesced stores.  No global atomics and no pre-zeroing of the grid.
//  diag    (steps 2b+3+4a): on the R2C half spectrum, a'[n] = A'[n] b[n] inside the
//          mode box |n_a| <= M, zero outside.  A' = A / psihat(n)^2 folds the
//          NUFFT deconvolution of both transforms into the tensor of Remark rem:step3.
//  interp  (steps 4b+5): one CTA per tile-bin; one warp per point gathers the
//          width^d cells of all C channels, reduces across the warp and combines
//          sum_k w_k(x_i) beta_k (+ shift * alpha_i).
//
// Fine-grid convention: grid coordinate g = (x - centre)/h + nf/2 with h = 1/(dw nf);
// the points never come within width/2 cells of the grid edge, so no wrap-around
// is needed.  Type 1: U = FFT(u) with u[l] = sum_i c_i psi(l - g_i) gives
// b[n] = (-1)^n U[n]/psihat(n); type 2 mirrors it, so the (-1)^n phases cancel in
// the composition and step 3 only needs the real factor 1/psihat(n)^2.
#include <cufft.h>

#include <cmath>

#include "plan.h"

namespace gpn {

namespace {

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

template <typename T>
__device__ __forceinline__ T es_psi(T s, int width, T beta, T inv_halfw) {
  T z = s * inv_halfw;
  T q = T(1) - z * z;
  return q > T(0) ? exp(beta * (sqrt(q) - T(1))) : T(0);
}

template <typename T>
struct SpreadArgs {
  const int* cell0[kMaxDim];
  const T* xi[kMaxDim];
  const T* wk;
  const int* bin_start;
  int nbins[kMaxDim];
  int ntiles[kMaxDim];
  const double* alpha;   // sorted order, N x R column-major
  long long n;
  T* grid;               // (R*C) x nf^d
  long long nf;
  long long G;           // nf^d
  int width;
  T beta;
  T inv_halfw;
  int tile;
  int C;
};

// Per-warp scratch layout in shared memory (after the tile):
//   psi[kMaxDim][kMaxWidth], str[kMaxChannels]
template <typename T>
struct WarpScratch {
  T psi[kMaxDim][kMaxWidth];
  T str[kMaxChannels];
};

template <typename T, int D>
__global__ void __launch_bounds__(256) k_spread(SpreadArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int TS = a.tile;
  int tvol = 1;
#pragma unroll
  for (int q = 0; q < D; ++q) tvol *= TS;
  T* tile = reinterpret_cast<T*>(smem_raw);
  WarpScratch<T>* ws = reinterpret_cast<WarpScratch<T>*>(tile + (size_t)a.C * tvol);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  WarpScratch<T>& my = ws[warp];
  const int r = blockIdx.y;

  for (int i = threadIdx.x; i < a.C * tvol; i += blockDim.x) tile[i] = T(0);

  // tile coordinates (last dimension fastest)
  int tc[kMaxDim] = {0, 0, 0};
  {
    long long rest = blockIdx.x;
    for (int q = D - 1; q >= 0; --q) {
      tc[q] = (int)(rest % a.ntiles[q]);
      rest /= a.ntiles[q];
    }
  }
  __syncthreads();

  const double* alpha_r = a.alpha + (size_t)r * a.n;
  for (int o = 0; o < (1 << D); ++o) {
    int b[kMaxDim] = {0, 0, 0};
    bool valid = true;
    long long lin = 0;
#pragma unroll
    for (int q = 0; q < D; ++q) {
      b[q] = tc[q] - ((o >> q) & 1);
      if (b[q] < 0) valid = false;
      lin = lin * a.nbins[q] + (b[q] < 0 ? 0 : b[q]);
    }
    if (!valid) continue;
    const int p0 = a.bin_start[lin], p1 = a.bin_start[lin + 1];
    for (int p = p0 + warp; p < p1; p += nwarps) {
      int lo[kMaxDim], cnt[kMaxDim], l0[kMaxDim];
      bool empty = false;
#pragma unroll
      for (int q = 0; q < D; ++q) {
        l0[q] = a.cell0[q][p];
        int base = tc[q] * TS;
        int l = max(0, base - l0[q]);
        int h = min(a.width, base + TS - l0[q]);
        lo[q] = l;
        cnt[q] = h - l;
        if (h <= l) empty = true;
      }
      if (empty) continue;
      // kernel values per dimension and the per-channel strengths w_k(x_p) alpha_p
      for (int t = lane; t < D * a.width; t += 32) {
        int q = t / a.width, i = t - q * a.width;
        my.psi[q][i] = es_psi<T>((T)i - a.xi[q][p], a.width, a.beta, a.inv_halfw);
      }
      if (lane < a.C) my.str[lane] = a.wk[(size_t)p * a.C + lane] * (T)alpha_r[p];
      __syncwarp();
      int total = 1;
#pragma unroll
      for (int q = 0; q < D; ++q) total *= cnt[q];
      for (int c = lane; c < total; c += 32) {
        int rem = c;
        T wgt = T(1);
        int cell = 0;
#pragma unroll
        for (int q = D - 1; q >= 0; --q) {
          int iq = lo[q] + rem % cnt[q];
          rem /= cnt[q];
          wgt *= my.psi[q][iq];
          int local = l0[q] + iq - tc[q] * TS;
          int stride = 1;
          for (int s = q + 1; s < D; ++s) stride *= TS;
          cell += local * stride;
        }
        for (int k = 0; k < a.C; ++k) atomicAdd(&tile[(size_t)k * tvol + cell], wgt * my.str[k]);
      }
      __syncwarp();
    }
  }
  __syncthreads();

  // write the tile (cells beyond nf in a partial last tile are dropped)
  for (int i = threadIdx.x; i < tvol; i += blockDim.x) {
    int rem = i;
    long long gidx = 0, gstride = 1;
    bool inside = true;
#pragma unroll
    for (int q = D - 1; q >= 0; --q) {
      int c = rem % TS;
      rem /= TS;
      long long g = (long long)tc[q] * TS + c;
      if (g >= a.nf) inside = false;
      gidx += g * gstride;
      gstride *= a.nf;
    }
    if (!inside) continue;
    for (int k = 0; k < a.C; ++k) a.grid[((size_t)r * a.C + k) * a.G + gidx] = tile[(size_t)k * tvol + i];
  }
}

template <typename T>
struct DiagArgs {
  typename Cplx<T>::type* spec;   // (R*C) x S
  const T* A;                     // packed upper triangle [p][f]
  long long S;                    // half-spectrum elements per channel
  long long half;                 // nf/2 + 1
  long long nf;
  long long M;
  long long n_freq;
  int C;
  int R;
};

template <typename T, int D>
__global__ void __launch_bounds__(256) k_diag(DiagArgs<T> a) {
  using C2 = typename Cplx<T>::type;
  long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (s >= a.S) return;
  long long il = s % a.half, rest = s / a.half;
  long long m[kMaxDim];
  m[D - 1] = il;
  for (int q = D - 2; q >= 0; --q) {
    long long i = rest % a.nf;
    rest /= a.nf;
    m[q] = (i <= a.nf / 2) ? i : i - a.nf;
  }
  bool inbox = il <= a.M;
  long long f = 0;
  for (int q = 0; q < D - 1; ++q) {
    if (m[q] < -a.M || m[q] > a.M) inbox = false;
    f = f * (2 * a.M + 1) + (m[q] + a.M);
  }
  f = f * (a.M + 1) + il;
  const int C = a.C;
  for (int r = 0; r < a.R; ++r) {
    C2* base = a.spec + (size_t)r * C * a.S + s;
    if (!inbox) {
      for (int k = 0; k < C; ++k) base[(size_t)k * a.S] = C2{T(0), T(0)};
      continue;
    }
    C2 b[kMaxChannels];
#pragma unroll
    for (int k = 0; k < kMaxChannels; ++k)
      if (k < C) b[k] = base[(size_t)k * a.S];
    for (int kp = 0; kp < C; ++kp) {
      T re = T(0), im = T(0);
#pragma unroll
      for (int k = 0; k < kMaxChannels; ++k) {
        if (k < C) {
          int lo = kp < k ? kp : k, hi = kp < k ? k : kp;
          int p = lo * C - (lo * (lo - 1)) / 2 + (hi - lo);
          T av = a.A[(size_t)p * a.n_freq + f];
          re += av * b[k].x;
          im += av * b[k].y;
        }
      }
      base[(size_t)kp * a.S] = C2{re, im};
    }
  }
}

template <typename T>
struct InterpArgs {
  const int* cell0[kMaxDim];
  const T* xi[kMaxDim];
  const T* wk;
  const int* bin_start;
  const int* perm;
  long long n;
  const T* grid;
  long long nf;
  long long G;
  int width;
  T beta;
  T inv_halfw;
  int C;
  const double* alpha;     // sorted order (may be null)
  double shift;
  double* out;             // sorted order, N x R
};

template <typename T, int D>
__global__ void __launch_bounds__(256) k_interp(InterpArgs<T> a) {
  __shared__ T psi_s[8][kMaxDim][kMaxWidth];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int r = blockIdx.y;
  const int p0 = a.bin_start[blockIdx.x], p1 = a.bin_start[blockIdx.x + 1];
  const T* grid_r = a.grid + (size_t)r * a.C * a.G;
  for (int p = p0 + warp; p < p1; p += nwarps) {
    int l0[kMaxDim];
#pragma unroll
    for (int q = 0; q < D; ++q) l0[q] = a.cell0[q][p];
    for (int t = lane; t < D * a.width; t += 32) {
      int q = t / a.width, i = t - q * a.width;
      psi_s[warp][q][i] = es_psi<T>((T)i - a.xi[q][p], a.width, a.beta, a.inv_halfw);
    }
    __syncwarp();
    T acc[kMaxChannels];
#pragma unroll
    for (int k = 0; k < kMaxChannels; ++k) acc[k] = T(0);
    int total = 1;
#pragma unroll
    for (int q = 0; q < D; ++q) total *= a.width;
    for (int c = lane; c < total; c += 32) {
      int rem = c;
      T wgt = T(1);
      long long gidx = 0, gstride = 1;
#pragma unroll
      for (int q = D - 1; q >= 0; --q) {
        int iq = rem % a.width;
        rem /= a.width;
        wgt *= psi_s[warp][q][iq];
        gidx += (long long)(l0[q] + iq) * gstride;
        gstride *= a.nf;
      }
#pragma unroll
      for (int k = 0; k < kMaxChannels; ++k)
        if (k < a.C) acc[k] += wgt * __ldg(grid_r + (size_t)k * a.G + gidx);
    }
    double res = 0.0;
#pragma unroll
    for (int k = 0; k < kMaxChannels; ++k) {
      if (k < a.C) {
        T v = acc[k];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        res += (double)a.wk[(size_t)p * a.C + k] * (double)v;
      }
    }
    if (lane == 0) {
      if (a.alpha) res += a.shift * a.alpha[(size_t)r * a.n + p];
      a.out[(size_t)r * a.n + p] = res;
    }
    __syncwarp();
  }
}

template <typename T>
struct ATensorArgs {
  const double* etab;   // [k][j][m]
  const double* vt;     // [j]
  T* A;
  long long n_freq;
  long long M;
  int C;
  int J;
  int d;
};

__global__ void k_build_a_f32(ATensorArgs<float> a);
__global__ void k_build_a_f64(ATensorArgs<double> a);

template <typename T>
__device__ void build_a_body(const ATensorArgs<T>& a) {
  long long f = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (f >= a.n_freq) return;
  long long m[kMaxDim];
  long long rest = f;
  m[a.d - 1] = rest % (a.M + 1);
  rest /= (a.M + 1);
  for (int q = a.d - 2; q >= 0; --q) {
    long long v = rest % (2 * a.M + 1) - a.M;
    rest /= (2 * a.M + 1);
    m[q] = v < 0 ? -v : v;
  }
  const long long Mp = a.M + 1;
  int p = 0;
  for (int k1 = 0; k1 < a.C; ++k1)
    for (int k2 = k1; k2 < a.C; ++k2, ++p) {
      double acc = 0.0;
      for (int j = 0; j < a.J; ++j) {
        const double* e1 = a.etab + ((size_t)k1 * a.J + j) * Mp;
        const double* e2 = a.etab + ((size_t)k2 * a.J + j) * Mp;
        double g = a.vt[j];
        for (int q = 0; q < a.d; ++q) g *= e1[m[q]] * e2[m[q]];
        acc += g;
      }
      a.A[(size_t)p * a.n_freq + f] = (T)acc;
    }
}

__global__ void k_build_a_f32(ATensorArgs<float> a) { build_a_body<float>(a); }
__global__ void k_build_a_f64(ATensorArgs<double> a) { build_a_body<double>(a); }

inline int blocks_for(long long n, int t) { return (int)((n + t - 1) / t); }

template <typename T>
void spread_impl(Plan& plan, const double* alpha_sorted, int R, cudaStream_t st) {
  const GridGeom& g = plan.geom;
  const PointSet& ps = plan.pts;
  SpreadArgs<T> a{};
  for (int q = 0; q < kMaxDim; ++q) {
    a.cell0[q] = ps.cell0[q];
    a.xi[q] = (const T*)ps.xi[q];
    a.nbins[q] = ps.nbins[q];
    a.ntiles[q] = ps.nbins[q];
  }
  a.wk = (const T*)ps.wk;
  a.bin_start = ps.bin_start;
  a.alpha = alpha_sorted;
  a.n = ps.n;
  a.grid = (T*)plan.grid;
  a.nf = g.nf;
  a.G = plan.grid_elems;
  a.width = g.width;
  a.beta = (T)g.beta;
  a.inv_halfw = (T)(2.0 / g.width);
  a.tile = g.tile;
  a.C = g.C;
  long long tvol = 1;
  for (int q = 0; q < g.d; ++q) tvol *= g.tile;
  size_t smem = sizeof(T) * (size_t)g.C * tvol + sizeof(WarpScratch<T>) * 8;
  dim3 grid((unsigned)ps.nbins_total, (unsigned)R);
  switch (g.d) {
    case 1:
      GPN_CUDA(cudaFuncSetAttribute(k_spread<T, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      k_spread<T, 1><<<grid, 256, smem, st>>>(a);
      break;
    case 2:
      GPN_CUDA(cudaFuncSetAttribute(k_spread<T, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      k_spread<T, 2><<<grid, 256, smem, st>>>(a);
      break;
    default:
      GPN_CUDA(cudaFuncSetAttribute(k_spread<T, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      k_spread<T, 3><<<grid, 256, smem, st>>>(a);
  }
  GPN_CUDA(cudaGetLastError());
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
  int nb = blocks_for(a.S, 256);
  switch (g.d) {
    case 1: k_diag<T, 1><<<nb, 256, 0, st>>>(a); break;
    case 2: k_diag<T, 2><<<nb, 256, 0, st>>>(a); break;
    default: k_diag<T, 3><<<nb, 256, 0, st>>>(a);
  }
  GPN_CUDA(cudaGetLastError());
}

template <typename T>
void interp_impl(Plan& plan, const PointSet& ps, const double* alpha_sorted, double shift, double* out_sorted, int R,
                 cudaStream_t st) {
  const GridGeom& g = plan.geom;
  InterpArgs<T> a{};
  for (int q = 0; q < kMaxDim; ++q) {
    a.cell0[q] = ps.cell0[q];
    a.xi[q] = (const T*)ps.xi[q];
  }
  a.wk = (const T*)ps.wk;
  a.bin_start = ps.bin_start;
  a.perm = ps.perm;
  a.n = ps.n;
  a.grid = (const T*)plan.grid;
  a.nf = g.nf;
  a.G = plan.grid_elems;
  a.width = g.width;
  a.beta = (T)g.beta;
  a.inv_halfw = (T)(2.0 / g.width);
  a.C = g.C;
  a.alpha = alpha_sorted;
  a.shift = shift;
  a.out = out_sorted;
  dim3 grid((unsigned)ps.nbins_total, (unsigned)R);
  switch (g.d) {
    case 1: k_interp<T, 1><<<grid, 256, 0, st>>>(a); break;
    case 2: k_interp<T, 2><<<grid, 256, 0, st>>>(a); break;
    default: k_interp<T, 3><<<grid, 256, 0, st>>>(a);
  }
  GPN_CUDA(cudaGetLastError());
}

}  // namespace

void build_a_tensor(Plan& plan, cudaStream_t st) {
  const Hyper& h = plan.h;
  const int C = plan.geom.C;
  const int J = (int)plan.tb.vt.size();
  double *etab = nullptr, *vt = nullptr;
  cudaError_t e = cudaMalloc(&etab, sizeof(double) * plan.tb.etab.size());
  if (e == cudaSuccess) e = cudaMalloc(&vt, sizeof(double) * J);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(etab, plan.tb.etab.data(), sizeof(double) * plan.tb.etab.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(vt, plan.tb.vt.data(), sizeof(double) * J, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) {
    int nb = blocks_for(plan.n_freq, 128);
    if (plan.precision == GP_FP32) {
      ATensorArgs<float> a{etab, vt, (float*)plan.a_tensor, plan.n_freq, h.M, C, J, h.d};
      k_build_a_f32<<<nb, 128, 0, st>>>(a);
    } else {
      ATensorArgs<double> a{etab, vt, (double*)plan.a_tensor, plan.n_freq, h.M, C, J, h.d};
      k_build_a_f64<<<nb, 128, 0, st>>>(a);
    }
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(etab);
  cudaFree(vt);
  GPN_CUDA(e);
}

void launch_spread(Plan& plan, const double* alpha_sorted, int R, cudaStream_t st) {
  if (plan.precision == GP_FP32)
    spread_impl<float>(plan, alpha_sorted, R, st);
  else
    spread_impl<double>(plan, alpha_sorted, R, st);
}

void launch_diag(Plan& plan, int R, cudaStream_t st) {
  if (plan.precision == GP_FP32)
    diag_impl<float>(plan, R, st);
  else
    diag_impl<double>(plan, R, st);
}

void launch_interp(Plan& plan, const PointSet& ps, const double* alpha_sorted, double shift, double* out_sorted,
                   int R, cudaStream_t st) {
  if (ps.n == 0) return;
  if (plan.precision == GP_FP32)
    interp_impl<float>(plan, ps, alpha_sorted, shift, out_sorted, R, st);
  else
    interp_impl<double>(plan, ps, alpha_sorted, shift, out_sorted, R, st);
}

#define GPN_CUFFT(call)                                                                                 \
  do {                                                                                                  \
    cufftResult r_ = (call);                                                                            \
    if (r_ != CUFFT_SUCCESS) ::gpn::fail(GP_ECUFFT, std::string(#call " failed: code ") + std::to_string((int)r_)); \
  } while (0)

cufftHandle Plan::fwd_plan(int R) {
  auto it = fft_fwd.find(R);
  if (it != fft_fwd.end()) return it->second;
  int n[3] = {(int)geom.nf, (int)geom.nf, (int)geom.nf};
  cufftHandle hdl;
  GPN_CUFFT(cufftPlanMany(&hdl, geom.d, n, nullptr, 1, 0, nullptr, 1, 0,
                          precision == GP_FP32 ? CUFFT_R2C : CUFFT_D2Z, geom.C * R));
  fft_fwd[R] = hdl;
  return hdl;
}

cufftHandle Plan::inv_plan(int R) {
  auto it = fft_inv.find(R);
  if (it != fft_inv.end()) return it->second;
  int n[3] = {(int)geom.nf, (int)geom.nf, (int)geom.nf};
  cufftHandle hdl;
  GPN_CUFFT(cufftPlanMany(&hdl, geom.d, n, nullptr, 1, 0, nullptr, 1, 0,
                          precision == GP_FP32 ? CUFFT_C2R : CUFFT_Z2D, geom.C * R));
  fft_inv[R] = hdl;
  return hdl;
}

void run_fft_forward(Plan& plan, int R, cudaStream_t st) {
  cufftHandle h = plan.fwd_plan(R);
  GPN_CUFFT(cufftSetStream(h, st));
  if (plan.precision == GP_FP32)
    GPN_CUFFT(cufftExecR2C(h, (cufftReal*)plan.grid, (cufftComplex*)plan.spec));
  else
    GPN_CUFFT(cufftExecD2Z(h, (cufftDoubleReal*)plan.grid, (cufftDoubleComplex*)plan.spec));
}

void run_fft_inverse(Plan& plan, int R, cudaStream_t st) {
  cufftHandle h = plan.inv_plan(R);
  GPN_CUFFT(cufftSetStream(h, st));
  if (plan.precision == GP_FP32)
    GPN_CUFFT(cufftExecC2R(h, (cufftComplex*)plan.spec, (cufftReal*)plan.grid));
  else
    GPN_CUFFT(cufftExecZ2D(h, (cufftDoubleComplex*)plan.spec, (cufftDoubleReal*)plan.grid));
}

void PhaseProfile::harvest() {
  if (!pending) return;
  GPN_CUDA(cudaEventSynchronize(ev[5]));
  for (int q = 0; q < 5; ++q) {
    float ms = 0.f;
    GPN_CUDA(cudaEventElapsedTime(&ms, ev[q], ev[q + 1]));
    acc[q] += ms;
  }
  ++count;
  pending = false;
}

void PhaseProfile::destroy() {
  if (!created) return;
  for (auto& e : ev) cudaEventDestroy(e);
  created = false;
}

void matvec_sorted(Plan& plan, const double* alpha_sorted, double* out_sorted, int R, double shift, cudaStream_t st) {
  PhaseProfile& pf = plan.prof;
  const bool rec = pf.on;
  if (rec) {
    pf.harvest();
    if (!pf.created) {
      for (auto& e : pf.ev) GPN_CUDA(cudaEventCreate(&e));
      pf.created = true;
    }
    GPN_CUDA(cudaEventRecord(pf.ev[0], st));
  }
  launch_spread(plan, alpha_sorted, R, st);
  if (rec) GPN_CUDA(cudaEventRecord(pf.ev[1], st));
  run_fft_forward(plan, R, st);
  if (rec) GPN_CUDA(cudaEventRecord(pf.ev[2], st));
  launch_diag(plan, R, st);
  if (rec) GPN_CUDA(cudaEventRecord(pf.ev[3], st));
  run_fft_inverse(plan, R, st);
  if (rec) GPN_CUDA(cudaEventRecord(pf.ev[4], st));
  launch_interp(plan, plan.pts, alpha_sorted, shift, out_sorted, R, st);
  if (rec) {
    GPN_CUDA(cudaEventRecord(pf.ev[5], st));
    pf.pending = true;
  }
}

}  // namespace gpn
