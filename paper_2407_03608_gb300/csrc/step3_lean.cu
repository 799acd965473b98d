// Step (3) of Sec. 4.2 without the tensor A' (memory-lean form):
//
//   a_k[n] = sum_j v~_j G^_{k,j}[n] sum_l G^_{l,j}[n] b_l[n],
//   G^_{k,j}[n] = prod_q E'_{k,j}(|n_q|),
//   E'_{k,j}(m) = sqrt(2 pi) sigma_k chi_j exp(-2 pi^2 (sigma_k chi_j dw m)^2) / psihat(m),
//
// i.e. the sequential processing over the quadrature nodes j and the channels k that
// the paper describes as the alternative to storing A[n] (Remark rem:step3 and the
// memory discussion of Sec. 5): the Gaussian transforms of Lemma stage3warmup are
// separable, so only the per-dimension factors E' (C (N_t+1) (M+1) values) are kept,
// and each frequency costs about 4.5 C (N_t+1) multiply-adds instead of one read of
// C(C+1)/2 tensor entries.  The deconvolution 1/psihat(n)^2 of both NUFFTs is inside
// the factors, as in A'.  sqrt(v~_j) (v~_j > 0) is folded into both sides, so
//   g_{k,j}[n] = sqrt(v~_j) prod_q E'_{k,j}(|n_q|),  t_j = sum_l g_{l,j} b_l,
//   a_k = sum_j g_{k,j} t_j.
//
// Table layout on the device: tab[j][m][CP] (m = 0..M, channels padded to CP, a
// multiple of 16 bytes), so a thread reads the CP factors of its own frequency
// coordinate with 16-byte loads; the factors of the coordinates a whole block shares
// are multiplied once into shared memory.
//
// Two kernels, one per spectrum layout:
//   k_step3_lean_t  (d = 2, transposed pruned transforms): columns Y[cr][m][nf]; one
//                   thread per (m, |n_1| <= M) serves n_1 and -n_1 with the same g.
//   k_step3_lean    (full-grid R2C half spectra, any d): one thread per half-spectrum
//                   element; the leading coordinates are per block row, the last one
//                   per thread; the spectrum outside the mode box is set to zero.
#include <algorithm>
#include <cmath>
#include <vector>

#include "fft_core.h"
#include "kernels.h"

namespace gpn {

namespace {

using fft::cpx;

// 16-byte vector of T
template <typename T>
struct Vec16;
template <>
struct Vec16<float> {
  using type = float4;
  static constexpr int n = 4;
};
template <>
struct Vec16<double> {
  using type = double2;
  static constexpr int n = 2;
};

template <typename T, int CPM>
__device__ __forceinline__ void load_factors(T (&g)[CPM], const T* p, int cp) {
  using V = typename Vec16<T>::type;
  constexpr int VW = Vec16<T>::n;
#pragma unroll
  for (int v = 0; v < CPM / VW; ++v) {
    if (v * VW < cp) {
      const V x = __ldg(reinterpret_cast<const V*>(p) + v);
      if constexpr (VW == 4) {
        g[4 * v] = x.x;
        g[4 * v + 1] = x.y;
        g[4 * v + 2] = x.z;
        g[4 * v + 3] = x.w;
      } else {
        g[2 * v] = x.x;
        g[2 * v + 1] = x.y;
      }
    }
  }
}

template <typename T, int CPM>
__device__ __forceinline__ void mul_shared(T (&g)[CPM], const T* s, int cp) {
  using V = typename Vec16<T>::type;
  constexpr int VW = Vec16<T>::n;
#pragma unroll
  for (int v = 0; v < CPM / VW; ++v) {
    if (v * VW < cp) {
      const V x = reinterpret_cast<const V*>(s)[v];
      if constexpr (VW == 4) {
        g[4 * v] *= x.x;
        g[4 * v + 1] *= x.y;
        g[4 * v + 2] *= x.z;
        g[4 * v + 3] *= x.w;
      } else {
        g[2 * v] *= x.x;
        g[2 * v + 1] *= x.y;
      }
    }
  }
}

__host__ __device__ constexpr int round_up(int a, int b) { return (a + b - 1) / b * b; }

// ---- transposed layout (d = 2) ---------------------------------------------------

template <typename T>
struct LeanTArgs {
  const cpx<T>* Y;   // column transforms [cr][M+1][nf]
  cpx<T>* Z;         // step-3 output, same layout
  const T* tab;      // [J][M+1][CP]
  const T* sqv;      // sqrt(v~_j), J
  long long nf;
  int M;
  int C;
  int CP;
  int J;
  int R;
};

constexpr int kTx = 64, kTy = 4;   // threads per block over n_1 and over m

// NC <= 16: C = NC (exact, the channel loops unroll without guards); NC = 32: runtime C.
template <typename T, int NC>
__global__ void __launch_bounds__(kTx * kTy, (sizeof(T) == 4 && NC <= 10) ? 2 : 1) k_step3_lean_t(LeanTArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* s_em = reinterpret_cast<T*>(smem_raw);   // [kTy][J][CP]: sqrt(v~_j) E'_{k,j}(m)
  constexpr int VW = Vec16<T>::n;
  constexpr int CPM = round_up(NC, VW);
  const int C = NC <= 16 ? NC : a.C;
  const int CP = NC <= 16 ? CPM : a.CP;
  const int J = a.J, Mp = a.M + 1;
  const int tid = threadIdx.y * kTx + threadIdx.x;
  const int m0 = blockIdx.y * kTy;
  for (int i = tid; i < kTy * J * CP; i += kTx * kTy) {
    const int t = i / (J * CP), rem = i - t * J * CP;
    const int j = rem / CP, k = rem - j * CP;
    const int m = m0 + t;
    s_em[i] = (m < Mp && k < C) ? a.sqv[j] * a.tab[((size_t)j * Mp + m) * CP + k] : T(0);
  }
  __syncthreads();
  const int n1 = blockIdx.x * kTx + threadIdx.x;
  const int m = m0 + threadIdx.y;
  if (n1 >= Mp || m >= Mp) return;
  const T* em = s_em + (size_t)threadIdx.y * J * CP;
  const size_t colstride = (size_t)Mp * a.nf;
  const size_t off_p = (size_t)m * a.nf + n1;
  const size_t off_n = (size_t)m * a.nf + (n1 == 0 ? 0 : a.nf - n1);
  const T* tn1 = a.tab + (size_t)n1 * CP;
  const size_t jstride = (size_t)Mp * CP;
  for (int r = 0; r < a.R; ++r) {
    const cpx<T>* Yr = a.Y + (size_t)r * C * colstride;
    cpx<T>* Zr = a.Z + (size_t)r * C * colstride;
    cpx<T> bp[CPM], bn[CPM], ap[CPM], an[CPM];
#pragma unroll
    for (int k = 0; k < CPM; ++k) {
      if (k < C) {
        bp[k] = Yr[k * colstride + off_p];
        bn[k] = Yr[k * colstride + off_n];
      }
      ap[k] = an[k] = cpx<T>{T(0), T(0)};
    }
    // the factors of node j + 1 are loaded while node j is processed
    T gn[CPM];
    load_factors<T, CPM>(gn, tn1, CP);
#pragma unroll 1
    for (int j = 0; j < J; ++j) {
      T g[CPM];
#pragma unroll
      for (int k = 0; k < CPM; ++k) g[k] = gn[k];
      if (j + 1 < J) load_factors<T, CPM>(gn, tn1 + (j + 1) * jstride, CP);
      mul_shared<T, CPM>(g, em + j * CP, CP);
      cpx<T> tp{T(0), T(0)}, tn{T(0), T(0)};
#pragma unroll
      for (int k = 0; k < CPM; ++k) {
        if (k < C) {
          tp.x += g[k] * bp[k].x;
          tp.y += g[k] * bp[k].y;
          tn.x += g[k] * bn[k].x;
          tn.y += g[k] * bn[k].y;
        }
      }
#pragma unroll
      for (int k = 0; k < CPM; ++k) {
        if (k < C) {
          ap[k].x += g[k] * tp.x;
          ap[k].y += g[k] * tp.y;
          an[k].x += g[k] * tn.x;
          an[k].y += g[k] * tn.y;
        }
      }
    }
#pragma unroll
    for (int k = 0; k < CPM; ++k) {
      if (k < C) {
        Zr[k * colstride + off_p] = ap[k];
        if (n1 != 0) Zr[k * colstride + off_n] = an[k];
      }
    }
  }
}

template <typename T, int NC>
void lean_t_dispatch(const LeanTArgs<T>& a, size_t smem, cudaStream_t st) {
  if constexpr (NC > 16) {
    GPN_CUDA(cudaFuncSetAttribute(k_step3_lean_t<T, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    dim3 grid((unsigned)((a.M + kTx) / kTx), (unsigned)((a.M + kTy) / kTy));
    k_step3_lean_t<T, 32><<<grid, dim3(kTx, kTy), smem, st>>>(a);
  } else {
    if (a.C == NC) {
      GPN_CUDA(cudaFuncSetAttribute(k_step3_lean_t<T, NC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      dim3 grid((unsigned)((a.M + kTx) / kTx), (unsigned)((a.M + kTy) / kTy));
      k_step3_lean_t<T, NC><<<grid, dim3(kTx, kTy), smem, st>>>(a);
    } else {
      lean_t_dispatch<T, NC + 1>(a, smem, st);
    }
  }
}

// ---- full-grid half spectra (any d) ------------------------------------------------

template <typename T>
struct LeanArgs {
  typename Cplx<T>::type* spec;   // (R*C) x S
  const T* tab;                   // [J][M+1][CP]
  const T* sqv;                   // sqrt(v~_j), J
  long long S;                    // half-spectrum elements per channel
  long long half;                 // nf/2 + 1
  long long nf;
  long long rows;                 // S / half
  long long row0;                 // first row of this launch
  int M;
  int C;
  int CP;
  int J;
  int R;
  int d;
};

constexpr int kRx = 128, kRy = 2;   // threads per block over the last coordinate and over rows

template <typename T, int CMAX>
__global__ void __launch_bounds__(kRx * kRy, (sizeof(T) == 4 && CMAX <= 12) ? 2 : 1) k_step3_lean(LeanArgs<T> a) {
  using C2 = typename Cplx<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* s_em = reinterpret_cast<T*>(smem_raw);   // [kRy][J][CP]
  __shared__ int s_mq[kRy][kMaxDim];          // |leading frequencies| of the block's rows, -1: outside the box
  const int C = a.C, CP = a.CP, J = a.J, Mp = a.M + 1;
  const int tid = threadIdx.y * kRx + threadIdx.x;
  const long long rbase = a.row0 + (long long)blockIdx.y * kRy;
  if (tid < kRy) {
    const long long row = rbase + tid;
    long long rest = row < a.rows ? row : 0;
    bool in = row < a.rows;
    for (int q = a.d - 2; q >= 0; --q) {
      const long long i = rest % a.nf;
      rest /= a.nf;
      const long long mq = (i <= a.nf / 2) ? i : a.nf - i;   // |signed frequency|
      in = in && mq <= a.M;
      s_mq[tid][q] = (int)mq;
    }
    s_mq[tid][kMaxDim - 1] = in ? 1 : -1;
  }
  __syncthreads();
  for (int i = tid; i < kRy * J * CP; i += kRx * kRy) {
    const int t = i / (J * CP), rem = i - t * J * CP;
    const int j = rem / CP, k = rem - j * CP;
    T v = T(0);
    if (s_mq[t][kMaxDim - 1] > 0 && k < C) {
      v = a.sqv[j];
      for (int q = 0; q < a.d - 1; ++q) v *= a.tab[((size_t)j * Mp + s_mq[t][q]) * CP + k];
    }
    s_em[i] = v;
  }
  __syncthreads();
  const long long row = rbase + threadIdx.y;
  const long long il = blockIdx.x * (long long)kRx + threadIdx.x;
  if (row >= a.rows || il >= a.half) return;
  const long long s = row * a.half + il;
  if (s_mq[threadIdx.y][kMaxDim - 1] < 0 || il > a.M) {
    for (int r = 0; r < a.R; ++r) {
      C2* base = a.spec + (size_t)r * C * a.S + s;
#pragma unroll
      for (int k = 0; k < CMAX; ++k)
        if (k < C) base[(size_t)k * a.S] = C2{T(0), T(0)};
    }
    return;
  }
  const T* em = s_em + (size_t)threadIdx.y * J * CP;
  const T* tl = a.tab + (size_t)il * CP;
  const size_t jstride = (size_t)Mp * CP;
  for (int r = 0; r < a.R; ++r) {
    C2* base = a.spec + (size_t)r * C * a.S + s;
    C2 b[CMAX], o[CMAX];
#pragma unroll
    for (int k = 0; k < CMAX; ++k) {
      b[k] = k < C ? base[(size_t)k * a.S] : C2{T(0), T(0)};
      o[k] = C2{T(0), T(0)};
    }
    T gn[CMAX];
    load_factors<T, CMAX>(gn, tl, CP);
#pragma unroll 1
    for (int j = 0; j < J; ++j) {
      T g[CMAX];
#pragma unroll
      for (int k = 0; k < CMAX; ++k) g[k] = gn[k];
      if (j + 1 < J) load_factors<T, CMAX>(gn, tl + (j + 1) * jstride, CP);
      mul_shared<T, CMAX>(g, em + j * CP, CP);
      T tx = T(0), ty = T(0);
#pragma unroll
      for (int k = 0; k < CMAX; ++k) {
        if (k < C) {
          tx += g[k] * b[k].x;
          ty += g[k] * b[k].y;
        }
      }
#pragma unroll
      for (int k = 0; k < CMAX; ++k) {
        if (k < C) {
          o[k].x += g[k] * tx;
          o[k].y += g[k] * ty;
        }
      }
    }
#pragma unroll
    for (int k = 0; k < CMAX; ++k)
      if (k < C) base[(size_t)k * a.S] = o[k];
  }
}

template <typename T, int CMAX>
void lean_launch(LeanArgs<T> a, size_t smem, cudaStream_t st) {
  GPN_CUDA(cudaFuncSetAttribute(k_step3_lean<T, CMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  // gridDim.y is limited to 65535: launch the rows in chunks
  const long long per = 65535ll * kRy;
  for (long long r0 = 0; r0 < a.rows; r0 += per) {
    a.row0 = r0;
    const long long nr = std::min(per, a.rows - r0);
    dim3 grid((unsigned)((a.half + kRx - 1) / kRx), (unsigned)((nr + kRy - 1) / kRy));
    k_step3_lean<T, CMAX><<<grid, dim3(kRx, kRy), smem, st>>>(a);
  }
}

template <typename T>
void lean_impl(Plan& plan, int R, cudaStream_t st) {
  const GridGeom& g = plan.geom;
  if (plan.tr3) {
    LeanTArgs<T> a{(const cpx<T>*)plan.fy, (cpx<T>*)plan.fz, (const T*)plan.lean_tab, (const T*)plan.lean_sqv,
                   g.nf, (int)g.M, g.C, plan.lean_cp, plan.lean_J, R};
    lean_t_dispatch<T, 1>(a, lean_smem_bytes(plan), st);
  } else {
    LeanArgs<T> a{};
    a.spec = (typename Cplx<T>::type*)plan.spec;
    a.tab = (const T*)plan.lean_tab;
    a.sqv = (const T*)plan.lean_sqv;
    a.S = plan.spec_elems;
    a.half = g.nf / 2 + 1;
    a.nf = g.nf;
    a.rows = a.S / a.half;
    a.M = (int)g.M;
    a.C = g.C;
    a.CP = plan.lean_cp;
    a.J = plan.lean_J;
    a.R = R;
    a.d = g.d;
    const size_t smem = lean_smem_bytes(plan);
    switch (cmax_bucket(g.C)) {
      case 8: lean_launch<T, 8>(a, smem, st); break;
      case 12: lean_launch<T, 12>(a, smem, st); break;
      case 16: lean_launch<T, 16>(a, smem, st); break;
      default: lean_launch<T, 32>(a, smem, st);
    }
  }
  GPN_CUDA(cudaGetLastError());
}

}  // namespace

int lean_channel_pitch(int C, size_t rs) { return round_up(C, (int)(16 / rs)); }

size_t lean_smem_bytes(const Plan& plan) {
  const int rows = plan.tr3 ? kTy : kRy;
  return (size_t)rows * plan.lean_J * plan.lean_cp * plan.real_size;
}

void build_lean_tables(Plan& plan) {
  const int C = plan.geom.C;
  const int J = (int)plan.tb.vt.size();
  const long long Mp = plan.h.M + 1;
  const int CP = lean_channel_pitch(C, plan.real_size);
  plan.lean_J = J;
  plan.lean_cp = CP;
  std::vector<double> tab((size_t)J * Mp * CP, 0.0), sqv(J);
  for (int j = 0; j < J; ++j) {
    GPN_CHECK(plan.tb.vt[j] > 0.0, GP_EUNSUPPORTED, "memory-lean step 3 needs positive quadrature weights");
    sqv[j] = std::sqrt(plan.tb.vt[j]);
    for (int k = 0; k < C; ++k)
      for (long long m = 0; m < Mp; ++m)
        tab[((size_t)j * Mp + m) * CP + k] = plan.tb.etab[((size_t)k * J + j) * Mp + m];
  }
  if (plan.precision == GP_FP32) {
    std::vector<float> tf(tab.begin(), tab.end()), sf(sqv.begin(), sqv.end());
    plan.lean_tab = plan.alloc(tf.size() * sizeof(float));
    plan.lean_sqv = plan.alloc(sf.size() * sizeof(float));
    GPN_CUDA(cudaMemcpy(plan.lean_tab, tf.data(), tf.size() * sizeof(float), cudaMemcpyHostToDevice));
    GPN_CUDA(cudaMemcpy(plan.lean_sqv, sf.data(), sf.size() * sizeof(float), cudaMemcpyHostToDevice));
  } else {
    plan.lean_tab = plan.alloc(tab.size() * sizeof(double));
    plan.lean_sqv = plan.alloc(sqv.size() * sizeof(double));
    GPN_CUDA(cudaMemcpy(plan.lean_tab, tab.data(), tab.size() * sizeof(double), cudaMemcpyHostToDevice));
    GPN_CUDA(cudaMemcpy(plan.lean_sqv, sqv.data(), sqv.size() * sizeof(double), cudaMemcpyHostToDevice));
  }
}

void launch_step3_lean(Plan& plan, int R, cudaStream_t st) {
  if (plan.precision == GP_FP32)
    lean_impl<float>(plan, R, st);
  else
    lean_impl<double>(plan, R, st);
}

}  // namespace gpn
