// Pruned 2-D transforms in transposed order (d = 2, nf = 2^a): the uniform FFTs of the
// type-1 and type-2 NUFFTs (App. D) with step (3) of Sec. 4.2 between them.
//
// Only the modes |n_a| <= M are used (the restriction Pi of Sec. 3.4), and only the
// rows [row_lo, row_hi) and columns [col_lo, col_hi) of the fine grid hold spread
// data or are read by the interpolation.  The transform is split by axis, and the
// row stage writes its output transposed, so every column transform reads and
// writes one contiguous column:
//   1. rows, forward (k_rows_fwd): each CTA transforms RB grid rows of length nf in
//      shared memory.  A real row is an nf/2-point complex FFT of its even/odd pairs
//      plus the real split (fft_core.h).  The CTA keeps the modes m = 0..M and writes
//      X[cr][m][y] (cr = rhs * C + channel), the RB rows side by side.  Rows outside
//      [row_lo, row_hi) are never written and stay zero.
//   2. columns, forward: cuFFT, batched 1-D C2C of length nf over the C R (M+1)
//      contiguous columns, from X into Y.
//   3. step 3 (k_diag_t): a_k = sum_l A'_kl b_l for |n_1| <= M, from Y into Z.  A'
//      depends on |n_1| and m only; one thread serves n_1 and -n_1 from the same A'
//      entries.  Rows |n_1| > M of Z stay zero from plan creation on.
//   4. columns, inverse: cuFFT, from Z into Y.
//   5. rows, inverse (k_rows_inv): each CTA reads the modes 0..M of RB rows, merges
//      them into the nf/2-point complex input, runs the inverse FFT and writes the
//      columns [col_lo, col_hi) of the grid rows.
// All transforms are unnormalised, forward e^{-2 pi i}, inverse e^{+2 pi i}, as with
// cuFFT's R2C/C2R, so A' is the same as for the full-grid path.
#include <cufft.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "fft_core.h"
#include "kernels.h"

namespace gpn {

namespace {

using fft::cpx;

template <typename T>
struct Vec2;
template <>
struct Vec2<float> {
  using type = float2;
};
template <>
struct Vec2<double> {
  using type = double2;
};

// RB adjacent complex values to global memory (16-byte stores where possible)
template <typename T, int RB>
__device__ __forceinline__ void store_rb(cpx<T>* o, const cpx<T> (&v)[RB]) {
  if constexpr (sizeof(T) == 4 && RB == 2) {
    *reinterpret_cast<float4*>(o) = make_float4(v[0].x, v[0].y, v[1].x, v[1].y);
  } else {
#pragma unroll
    for (int r = 0; r < RB; ++r) *reinterpret_cast<typename Vec2<T>::type*>(o + r) = {v[r].x, v[r].y};
  }
}

template <typename T, int RB>
__device__ __forceinline__ void load_rb(const cpx<T>* o, cpx<T> (&v)[RB]) {
  if constexpr (sizeof(T) == 4 && RB == 2) {
    const float4 u = *reinterpret_cast<const float4*>(o);
    v[0] = {u.x, u.y};
    v[1] = {u.z, u.w};
  } else {
#pragma unroll
    for (int r = 0; r < RB; ++r) {
      const typename Vec2<T>::type u = *reinterpret_cast<const typename Vec2<T>::type*>(o + r);
      v[r] = {u.x, u.y};
    }
  }
}

// shared-memory elements of one row buffer: the padded length-N2 FFT plus the slot N2
__host__ __device__ constexpr int row_buf(int n2) { return n2 + n2 / 16 + 1; }
// entries of one high-part twiddle table (W^{64 q}, q <= N2 / 64)
__host__ __device__ constexpr int tw_hi(int n2) { return n2 / 64 + 1; }
// dynamic shared memory of a row kernel: RB row buffers, then the two-level twiddles of
// the length-N2 FFT ([hi][lo]) and of the real split ([hi][lo])
constexpr size_t row_smem(int n2, int rb, size_t cs) { return ((size_t)rb * row_buf(n2) + 2 * (tw_hi(n2) + 64)) * cs; }

// the twiddle functors over the tables staged in shared memory
template <typename T>
__device__ __forceinline__ void stage_twiddles(cpx<T>* s_tw, const cpx<T>* __restrict__ g, int n2) {
  for (int i = threadIdx.x; i < 2 * (tw_hi(n2) + 64); i += blockDim.x) s_tw[i] = g[i];
}

template <typename T>
struct RowsArgs {
  const T* gin;            // spreading grids (forward input), (R*C) x nf x nf
  T* gout;                 // interp grids (inverse output)
  cpx<T>* X;               // forward row output / inverse row input: [cr][M+1][nf]
  const cpx<T>* tw;        // two-level tables: W_{N2} (hi, lo), then W_nf (hi, lo)
  long long nf;
  long long G;             // nf^2
  int M;
  int row0;                // first row of block 0 (a multiple of RB)
  int row_hi;
  int col_lo, col_hi;
};

// In-place complex FFT of length 2^L on the row buffer b, NT = 2^L / 16 threads per
// row (t = 0..NT-1), every thread of the block taking part in the barriers.
template <bool INV, int L, typename T>
__device__ __forceinline__ void fft_block(cpx<T>* b, const fft::Twiddle2<T>& tw, int t) {
  constexpr int N = 1 << L, NT = N / 16;
  int Ns = 1;
  if constexpr (L % 4 != 0) {
    constexpr int R = 1 << (L % 4);
    fft::Pass<R, 16 / R, T> p;
    p.load(b, N, t, NT);
    __syncthreads();
    p.template store<INV>(b, tw, N, Ns, t, NT);
    __syncthreads();
    Ns *= R;
  }
#pragma unroll 1
  for (int s = 0; s < L / 4; ++s) {
    fft::Pass<16, 1, T> p;
    p.load(b, N, t, NT);
    __syncthreads();
    p.template store<INV>(b, tw, N, Ns, t, NT);
    __syncthreads();
    Ns *= 16;
  }
}

// Blocks of RB * 2^L / 16 threads; in FP32 at most 64 registers a thread, so that two
// 512-thread blocks fit an SM.
template <typename T, int L, int RB>
constexpr int rows_min_blocks() {
  return sizeof(T) == 4 ? ((1024 / (RB * (1 << L) / 16)) > 0 ? 1024 / (RB * (1 << L) / 16) : 1) : 1;
}

// RB rows per CTA, NT = 2^L / 16 threads per row.
template <typename T, int L, int RB>
__global__ void __launch_bounds__(RB*(1 << L) / 16, (rows_min_blocks<T, L, RB>())) k_rows_fwd(RowsArgs<T> a) {
  constexpr int N2 = 1 << L, NT = N2 / 16, BUF = row_buf(N2);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<T>* buf = reinterpret_cast<cpx<T>*>(smem_raw);
  const int q = threadIdx.x / NT, t = threadIdx.x - q * NT;
  const int cr = blockIdx.y;
  const long long y0 = a.row0 + (long long)blockIdx.x * RB;
  const long long y = y0 + q;
  cpx<T>* b = buf + q * BUF;
  cpx<T>* s_tw = buf + RB * BUF;
  stage_twiddles(s_tw, a.tw, N2);
  const fft::Twiddle2<T> tw{s_tw, s_tw + tw_hi(N2)};
  const fft::Twiddle2<T> wn{s_tw + tw_hi(N2) + 64, s_tw + 2 * tw_hi(N2) + 64};
  {
    const T* src = a.gin + (size_t)cr * a.G + y * a.nf;
    const bool rin = y < a.row_hi;
    for (int i = t; i < N2; i += NT) {
      cpx<T> v{T(0), T(0)};
      if (rin && 2 * i + 1 >= a.col_lo && 2 * i < a.col_hi) {
        const typename Vec2<T>::type u = *reinterpret_cast<const typename Vec2<T>::type*>(src + 2 * i);
        v = {u.x, u.y};
      }
      b[fft::pad(i)] = v;  // z[i] = x[2i] + i x[2i+1]
    }
  }
  __syncthreads();
  fft_block<false, L>(b, tw, t);
  // real split of the RB rows at m = 0..M; the RB values of one m are adjacent in X
  cpx<T>* dst = a.X + (size_t)cr * (a.M + 1) * a.nf + y0;
  for (int m = threadIdx.x; m <= a.M; m += blockDim.x) {
    const cpx<T> w = wn(m);
    cpx<T> out[RB];
#pragma unroll
    for (int r = 0; r < RB; ++r) {
      const cpx<T>* br = buf + r * BUF;
      out[r] = fft::r2c_split(br[fft::pad(m)], br[fft::pad((N2 - m) & (N2 - 1))], w);
    }
    store_rb<T, RB>(dst + (size_t)m * a.nf, out);
  }
}

// Inverse of k_rows_fwd: modes 0..M of RB rows (zero above M; the imaginary part of
// mode 0 is dropped, as a C2R transform does) to the grid columns [col_lo, col_hi).
template <typename T, int L, int RB>
__global__ void __launch_bounds__(RB*(1 << L) / 16, (rows_min_blocks<T, L, RB>())) k_rows_inv(RowsArgs<T> a) {
  constexpr int N2 = 1 << L, NT = N2 / 16, BUF = row_buf(N2), H = N2 / 2 + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<T>* buf = reinterpret_cast<cpx<T>*>(smem_raw);
  const int q = threadIdx.x / NT, t = threadIdx.x - q * NT;
  const int cr = blockIdx.y;
  const long long y0 = a.row0 + (long long)blockIdx.x * RB;
  const long long y = y0 + q;
  const cpx<T>* src = a.X + (size_t)cr * (a.M + 1) * a.nf + y0;
  cpx<T>* s_tw = buf + RB * BUF;
  stage_twiddles(s_tw, a.tw, N2);
  const fft::Twiddle2<T> tw{s_tw, s_tw + tw_hi(N2)};
  const fft::Twiddle2<T> wn{s_tw + tw_hi(N2) + 64, s_tw + 2 * tw_hi(N2) + 64};
  for (int m = threadIdx.x; m <= N2; m += blockDim.x) {
    cpx<T> v[RB];
    if (m <= a.M) {
      load_rb<T, RB>(src + (size_t)m * a.nf, v);
    } else {
#pragma unroll
      for (int r = 0; r < RB; ++r) v[r] = {T(0), T(0)};
    }
#pragma unroll
    for (int r = 0; r < RB; ++r) {
      if (m == 0) v[r].y = T(0);
      buf[r * BUF + fft::pad(m)] = v[r];
    }
  }
  __syncthreads();
  // merge the pairs (k, N2 - k) in place: thread-private slots, no barrier needed inside
  for (int kk = threadIdx.x; kk < RB * H; kk += blockDim.x) {
    const int r = kk / H, k = kk - r * H;
    cpx<T>* br = buf + r * BUF;
    const cpx<T> xk = br[fft::pad(k)], xn = br[fft::pad(N2 - k)];
    const cpx<T> zk = fft::c2r_merge(xk, xn, wn(k));
    if (k != 0 && k != N2 / 2) br[fft::pad(N2 - k)] = fft::c2r_merge(xn, xk, wn(N2 - k));
    br[fft::pad(k)] = zk;
  }
  __syncthreads();
  cpx<T>* b = buf + q * BUF;
  fft_block<true, L>(b, tw, t);
  if (y < a.row_hi) {
    T* dst = a.gout + (size_t)cr * a.G + y * a.nf;
    for (int i = t; i < N2; i += NT) {
      if (2 * i + 1 >= a.col_lo && 2 * i < a.col_hi) {
        const cpx<T> v = b[fft::pad(i)];
        *reinterpret_cast<typename Vec2<T>::type*>(dst + 2 * i) = {v.x, v.y};
      }
    }
  }
}


template <typename T>
struct DiagTArgs {
  const cpx<T>* Y;         // column transforms [cr][M+1][nf]
  cpx<T>* Z;               // step-3 output, same layout
  const T* A;              // A' on the quadrant: [pair][m][|n1|], pairs (k <= l) packed
  long long nf;
  int M;
  int C;
  int R;
};

// One thread per (m, n1 >= 0): b_l at the rows n1 and nf - n1 of every channel's
// column m, then a_k = sum_l A'_kl b_l for both rows, output channel by output
// channel, with the same A' entries (A'_kl = A'_lk is stored once, packed for k <= l).
// NC: channels known at compile time (C itself up to 16, inputs in registers); NC = 32
// takes a runtime C and re-reads the inputs through the L1 cache.
template <typename T, int NC>
__global__ void __launch_bounds__(128) k_diag_t(DiagTArgs<T> a) {
  const int n1 = blockIdx.x * blockDim.x + threadIdx.x;
  const int m = blockIdx.y;
  if (n1 > a.M) return;
  constexpr bool kReg = NC <= 16;
  const int C = kReg ? NC : a.C;
  const size_t Mp = (size_t)a.M + 1;
  const size_t colstride = Mp * a.nf;          // between channels
  const size_t off_p = (size_t)m * a.nf + n1;
  const size_t off_n = (size_t)m * a.nf + (n1 == 0 ? 0 : a.nf - n1);
  const T* Am = a.A + (size_t)m * Mp + n1;
  const size_t pstride = Mp * Mp;
  for (int r = 0; r < a.R; ++r) {
    const cpx<T>* Yr = a.Y + (size_t)r * C * colstride;
    cpx<T>* Zr = a.Z + (size_t)r * C * colstride;
    cpx<T> bp[kReg ? NC : 1], bn[kReg ? NC : 1];
    if constexpr (kReg) {
#pragma unroll
      for (int l = 0; l < NC; ++l) {
        bp[l] = Yr[l * colstride + off_p];
        bn[l] = Yr[l * colstride + off_n];
      }
    }
#pragma unroll 1
    for (int k = 0; k < C; ++k) {
      cpx<T> ap{T(0), T(0)}, an{T(0), T(0)};
#pragma unroll(kReg ? NC : 1)
      for (int l = 0; l < C; ++l) {
        const int lo = k < l ? k : l, hi = k < l ? l : k;
        const int p = lo * C - lo * (lo - 1) / 2 + (hi - lo);
        const T w = Am[(size_t)p * pstride];
        cpx<T> xp, xn;
        if constexpr (kReg) {
          xp = bp[l];
          xn = bn[l];
        } else {
          xp = Yr[l * colstride + off_p];
          xn = Yr[l * colstride + off_n];
        }
        ap.x += w * xp.x;
        ap.y += w * xp.y;
        an.x += w * xn.x;
        an.y += w * xn.y;
      }
      Zr[k * colstride + off_p] = ap;
      if (n1 != 0) Zr[k * colstride + off_n] = an;
    }
  }
}

template <typename T, int NC>
void diag_dispatch(const DiagTArgs<T>& a, cudaStream_t st) {
  if constexpr (NC > 16) {
    dim3 grid((unsigned)((a.M + 128) / 128), (unsigned)(a.M + 1));
    k_diag_t<T, 32><<<grid, 128, 0, st>>>(a);
  } else {
    if (a.C == NC) {
      dim3 grid((unsigned)((a.M + 128) / 128), (unsigned)(a.M + 1));
      k_diag_t<T, NC><<<grid, 128, 0, st>>>(a);
    } else {
      diag_dispatch<T, NC + 1>(a, st);
    }
  }
}

constexpr int kMinLog = 4, kMaxLog = 13;       // nf = 32 .. 16384
constexpr size_t kRowSmemMax = size_t(150) << 10;

template <typename T, int L, int RB>
void rows_launch(bool inv, const RowsArgs<T>& a, unsigned nblk, unsigned ncr, cudaStream_t st) {
  const size_t smem = row_smem(1 << L, RB, sizeof(cpx<T>));
  void (*k)(RowsArgs<T>) = inv ? k_rows_inv<T, L, RB> : k_rows_fwd<T, L, RB>;
  GPN_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k<<<dim3(nblk, ncr), RB * (1 << L) / 16, smem, st>>>(a);
}

template <typename T, int L>
void rows_rb(bool inv, int rb, const RowsArgs<T>& a, unsigned nblk, unsigned ncr, cudaStream_t st) {
  // two rows per CTA only where tr3_setup allows it (shared memory and block size)
  if constexpr (row_smem(1 << L, 2, sizeof(cpx<T>)) <= kRowSmemMax && 2 * (1 << L) / 16 <= 1024) {
    if (rb == 2) return rows_launch<T, L, 2>(inv, a, nblk, ncr, st);
  }
  rows_launch<T, L, 1>(inv, a, nblk, ncr, st);
}

template <typename T>
void rows(bool inv, int L, int rb, const RowsArgs<T>& a, unsigned nblk, unsigned ncr, cudaStream_t st) {
  switch (L) {
    case 4: rows_rb<T, 4>(inv, rb, a, nblk, ncr, st); break;
    case 5: rows_rb<T, 5>(inv, rb, a, nblk, ncr, st); break;
    case 6: rows_rb<T, 6>(inv, rb, a, nblk, ncr, st); break;
    case 7: rows_rb<T, 7>(inv, rb, a, nblk, ncr, st); break;
    case 8: rows_rb<T, 8>(inv, rb, a, nblk, ncr, st); break;
    case 9: rows_rb<T, 9>(inv, rb, a, nblk, ncr, st); break;
    case 10: rows_rb<T, 10>(inv, rb, a, nblk, ncr, st); break;
    case 11: rows_rb<T, 11>(inv, rb, a, nblk, ncr, st); break;
    case 12: rows_rb<T, 12>(inv, rb, a, nblk, ncr, st); break;
    default: rows_rb<T, 13>(inv, rb, a, nblk, ncr, st);
  }
}

int log2_exact(long long n) {
  int L = 0;
  while ((1ll << L) < n) ++L;
  return (1ll << L) == n ? L : -1;
}

template <typename T>
RowsArgs<T> rows_args(Plan& plan, const void* X) {
  RowsArgs<T> a{};
  a.gin = (const T*)plan.grid;
  a.gout = (T*)plan.grid_out;
  a.X = (cpx<T>*)X;
  a.tw = (const cpx<T>*)plan.tw_half;
  a.nf = plan.geom.nf;
  a.G = plan.grid_elems;
  a.M = (int)plan.geom.M;
  a.row0 = plan.row_lo / plan.t3_rb * plan.t3_rb;
  a.row_hi = plan.row_hi;
  a.col_lo = plan.col_lo;
  a.col_hi = plan.col_hi;
  return a;
}

template <typename T>
void rows_run(Plan& plan, bool inv, const void* X, int R, cudaStream_t st) {
  const RowsArgs<T> a = rows_args<T>(plan, X);
  if (plan.row_hi <= a.row0) return;
  const unsigned nblk = (unsigned)((plan.row_hi - a.row0 + plan.t3_rb - 1) / plan.t3_rb);
  rows<T>(inv, log2_exact(plan.geom.nf / 2), plan.t3_rb, a, nblk, (unsigned)(plan.geom.C * R), st);
  GPN_CUDA(cudaGetLastError());
}

#define GPN_CUFFT3(call)                                                                                \
  do {                                                                                                  \
    cufftResult r_ = (call);                                                                            \
    if (r_ != CUFFT_SUCCESS) ::gpn::fail(GP_ECUFFT, std::string(#call " failed: code ") + std::to_string((int)r_)); \
  } while (0)

}  // namespace

bool tr3_supported(int d, long long nf, size_t rs) {
  if (d != 2) return false;
  const int L = log2_exact(nf / 2);
  if (nf % 2 || L < kMinLog || L > kMaxLog) return false;
  return row_smem(1 << L, 1, 2 * rs) <= kRowSmemMax;
}

void tr3_setup(Plan& plan) {
  const long long nf = plan.geom.nf, N2 = nf / 2;
  const int L = log2_exact(N2);
  const size_t cs = 2 * plan.real_size;
  plan.t3_rb = (row_smem(1 << L, 2, cs) <= kRowSmemMax && 2 * (N2 / 16) <= 1024) ? 2 : 1;
  // two-level tables, computed in float64: W_{N2}^{64 q} (q < H), W_{N2}^j (j < 64),
  // W_nf^{64 q} (q < H), W_nf^j (j < 64), with H = N2 / 64 + 1
  const int H = tw_hi((int)N2);
  std::vector<double> w;
  w.reserve(4 * (H + 64));
  auto put = [&](long long i, long long n) {
    const double th = 2.0 * M_PI * (double)(i % n) / (double)n;
    w.push_back(std::cos(th));
    w.push_back(-std::sin(th));
  };
  for (int q = 0; q < H; ++q) put(64ll * q, N2);
  for (int j = 0; j < 64; ++j) put(j, N2);
  for (int q = 0; q < H; ++q) put(64ll * q, nf);
  for (int j = 0; j < 64; ++j) put(j, nf);
  plan.tw_half = plan.alloc(w.size() * plan.real_size);
  if (plan.precision == GP_FP32) {
    std::vector<float> f(w.begin(), w.end());
    GPN_CUDA(cudaMemcpy(plan.tw_half, f.data(), f.size() * sizeof(float), cudaMemcpyHostToDevice));
  } else {
    GPN_CUDA(cudaMemcpy(plan.tw_half, w.data(), w.size() * sizeof(double), cudaMemcpyHostToDevice));
  }
}

cufftHandle Plan::t3_plan(int R) {
  auto it = fft_t3.find(R);
  if (it != fft_t3.end()) return it->second;
  int n[1] = {(int)geom.nf};
  cufftHandle hdl;
  GPN_CUFFT3(cufftPlanMany(&hdl, 1, n, n, 1, (int)geom.nf, n, 1, (int)geom.nf,
                           precision == GP_FP32 ? CUFFT_C2C : CUFFT_Z2Z, (int)(geom.C * R * (geom.M + 1))));
  fft_t3[R] = hdl;
  return hdl;
}

void tr3_forward(Plan& plan, int R, cudaStream_t st) {
  cufftHandle h = plan.t3_plan(R);
  if (plan.precision == GP_FP32) {
    rows_run<float>(plan, false, plan.fx, R, st);
    GPN_CUFFT3(cufftSetStream(h, st));
    GPN_CUFFT3(cufftExecC2C(h, (cufftComplex*)plan.fx, (cufftComplex*)plan.fy, CUFFT_FORWARD));
  } else {
    rows_run<double>(plan, false, plan.fx, R, st);
    GPN_CUFFT3(cufftSetStream(h, st));
    GPN_CUFFT3(cufftExecZ2Z(h, (cufftDoubleComplex*)plan.fx, (cufftDoubleComplex*)plan.fy, CUFFT_FORWARD));
  }
}

void tr3_diag(Plan& plan, int R, cudaStream_t st) {
  if (plan.precision == GP_FP32) {
    DiagTArgs<float> a{(const cpx<float>*)plan.fy, (cpx<float>*)plan.fz, (const float*)plan.a_tensor,
                       plan.geom.nf, (int)plan.geom.M, plan.geom.C, R};
    diag_dispatch<float, 1>(a, st);
  } else {
    DiagTArgs<double> a{(const cpx<double>*)plan.fy, (cpx<double>*)plan.fz, (const double*)plan.a_tensor,
                        plan.geom.nf, (int)plan.geom.M, plan.geom.C, R};
    diag_dispatch<double, 1>(a, st);
  }
  GPN_CUDA(cudaGetLastError());
}

void tr3_inverse(Plan& plan, int R, cudaStream_t st) {
  cufftHandle h = plan.t3_plan(R);
  GPN_CUFFT3(cufftSetStream(h, st));
  if (plan.precision == GP_FP32) {
    GPN_CUFFT3(cufftExecC2C(h, (cufftComplex*)plan.fz, (cufftComplex*)plan.fy, CUFFT_INVERSE));
    rows_run<float>(plan, true, plan.fy, R, st);
  } else {
    GPN_CUFFT3(cufftExecZ2Z(h, (cufftDoubleComplex*)plan.fz, (cufftDoubleComplex*)plan.fy, CUFFT_INVERSE));
    rows_run<double>(plan, true, plan.fy, R, st);
  }
}

}  // namespace gpn
