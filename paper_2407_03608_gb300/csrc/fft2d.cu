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
//   2. columns, forward: batched 1-D C2C of length nf over the C R (M+1) contiguous
//      columns, from X into Y: cuFFT for float and double plans, the library's own
//      k_cols for float-float plans (cuFFT has no float-float type).
//   3. step 3 (k_diag_t): a_k = sum_l A'_kl b_l for |n_1| <= M, from Y into Z.  A'
//      depends on |n_1| and m only; one thread serves n_1 and -n_1 from the same A'
//      entries.  Rows |n_1| > M of Z stay zero from plan creation on.
//   4. columns, inverse: cuFFT or k_cols, from Z into Y.
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
template <>
struct Vec2<dd> {
  using type = cpx<dd>;
};

// RB adjacent complex values to global memory (16-byte stores where possible)
template <typename T, int RB>
__device__ __forceinline__ void store_rb(cpx<T>* o, const cpx<T> (&v)[RB]) {
  if constexpr (sizeof(T) == 4 && RB % 2 == 0) {
#pragma unroll
    for (int r = 0; r < RB; r += 2)
      *reinterpret_cast<float4*>(o + r) = make_float4(v[r].x, v[r].y, v[r + 1].x, v[r + 1].y);
  } else {
#pragma unroll
    for (int r = 0; r < RB; ++r) *reinterpret_cast<typename Vec2<T>::type*>(o + r) = {v[r].x, v[r].y};
  }
}

template <typename T, int RB>
__device__ __forceinline__ void load_rb(const cpx<T>* o, cpx<T> (&v)[RB]) {
  if constexpr (sizeof(T) == 4 && RB % 2 == 0) {
#pragma unroll
    for (int r = 0; r < RB; r += 2) {
      const float4 u = *reinterpret_cast<const float4*>(o + r);
      v[r] = {u.x, u.y};
      v[r + 1] = {u.z, u.w};
    }
  } else {
#pragma unroll
    for (int r = 0; r < RB; ++r) {
      const typename Vec2<T>::type u = *reinterpret_cast<const typename Vec2<T>::type*>(o + r);
      v[r] = {u.x, u.y};
    }
  }
}

// Radix-16 passes are unrolled (measured: running the float-float passes as a loop, to
// shrink the code, made the column kernels 27 % slower)
template <typename T>
constexpr int kPassUnroll = 4;

// shared-memory elements of one row buffer: the padded length-N2 FFT plus the slot N2,
// rounded up to an even count (16-byte alignment of what follows)
__host__ __device__ constexpr int row_buf(int n2) { return (n2 + n2 / 16 + 2) & ~1; }
// entries of one high-part twiddle table (W^{64 q}, q <= N2 / 64)
__host__ __device__ constexpr int tw_hi(int n2) { return n2 / 64 + 1; }
// The FP32 forward kernel reads per-pass twiddle tables (fft::pass_tables) staged in
// shared memory, one load a twiddle; the others form the FFT twiddles from the
// two-level tables (measured: the inverse kernel runs faster with the smaller
// shared-memory footprint).
template <typename T, bool INV>
__host__ __device__ constexpr bool pass_tables_in_smem() { return (sizeof(T) == 4 && !INV) || is_dd<T>::value; }
// twiddle entries staged by a row kernel: the two-level tables of the length-N2 FFT
// ([hi][lo]) and of the real split ([hi][lo]), then (FP32) the pass tables; padded to
// whole 16-byte chunks
template <typename T, bool INV>
__host__ __device__ constexpr int tw_count(int L) {
  return (2 * (tw_hi(1 << L) + 64) + (pass_tables_in_smem<T, INV>() ? fft::pass_table_size(L) : 0) + 1) & ~1;
}
// dynamic shared memory of a row kernel: RB row buffers, then the twiddles
template <typename T, bool INV>
constexpr size_t row_smem(int L, int rb) {
  return ((size_t)rb * row_buf(1 << L) + tw_count<T, INV>(L)) * sizeof(cpx<T>);
}

// the twiddle functors over the tables staged in shared memory
template <typename T>
struct RowsArgs {
  const T* gin;            // spreading grids (forward input), (R*C) x nf x nf
  T* gout;                 // interp grids (inverse output)
  cpx<T>* X;               // forward row output / inverse row input: [cr][M+1][nf]
  const cpx<T>* tw;        // two-level tables: W_{N2} (hi, lo), then W_nf (hi, lo)
  long long nf;
  long long G;             // nf^2
  int M;
  int row0;                // first row of item 0 (a multiple of RB)
  int row_hi;
  long long npairs;        // RB-row groups per grid
  long long nitems;        // npairs * C * R
  int col_lo, col_hi;
};

// In-place complex FFT of length N = 2^L on the row buffer b by Stockham passes (one of
// radix 2^(L mod 4) when L is not a multiple of 4, then radix 16), NT = N / 16 threads per
// row (t = 0..NT-1), every thread of the block taking part in the barriers.  The first
// pass takes its inputs from x[u] = element t + u N/16 (the values the thread loaded
// from global memory), which skips a shared-memory round trip.  tw2: the two-level
// twiddle; ptab: the staged pass tables (FP32 forward).
template <bool INV, int L, typename T>
__device__ __forceinline__ void fft_block_from_regs(cpx<T>* b, const cpx<T> (&x)[16], const fft::Twiddle2<T>& tw2,
                                                    const cpx<T>* ptab, int t) {
  constexpr int N = 1 << L, NT = N / 16;
  constexpr int R0 = (L % 4 == 0) ? 16 : (1 << (L % 4));
  {
    fft::Pass<R0, 16 / R0, T> p;
    fft::first_pass_inputs(p, x);
    p.template compute<INV>(tw2, N, 1, t, NT);  // span 1: no twiddles
    p.write(b, 1, t, NT);
  }
  __syncthreads();
  int Ns = R0;
#pragma unroll (kPassUnroll<T>)
  for (int s = (L % 4 == 0) ? 1 : 0; s < L / 4; ++s) {
    fft::Pass<16, 1, T> p;
    p.load(b, N, t, NT);
    __syncthreads();
    if constexpr (pass_tables_in_smem<T, INV>()) {
      const fft::PassTwiddle<T> tw{ptab + fft::pass_table_offset(L, Ns), Ns};
      p.template store<INV>(b, tw, N, Ns, t, NT);
    } else {
      p.template store<INV>(b, tw2, N, Ns, t, NT);
    }
    __syncthreads();
    Ns *= 16;
  }
}

// The same transform from the buffer, except that the last pass (radix 16 at span N/16)
// hands its outputs to out(r, v) instead of the buffer: output r of thread t is element
// t + r N/16 of the transform.  No barrier follows.
template <bool INV, int L, typename T, typename Out>
__device__ __forceinline__ void fft_block_to(cpx<T>* b, const fft::Twiddle2<T>& tw2, const cpx<T>* ptab, int t,
                                             Out out) {
  constexpr int N = 1 << L, NT = N / 16;
  int Ns = 1;
  if constexpr (L % 4 != 0) {
    constexpr int R = 1 << (L % 4);
    fft::Pass<R, 16 / R, T> p;
    p.load(b, N, t, NT);
    __syncthreads();
    p.template store<INV>(b, tw2, N, Ns, t, NT);  // span 1: no twiddles
    __syncthreads();
    Ns *= R;
  }
#pragma unroll (kPassUnroll<T>)
  for (int s = 0; s < L / 4; ++s) {
    fft::Pass<16, 1, T> p;
    p.load(b, N, t, NT);
    __syncthreads();
    if constexpr (pass_tables_in_smem<T, INV>()) {
      const fft::PassTwiddle<T> tw{ptab + fft::pass_table_offset(L, Ns), Ns};
      p.template compute<INV>(tw, N, Ns, t, NT);
    } else {
      p.template compute<INV>(tw2, N, Ns, t, NT);
    }
    if (s + 1 < L / 4) {
      p.write(b, Ns, t, NT);
      __syncthreads();
    } else {
#pragma unroll
      for (int r = 0; r < 16; ++r) out(r, p.v[0][r]);
    }
    Ns *= 16;
  }
}

// async 16-byte copy global -> shared (no registers), completed by cp_async_wait_all
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// stage the twiddle tables (global layout: two-level tables, then the pass tables; the
// count padded to whole 16-byte chunks)
template <typename T, bool INV>
__device__ __forceinline__ void stage_twiddles_async(cpx<T>* s_tw, const cpx<T>* __restrict__ g, int L) {
  const int chunks = (int)(tw_count<T, INV>(L) * sizeof(cpx<T>) / 16);
  for (int i = threadIdx.x; i < chunks; i += blockDim.x)
    cp_async16(reinterpret_cast<char*>(s_tw) + 16 * i, reinterpret_cast<const char*>(g) + 16 * i);
}

// Blocks of RB * 2^L / 16 threads; for the long FP32 rows at most 64 registers a
// thread, so that two 512-thread blocks fit an SM.
template <typename T, int L, int RB>
constexpr int rows_min_blocks() {
  return (sizeof(T) == 4 && L >= 11) ? 1024 / (RB * (1 << L) / 16) : 1;
}

// Each CTA stages the twiddles (asynchronously, overlapping its first loads), then
// takes the work items blockIdx.x, blockIdx.x + gridDim.x, ... (the launch uses one
// item per CTA); an item is RB consecutive rows of one (rhs, channel) grid, the row
// groups of one grid being consecutive items.  NT = 2^L / 16 threads per row.
template <typename T, int L, int RB>
__global__ void __launch_bounds__(RB*(1 << L) / 16, (rows_min_blocks<T, L, RB>())) k_rows_fwd(RowsArgs<T> a) {
  constexpr int N2 = 1 << L, NT = N2 / 16, BUF = row_buf(N2);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<T>* buf = reinterpret_cast<cpx<T>*>(smem_raw);
  const int q = threadIdx.x / NT, t = threadIdx.x - q * NT;
  cpx<T>* b = buf + q * BUF;
  cpx<T>* s_tw = buf + RB * BUF;
  stage_twiddles_async<T, false>(s_tw, a.tw, L);
  const fft::Twiddle2<T> tw{s_tw, s_tw + tw_hi(N2)};
  const fft::Twiddle2<T> wn{s_tw + tw_hi(N2) + 64, s_tw + 2 * tw_hi(N2) + 64};
  const cpx<T>* ptab = s_tw + 2 * (tw_hi(N2) + 64);
  bool first = true;
  for (long long item = blockIdx.x; item < a.nitems; item += gridDim.x) {
    const int cr = (int)(item / a.npairs);
    const long long y0 = a.row0 + (item - (long long)cr * a.npairs) * RB;
    const long long y = y0 + q;
    {
      // 16 elements a thread: every load is issued before the first shared-memory store
      const T* src = a.gin + (size_t)cr * a.G + y * a.nf;
      const bool rin = y < a.row_hi;
      cpx<T> v[16];
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        const int i = t + u * NT;
        v[u] = {T(0), T(0)};
        if (rin && 2 * i + 1 >= a.col_lo && 2 * i < a.col_hi) {
          const typename Vec2<T>::type w = *reinterpret_cast<const typename Vec2<T>::type*>(src + 2 * i);
          v[u] = {w.x, w.y};
        }
      }
      if (first) {
        cp_async_wait_all();
        first = false;
      }
      __syncthreads();  // twiddles staged; the previous item's buffers are free
      fft_block_from_regs<false, L>(b, v, tw, ptab, t);  // z[i] = x[2i] + i x[2i+1]
    }
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
    __syncthreads();  // the buffers are refilled by the next item
  }
  if (first) cp_async_wait_all();
}

// Inverse of k_rows_fwd: modes 0..M of RB rows (zero above M; the imaginary part of
// mode 0 is dropped, as a C2R transform does) to the grid columns [col_lo, col_hi).
template <typename T, int L, int RB>
__global__ void __launch_bounds__(RB*(1 << L) / 16, (rows_min_blocks<T, L, RB>())) k_rows_inv(RowsArgs<T> a) {
  constexpr int N2 = 1 << L, NT = N2 / 16, BUF = row_buf(N2), H = N2 / 2 + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<T>* buf = reinterpret_cast<cpx<T>*>(smem_raw);
  const int q = threadIdx.x / NT, t = threadIdx.x - q * NT;
  cpx<T>* b = buf + q * BUF;
  cpx<T>* s_tw = buf + RB * BUF;
  stage_twiddles_async<T, true>(s_tw, a.tw, L);
  const fft::Twiddle2<T> tw{s_tw, s_tw + tw_hi(N2)};
  const fft::Twiddle2<T> wn{s_tw + tw_hi(N2) + 64, s_tw + 2 * tw_hi(N2) + 64};
  const cpx<T>* ptab = s_tw + 2 * (tw_hi(N2) + 64);
  bool first = true;
  for (long long item = blockIdx.x; item < a.nitems; item += gridDim.x) {
    const int cr = (int)(item / a.npairs);
    const long long y0 = a.row0 + (item - (long long)cr * a.npairs) * RB;
    const long long y = y0 + q;
    const cpx<T>* src = a.X + (size_t)cr * (a.M + 1) * a.nf + y0;
    {
      // modes m = threadIdx.x + u * blockDim (U rounds cover 0..N2); loads first, then stores
      constexpr int NTH = RB * NT, U = (N2 + 1 + NTH - 1) / NTH;
      cpx<T> v[U][RB];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int m = threadIdx.x + u * NTH;
        if (m <= a.M) {
          load_rb<T, RB>(src + (size_t)m * a.nf, v[u]);
        } else {
#pragma unroll
          for (int r = 0; r < RB; ++r) v[u][r] = {T(0), T(0)};
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int m = threadIdx.x + u * NTH;
        if (m <= N2) {
#pragma unroll
          for (int r = 0; r < RB; ++r) {
            if (m == 0) v[u][r].y = T(0);
            buf[r * BUF + fft::pad(m)] = v[u][r];
          }
        }
      }
    }
    if (first) {
      cp_async_wait_all();
      first = false;
    }
    __syncthreads();
    // merge the pairs (k, N2 - k) in place: thread-private slots, no barrier needed inside
    for (int kk = threadIdx.x; kk < RB * H; kk += blockDim.x) {
      const int r = kk / H, k = kk - r * H;
      cpx<T>* br = buf + r * BUF;
      const cpx<T> xk = br[fft::pad(k)], xn = br[fft::pad(N2 - k)];
      // W_nf^(N2 - k) = W_nf^(N2) W_nf^(-k) = -conj(W_nf^k): one twiddle serves the pair
      const cpx<T> w = wn(k);
      const cpx<T> zk = fft::c2r_merge(xk, xn, w);
      if (k != 0 && k != N2 / 2) br[fft::pad(N2 - k)] = fft::c2r_merge(xn, xk, cpx<T>{-w.x, w.y});
      br[fft::pad(k)] = zk;
    }
    __syncthreads();
    {
      // the last pass writes x[2i], x[2i+1] (i = t + r NT) straight to the grid row
      T* dst = a.gout + (size_t)cr * a.G + y * a.nf;
      const bool rin = y < a.row_hi;
      const int clo = a.col_lo, chi = a.col_hi;
      fft_block_to<true, L>(b, tw, ptab, t, [&](int r, const cpx<T>& v) {
        const int i = t + r * NT;
        if (rin && 2 * i + 1 >= clo && 2 * i < chi)
          *reinterpret_cast<typename Vec2<T>::type*>(dst + 2 * i) = {v.x, v.y};
      });
    }
    __syncthreads();  // the buffers are refilled by the next item
  }
  if (first) cp_async_wait_all();
}

// ---- column transforms (float-float plans) -------------------------------------------
//
// The first-axis transforms of the transposed layout: every (rhs, channel, mode m)
// column of nf complex values is contiguous, so one CTA takes one column, loads it
// into registers (16 values a thread, coalesced), runs the Stockham passes through
// shared memory and writes the last pass straight back.  Rows known to be zero are
// not read, and only the rows the next stage reads are written:
//   forward (X -> Y): input rows [row_lo, row_hi) (the data extent; the row stage
//     writes no others), output rows |n_1| <= M (what step 3 reads);
//   inverse (Z -> Y): input rows |n_1| <= M (step 3 writes no others), output rows
//     [out_lo, out_hi) (the row groups the inverse row kernel reads).
// Twiddles come from the pass tables of the length-nf FFT in global memory (L1/L2
// resident; too large for shared memory next to a 16-byte-per-value column).

// one complex value through the read-only path
template <typename T>
__device__ __forceinline__ cpx<T> ldg_c(const cpx<T>* p) {
  return *p;
}
template <>
__device__ __forceinline__ cpx<dd> ldg_c<dd>(const cpx<dd>* p) {
  const float4 u = __ldg(reinterpret_cast<const float4*>(p));
  return {dd(u.x, u.y), dd(u.z, u.w)};
}

// twiddles of one radix-16 pass from a pass table in global memory ([r - 1][k])
template <typename T>
struct GPassTwiddle {
  const cpx<T>* tab;
  int Ns;
  __device__ __forceinline__ cpx<T> operator()(int r, int k, int) const { return ldg_c(tab + (r - 1) * Ns + k); }
};

// In-place complex FFT of length N = 2^L (L >= 5) with NT = N / 16 threads: the first
// pass (radix 2^(L mod 4), or 16) from the registers x[u] = element t + u NT, the
// middle passes through the buffer, and the last pass (radix 16 at span N/16) handed to
// out(r, v), output r of thread t being element t + r NT.  No barrier follows.
template <bool INV, int L, typename T, typename Out>
__device__ __forceinline__ void fft_block_regs_to(cpx<T>* b, const cpx<T> (&x)[16], const cpx<T>* ptab, int t,
                                                  Out out) {
  constexpr int N = 1 << L, NT = N / 16;
  constexpr int R0 = (L % 4 == 0) ? 16 : (1 << (L % 4));
  constexpr int S = (L % 4 == 0) ? L / 4 - 1 : L / 4;   // radix-16 passes after the first
  static_assert(L >= 5, "at least one radix-16 pass after the first");
  {
    fft::Pass<R0, 16 / R0, T> p;
    fft::first_pass_inputs(p, x);
    p.template compute<INV>(GPassTwiddle<T>{ptab, 1}, N, 1, t, NT);   // span 1: no twiddles
    p.write(b, 1, t, NT);
  }
  __syncthreads();
  int Ns = R0;
#pragma unroll (kPassUnroll<T>)
  for (int s = 0; s < S; ++s) {
    fft::Pass<16, 1, T> p;
    p.load(b, N, t, NT);
    __syncthreads();
    p.template compute<INV>(GPassTwiddle<T>{ptab + fft::pass_table_offset(L, Ns), Ns}, N, Ns, t, NT);
    if (s + 1 < S) {
      p.write(b, Ns, t, NT);
      __syncthreads();
    } else {
#pragma unroll
      for (int r = 0; r < 16; ++r) out(r, p.v[0][r]);
    }
    Ns *= 16;
  }
}

template <typename T>
struct ColsArgs {
  const cpx<T>* in;        // [col][nf]
  cpx<T>* out;             // [col][nf]
  const cpx<T>* ptab;      // pass tables of the length-nf FFT
  long long ncols;         // C R (M + 1)
  int in_lo0, in_hi0, in_lo1, in_hi1;     // input rows that may be nonzero: two ranges
  int out_lo0, out_hi0, out_lo1, out_hi1; // output rows written: two ranges
};

__device__ __forceinline__ bool in_ranges(int y, int a0, int a1, int b0, int b1) {
  return (y >= a0 && y < a1) || (y >= b0 && y < b1);
}

template <typename T, int L, bool INV>
__global__ void __launch_bounds__((1 << L) / 16, 1) k_cols(ColsArgs<T> a) {
  constexpr int N = 1 << L, NT = N / 16;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<T>* b = reinterpret_cast<cpx<T>*>(smem_raw);
  const int t = threadIdx.x;
  for (long long col = blockIdx.x; col < a.ncols; col += gridDim.x) {
    const cpx<T>* src = a.in + (size_t)col * N;
    cpx<T>* dst = a.out + (size_t)col * N;
    cpx<T> v[16];
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      const int y = t + u * NT;
      v[u] = in_ranges(y, a.in_lo0, a.in_hi0, a.in_lo1, a.in_hi1) ? ldg_c(src + y) : cpx<T>{T(0), T(0)};
    }
    __syncthreads();   // the previous column's last pass has read the buffer
    fft_block_regs_to<INV, L>(b, v, a.ptab, t, [&](int r, const cpx<T>& val) {
      const int y = t + r * NT;
      if (in_ranges(y, a.out_lo0, a.out_hi0, a.out_lo1, a.out_hi1)) dst[y] = val;
    });
  }
}

template <typename T>
constexpr size_t cols_smem(int L) {
  return (size_t)((1 << L) + (1 << L) / 16) * sizeof(cpx<T>);
}

template <typename T, int L>
void cols_launch(bool inv, const ColsArgs<T>& a, cudaStream_t st) {
  const size_t smem = cols_smem<T>(L);
  void (*k)(ColsArgs<T>) = inv ? k_cols<T, L, true> : k_cols<T, L, false>;
  GPN_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k<<<(unsigned)a.ncols, (1 << L) / 16, smem, st>>>(a);
}

template <typename T>
void cols(bool inv, int L, const ColsArgs<T>& a, cudaStream_t st) {
  switch (L) {
    case 5: cols_launch<T, 5>(inv, a, st); break;
    case 6: cols_launch<T, 6>(inv, a, st); break;
    case 7: cols_launch<T, 7>(inv, a, st); break;
    case 8: cols_launch<T, 8>(inv, a, st); break;
    case 9: cols_launch<T, 9>(inv, a, st); break;
    case 10: cols_launch<T, 10>(inv, a, st); break;
    case 11: cols_launch<T, 11>(inv, a, st); break;
    case 12: cols_launch<T, 12>(inv, a, st); break;
    default: cols_launch<T, 13>(inv, a, st);
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
  // up to 11 channels: all C(C+1)/2 entries of A' at this frequency are loaded at once,
  // before the right-hand sides (many loads in flight; A' read once for every rhs)
  constexpr int NP = NC * (NC + 1) / 2;
  if constexpr (kReg && NC <= 11) {
    T av[NP];
#pragma unroll
    for (int p = 0; p < NP; ++p) av[p] = ldg_val(Am + (size_t)p * pstride);
    for (int r = 0; r < a.R; ++r) {
      const cpx<T>* Yr = a.Y + (size_t)r * NC * colstride;
      cpx<T>* Zr = a.Z + (size_t)r * NC * colstride;
      cpx<T> bp[NC], bn[NC];
#pragma unroll
      for (int l = 0; l < NC; ++l) {
        bp[l] = Yr[l * colstride + off_p];
        bn[l] = Yr[l * colstride + off_n];
      }
#pragma unroll
      for (int k = 0; k < NC; ++k) {
        cpx<T> ap{T(0), T(0)}, an{T(0), T(0)};
#pragma unroll
        for (int l = 0; l < NC; ++l) {
          const int lo = k < l ? k : l, hi = k < l ? l : k;
          const T w = av[lo * NC - lo * (lo - 1) / 2 + (hi - lo)];
          madd_lazy(ap.x, w, bp[l].x);
          madd_lazy(ap.y, w, bp[l].y);
          madd_lazy(an.x, w, bn[l].x);
          madd_lazy(an.y, w, bn[l].y);
        }
        Zr[k * colstride + off_p] = {renorm_val(ap.x), renorm_val(ap.y)};
        if (n1 != 0) Zr[k * colstride + off_n] = {renorm_val(an.x), renorm_val(an.y)};
      }
    }
    return;
  }
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
        madd(ap.x, w, xp.x);
        madd(ap.y, w, xp.y);
        madd(an.x, w, xn.x);
        madd(an.y, w, xn.y);
      }
      Zr[k * colstride + off_p] = ap;
      if (n1 != 0) Zr[k * colstride + off_n] = an;
    }
  }
}

// 8-byte async copy global -> shared (no registers), completed by cp_async_wait_all
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}

// k_diag_t for float-float plans with up to 9 channels: the C(C+1)/2 entries of A' at the
// thread's frequency go to shared memory by asynchronous copies (one column of
// s_av per thread, so a warp's reads are consecutive) instead of registers, which keeps
// the thread at about 100 registers and four CTAs an SM; the entries are then read once
// per (k, l) like the register form reads them.
constexpr int kDiagDDMaxC = 9;
constexpr int kDiagThreads = 128;
template <int NC>
__global__ void __launch_bounds__(kDiagThreads, 4) k_diag_t_dd(DiagTArgs<dd> a) {
  constexpr int NP = NC * (NC + 1) / 2;
  __shared__ dd s_av[NP][kDiagThreads];
  const int n1 = blockIdx.x * blockDim.x + threadIdx.x;
  const int m = blockIdx.y;
  if (n1 > a.M) return;   // no barrier below: each thread reads only its own column
  const size_t Mp = (size_t)a.M + 1;
  const size_t colstride = Mp * a.nf;
  const size_t off_p = (size_t)m * a.nf + n1;
  const size_t off_n = (size_t)m * a.nf + (n1 == 0 ? 0 : a.nf - n1);
  const dd* Am = a.A + (size_t)m * Mp + n1;
  const size_t pstride = Mp * Mp;
#pragma unroll
  for (int p = 0; p < NP; ++p) cp_async8(&s_av[p][threadIdx.x], Am + (size_t)p * pstride);
  for (int r = 0; r < a.R; ++r) {
    const cpx<dd>* Yr = a.Y + (size_t)r * NC * colstride;
    cpx<dd>* Zr = a.Z + (size_t)r * NC * colstride;
    cpx<dd> bp[NC], bn[NC];
#pragma unroll
    for (int l = 0; l < NC; ++l) {
      bp[l] = Yr[l * colstride + off_p];
      bn[l] = Yr[l * colstride + off_n];
    }
    if (r == 0) cp_async_wait_all();
#pragma unroll 1
    for (int k = 0; k < NC; ++k) {
      cpx<dd> ap{dd(0), dd(0)}, an{dd(0), dd(0)};
#pragma unroll
      for (int l = 0; l < NC; ++l) {
        const int lo = k < l ? k : l, hi = k < l ? l : k;
        const dd w = s_av[lo * NC - lo * (lo - 1) / 2 + (hi - lo)][threadIdx.x];
        madd_lazy(ap.x, w, bp[l].x);
        madd_lazy(ap.y, w, bp[l].y);
        madd_lazy(an.x, w, bn[l].x);
        madd_lazy(an.y, w, bn[l].y);
      }
      Zr[k * colstride + off_p] = {renorm_val(ap.x), renorm_val(ap.y)};
      if (n1 != 0) Zr[k * colstride + off_n] = {renorm_val(an.x), renorm_val(an.y)};
    }
  }
}

template <typename T, int NC>
void diag_dispatch(const DiagTArgs<T>& a, cudaStream_t st) {
  if constexpr (is_dd<T>::value && NC <= kDiagDDMaxC) {
    if (a.C == NC) {
      dim3 grid((unsigned)((a.M + kDiagThreads) / kDiagThreads), (unsigned)(a.M + 1));
      k_diag_t_dd<NC><<<grid, kDiagThreads, 0, st>>>(a);
      return;
    }
  }
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
// float-float row kernels also stage their pass tables (one 16-byte load a twiddle
// instead of a float-float complex product)
constexpr size_t kRowSmemMaxDD = size_t(215) << 10;
template <typename T>
constexpr size_t row_smem_max() { return is_dd<T>::value ? kRowSmemMaxDD : kRowSmemMax; }

template <typename T, int L, int RB>
void rows_launch(bool inv, const RowsArgs<T>& a, cudaStream_t st) {
  const size_t smem = inv ? row_smem<T, true>(L, RB) : row_smem<T, false>(L, RB);
  const int threads = RB * (1 << L) / 16;
  void (*k)(RowsArgs<T>) = inv ? k_rows_inv<T, L, RB> : k_rows_fwd<T, L, RB>;
  GPN_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  // one item per block: adjacent row groups run together, so the two halves of a
  // 32-byte sector of the transposed output meet in L2 (a persistent grid, tried,
  // spread them apart and raised DRAM traffic by a quarter)
  const long long grid = a.nitems;
  k<<<(unsigned)grid, threads, smem, st>>>(a);
}

// RB rows per CTA where the shared memory and the block size allow it (the same
// test as rows_per_block)
template <typename T, int L, int RB>
constexpr bool rows_fit() {
  return std::max(row_smem<T, false>(L, RB), row_smem<T, true>(L, RB)) <= row_smem_max<T>() &&
         RB * (1 << L) / 16 <= 1024;
}

template <typename T, int L>
void rows_rb(bool inv, int rb, const RowsArgs<T>& a, cudaStream_t st) {
  if constexpr (rows_fit<T, L, 2>()) {
    if (rb == 2) return rows_launch<T, L, 2>(inv, a, st);
  }
  rows_launch<T, L, 1>(inv, a, st);
}

template <typename T>
void rows(bool inv, int L, int rb, const RowsArgs<T>& a, cudaStream_t st) {
  switch (L) {
    case 4: rows_rb<T, 4>(inv, rb, a, st); break;
    case 5: rows_rb<T, 5>(inv, rb, a, st); break;
    case 6: rows_rb<T, 6>(inv, rb, a, st); break;
    case 7: rows_rb<T, 7>(inv, rb, a, st); break;
    case 8: rows_rb<T, 8>(inv, rb, a, st); break;
    case 9: rows_rb<T, 9>(inv, rb, a, st); break;
    case 10: rows_rb<T, 10>(inv, rb, a, st); break;
    case 11: rows_rb<T, 11>(inv, rb, a, st); break;
    case 12: rows_rb<T, 12>(inv, rb, a, st); break;
    default: rows_rb<T, 13>(inv, rb, a, st);
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
  RowsArgs<T> a = rows_args<T>(plan, X);
  if (plan.row_hi <= a.row0) return;
  a.npairs = (plan.row_hi - a.row0 + plan.t3_rb - 1) / plan.t3_rb;
  a.nitems = a.npairs * plan.geom.C * R;
  rows<T>(inv, log2_exact(plan.geom.nf / 2), plan.t3_rb, a, st);
  GPN_CUDA(cudaGetLastError());
}

#define GPN_CUFFT3(call)                                                                                \
  do {                                                                                                  \
    cufftResult r_ = (call);                                                                            \
    if (r_ != CUFFT_SUCCESS) ::gpn::fail(GP_ECUFFT, std::string(#call " failed: code ") + std::to_string((int)r_)); \
  } while (0)

}  // namespace

bool tr3_supported(int d, long long nf, int precision) {
  if (d != 2) return false;
  const int L = log2_exact(nf / 2);
  if (nf % 2 || L < kMinLog || L > kMaxLog) return false;
  if (precision == GP_DF64)   // the float-float column kernel holds a column of nf values
    return L + 1 >= 5 && L + 1 <= 13 && row_smem<dd, false>(L, 1) <= kRowSmemMaxDD &&
           cols_smem<dd>(L + 1) <= kRowSmemMaxDD;
  return (precision == GP_FP32 ? row_smem<float, false>(L, 1) : row_smem<double, false>(L, 1)) <= kRowSmemMax;
}

void tr3_setup(Plan& plan) {
  const long long nf = plan.geom.nf, N2 = nf / 2;
  const int L = log2_exact(N2);
  const bool f32 = plan.precision == GP_FP32, ddp = plan.precision == GP_DF64;
  const size_t sm2 = f32 ? row_smem<float, false>(L, 2) : (ddp ? row_smem<dd, false>(L, 2) : row_smem<double, false>(L, 2));
  const size_t smax = ddp ? kRowSmemMaxDD : kRowSmemMax;
  plan.t3_rb = (sm2 <= smax && 2 * (N2 / 16) <= 1024) ? 2 : 1;
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
  if (f32 || ddp) {
    const std::vector<double> pt = fft::pass_tables(L);
    w.insert(w.end(), pt.begin(), pt.end());
  }
  const size_t count = f32 ? tw_count<float, false>(L) : (ddp ? tw_count<dd, false>(L) : tw_count<double, false>(L));
  w.resize(2 * count, 0.0);  // padded to whole 16-byte chunks
  plan.tw_half = plan.alloc(w.size() * plan.real_size);
  auto upload_dd = [&](void* dst, const std::vector<double>& v) {
    std::vector<dd> f(v.size());
    for (size_t i = 0; i < v.size(); ++i) f[i] = dd(v[i]);
    GPN_CUDA(cudaMemcpy(dst, f.data(), f.size() * sizeof(dd), cudaMemcpyHostToDevice));
  };
  if (f32) {
    std::vector<float> f(w.begin(), w.end());
    GPN_CUDA(cudaMemcpy(plan.tw_half, f.data(), f.size() * sizeof(float), cudaMemcpyHostToDevice));
  } else if (ddp) {
    upload_dd(plan.tw_half, w);
    // the column transforms' pass tables (length nf), read from global memory
    const std::vector<double> ct = fft::pass_tables(L + 1);
    plan.col_tw = plan.alloc(std::max<size_t>(ct.size(), 2) * sizeof(dd));
    if (!ct.empty()) upload_dd(plan.col_tw, ct);
  } else {
    GPN_CUDA(cudaMemcpy(plan.tw_half, w.data(), w.size() * sizeof(double), cudaMemcpyHostToDevice));
  }
}

namespace {
// the column transforms of the float-float plans (cuFFT has no float-float type)
void cols_run_dd(Plan& plan, bool inv, const void* in, void* out, int R, cudaStream_t st) {
  ColsArgs<dd> a{};
  a.in = (const cpx<dd>*)in;
  a.out = (cpx<dd>*)out;
  a.ptab = (const cpx<dd>*)plan.col_tw;
  a.ncols = (long long)plan.geom.C * R * (plan.geom.M + 1);
  const int nf = (int)plan.geom.nf, M = (int)plan.geom.M;
  // the row groups of the inverse row kernel: [row0, row0 + npairs RB)
  const int row0 = plan.row_lo / plan.t3_rb * plan.t3_rb;
  const int rows_end = std::min(nf, row0 + (plan.row_hi - row0 + plan.t3_rb - 1) / plan.t3_rb * plan.t3_rb);
  if (!inv) {
    a.in_lo0 = plan.row_lo, a.in_hi0 = plan.row_hi, a.in_lo1 = 0, a.in_hi1 = 0;
    a.out_lo0 = 0, a.out_hi0 = M + 1, a.out_lo1 = nf - M, a.out_hi1 = nf;
  } else {
    a.in_lo0 = 0, a.in_hi0 = M + 1, a.in_lo1 = nf - M, a.in_hi1 = nf;
    a.out_lo0 = row0, a.out_hi0 = rows_end, a.out_lo1 = 0, a.out_hi1 = 0;
  }
  if (a.ncols == 0) return;
  cols<dd>(inv, log2_exact(nf), a, st);
  GPN_CUDA(cudaGetLastError());
}
}  // namespace

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
  if (plan.precision == GP_DF64) {
    rows_run<dd>(plan, false, plan.fx, R, st);
    prof_mark(plan, 0, st);
    cols_run_dd(plan, false, plan.fx, plan.fy, R, st);
    return;
  }
  cufftHandle h = plan.t3_plan(R);
  if (plan.precision == GP_FP32) {
    rows_run<float>(plan, false, plan.fx, R, st);
    prof_mark(plan, 0, st);
    GPN_CUFFT3(cufftSetStream(h, st));
    GPN_CUFFT3(cufftExecC2C(h, (cufftComplex*)plan.fx, (cufftComplex*)plan.fy, CUFFT_FORWARD));
  } else {
    rows_run<double>(plan, false, plan.fx, R, st);
    prof_mark(plan, 0, st);
    GPN_CUFFT3(cufftSetStream(h, st));
    GPN_CUFFT3(cufftExecZ2Z(h, (cufftDoubleComplex*)plan.fx, (cufftDoubleComplex*)plan.fy, CUFFT_FORWARD));
  }
}

void tr3_diag(Plan& plan, int R, cudaStream_t st) {
  if (plan.precision == GP_DF64) {
    DiagTArgs<dd> a{(const cpx<dd>*)plan.fy, (cpx<dd>*)plan.fz, (const dd*)plan.a_tensor, plan.geom.nf,
                    (int)plan.geom.M, plan.geom.C, R};
    diag_dispatch<dd, 1>(a, st);
  } else if (plan.precision == GP_FP32) {
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
  if (plan.precision == GP_DF64) {
    cols_run_dd(plan, true, plan.fz, plan.fy, R, st);
    prof_mark(plan, 1, st);
    rows_run<dd>(plan, true, plan.fy, R, st);
    return;
  }
  cufftHandle h = plan.t3_plan(R);
  GPN_CUFFT3(cufftSetStream(h, st));
  if (plan.precision == GP_FP32) {
    GPN_CUFFT3(cufftExecC2C(h, (cufftComplex*)plan.fz, (cufftComplex*)plan.fy, CUFFT_INVERSE));
    prof_mark(plan, 1, st);
    rows_run<float>(plan, true, plan.fy, R, st);
  } else {
    GPN_CUFFT3(cufftExecZ2Z(h, (cufftDoubleComplex*)plan.fz, (cufftDoubleComplex*)plan.fy, CUFFT_INVERSE));
    prof_mark(plan, 1, st);
    rows_run<double>(plan, true, plan.fy, R, st);
  }
}

}  // namespace gpn
