// Steps (1) + (2a) of Sec. 4.2: spread c_k,i = w_k(x_i) alpha_i onto the fine grids,
// for all Chebyshev channels k at once (the type-1 NUFFTs of step (2) share the
// spreading pass).
//
// Output-stationary tiling.  One CTA owns one tile of tile^d fine-grid cells for
// one right-hand side and accumulates, in shared memory, the contributions of
// every point whose support meets the tile: with points binned by the first cell
// of their support, those are the points of the 2^d bins at offsets {0,-1}^d,
// which form 2^(d-1) contiguous ranges of the sorted points.  For each batch of
// candidates the CTA keeps the points whose support actually meets the tile
// (compacted through a shared counter) and tabulates their kernel values per axis
// in shared memory; then a group of lanes works on each point: in 2-D one lane per
// support row (a "pencil" of `width` cells along the last axis), in 3-D the warp's
// lanes over the width^2 pencils, in 1-D one lane per point.  The tile is written
// once with coalesced stores.  Only tiles
// some point can reach are launched (the plan's active-tile list): the other
// cells of the spreading grid are zeroed once when the plan is built, and the
// forward R2C transform leaves its input untouched.  No global atomics; the
// shared tile of the FP32 path accumulates in int32 fixed point (see SpreadAcc).
// The shared tile's last dimension is padded to an odd pitch so that the rows a
// warp touches fall in different banks.
#include "kernels.h"

namespace gpn {

namespace {

constexpr int kBatch = 128;  // points staged per batch

template <typename T>
struct SpreadArgs {
  const int* cell0[kMaxDim];
  const T* xi[kMaxDim];
  const T* wk;
  const float* wabs;     // max_k |w_k(x_i)|
  const int* bin_start;
  const int* tiles;      // active tile ids
  int nbins[kMaxDim];
  const double* alpha;   // sorted order, N x R column-major
  long long n;
  T* grid;               // (R*C) x nf^d
  long long nf;
  long long G;           // nf^d
  int width;
  T beta;
  T inv_halfw;
  int tile;
  int pitch;             // padded extent of the last tile dimension in shared memory
  int C;                 // channels of one chunk (blockIdx.z = chunk)
  int Ctot;              // channels in total
  unsigned pmagic;       // ceil(2^24 / P): (g * pmagic) >> 24 == g / P for g < 2^24 / P
  unsigned wmagic;       // ceil(2^12 / width): (x * wmagic) >> 12 == x / width for x < 256
};

// Accumulator of the shared tile.  Float atomics on shared memory are emulated on
// sm_103 (compare-and-swap; measured 2.9 T/s and slowing with every address
// collision), and so are 64-bit integer atomics, while 32-bit integer atomics are
// native (8.2 T/s, collisions combined in hardware).  The FP32 path therefore
// accumulates in fixed point held as two int32 words per cell.  Each contribution
// v, already scaled by 2^e, is split with float arithmetic only:
//   hi = floor(v / 2^16)          (|hi| < 2^22, so hi is exact as a float)
//   lo = round(v - hi * 2^16)     (one FMA, exact; 0 <= lo <= 2^16)
// both converted to int32 by adding 1.5 * 2^23, which leaves round(x) in the low
// mantissa bits for |x| < 2^22, and the cell is sum(hi) * 2^16 + sum(lo).  e is
// chosen per tile so that S 2^e <= 2^38 with S = sum over the points reaching the
// tile of max_k |w_k| |alpha| (a bound on every cell since psi <= 1); the hi sums
// stay inside int32 and the lo sums below 2^31 for up to 32768 contributions per
// cell.  The resolution is S 2^-38, far below the float rounding of the products.  The FP64 path
// keeps float64 atomics (it is bound by its FFTs).
template <typename T>
struct SpreadAcc {
  using type = T;
};
template <>
struct SpreadAcc<float> {
  using type = int;  // two words per cell: hi block then lo block
};

template <typename T, int D, int CMAX>
__global__ void __launch_bounds__(256) k_spread(SpreadArgs<T> a) {
  using Acc = typename SpreadAcc<T>::type;
  constexpr bool kFixed = sizeof(Acc) == 4 && sizeof(T) == 4;
  constexpr int kWords = kFixed ? 2 : 1;  // accumulator words per cell and channel
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_count[2];
  __shared__ float s_red[8];
  const int ch0 = blockIdx.z * a.C;                 // first channel of this chunk
  const int TS = a.tile, TP = a.pitch, W = a.width, C = min(a.C, a.Ctot - ch0);
  int lead = 1;  // cells in the leading D-1 dimensions
#pragma unroll
  for (int q = 0; q < D - 1; ++q) lead *= TS;
  const int TV = lead * TP;  // padded tile volume
  const int PSTR = (D * W) | 1;  // odd stride of a point's kernel-value table
  Acc* tile = reinterpret_cast<Acc*>(smem_raw);           // [kWords][C][TV]
  T* s_psi = reinterpret_cast<T*>(tile + (size_t)kWords * C * TV);  // [kBatch][PSTR]: psi_q(j - xi_q), q-major
  T* s_wk = s_psi + (size_t)kBatch * PSTR;               // [C][kBatch]: w_k(x) alpha
  int* s_l0 = reinterpret_cast<int*>(s_wk + (size_t)C * kBatch);  // [D][kBatch]
  const int r = blockIdx.y;

  for (int i = threadIdx.x; i < kWords * C * TV; i += blockDim.x) tile[i] = Acc(0);
  if (threadIdx.x == 0) s_count[0] = 0;

  int tc[kMaxDim] = {0, 0, 0}, base[kMaxDim] = {0, 0, 0};
  {
    long long rest = a.tiles[blockIdx.x];
#pragma unroll
    for (int q = D - 1; q >= 0; --q) {
      tc[q] = (int)(rest % a.nbins[q]);
      rest /= a.nbins[q];
      base[q] = tc[q] * TS;
    }
  }
  // candidate ranges: bins (lead - o, last - 1 .. last) are consecutive in sorted order
  constexpr int NR = 1 << (D - 1);
  int rs[NR], rl[NR];
  int total = 0;
#pragma unroll
  for (int o = 0; o < NR; ++o) {
    long long lin = 0;
    bool valid = true;
#pragma unroll
    for (int q = 0; q < D - 1; ++q) {
      const int b = tc[q] - ((o >> q) & 1);
      valid = valid && b >= 0;
      lin = lin * a.nbins[q] + (b < 0 ? 0 : b);
    }
    const long long lin_hi = lin * a.nbins[D - 1] + tc[D - 1];
    const long long lin_lo = lin_hi - (tc[D - 1] > 0 ? 1 : 0);
    rs[o] = valid ? a.bin_start[lin_lo] : 0;
    rl[o] = valid ? a.bin_start[lin_hi + 1] - rs[o] : 0;
    total += rl[o];
  }
  int P = 1;  // pencils per point
#pragma unroll
  for (int q = 0; q < D - 1; ++q) P *= W;
  const double* alpha_r = a.alpha + (size_t)r * a.n;
  T scale = T(1), inv_scale = T(1);
  if (kFixed) {
    // tile bound S = sum over the candidates reaching the tile of max_k |w_k| |alpha|
    float part = 0.f;
    for (int i = threadIdx.x; i < total; i += blockDim.x) {
      int c = i, p = 0;
#pragma unroll
      for (int o = 0; o < NR; ++o) {
        if (c >= 0 && c < rl[o]) p = rs[o] + c;
        c -= rl[o];
      }
      bool meets = true;
#pragma unroll
      for (int q = 0; q < D; ++q) {
        const int l0 = a.cell0[q][p];
        meets = meets && l0 + W > base[q] && l0 < base[q] + TS;
      }
      if (meets) part += a.wabs[p] * (float)fabs(alpha_r[p]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = part;
    __syncthreads();
    float S = 0.f;
#pragma unroll
    for (int w = 0; w < 8; ++w) S += s_red[w];
    if (S > 0.f) {
      int ex;
      frexpf(S, &ex);          // S < 2^ex
      scale = ldexpf(1.f, 38 - ex);
      inv_scale = ldexpf(1.f, ex - 38);
    }
  }
  __syncthreads();

  int round = 0;
  for (int c0 = 0; c0 < total; c0 += kBatch, ++round) {
    const int par = round & 1;
    const int nc = min(kBatch, total - c0);
    // keep the candidates whose support meets this tile; their slot gets l0, the
    // kernel values along every axis and w_k(x) alpha
    for (int i = threadIdx.x; i < nc; i += blockDim.x) {
      int c = c0 + i, p = 0;
#pragma unroll
      for (int o = 0; o < NR; ++o) {
        if (c >= 0 && c < rl[o]) p = rs[o] + c;
        c -= rl[o];
      }
      int l0[kMaxDim];
      bool meets = true;
#pragma unroll
      for (int q = 0; q < D; ++q) {
        l0[q] = a.cell0[q][p];
        meets = meets && l0[q] + W > base[q] && l0[q] < base[q] + TS;
      }
      if (!meets) continue;
      const int slot = atomicAdd(&s_count[par], 1);
#pragma unroll
      for (int q = 0; q < D; ++q) s_l0[q * kBatch + slot] = l0[q];
      T* psi = s_psi + slot * PSTR;
#pragma unroll
      for (int q = 0; q < D; ++q) {
        const T xq = a.xi[q][p];
        for (int j = 0; j < W; ++j) psi[q * W + j] = es_psi<T>((T)j - xq, a.beta, a.inv_halfw);
      }
      const T amp = (T)alpha_r[p] * scale;
      const T* wkp = a.wk + (size_t)p * a.Ctot + ch0;
#pragma unroll
      for (int k = 0; k < CMAX; ++k)
        if (k < C) s_wk[k * kBatch + slot] = wkp[k] * amp;
    }
    if (threadIdx.x == 0) s_count[par ^ 1] = 0;  // the other counter is idle this round
    __syncthreads();
    const int nrel = s_count[par];
    // (slot, pencil) work items, spread evenly over the block
    const int items = nrel * P;
    for (int g = threadIdx.x; g < items; g += blockDim.x) {
      const int i = (int)(((unsigned long long)g * a.pmagic) >> 24);  // g / P
      int pen = g - i * P;
      const T* psi = s_psi + i * PSTR;
      int off = 0;
      bool inside = true;
      T amp = T(1);
      int iq[kMaxDim];
#pragma unroll
      for (int q = D - 2; q >= 0; --q) {
        const int qq = (int)(((unsigned)pen * a.wmagic) >> 12);  // pen / W
        iq[q] = pen - qq * W;
        pen = qq;
      }
#pragma unroll
      for (int q = 0; q < D - 1; ++q) {
        const int c = s_l0[q * kBatch + i] + iq[q] - base[q];
        inside = inside && c >= 0 && c < TS;
        off = off * TS + c;
        amp *= psi[q * W + iq[q]];
      }
      if (!inside) continue;
      const int l0 = s_l0[(D - 1) * kBatch + i];
      const int lo = max(0, base[D - 1] - l0), hi = min(W, base[D - 1] + TS - l0);
      T wk[CMAX];
#pragma unroll
      for (int k = 0; k < CMAX; ++k) wk[k] = k < C ? s_wk[k * kBatch + i] * amp : T(0);
      const T* plast = psi + (D - 1) * W;
      Acc* rowp = tile + off * TP + (l0 - base[D - 1]);
      for (int c = lo; c < hi; ++c) {
        const T ps = plast[c];
#pragma unroll
        for (int k = 0; k < CMAX; ++k) {
          if (k < C) {
            if constexpr (kFixed) {
              const float v = ps * wk[k];
              const float hf = floorf(v * (1.f / 65536.f));
              const float lf = fmaf(-hf, 65536.f, v);
              const int hi = __float_as_int(hf + 12582912.f) - 0x4B400000;
              const int lo = __float_as_int(lf + 12582912.f) - 0x4B400000;
              atomicAdd(rowp + c + (size_t)k * TV, hi);
              atomicAdd(rowp + c + (size_t)(C + k) * TV, lo);
            } else
              atomicAdd(rowp + c + (size_t)k * TV, ps * wk[k]);
          }
        }
      }
    }
    __syncthreads();  // slots are reused by the next round
  }

  // write the tile once (cells past nf in a partial last tile are dropped)
  const int vol = lead * TS;
  for (int i = threadIdx.x; i < vol; i += blockDim.x) {
    int rem = i;
    long long gidx = 0, gstride = 1;
    int sidx = 0, sstride = 1;
    bool in = true;
#pragma unroll
    for (int q = D - 1; q >= 0; --q) {
      const int c = rem % TS;
      rem /= TS;
      const long long gq = (long long)base[q] + c;
      in = in && gq < a.nf;
      gidx += gq * gstride;
      gstride *= a.nf;
      sidx += c * sstride;
      sstride *= (q == D - 1) ? TP : TS;
    }
    if (!in) continue;
    T* dst = a.grid + ((size_t)r * a.Ctot + ch0) * a.G + gidx;
#pragma unroll
    for (int k = 0; k < CMAX; ++k) {
      if (k < C) {
        if constexpr (kFixed) {
          const long long v = ((long long)tile[(size_t)k * TV + sidx] << 16) + tile[(size_t)(C + k) * TV + sidx];
          dst[(size_t)k * a.G] = __ll2float_rn(v) * inv_scale;
        } else {
          dst[(size_t)k * a.G] = tile[(size_t)k * TV + sidx];
        }
      }
    }
  }
}

template <typename T, int D, int CMAX>
void launch(const SpreadArgs<T>& a, dim3 grid, size_t smem, cudaStream_t st) {
  GPN_CUDA(cudaFuncSetAttribute(k_spread<T, D, CMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_spread<T, D, CMAX><<<grid, 256, smem, st>>>(a);
}

template <typename T, int D>
void launch_c(const SpreadArgs<T>& a, dim3 grid, size_t smem, cudaStream_t st) {
  switch (cmax_bucket(a.C)) {
    case 8: launch<T, D, 8>(a, grid, smem, st); break;
    case 12: launch<T, D, 12>(a, grid, smem, st); break;
    case 16: launch<T, D, 16>(a, grid, smem, st); break;
    default: launch<T, D, 32>(a, grid, smem, st);
  }
}

template <typename T>
void spread_impl(Plan& plan, const double* alpha_sorted, int R, cudaStream_t st) {
  const GridGeom& g = plan.geom;
  const PointSet& ps = plan.pts;
  if (plan.n_active_tiles == 0) return;
  SpreadArgs<T> a{};
  for (int q = 0; q < kMaxDim; ++q) {
    a.cell0[q] = ps.cell0[q];
    a.xi[q] = (const T*)ps.xi[q];
    a.nbins[q] = ps.nbins[q];
  }
  a.wk = (const T*)ps.wk;
  a.wabs = ps.wabs;
  a.bin_start = ps.bin_start;
  a.tiles = plan.active_tiles;
  a.alpha = alpha_sorted;
  a.n = ps.n;
  a.grid = (T*)plan.grid;
  a.nf = g.nf;
  a.G = plan.grid_elems;
  a.width = g.width;
  a.beta = es_beta_arg<T>(g.beta);
  a.inv_halfw = (T)(2.0 / g.width);
  a.tile = g.tile;
  a.pitch = spread_pitch(g.d, g.tile);
  // channels per launch chunk: all of them when the shared tile fits, else fewer
  int cc = g.C;
  while (cc > 1 && spread_smem_bytes(g.d, g.tile, cc, sizeof(T), g.width) > kSpreadSmemMax) --cc;
  GPN_CHECK(spread_smem_bytes(g.d, g.tile, cc, sizeof(T), g.width) <= kSpreadSmemMax, GP_EUNSUPPORTED,
            "spreading tile does not fit in shared memory");
  a.C = cc;
  a.Ctot = g.C;
  {
    unsigned P = 1;
    for (int q = 0; q < g.d - 1; ++q) P *= (unsigned)g.width;
    a.pmagic = (unsigned)(((1ull << 24) + P - 1) / P);
    a.wmagic = (unsigned)(((1u << 12) + g.width - 1) / g.width);
  }
  size_t smem = spread_smem_bytes(g.d, g.tile, cc, sizeof(T), g.width);
  dim3 grid((unsigned)plan.n_active_tiles, (unsigned)R, (unsigned)((g.C + cc - 1) / cc));
  switch (g.d) {
    case 1: launch_c<T, 1>(a, grid, smem, st); break;
    case 2: launch_c<T, 2>(a, grid, smem, st); break;
    default: launch_c<T, 3>(a, grid, smem, st);
  }
  GPN_CUDA(cudaGetLastError());
}

}  // namespace

// d = 1 in FP64 with fewer active tiles than SMs (short point sets): the tiled kernel
// would run a handful of CTAs, and float64 shared-memory atomics are emulated on sm_103.
// Instead one thread per point evaluates its W kernel values once and adds every
// (cell, channel) contribution with a native float64 atomic in L2 to the zeroed grid.
// The summation order varies from run to run at the level of float64 rounding.
__global__ void __launch_bounds__(128) k_spread1d_atomic(const int* __restrict__ cell0,
                                                         const double* __restrict__ xi,
                                                         const double* __restrict__ wk,
                                                         const double* __restrict__ alpha, long long n, double* grid,
                                                         long long G, int W, double beta, double inv_halfw, int C) {
  const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const int r = blockIdx.y;
  if (p >= n) return;
  double psi[kMaxWidth];
  const double x = xi[p];
#pragma unroll
  for (int c = 0; c < kMaxWidth; ++c) psi[c] = c < W ? es_psi<double>((double)c - x, beta, inv_halfw) : 0.0;
  const double amp = alpha[(size_t)r * n + p];
  double* g = grid + (size_t)r * C * G + cell0[p];
  for (int k = 0; k < C; ++k) {
    const double v = wk[(size_t)p * C + k] * amp;
    double* gk = g + (size_t)k * G;
#pragma unroll
    for (int c = 0; c < kMaxWidth; ++c)
      if (c < W) atomicAdd(gk + c, psi[c] * v);
  }
}

int spread_pitch(int d, int tile) { return d == 1 ? tile : tile + 1; }

size_t spread_smem_bytes(int d, int tile, int C, size_t rs, int width) {
  size_t lead = 1;
  for (int q = 0; q < d - 1; ++q) lead *= tile;
  size_t tilev = lead * spread_pitch(d, tile) * (size_t)C * 8;  // two int32 words (FP32) or one double
  size_t batch = (size_t)kBatch * ((((size_t)d * width) | 1) * rs + C * rs + d * sizeof(int));
  return tilev + batch;
}

void launch_spread(Plan& plan, const double* alpha_sorted, int R, cudaStream_t st) {
  if (plan.sp2_tiles) return launch_spread2d(plan, alpha_sorted, R, st);
  const GridGeom& g = plan.geom;
  if (g.d == 1 && plan.precision == GP_FP64 && plan.n_active_tiles < 152) {
    const PointSet& ps = plan.pts;
    GPN_CUDA(cudaMemsetAsync(plan.grid, 0, sizeof(double) * (size_t)g.C * R * plan.grid_elems, st));
    if (ps.n == 0) return;
    dim3 grid((unsigned)((ps.n + 127) / 128), (unsigned)R);
    k_spread1d_atomic<<<grid, 128, 0, st>>>(ps.cell0[0], (const double*)ps.xi[0], (const double*)ps.wk, alpha_sorted,
                                            ps.n, (double*)plan.grid, plan.grid_elems, g.width, g.beta,
                                            2.0 / g.width, g.C);
    GPN_CUDA(cudaGetLastError());
    return;
  }
  if (plan.precision == GP_FP32)
    spread_impl<float>(plan, alpha_sorted, R, st);
  else
    spread_impl<double>(plan, alpha_sorted, R, st);
}

}  // namespace gpn
