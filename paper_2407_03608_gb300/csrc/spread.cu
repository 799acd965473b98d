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
// forward R2C transform leaves its input untouched.  No global atomics.
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
  int C;
};

template <typename T, int D, int CMAX>
__global__ void __launch_bounds__(256) k_spread(SpreadArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_count;
  const int TS = a.tile, TP = a.pitch, W = a.width, C = a.C;
  int lead = 1;  // cells in the leading D-1 dimensions
#pragma unroll
  for (int q = 0; q < D - 1; ++q) lead *= TS;
  const int TV = lead * TP;  // padded tile volume
  const int PSTR = (D * W) | 1;  // odd stride of a point's kernel-value table
  T* tile = reinterpret_cast<T*>(smem_raw);
  T* s_psi = tile + (size_t)C * TV;                      // [kBatch][PSTR]: psi_q(j - xi_q), q-major
  T* s_amp = s_psi + (size_t)kBatch * PSTR;              // [kBatch] alpha of the point
  T* s_wk = s_amp + kBatch;                              // [C][kBatch]
  int* s_l0 = reinterpret_cast<int*>(s_wk + (size_t)C * kBatch);  // [D][kBatch]
  int* s_pid = s_l0 + D * kBatch;                        // [kBatch] sorted point index
  const int r = blockIdx.y;

  for (int i = threadIdx.x; i < C * TV; i += blockDim.x) tile[i] = T(0);

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
  // lane groups: one point per group; in 2-D a lane is a support row, in 3-D the
  // warp's lanes run over the width^2 pencils, in 1-D a lane is a whole point
  constexpr int kGroup = D == 1 ? 1 : (D == 2 ? 0 : 32);
  const int Gs = kGroup == 0 ? W : kGroup;
  const int ppw = 32 / Gs;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int grp = lane / Gs, gl = lane - grp * Gs;
  int P = 1;  // pencils per point
#pragma unroll
  for (int q = 0; q < D - 1; ++q) P *= W;
  const double* alpha_r = a.alpha + (size_t)r * a.n;

#pragma unroll 1
  for (int o = 0; o < (1 << (D - 1)); ++o) {
    // bins (lead - o, last - 1 .. last) are consecutive in the sorted order
    long long lin = 0;
    bool valid = true;
#pragma unroll
    for (int q = 0; q < D - 1; ++q) {
      int b = tc[q] - ((o >> q) & 1);
      valid = valid && b >= 0;
      lin = lin * a.nbins[q] + (b < 0 ? 0 : b);
    }
    if (!valid) continue;
    const long long lin_hi = lin * a.nbins[D - 1] + tc[D - 1];
    const long long lin_lo = lin_hi - (tc[D - 1] > 0 ? 1 : 0);
    const int r0 = a.bin_start[lin_lo], r1 = a.bin_start[lin_hi + 1];
    for (int b0 = r0; b0 < r1; b0 += kBatch) {
      const int nb = min(kBatch, r1 - b0);
      __syncthreads();  // previous batch consumed (and the tile zeroed)
      if (threadIdx.x == 0) s_count = 0;
      __syncthreads();
      // keep only the candidates whose support meets this tile
      for (int i = threadIdx.x; i < nb; i += blockDim.x) {
        const int p = b0 + i;
        int l0[kMaxDim];
        bool meets = true;
#pragma unroll
        for (int q = 0; q < D; ++q) {
          l0[q] = a.cell0[q][p];
          meets = meets && l0[q] + W > base[q] && l0[q] < base[q] + TS;
        }
        if (meets) {
          const int slot = atomicAdd(&s_count, 1);
#pragma unroll
          for (int q = 0; q < D; ++q) s_l0[q * kBatch + slot] = l0[q];
          s_pid[slot] = p;
          s_amp[slot] = (T)alpha_r[p];
        }
      }
      __syncthreads();
      const int nrel = s_count;
      for (int slot = threadIdx.x; slot < nrel; slot += blockDim.x) {
        const int p = s_pid[slot];
        const T* wkp = a.wk + (size_t)p * C;
#pragma unroll
        for (int k = 0; k < CMAX; ++k)
          if (k < C) s_wk[k * kBatch + slot] = wkp[k];
        T* psi = s_psi + slot * PSTR;
#pragma unroll
        for (int q = 0; q < D; ++q) {
          const T xq = a.xi[q][p];
          for (int j = 0; j < W; ++j) psi[q * W + j] = es_psi<T>((T)j - xq, a.beta, a.inv_halfw);
        }
      }
      __syncthreads();
      for (int pb = warp * ppw; pb < nrel; pb += nwarps * ppw) {
        const int i = pb + grp;
        if (grp >= ppw || i >= nrel) continue;
        const T* psi = s_psi + i * PSTR;
        const int l0 = s_l0[(D - 1) * kBatch + i];
        const int lo = max(0, base[D - 1] - l0), hi = min(W, base[D - 1] + TS - l0);
        T wk[CMAX];
#pragma unroll
        for (int k = 0; k < CMAX; ++k) wk[k] = k < C ? s_wk[k * kBatch + i] * s_amp[i] : T(0);
        for (int pen = gl; pen < P; pen += Gs) {
          int rem = pen, off = 0;
          bool inside = true;
          T amp = T(1);
          int iq[kMaxDim];
#pragma unroll
          for (int q = D - 2; q >= 0; --q) {
            iq[q] = rem % W;
            rem /= W;
          }
#pragma unroll
          for (int q = 0; q < D - 1; ++q) {
            const int c = s_l0[q * kBatch + i] + iq[q] - base[q];
            inside = inside && c >= 0 && c < TS;
            off = off * TS + c;
            amp *= psi[q * W + iq[q]];
          }
          if (!inside) continue;
          const T* plast = psi + (D - 1) * W;
          T* rowp = tile + off * TP + (l0 - base[D - 1]);
          for (int c = lo; c < hi; ++c) {
            const T ps = amp * plast[c];
#pragma unroll
            for (int k = 0; k < CMAX; ++k)
              if (k < C) atomicAdd(rowp + c + (size_t)k * TV, ps * wk[k]);
          }
        }
      }
    }
  }
  __syncthreads();

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
    T* dst = a.grid + (size_t)r * C * a.G + gidx;
#pragma unroll
    for (int k = 0; k < CMAX; ++k)
      if (k < C) dst[(size_t)k * a.G] = tile[(size_t)k * TV + sidx];
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
  a.C = g.C;
  size_t smem = spread_smem_bytes(g.d, g.tile, g.C, sizeof(T), g.width);
  dim3 grid((unsigned)plan.n_active_tiles, (unsigned)R);
  switch (g.d) {
    case 1: launch_c<T, 1>(a, grid, smem, st); break;
    case 2: launch_c<T, 2>(a, grid, smem, st); break;
    default: launch_c<T, 3>(a, grid, smem, st);
  }
  GPN_CUDA(cudaGetLastError());
}

}  // namespace

int spread_pitch(int d, int tile) { return d == 1 ? tile : tile + 1; }

size_t spread_smem_bytes(int d, int tile, int C, size_t rs, int width) {
  size_t lead = 1;
  for (int q = 0; q < d - 1; ++q) lead *= tile;
  size_t tilev = lead * spread_pitch(d, tile) * (size_t)C * rs;
  size_t batch = (size_t)kBatch * ((((size_t)d * width) | 1) * rs + (1 + C) * rs + (d + 1) * sizeof(int));
  return tilev + batch;
}

void launch_spread(Plan& plan, const double* alpha_sorted, int R, cudaStream_t st) {
  if (plan.precision == GP_FP32)
    spread_impl<float>(plan, alpha_sorted, R, st);
  else
    spread_impl<double>(plan, alpha_sorted, R, st);
}

}  // namespace gpn
