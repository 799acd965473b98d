// Steps (1) + (2a) of Sec. 4.2 in two dimensions: spread c_k,i = w_k(x_i) alpha_i onto
// the fine grids of all Chebyshev channels k at once, accumulating in registers.
//
// Output-stationary tiles of 32 columns (last axis) by TY = 8 * RPW rows.  Warp w of
// the CTA owns the band of rows w*RPW .. w*RPW + RPW - 1; its lanes form four groups
// of eight, and group g owns the strip of columns 8g .. 8g + 7.  Each lane keeps the
// RPW x C sums of its column in registers.  A point's support (width <= 16 cells per
// axis) meets a few (band, strip) pairs of the tile; the CTA builds, for every pair,
// the ordered list of the points that meet it, so that each group walks only its own
// list and the four groups of a warp spread four different points per instruction.
//
// Per round the CTA scans up to 256 points of the bins that can reach the tile (one
// per thread), keeps those whose support meets the tile in sorted order, tabulates
// their kernel values psi(j - xi) per axis and their w_k alpha in shared memory, and
// fills the 32 lists with ballots (the order, and so the FP32 summation order, is
// fixed: results are reproducible bit for bit).  No atomics and no shared
// accumulator: every grid value is one register sum, written once with 128-byte
// coalesced stores.  Tiles whose candidate bins are empty are never launched; their
// cells stay zero from plan creation on.
#include <algorithm>
#include <type_traits>

#include "fft_core.h"
#include "kernels.h"

namespace gpn {

namespace {

constexpr int kStrip = 8;                    // columns per lane group
constexpr int kGroups = 4;                   // lane groups per warp
constexpr int kTX = kStrip * kGroups;        // tile columns
constexpr int kWarps = 8;
constexpr int kLists = kWarps * kGroups;     // (band, strip) lists
constexpr int kSlots = 256;                  // candidates scanned per round (one per thread)
constexpr int kMaxRanges = 8;                // bin rows a tile's candidates can come from
constexpr int kMaxW = 16;                    // widest kernel support the tables hold

// Per-slot shared tables, strides odd against bank conflicts: the x table holds
// psi(j - xi) for j < W; the row table holds psi(j - xi) at j + RPW - 1 with zeros around,
// so a band row just outside the support reads zero without a test.
__host__ __device__ constexpr int col_stride(int w) { return w | 1; }
__host__ __device__ constexpr int row_stride(int w, int rpw) { return (w + 2 * (rpw - 1)) | 1; }
// w_k alpha of a slot: NC channels padded to whole 16-byte vectors
template <typename T>
__host__ __device__ constexpr int wk_pitch(int nc) { return (nc + (int)(16 / sizeof(T)) - 1) / (int)(16 / sizeof(T)) * (int)(16 / sizeof(T)); }

template <typename T>
struct Spread2Args {
  const int* l0y;        // first support cell along the first axis (sorted order)
  const int* l0x;        // ... along the last axis
  const T* xiy;
  const T* xix;
  const T* wk;           // [n][C]
  const T* psy;          // tabulated kernel values [n][width] per axis (null: evaluate)
  const T* psx;
  const int* bin_start;
  const int* tiles;      // active tile ids, ty * ntx + tx
  int ntx;
  int nby, nbx;          // bins per axis
  int bt;                // bin edge in cells
  const double* alpha;   // sorted order, n x R column-major
  long long n;
  T* grid;               // (R*C) x nf^2
  long long nf;
  long long G;
  int width;
  T beta;
  T inv_halfw;
  int C;
};

// NC: channels held in registers (C itself up to 16, else 32 with the extra ones zero).
template <typename T, int NC, int RPW>
__global__ void __launch_bounds__(256) k_spread2d(Spread2Args<T> a) {
  constexpr int TY = kWarps * RPW;
  constexpr int WP = wk_pitch<T>(NC);
  constexpr int VW = (int)(16 / sizeof(T));
  // 16-byte vector of VW values: four floats, two doubles or two float-float values
  using V = typename std::conditional<sizeof(T) == 4, float4,
                                      typename std::conditional<is_dd<T>::value, fft::cpx<dd>, double2>::type>::type;
  const int PSX = col_stride(a.width), SY = row_stride(a.width, RPW);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* s_wk = reinterpret_cast<T*>(smem_raw);                      // [kSlots][WP]
  int2* s_l0 = reinterpret_cast<int2*>(s_wk + kSlots * WP);      // [kSlots]: (l0y, l0x)
  T* s_psx = reinterpret_cast<T*>(s_l0 + kSlots);                // [kSlots][PSX]
  T* s_psy = s_psx + kSlots * PSX;                               // [kSlots][SY]
  unsigned char* s_list = reinterpret_cast<unsigned char*>(s_psy + kSlots * SY);  // [kLists][kSlots]
  __shared__ int s_rs[kMaxRanges], s_rl[kMaxRanges], s_wcnt[kWarps];
  __shared__ int s_cnt[kLists][kWarps], s_len[kLists];

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int tile = a.tiles[blockIdx.x];
  const int ty = tile / a.ntx, tx = tile - ty * a.ntx;
  const int y0 = ty * TY, x0 = tx * kTX;
  const int W = a.width, C = a.C, r = blockIdx.y;

  // candidates: points with l0y in [y0 - W + 1, y0 + TY - 1] and l0x in
  // [x0 - W + 1, x0 + kTX - 1]; per bin row one contiguous run of sorted points
  const int ylo = y0 - W + 1, xlo = x0 - W + 1;
  const int by0 = ylo < 0 ? 0 : ylo / a.bt, by1 = min(a.nby - 1, (y0 + TY - 1) / a.bt);
  const int bx0 = xlo < 0 ? 0 : xlo / a.bt, bx1 = min(a.nbx - 1, (x0 + kTX - 1) / a.bt);
  const int nr = min(kMaxRanges, by1 - by0 + 1);
  if (tid < nr) {
    const long long row = (long long)(by0 + tid) * a.nbx;
    const int lo = a.bin_start[row + bx0];
    s_rs[tid] = lo;
    s_rl[tid] = a.bin_start[row + bx1 + 1] - lo;
  }
  __syncthreads();
  int total = 0;
  for (int q = 0; q < nr; ++q) total += s_rl[q];

  T acc[RPW][NC];
#pragma unroll
  for (int rr = 0; rr < RPW; ++rr)
#pragma unroll
    for (int k = 0; k < NC; ++k) acc[rr][k] = T(0);
  const int grp = lane >> 3;
  const int xg = x0 + grp * kStrip + (lane & 7);  // this lane's column
  const int rw0 = y0 + warp * RPW;                 // the warp's first row
  const int my_list = warp * kGroups + grp;
  const unsigned lt = (1u << lane) - 1u;
  const double* alpha_r = a.alpha + (size_t)r * a.n;

  for (int c0 = 0; c0 < total; c0 += kSlots) {
    // scan: one candidate per thread; the ones meeting the tile are compacted in order
    const int c = c0 + tid;
    int p = 0, l0y = 0, l0x = 0;
    bool meets = false;
    if (c < total) {
      int cc = c;
      for (int q = 0; q < nr; ++q) {
        if (cc < s_rl[q]) {
          p = s_rs[q] + cc;
          break;
        }
        cc -= s_rl[q];
      }
      l0y = a.l0y[p];
      l0x = a.l0x[p];
      meets = l0y + W > y0 && l0y < y0 + TY && l0x + W > x0 && l0x < x0 + kTX;
    }
    const unsigned bal = __ballot_sync(0xffffffffu, meets);
    if (lane == 0) s_wcnt[warp] = __popc(bal);
    // the (band, strip) pairs the support meets, as a bit mask over the lists
    unsigned mask = 0u;
    if (meets) {
      const int b0 = l0y <= y0 ? 0 : (l0y - y0) / RPW, b1 = min(kWarps - 1, (l0y + W - 1 - y0) / RPW);
      const int s0 = l0x <= x0 ? 0 : (l0x - x0) / kStrip, s1 = min(kGroups - 1, (l0x + W - 1 - x0) / kStrip);
      const unsigned smask = ((1u << (s1 + 1)) - 1u) & ~((1u << s0) - 1u);
      for (int b = b0; b <= b1; ++b) mask |= smask << (b * kGroups);
    }
#pragma unroll
    for (int L = 0; L < kLists; ++L) {
      const unsigned bl = __ballot_sync(0xffffffffu, (mask >> L) & 1u);
      if (lane == 0) s_cnt[L][warp] = __popc(bl);
    }
    __syncthreads();
    int off = 0, nrel = 0;
#pragma unroll
    for (int q = 0; q < kWarps; ++q) {
      const int v = s_wcnt[q];
      off += q < warp ? v : 0;
      nrel += v;
    }
    // exclusive prefix over warps of every list count: warp w scans lists 4w .. 4w + 3
    {
      const int L = warp * kGroups + (lane >> 3), q = lane & 7;
      const int v = s_cnt[L][q];
      int inc = v;
#pragma unroll
      for (int o = 1; o < 8; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, inc, o, 8);
        if (q >= o) inc += u;
      }
      __syncwarp();
      s_cnt[L][q] = inc - v;
      if (q == 7) s_len[L] = inc;
    }
    const int slot = off + __popc(bal & lt);
    if (meets) {
      s_l0[slot] = make_int2(l0y, l0x);
      const T yq = a.xiy[p], xq = a.xix[p];
      T* py = s_psy + slot * SY;
      T* px = s_psx + slot * PSX;
      if (a.psx) {
        const T* tx = a.psx + (size_t)p * W;
        const T* ty = a.psy + (size_t)p * W;
        for (int j = 0; j < W; ++j) px[j] = tx[j];
        for (int j = 0; j < SY; ++j) {
          const int jj = j - (RPW - 1);
          py[j] = (jj >= 0 && jj < W) ? ty[jj] : T(0);
        }
      } else {
        for (int j = 0; j < W; ++j) px[j] = psi_at<T>(j, xq, a.beta, a.inv_halfw);
        for (int j = 0; j < SY; ++j) {
          const int jj = j - (RPW - 1);
          py[j] = (jj >= 0 && jj < W) ? psi_at<T>(jj, yq, a.beta, a.inv_halfw) : T(0);
        }
      }
      const T amp = (T)alpha_r[p];
      const T* wkp = a.wk + (size_t)p * C;
#pragma unroll
      for (int k = 0; k < WP; ++k) s_wk[slot * WP + k] = k < C ? wkp[k] * amp : T(0);
    }
    __syncthreads();
    // fill the lists in candidate order
#pragma unroll
    for (int L = 0; L < kLists; ++L) {
      const unsigned hit = (mask >> L) & 1u;
      const unsigned bl = __ballot_sync(0xffffffffu, hit);
      if (hit) s_list[L * kSlots + s_cnt[L][warp] + __popc(bl & lt)] = (unsigned char)slot;
    }
    __syncthreads();
    // accumulate: group g walks the list of (its warp's band, strip g)
    const int len = s_len[my_list];
    int steps = 0;
#pragma unroll
    for (int q = 0; q < kGroups; ++q) steps = max(steps, s_len[warp * kGroups + q]);
    const unsigned char* lst = s_list + my_list * kSlots;
    for (int j = 0; j < steps; ++j) {
      const bool valid = j < len;
      const int is = valid ? lst[j] : 0;   // slot 0 exists whenever some list is non-empty
      const int2 l0 = s_l0[is];
      const int dyo = valid ? rw0 - l0.x : 0;   // in [1 - RPW, W - 1] for list members
      const int dx = xg - l0.y;
      const T px = (valid && (unsigned)dx < (unsigned)W) ? s_psx[is * PSX + dx] : T(0);
      T wk[WP];
#pragma unroll
      for (int v = 0; v < WP / VW; ++v) {
        const V u = reinterpret_cast<const V*>(s_wk + is * WP)[v];
        if constexpr (VW == 4) {
          wk[4 * v] = u.x;
          wk[4 * v + 1] = u.y;
          wk[4 * v + 2] = u.z;
          wk[4 * v + 3] = u.w;
        } else {
          wk[2 * v] = u.x;
          wk[2 * v + 1] = u.y;
        }
      }
      const T* pyr = s_psy + is * SY + (RPW - 1) + dyo;
#pragma unroll
      for (int rr = 0; rr < RPW; ++rr) {
        const T v = px * pyr[rr];
#pragma unroll
        for (int k = 0; k < NC; ++k) madd_lazy(acc[rr][k], v, wk[k]);
      }
      if constexpr (is_dd<T>::value) {
        // float-float sums: renormalise every eight points (the low word then stays within a
        // few ulps of the high one)
        if ((j & 7) == 7) {
#pragma unroll
          for (int rr = 0; rr < RPW; ++rr)
#pragma unroll
            for (int k = 0; k < NC; ++k) acc[rr][k] = renorm_val(acc[rr][k]);
        }
      }
    }
    if constexpr (is_dd<T>::value) {
#pragma unroll
      for (int rr = 0; rr < RPW; ++rr)
#pragma unroll
        for (int k = 0; k < NC; ++k) acc[rr][k] = renorm_val(acc[rr][k]);
    }
    __syncthreads();  // slots, lists and counters are refilled by the next round
  }

  // every lane holds the complete sums of its column over the warp's rows
  if (xg >= a.nf) return;
  T* gr = a.grid + (size_t)r * C * a.G + xg;
#pragma unroll
  for (int rr = 0; rr < RPW; ++rr) {
    const long long row = rw0 + rr;
    if (row < a.nf) {
#pragma unroll
      for (int k = 0; k < NC; ++k)
        if (k < C) gr[(size_t)k * a.G + row * a.nf] = acc[rr][k];
    }
  }
}

// channels held in registers: C itself up to 16, else 32
constexpr int reg_channels(int C) { return C <= 16 ? C : 32; }

template <typename T>
constexpr int rows_per_warp(int nc) {
  // float64 and float-float sums take two registers each: two rows a warp (four rows of
  // float-float sums held 156 registers at 9 channels, one CTA an SM, and the spread ran
  // 4.29 ms at the 2-D benchmark size against 3.14 ms with two rows and 80 registers);
  // FP32 keeps four
  return (sizeof(T) == 8 || nc > 16) ? 2 : 4;
}

size_t smem_bytes(size_t rs, int nc, int rpw, int w) {
  const int wp = rs == 4 ? wk_pitch<float>(nc) : wk_pitch<double>(nc);
  return (size_t)kSlots * ((col_stride(w) + row_stride(w, rpw)) * rs + wp * rs + sizeof(int2) + kLists);
}

template <typename T, int NC>
void launch(const Spread2Args<T>& a, dim3 grid, cudaStream_t st) {
  constexpr int RPW = rows_per_warp<T>(NC);
  const size_t smem = smem_bytes(sizeof(T), NC, RPW, a.width);
  GPN_CUDA(cudaFuncSetAttribute(k_spread2d<T, NC, RPW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_spread2d<T, NC, RPW><<<grid, kWarps * 32, smem, st>>>(a);
}

template <typename T, int NC>
void dispatch(const Spread2Args<T>& a, dim3 grid, cudaStream_t st) {
  if constexpr (NC > 16) {
    launch<T, 32>(a, grid, st);
  } else {
    if (a.C == NC)
      launch<T, NC>(a, grid, st);
    else
      dispatch<T, NC + 1>(a, grid, st);
  }
}

template <typename T>
void impl(Plan& plan, const double* alpha_sorted, int R, cudaStream_t st) {
  if (plan.n_sp2_tiles == 0) return;
  const GridGeom& g = plan.geom;
  const PointSet& ps = plan.pts;
  Spread2Args<T> a{};
  a.l0y = ps.cell0[0];
  a.l0x = ps.cell0[1];
  a.xiy = (const T*)ps.xi[0];
  a.xix = (const T*)ps.xi[1];
  a.psy = (const T*)ps.psi[0];
  a.psx = (const T*)ps.psi[1];
  a.wk = (const T*)ps.wk;
  a.bin_start = ps.bin_start;
  a.tiles = plan.sp2_tiles;
  a.ntx = (int)((g.nf + kTX - 1) / kTX);
  a.nby = ps.nbins[0];
  a.nbx = ps.nbins[1];
  a.bt = g.tile;
  a.alpha = alpha_sorted;
  a.n = ps.n;
  a.grid = (T*)plan.grid;
  a.nf = g.nf;
  a.G = plan.grid_elems;
  a.width = g.width;
  a.beta = es_beta_arg<T>(g.beta);
  a.inv_halfw = (T)(2.0 / g.width);
  a.C = g.C;
  dim3 grid((unsigned)plan.n_sp2_tiles, (unsigned)R);
  dispatch<T, 1>(a, grid, st);
  GPN_CUDA(cudaGetLastError());
}

}  // namespace

int spread2d_rows(const Plan& plan) {
  const int nc = reg_channels(plan.geom.C);
  const int rpw = plan.precision == GP_FP32   ? rows_per_warp<float>(nc)
                  : plan.precision == GP_DF64 ? rows_per_warp<dd>(nc)
                                              : rows_per_warp<double>(nc);
  return kWarps * rpw;
}

bool spread2d_supported(const Plan& plan) {
  const GridGeom& g = plan.geom;
  if (g.d != 2 || g.width > kMaxW || g.C > kMaxChannels) return false;
  const int TY = spread2d_rows(plan);
  const int bin_rows = (TY + g.width - 2) / g.tile + 2;
  const int nc = reg_channels(g.C);
  return bin_rows <= kMaxRanges && smem_bytes(plan.real_size, nc, TY / kWarps, g.width) <= 200 * 1024;
}

// Tiles whose candidate bins hold at least one point; the others stay zero.
void build_spread2d_tiles(Plan& plan, const std::vector<int>& bstart) {
  const GridGeom& g = plan.geom;
  const PointSet& ps = plan.pts;
  const int TY = spread2d_rows(plan), W = g.width, bt = g.tile;
  const int nty = (int)((g.nf + TY - 1) / TY), ntx = (int)((g.nf + kTX - 1) / kTX);
  const int nby = ps.nbins[0], nbx = ps.nbins[1];
  std::vector<int> act;
  for (int ty = 0; ty < nty; ++ty) {
    const int y0 = ty * TY, ylo = y0 - W + 1;
    const int by0 = ylo < 0 ? 0 : ylo / bt, by1 = std::min(nby - 1, (y0 + TY - 1) / bt);
    for (int tx = 0; tx < ntx; ++tx) {
      const int x0 = tx * kTX, xlo = x0 - W + 1;
      const int bx0 = xlo < 0 ? 0 : xlo / bt, bx1 = std::min(nbx - 1, (x0 + kTX - 1) / bt);
      bool any = false;
      for (int by = by0; by <= by1 && !any; ++by)
        any = bstart[(size_t)by * nbx + bx1 + 1] > bstart[(size_t)by * nbx + bx0];
      if (any) act.push_back(ty * ntx + tx);
    }
  }
  plan.n_sp2_tiles = (long long)act.size();
  plan.sp2_tiles = (int*)plan.alloc(sizeof(int) * std::max<size_t>(act.size(), 1));
  if (!act.empty())
    GPN_CUDA(cudaMemcpy(plan.sp2_tiles, act.data(), sizeof(int) * act.size(), cudaMemcpyHostToDevice));
}

void launch_spread2d(Plan& plan, const double* alpha_sorted, int R, cudaStream_t st) {
  if (plan.precision == GP_FP32)
    impl<float>(plan, alpha_sorted, R, st);
  else if (plan.precision == GP_DF64)
    impl<dd>(plan, alpha_sorted, R, st);
  else
    impl<double>(plan, alpha_sorted, R, st);
}

}  // namespace gpn
