// Steps (4b) + (5) of Sec. 4.2: interpolate the inverse-transformed fine grids at
// the points (the type-2 NUFFTs of step (4) share this pass) and combine
//   out_i = sum_k w_k(x_i) beta_k(x_i)  (+ shift * alpha_i).
//
// One CTA per non-empty tile bin and right-hand side.  The bin's points need the
// cells [b*tile, b*tile + tile + width - 1) in every dimension.  For d >= 2 the
// CTA brings that block of `cc` channels into shared memory with one TMA tile
// copy (cp.async.bulk.tensor, completion on an mbarrier; out-of-range cells read
// as zero); for d = 1 with a plain coalesced loop.  Then a group of lanes handles
// each point:
//   d = 1: one lane per point;  d = 2: one lane per support row (width lanes);
//   d = 3: one warp per point, lanes over the width^2 pencils.
// Each lane accumulates its channels in registers.  d = 2: the lanes of a point write
// their per-row sums to shared memory and lane k of the point adds up channel k's rows
// (a transpose instead of one shuffle tree per channel), forms w_k(x_i) beta_k in FP32 and
// the group sums the products in float64.  d = 1, 3: the group is reduced with shuffles
// and the group leader applies w_k(x_i) in float64.
// The mbarrier wait is bounded: when it runs out the CTA records a timeout in the
// plan's device status word and returns.
#include <algorithm>
#include <type_traits>

#include "kernels.h"

namespace gpn {

namespace {

constexpr long long kMaxPolls = 1ll << 22;

template <typename T>
struct InterpArgs {
  const int* cell0[kMaxDim];
  const T* xi[kMaxDim];
  const T* psi[kMaxDim];   // tabulated kernel values [n][width] per axis (null: evaluate)
  const T* wk;
  const int* bin_start;
  const int* bins;       // non-empty bins
  int nbins[kMaxDim];
  long long n;
  const T* grid;
  long long nf;
  long long G;
  int width;
  T beta;
  T inv_halfw;
  int tile;
  int ext;       // staged extent per dimension: tile + width - 1
  int epitch;    // last-dimension pitch of the staged block in shared memory
  int cc;        // channels per staging chunk
  int C;
  unsigned box_bytes;    // bytes of one TMA box
  const double* alpha;   // sorted order (may be null)
  double shift;
  const double* dcorr;   // per-point addition to the shift (sorted order, may be null)
  double* out;           // sorted order, N x R
  int* status;
};

// d = 2 channel-sum transpose: per warp, 32 lanes x (CMAX | 1) values (odd row pitch)
template <typename T, int D, int CMAX>
__host__ __device__ constexpr bool use_transpose() { return D == 2 && CMAX <= 16; }
template <typename T, int D, int CMAX>
__host__ __device__ constexpr size_t transpose_bytes() { return use_transpose<T, D, CMAX>() ? 8 * 32 * (CMAX | 1) * sizeof(T) : 0; }

// EXACT: every channel chunk holds exactly CMAX channels (C = cc = CMAX), so the
// channel loops run without guards.
template <typename T, int D, int CMAX, bool TMA, bool EXACT>
__global__ void __launch_bounds__(256) k_interp(InterpArgs<T> a, const __grid_constant__ CUtensorMap tmap) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(smem_raw);
  T* st = reinterpret_cast<T*>(smem_raw + 128);
  // after the staged block (box_bytes, a multiple of 16)
  T* s_red = reinterpret_cast<T*>(smem_raw + 128 + a.box_bytes);
  const int bin = a.bins[blockIdx.x];
  const int p0 = a.bin_start[bin], p1 = a.bin_start[bin + 1];
  const int npts = p1 - p0;
  const int r = blockIdx.y, W = a.width, C = a.C, E = a.ext, EP = a.epitch;
  int base[kMaxDim] = {0, 0, 0};
  {
    long long rest = bin;
#pragma unroll
    for (int q = D - 1; q >= 0; --q) {
      base[q] = (int)(rest % a.nbins[q]) * a.tile;
      rest /= a.nbins[q];
    }
  }
  int lead_e = 1;
#pragma unroll
  for (int q = 0; q < D - 1; ++q) lead_e *= E;
  const int SV = lead_e * EP;  // staged volume per channel

  constexpr int kGroup = D == 1 ? 1 : (D == 2 ? 0 : 32);  // 0: width lanes
  const int Gs = kGroup == 0 ? W : kGroup;
  const int ppw = 32 / Gs;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int grp = lane / Gs, gl = lane - grp * Gs;
  int P = 1;
#pragma unroll
  for (int q = 0; q < D - 1; ++q) P *= W;
  const T* grid_r = a.grid + (size_t)r * C * a.G;
  double* out_r = a.out + (size_t)r * a.n;
  const double* alpha_r = a.alpha ? a.alpha + (size_t)r * a.n : nullptr;

  if (TMA && threadIdx.x == 0) mbar_init(bar, 1);
  unsigned phase = 0;

  // a batch's per-point data (first support cell relative to the block, offset xi);
  // the next batch's is loaded while the current one is processed, the first one while
  // the staging copy is in flight
  auto load_pt = [&](int pb_, int (&L)[kMaxDim], T (&X)[kMaxDim]) {
    const int pi_ = pb_ + grp;
    const int p_ = p0 + ((grp < ppw && pi_ < npts) ? pi_ : 0);
#pragma unroll
    for (int q = 0; q < D; ++q) {
      L[q] = a.cell0[q][p_] - base[q];
      X[q] = a.xi[q][p_];
    }
  };
  for (int c0 = 0; c0 < C; c0 += a.cc) {
    const int ncur = min(a.cc, C - c0);
    __syncthreads();  // the previous chunk has been read (and the barrier initialised)
    int nl0[kMaxDim];
    T nx[kMaxDim];
    load_pt(warp * ppw, nl0, nx);
    if (TMA) {
      if (threadIdx.x == 0) {
        mbar_expect_tx(bar, a.box_bytes);
        if (D == 2)
          tma_load_3d(st, &tmap, base[1], base[0], r * C + c0, bar);
        else
          tma_load_4d(st, &tmap, base[2], base[1], base[0], r * C + c0, bar);
      }
      const bool ok = mbar_wait_bounded(bar, phase, kMaxPolls);
      if (__syncthreads_or(!ok)) {
        if (threadIdx.x == 0) {
          atomicExch(a.status, kStatusTimeout);
          mbar_wait_bounded(bar, phase, kMaxPolls);  // let an in-flight copy land before exiting
        }
        return;
      }
      phase ^= 1u;
    } else {
      const int total = ncur * lead_e * E;
      for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
        int rem = idx;
        const int last = rem % E;
        rem /= E;
        int soff = 0;
        long long goff = 0;
        bool in = (long long)base[D - 1] + last < a.nf;
        int lcoord[kMaxDim];
#pragma unroll
        for (int q = D - 2; q >= 0; --q) {
          lcoord[q] = rem % E;
          rem /= E;
        }
        const int k = rem;
#pragma unroll
        for (int q = 0; q < D - 1; ++q) {
          const long long gq = (long long)base[q] + lcoord[q];
          in = in && gq < a.nf;
          soff = soff * E + lcoord[q];
          goff = goff * a.nf + gq;
        }
        goff = goff * a.nf + base[D - 1] + last;
        st[(size_t)k * SV + soff * EP + last] = in ? grid_r[(size_t)(c0 + k) * a.G + goff] : T(0);
      }
      __syncthreads();
    }

    for (int pb = warp * ppw; pb < npts; pb += nwarps * ppw) {
      const int pi = pb + grp;
      const bool active = grp < ppw && pi < npts;
      T acc[CMAX];
#pragma unroll
      for (int k = 0; k < CMAX; ++k) acc[k] = T(0);
      const int p = p0 + (active ? pi : 0);
      int l0[kMaxDim];
      T x[kMaxDim];
#pragma unroll
      for (int q = 0; q < D; ++q) {
        l0[q] = nl0[q];
        x[q] = nx[q];
      }
      if (pb + nwarps * ppw < npts) load_pt(pb + nwarps * ppw, nl0, nx);
      // the epilogue's own inputs, loaded before the accumulation so their latency is hidden
      T wk_gl = T(0);
      double shift_al = 0.0;
      if constexpr (use_transpose<T, D, CMAX>()) {
        if (grp < ppw && gl < ncur) wk_gl = a.wk[(size_t)p * C + c0 + gl];
        if (active && gl == 0 && c0 == 0 && alpha_r)
          shift_al = (a.dcorr ? a.shift + a.dcorr[p] : a.shift) * alpha_r[p];
      }
      if (D == 1) {
        if (active) {
          const T* rowp = st + l0[0];
          for (int i = 0; i < W; ++i) {
            const T wgt = psi_at<T>(i, x[0], a.beta, a.inv_halfw);
#pragma unroll
            for (int k = 0; k < CMAX; ++k)
              if (EXACT || k < ncur) madd_lazy(acc[k], wgt, rowp[(size_t)k * SV + i]);
          }
        }
      } else {
        // lane j of the group holds psi_q(j - xi_q) for every axis q; the others
        // fetch them by shuffles (every lane executes every shuffle)
        const int src = kGroup == 0 ? grp * Gs : 0;
        T pq[kMaxDim];
#pragma unroll
        for (int q = 0; q < D; ++q)
          pq[q] = gl < W ? (a.psi[q] ? a.psi[q][(size_t)p * W + gl] : psi_at<T>(gl, x[q], a.beta, a.inv_halfw))
                         : T(0);
        for (int pen0 = 0; pen0 < P; pen0 += Gs) {
          const int pen = pen0 + gl;
          const bool valid = active && pen < P;
          int rem = valid ? pen : 0, off = 0;
          T plead = T(1);
          int iq[kMaxDim];
#pragma unroll
          for (int q = D - 2; q >= 0; --q) {
            iq[q] = rem % W;
            rem /= W;
          }
#pragma unroll
          for (int q = 0; q < D - 1; ++q) {
            plead *= shfl_val(pq[q], src + iq[q]);
            off = off * E + l0[q] + iq[q];
          }
          const T* rowp = st + (size_t)off * EP + l0[D - 1];
#pragma unroll 3
          for (int i = 0; i < W; ++i) {
            const T wgt = plead * shfl_val(pq[D - 1], src + i);
            if (valid) {
#pragma unroll
              for (int k = 0; k < CMAX; ++k)
                if (EXACT || k < ncur) madd_lazy(acc[k], wgt, rowp[(size_t)k * SV + i]);
            }
          }
        }
      }
      // (float-float: the per-lane sums of at most width x width terms close here)
#pragma unroll
      for (int k = 0; k < CMAX; ++k) acc[k] = renorm_val(acc[k]);
      // reduce within the point's lane group
      if constexpr (use_transpose<T, D, CMAX>()) {
        constexpr int RP = CMAX | 1;   // odd pitch: the 32 lanes write to 32 banks
        T* red = s_red + (size_t)warp * 32 * RP;
#pragma unroll
        for (int k = 0; k < CMAX; ++k)
          if (EXACT || k < ncur) red[lane * RP + k] = acc[k];
        __syncwarp();
        // w_k beta_k summed in float64, or for float-float plans in float-float (converted
        // once at the end: float64 operations run at a small fraction of the FP32 rate)
        using PartT = typename std::conditional<is_dd<T>::value, dd, double>::type;
        PartT part{};
        if (grp < ppw) {   // lanes past the last full group hold no point
          for (int k = gl; k < ncur; k += Gs) {
            T sum = T(0);
            for (int row = 0; row < Gs; ++row) sum += red[(grp * Gs + row) * RP + k];
            const T wkv = k == gl ? wk_gl : a.wk[(size_t)p * C + c0 + k];
            if constexpr (is_dd<T>::value)
              madd(part, wkv, sum);
            else
              part += (double)(wkv * sum);
          }
        }
        __syncwarp();   // red is rewritten by the next point batch
        for (int o = 1; o < Gs; o <<= 1) {
          const PartT v = shfl_down_val(part, o);
          if (gl + o < Gs) part += v;
        }
        if (active && gl == 0) {
          if (c0 == 0)
            out_r[p] = to_f64(part) + shift_al;
          else
            out_r[p] += to_f64(part);
        }
        continue;
      } else if (kGroup == 32) {
#pragma unroll
        for (int k = 0; k < CMAX; ++k) {
          if (k < ncur) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc[k] += shfl_xor_val(acc[k], o);
          }
        }
      } else if (kGroup == 0) {
#pragma unroll
        for (int k = 0; k < CMAX; ++k) {
          if (k < ncur) {
            for (int o = 1; o < Gs; o <<= 1) {
              const T v = shfl_down_val(acc[k], o);
              if (gl + o < Gs) acc[k] += v;
            }
          }
        }
      }
      if (active && gl == 0) {
        double res = 0.0;
#pragma unroll
        for (int k = 0; k < CMAX; ++k)
          if (k < ncur) res += (double)a.wk[(size_t)p * C + c0 + k] * (double)acc[k];
        if (c0 == 0) {
          if (alpha_r) res += (a.dcorr ? a.shift + a.dcorr[p] : a.shift) * alpha_r[p];
          out_r[p] = res;
        } else {
          out_r[p] += res;
        }
      }
    }
  }
}

template <typename T, int D, int CMAX, bool TMA, bool EXACT = false>
void launch(const InterpArgs<T>& a, const CUtensorMap& tm, dim3 grid, size_t smem0, cudaStream_t st) {
  const size_t smem = smem0 + transpose_bytes<T, D, CMAX>();
  GPN_CUDA(cudaFuncSetAttribute(k_interp<T, D, CMAX, TMA, EXACT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem));
  k_interp<T, D, CMAX, TMA, EXACT><<<grid, 256, smem, st>>>(a, tm);
}

// d = 2 with all channels in one chunk and C <= 16: the exact channel count
template <typename T, int NC>
void launch_exact2(const InterpArgs<T>& a, const CUtensorMap& tm, dim3 grid, size_t smem, cudaStream_t st) {
  if constexpr (NC <= 16) {
    if (a.C == NC) return launch<T, 2, NC, true, true>(a, tm, grid, smem, st);
    launch_exact2<T, NC + 1>(a, tm, grid, smem, st);
  }
}

template <typename T, int D, bool TMA>
void launch_c(const InterpArgs<T>& a, const CUtensorMap& tm, dim3 grid, size_t smem, cudaStream_t st) {
  if (D == 2 && a.cc == a.C && a.C <= 16) return launch_exact2<T, 1>(a, tm, grid, smem, st);
  switch (cmax_bucket(a.cc)) {
    case 8: launch<T, D, 8, TMA>(a, tm, grid, smem, st); break;
    case 12: launch<T, D, 12, TMA>(a, tm, grid, smem, st); break;
    case 16: launch<T, D, 16, TMA>(a, tm, grid, smem, st); break;
    default: launch<T, D, 32, TMA>(a, tm, grid, smem, st);
  }
}

template <typename T>
void interp_impl(Plan& plan, const PointSet& ps, const double* alpha_sorted, double shift, double* out_sorted, int R,
                 cudaStream_t st) {
  if (ps.n_active_bins == 0) return;
  const GridGeom& g = plan.geom;
  InterpArgs<T> a{};
  for (int q = 0; q < kMaxDim; ++q) {
    a.cell0[q] = ps.cell0[q];
    a.xi[q] = (const T*)ps.xi[q];
    a.psi[q] = (const T*)ps.psi[q];
    a.nbins[q] = ps.nbins[q];
  }
  a.wk = (const T*)ps.wk;
  a.bin_start = ps.bin_start;
  a.bins = ps.active_bins;
  a.n = ps.n;
  a.grid = (const T*)plan.grid_out;
  a.nf = g.nf;
  a.G = plan.grid_elems;
  a.width = g.width;
  a.beta = es_beta_arg<T>(g.beta);
  a.inv_halfw = (T)(2.0 / g.width);
  a.tile = g.tile;
  a.ext = g.tile + g.width - 1;
  a.epitch = interp_pitch(g.d, g.tile, g.width, sizeof(T));
  a.C = g.C;
  a.cc = plan.interp_cc;
  a.box_bytes = (unsigned)(interp_stage_bytes(g.d, g.tile, g.width, sizeof(T)) * a.cc);
  a.alpha = alpha_sorted;
  a.shift = shift;
  a.dcorr = (&ps == &plan.pts) ? plan.dcorr : nullptr;
  a.out = out_sorted;
  a.status = plan.dev_status;
  // a TMA tile copy must start on a 16-byte boundary along x (x = bin * tile)
  GPN_CHECK(g.d == 1 || (g.tile * sizeof(T)) % 16 == 0, GP_EUNSUPPORTED,
            "interp tile must be a multiple of 16 bytes of grid values for the TMA copies");
  const size_t smem = 128 + (size_t)a.box_bytes;
  dim3 grid((unsigned)ps.n_active_bins, (unsigned)R);
  switch (g.d) {
    case 1: launch_c<T, 1, false>(a, plan.tmap_out, grid, smem, st); break;
    case 2: launch_c<T, 2, true>(a, plan.tmap_out, grid, smem, st); break;
    default: launch_c<T, 3, true>(a, plan.tmap_out, grid, smem, st);
  }
  GPN_CUDA(cudaGetLastError());
}

}  // namespace

// Last-dimension pitch of the staged block: for d >= 2 the TMA box width, a
// multiple of 16 bytes chosen congruent to 4 words mod 8 so that the support rows
// a lane group reads spread over the banks; for d = 1 the extent itself.
int interp_pitch(int d, int tile, int width, size_t rs) {
  int e = tile + width - 1;
  if (d == 1) return e;
  const int q = (int)(16 / rs);          // elements per 16 bytes
  int p = (e + q - 1) / q * q;
  const int words = (int)(rs / 4);
  while (((p * words) % 8) != 4) p += q;
  return p;
}

size_t interp_stage_bytes(int d, int tile, int width, size_t rs) {
  size_t e = (size_t)tile + width - 1;
  size_t lead = 1;
  for (int q = 0; q < d - 1; ++q) lead *= e;
  return lead * (size_t)interp_pitch(d, tile, width, rs) * rs;
}

void launch_interp(Plan& plan, const PointSet& ps, const double* alpha_sorted, double shift, double* out_sorted,
                   int R, cudaStream_t st) {
  if (ps.n == 0) return;
  if (plan.precision == GP_FP32)
    interp_impl<float>(plan, ps, alpha_sorted, shift, out_sorted, R, st);
  else if (plan.precision == GP_DF64)
    interp_impl<dd>(plan, ps, alpha_sorted, shift, out_sorted, R, st);
  else
    interp_impl<double>(plan, ps, alpha_sorted, shift, out_sorted, R, st);
}

}  // namespace gpn
