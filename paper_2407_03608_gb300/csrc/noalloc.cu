// Posterior mean at a batch of query points without any device allocation
// (gp_posterior_mean_noalloc).  The paper has no counterpart: this is a serving
// variant of step (4b)+(5) of Sec. 4.2 evaluated at query points.
//
// Why it exists: gp_posterior_mean builds a binned, sorted copy of the queries
// and frees it on return.  Its cudaMalloc/cudaFree calls synchronise the whole
// device (cudaFree waits for all work on it) and can fail when the device
// memory is already committed.  A serving loop that answers small query batches
// between other streams' work, or a process that has reserved the device memory
// up front, cannot afford either.  This variant keeps its scratch (host-input
// staging, the host-output staging and an error counter) in one file-scope
// __device__ array and evaluates each query straight from the fine grid, one warp
// per query point, with the query's fields, cell, offsets and Chebyshev weights
// computed in the kernel.  So nothing needs binning or sorting.
//
// The scratch is shared by every call on a device: calls whose GPU work overlaps
// (other streams, other host threads, other plans) race on it.
#include <cuda.h>

#include <mutex>

#include "kernels.h"

namespace gpn {

namespace {

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
// per device: the context the address was looked up in, the address and the SM count
CUcontext g_scratch_ctx[kMaxDevices] = {};
NoAllocScratch g_scratch[kMaxDevices] = {};

// The current context, through the runtime's driver entry point (the library does not
// link libcuda).  A reset device gets a new primary context, which loads the module, and
// so the array, again.
CUcontext current_context() {
  using GetCtx = CUresult (*)(CUcontext*);
  static GetCtx get = nullptr;
  if (!get) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    GPN_CUDA(cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 12000, cudaEnableDefault, &q));
    GPN_CHECK(q == cudaDriverEntryPointSuccess && fn, GP_ECUDA, "cuCtxGetCurrent unavailable");
    get = (GetCtx)fn;
  }
  CUcontext c = nullptr;
  GPN_CHECK(get(&c) == CUDA_SUCCESS, GP_ECUDA, "cuCtxGetCurrent failed");
  return c;
}

constexpr double kTwoPi = 6.283185307179586476925286766559;

template <typename T>
struct QueryArgs {
  const double* x;     // nq x d row-major
  const double* fa;    // field a (param_mode)
  const double* fb;    // field b
  double* mu;          // nq
  long long nq;
  int mode;
  double centre[kMaxDim];
  double box_lo[kMaxDim];
  double box_hi[kMaxDim];
  double inv_h;
  double half_nf;
  double half_w;
  double sig_lo;
  double sig_hi;
  double nodes[kMaxChannels];
  double bary[kMaxChannels];
  int C;
  const T* grid;       // inverse-transformed fine grids, channel k at k * G
  long long nf;
  long long G;
  int width;
  T beta;
  T inv_halfw;
  unsigned* bad;       // count of rejected queries (starts at zero)
};

// One warp per query.  Every lane computes the query's scalars (same inputs, so
// the branches are warp-uniform); the lanes then split the width^d support cells,
// each lane summing psi-weighted grid values per channel, and a shuffle reduction
// gives beta_k(x_q).  Lane 0 forms mu_q = sum_k w_k(x_q) beta_k(x_q) in float64.
template <typename T, int D, int CMAX>
__global__ void __launch_bounds__(256) k_query_interp(QueryArgs<T> a) {
  const int lane = threadIdx.x & 31;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  const int W = a.width;
  int total = 1;
#pragma unroll
  for (int q = 0; q < D; ++q) total *= W;
  for (long long qi = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; qi < a.nq; qi += nw) {
    const double fa = a.fa[qi], fb = a.fb[qi];
    double w, s;
    if (a.mode == GP_PARAMS_SCALES) {
      s = fb * 0.70710678118654752440;
      w = fa * pow(kTwoPi, 0.25 * D) * pow(fb, 0.5 * D);
    } else {
      w = fa;
      s = fb;
    }
    bool ok = s > 0.0 && isfinite(s) && w >= 0.0 && isfinite(w) && s >= a.sig_lo * (1.0 - 1e-12) &&
              s <= a.sig_hi * (1.0 + 1e-12);
    long long l0[D];
    T xi[D];
#pragma unroll
    for (int q = 0; q < D; ++q) {
      const double xa = a.x[qi * D + q];
      ok = ok && isfinite(xa) && xa >= a.box_lo[q] && xa <= a.box_hi[q];
      const double g = (xa - a.centre[q]) * a.inv_h + a.half_nf;
      const double l0d = ceil(g - a.half_w);
      // The plan centres the box on the grid with a margin of at least width/2 + 2 cells
      // per side, so for a query inside the box the support lies inside the grid and
      // this test never rejects it; it only guards the grid reads below.
      ok = ok && l0d >= 0.0 && l0d + W <= (double)a.nf;
      l0[q] = ok ? (long long)l0d : 0;
      xi[q] = ok ? (T)(g - l0d) : T(0);
    }
    if (!ok) {
      if (lane == 0) {
        atomicAdd(a.bad, 1u);
        a.mu[qi] = __longlong_as_double(0x7ff8000000000000ll);  // quiet NaN
      }
      continue;
    }
    // lane j < W holds psi(j - xi_q) for every axis q
    T pq[D];
#pragma unroll
    for (int q = 0; q < D; ++q) pq[q] = lane < W ? psi_at<T>(lane, xi[q], a.beta, a.inv_halfw) : T(0);
    T acc[CMAX];
#pragma unroll
    for (int k = 0; k < CMAX; ++k) acc[k] = T(0);
    for (int c0 = 0; c0 < total; c0 += 32) {
      const int c = c0 + lane;
      const bool valid = c < total;
      int rem = valid ? c : 0;
      int iq[D];
#pragma unroll
      for (int q = D - 1; q >= 0; --q) {
        iq[q] = rem % W;
        rem /= W;
      }
      T wgt = T(1);
      long long off = 0;
#pragma unroll
      for (int q = 0; q < D; ++q) {
        wgt *= shfl_val(pq[q], iq[q]);
        off = off * a.nf + l0[q] + iq[q];
      }
      if (valid) {
        const T* gp = a.grid + off;
#pragma unroll
        for (int k = 0; k < CMAX; ++k)
          if (k < a.C) madd(acc[k], wgt, ldg_val(gp + (size_t)k * a.G));
      }
    }
#pragma unroll
    for (int k = 0; k < CMAX; ++k) {
      if (k < a.C) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc[k] += shfl_xor_val(acc[k], o);
      }
    }
    if (lane == 0) {
      // w_k = w (2 pi sigma^2)^(-d/2) P_k(sigma), P_k barycentric on the Chebyshev-Lobatto nodes
      const double pre = w * pow(kTwoPi * s * s, -0.5 * D);
      int hit = -1;
      for (int k = 0; k < a.C; ++k)
        if (s == a.nodes[k]) hit = k;
      double den = 0.0;
      if (hit < 0 && a.C > 1)
        for (int k = 0; k < a.C; ++k) den += a.bary[k] / (s - a.nodes[k]);
      double res = 0.0;
#pragma unroll
      for (int k = 0; k < CMAX; ++k) {
        if (k < a.C) {
          double wk;
          if (hit >= 0 || a.C == 1)
            wk = (k == hit || a.C == 1) ? pre : 0.0;
          else
            wk = pre * (a.bary[k] / (s - a.nodes[k])) / den;
          res += (double)(T)wk * (double)acc[k];
        }
      }
      a.mu[qi] = res;
    }
  }
}

template <typename T, int D>
void launch_d(const QueryArgs<T>& a, int blocks, cudaStream_t st) {
  switch (cmax_bucket(a.C)) {
    case 8: k_query_interp<T, D, 8><<<blocks, 256, 0, st>>>(a); break;
    case 12: k_query_interp<T, D, 12><<<blocks, 256, 0, st>>>(a); break;
    case 16: k_query_interp<T, D, 16><<<blocks, 256, 0, st>>>(a); break;
    default: k_query_interp<T, D, 32><<<blocks, 256, 0, st>>>(a);
  }
}

template <typename T>
void query_impl(Plan& plan, const double* x, const double* fa, const double* fb, long long nq, double* mu,
                unsigned* bad, int sms, cudaStream_t st) {
  const Hyper& h = plan.h;
  const GridGeom& g = plan.geom;
  QueryArgs<T> a{};
  a.x = x;
  a.fa = fa;
  a.fb = fb;
  a.mu = mu;
  a.nq = nq;
  a.mode = plan.param_mode;
  for (int q = 0; q < h.d; ++q) {
    a.centre[q] = 0.5 * (h.box_lo[q] + h.box_hi[q]);
    a.box_lo[q] = h.box_lo[q];
    a.box_hi[q] = h.box_hi[q];
  }
  const double P = 1.0 / h.dw;  // the same operations as the training points' binning
  a.inv_h = h.nf / P;
  a.half_nf = 0.5 * h.nf;
  a.half_w = 0.5 * h.width;
  a.sig_lo = h.sig_lo;
  a.sig_hi = h.sig_hi;
  a.C = g.C;
  for (int k = 0; k < g.C; ++k) {
    a.nodes[k] = plan.tb.nodes[k];
    a.bary[k] = plan.tb.bary[k];
  }
  a.grid = (const T*)plan.grid_out;
  a.nf = g.nf;
  a.G = plan.grid_elems;
  a.width = g.width;
  a.beta = es_beta_arg<T>(g.beta);
  a.inv_halfw = (T)(2.0 / g.width);
  a.bad = bad;
  // eight warps (queries) a block; at most eight blocks an SM, the rest by the grid-stride loop
  const int blocks = (int)std::min<long long>((nq + 7) / 8, (long long)sms * 8);
  switch (h.d) {
    case 1: launch_d<T, 1>(a, blocks, st); break;
    case 2: launch_d<T, 2>(a, blocks, st); break;
    default: launch_d<T, 3>(a, blocks, st);
  }
  GPN_CUDA(cudaGetLastError());
}

}  // namespace

NoAllocScratch noalloc_scratch(int device) {
  GPN_CHECK(device >= 0 && device < kMaxDevices, GP_EUNSUPPORTED, "device ordinal beyond the scratch table");
  std::lock_guard<std::mutex> lk(g_setup_mu);
  // the caller has made `device` current; the symbol's address is per device (and per
  // context: after a reset of the device it is looked up again)
  const CUcontext ctx = current_context();
  if (!g_scratch[device].ptr || g_scratch_ctx[device] != ctx) {
    NoAllocScratch s{};
    GPN_CUDA(cudaGetSymbolAddress(&s.ptr, g_noalloc_scratch));
    GPN_CUDA(cudaDeviceGetAttribute(&s.sms, cudaDevAttrMultiProcessorCount, device));
    GPN_CHECK(s.ptr && s.sms > 0, GP_ECUDA, "no device address or SM count for the static scratch");
    g_scratch[device] = s;
    g_scratch_ctx[device] = ctx;
  }
  return g_scratch[device];
}

void launch_query_interp(Plan& plan, const double* x, const double* fa, const double* fb, long long nq, double* mu,
                         unsigned* bad, int sms, cudaStream_t st) {
  if (nq == 0) return;
  if (plan.precision == GP_FP32)
    query_impl<float>(plan, x, fa, fb, nq, mu, bad, sms, st);
  else if (plan.precision == GP_DF64)
    query_impl<dd>(plan, x, fa, fb, nq, mu, bad, sms, st);
  else
    query_impl<double>(plan, x, fa, fb, nq, mu, bad, sms, st);
}

}  // namespace gpn
