// Plan-time point processing: scale-field conversion, statistics, binning/sorting of
// the points into fine-grid tiles, and the per-point Chebyshev weights w_k(x_i) (Eq. Wk).
#include <cub/cub.cuh>

#include <cmath>
#include <vector>

#include "ff64.h"
#include "kernels.h"
#include "plan.h"

namespace gpn {

namespace {

constexpr double kPi = 3.14159265358979323846264338327950;
constexpr double kTwoPi = 6.283185307179586476925286766559;

__global__ void k_fields_to_paper(const double* __restrict__ a, const double* __restrict__ b, double* __restrict__ w,
                                  double* __restrict__ sig, long long n, int d, int mode) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  double fa = a[i], fb = b[i];
  if (mode == GP_PARAMS_SCALES) {
    // sigma = l / sqrt(2), w = s (2 pi)^(d/4) l^(d/2): Eq. (nonstat2) equals the Paciorek form.
    sig[i] = fb * 0.70710678118654752440;
    w[i] = fa * pow(kTwoPi, 0.25 * d) * pow(fb, 0.5 * d);
  } else {
    w[i] = fa;
    sig[i] = fb;
  }
}

// Per-block partial statistics: [sig_min, sig_max, x_min[d], x_max[d], bad]
__global__ void k_stats(const double* __restrict__ x, const double* __restrict__ w, const double* __restrict__ sig,
                        long long n, int d, double* __restrict__ part) {
  __shared__ double sh[8][256];
  double v[8];
  v[0] = INFINITY;
  v[1] = -INFINITY;
  for (int a = 0; a < 3; ++a) {
    v[2 + a] = INFINITY;
    v[5 + a] = -INFINITY;
  }
  double bad = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    double s = sig[i], ww = w[i];
    if (!(s > 0.0) || !isfinite(s) || !(ww >= 0.0) || !isfinite(ww)) bad += 1.0;
    v[0] = fmin(v[0], s);
    v[1] = fmax(v[1], s);
    for (int a = 0; a < d; ++a) {
      double xa = x[i * d + a];
      if (!isfinite(xa)) bad += 1.0;
      v[2 + a] = fmin(v[2 + a], xa);
      v[5 + a] = fmax(v[5 + a], xa);
    }
  }
  int t = threadIdx.x;
  for (int q = 0; q < 8; ++q) sh[q][t] = v[q];
  __shared__ double shb[256];
  shb[t] = bad;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (t < s) {
      sh[0][t] = fmin(sh[0][t], sh[0][t + s]);
      sh[1][t] = fmax(sh[1][t], sh[1][t + s]);
      for (int a = 0; a < 3; ++a) {
        sh[2 + a][t] = fmin(sh[2 + a][t], sh[2 + a][t + s]);
        sh[5 + a][t] = fmax(sh[5 + a][t], sh[5 + a][t + s]);
      }
      shb[t] += shb[t + s];
    }
    __syncthreads();
  }
  if (t == 0) {
    for (int q = 0; q < 8; ++q) part[blockIdx.x * 9 + q] = sh[q][0];
    part[blockIdx.x * 9 + 8] = shb[0];
  }
}

struct CellArgs {
  double centre[kMaxDim];
  double inv_h;
  double half_nf;
  double half_w;
  int width;
  long long nf;
  int tile;
  int nb[kMaxDim];
  int d;
};

// Fine-grid coordinate g = (x - centre)/h + nf/2; support starts at l0 = ceil(g - width/2);
// bin = floor(l0 / tile) per dimension.  bad[0] counts points whose support leaves the grid.
__global__ void k_cells(const double* __restrict__ x, long long n, CellArgs ca, int* __restrict__ l0_out,
                        double* __restrict__ xi_out, int* __restrict__ key, int* __restrict__ idx,
                        unsigned long long* __restrict__ bad) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  long long lin = 0;
  bool ok = true;
  for (int a = 0; a < ca.d; ++a) {
    double g = (x[i * ca.d + a] - ca.centre[a]) * ca.inv_h + ca.half_nf;
    double l0d = ceil(g - ca.half_w);
    long long l0 = (long long)l0d;
    if (!(l0 >= 0 && l0 + ca.width <= ca.nf)) {
      ok = false;
      l0 = 0;
    }
    l0_out[a * n + i] = (int)l0;
    xi_out[a * n + i] = g - (double)l0;
    int b = (int)(l0 / ca.tile);
    if (b >= ca.nb[a]) b = ca.nb[a] - 1;
    lin = lin * ca.nb[a] + b;
  }
  if (!ok) atomicAdd(bad, 1ull);
  key[i] = (int)lin;
  idx[i] = (int)i;
}

// bin_start[b] = first sorted position whose key >= b (lower bound).
__global__ void k_bin_start(const int* __restrict__ keys, long long n, long long nbins, int* __restrict__ start) {
  long long b = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (b > nbins) return;
  long long lo = 0, hi = n;
  while (lo < hi) {
    long long mid = (lo + hi) >> 1;
    if (keys[mid] < b)
      lo = mid + 1;
    else
      hi = mid;
  }
  start[b] = (int)lo;
}

// Diagonal defect K_ii - K~_ii per sorted point (see build_diag_correction).
__global__ void k_diag_defect(const int* __restrict__ perm, long long n, const double* __restrict__ w,
                              const double* __restrict__ sig, ChebArgs cb, const double* __restrict__ S,
                              double* __restrict__ out) {
  long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (p >= n) return;
  const long long i = perm[p];
  const double s = sig[i];
  double wk[kMaxChannels];
  cheb_weights(w[i], s, cb, wk);
  double q = 0.0;
  for (int k = 0; k < cb.C; ++k) {
    double row = 0.0;
    for (int l = 0; l < cb.C; ++l) row += S[k * cb.C + l] * wk[l];
    q += wk[k] * row;
  }
  out[p] = w[i] * w[i] * pow(2.0 * kTwoPi * s * s, -0.5 * cb.d) - q;
}

template <typename T>
__global__ void k_gather_points(const int* __restrict__ perm, long long n, int d, const int* __restrict__ l0_in,
                                const double* __restrict__ xi_in, int* c0, int* c1, int* c2, T* x0, T* x1, T* x2,
                                const double* __restrict__ w, const double* __restrict__ sig, ChebArgs cb,
                                T* __restrict__ wk, float* __restrict__ wabs) {
  long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (p >= n) return;
  long long i = perm[p];
  int* cs[3] = {c0, c1, c2};
  T* xs[3] = {x0, x1, x2};
  for (int a = 0; a < d; ++a) {
    cs[a][p] = l0_in[a * n + i];
    xs[a][p] = (T)xi_in[a * n + i];
  }
  double v[kMaxChannels];
  cheb_weights(w[i], sig[i], cb, v);
  double m = 0.0;
  for (int k = 0; k < cb.C; ++k) {
    wk[p * cb.C + k] = (T)v[k];
    m = fmax(m, fabs(v[k]));
  }
  wabs[p] = (float)m;
}

// psi(j - xi_a(p)) for every sorted point p, axis a < d and j < W (the values the spread and
// the interpolation would otherwise evaluate at every visit of the point)
template <typename T>
__global__ void k_psi_tables(long long n, int d, int W, const T* __restrict__ x0, const T* __restrict__ x1,
                             const T* __restrict__ x2, T beta, T inv_halfw, T* t0, T* t1, T* t2) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n * W) return;
  const long long p = i / W;
  const int j = (int)(i - p * W);
  const T* xs[3] = {x0, x1, x2};
  T* ts[3] = {t0, t1, t2};
  for (int a = 0; a < d; ++a) ts[a][i] = psi_at<T>(j, xs[a][p], beta, inv_halfw);
}

// dst[p + r N] = src[perm[p] + r N]
__global__ void k_gather(const int* __restrict__ perm, const double* __restrict__ src, double* __restrict__ dst,
                         long long n, int R) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= n * R) return;
  long long r = t / n, p = t - r * n;
  dst[t] = src[r * n + perm[p]];
}

// dst[perm[p] + r N] = src[p + r N]
__global__ void k_scatter(const int* __restrict__ perm, const double* __restrict__ src, double* __restrict__ dst,
                          long long n, int R) {
  long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= n * R) return;
  long long r = t / n, p = t - r * n;
  dst[r * n + perm[p]] = src[t];
}

}  // namespace

void gather_sorted(const PointSet& ps, const double* src, double* dst, int R, cudaStream_t st) {
  if (ps.n == 0) return;
  k_gather<<<blocks_for(ps.n * R, 256), 256, 0, st>>>(ps.perm, src, dst, ps.n, R);
  GPN_CUDA(cudaGetLastError());
}

void scatter_sorted(const PointSet& ps, const double* src, double* dst, int R, cudaStream_t st) {
  if (ps.n == 0) return;
  k_scatter<<<blocks_for(ps.n * R, 256), 256, 0, st>>>(ps.perm, src, dst, ps.n, R);
  GPN_CUDA(cudaGetLastError());
}

void fields_to_paper(const double* a, const double* b, double* w_out, double* sig_out, long long n, int d, int mode,
                     cudaStream_t st) {
  if (n == 0) return;
  k_fields_to_paper<<<blocks_for(n, 256), 256, 0, st>>>(a, b, w_out, sig_out, n, d, mode);
  GPN_CUDA(cudaGetLastError());
}

void field_stats(const double* x, const double* w, const double* sig, long long n, int d, double* host_out,
                 cudaStream_t st) {
  int nb = (int)std::min<long long>(1024, (n + 255) / 256);
  if (nb < 1) nb = 1;
  double* part = nullptr;
  GPN_CUDA(cudaMalloc(&part, sizeof(double) * 9 * nb));
  k_stats<<<nb, 256, 0, st>>>(x, w, sig, n, d, part);
  std::vector<double> h(9 * nb);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), part, sizeof(double) * 9 * nb, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(part);
  GPN_CUDA(e);
  double out[9] = {INFINITY, -INFINITY, INFINITY, INFINITY, INFINITY, -INFINITY, -INFINITY, -INFINITY, 0.0};
  for (int b = 0; b < nb; ++b) {
    out[0] = std::fmin(out[0], h[b * 9 + 0]);
    out[1] = std::fmax(out[1], h[b * 9 + 1]);
    for (int a = 0; a < 3; ++a) {
      out[2 + a] = std::fmin(out[2 + a], h[b * 9 + 2 + a]);
      out[5 + a] = std::fmax(out[5 + a], h[b * 9 + 5 + a]);
    }
    out[8] += h[b * 9 + 8];
  }
  for (int q = 0; q < 9; ++q) host_out[q] = out[q];
}

void build_pointset(Plan& plan, PointSet& ps, const double* x_dev, const double* w_dev, const double* sig_dev,
                    long long n, cudaStream_t st, DevAlloc alloc, void* actx, std::vector<int>* bin_start_host) {
  const Hyper& h = plan.h;
  const int d = h.d;
  ps.n = n;
  ps.nbins_total = 1;
  for (int a = 0; a < kMaxDim; ++a) ps.nbins[a] = 1;
  for (int a = 0; a < d; ++a) {
    ps.nbins[a] = (int)((h.nf + h.tile - 1) / h.tile);
    ps.nbins_total *= ps.nbins[a];
  }
  GPN_CHECK(ps.nbins_total < (1ll << 30), GP_EINVAL, "too many tiles");
  GPN_CHECK(n < (1ll << 31), GP_EINVAL, "at most 2^31 - 1 points");
  CellArgs ca{};
  double P = 1.0 / h.dw;
  ca.inv_h = h.nf / P;
  ca.half_nf = 0.5 * h.nf;
  ca.half_w = 0.5 * h.width;
  ca.width = h.width;
  ca.nf = h.nf;
  ca.tile = h.tile;
  ca.d = d;
  for (int a = 0; a < d; ++a) {
    ca.centre[a] = 0.5 * (h.box_lo[a] + h.box_hi[a]);
    ca.nb[a] = ps.nbins[a];
  }
  // temporaries (caller order)
  int *l0_tmp = nullptr, *keys = nullptr, *keys_sorted = nullptr, *idx = nullptr;
  double* xi_tmp = nullptr;
  unsigned long long* bad = nullptr;
  void* cub_tmp = nullptr;
  size_t cub_bytes = 0;
  cudaError_t e = cudaSuccess;
  auto chk = [&](cudaError_t x) {
    if (e == cudaSuccess) e = x;
  };
  size_t nn = (size_t)std::max<long long>(n, 1);
  chk(cudaMalloc(&l0_tmp, sizeof(int) * nn * d));
  chk(cudaMalloc(&xi_tmp, sizeof(double) * nn * d));
  chk(cudaMalloc(&keys, sizeof(int) * nn));
  chk(cudaMalloc(&keys_sorted, sizeof(int) * nn));
  chk(cudaMalloc(&idx, sizeof(int) * nn));
  chk(cudaMalloc(&bad, sizeof(unsigned long long)));
  const size_t rs = plan.real_size;
  for (int a = 0; a < d; ++a) {
    ps.cell0[a] = (int*)alloc(actx, sizeof(int) * nn);
    ps.xi[a] = alloc(actx, rs * nn);
  }
  ps.perm = (int*)alloc(actx, sizeof(int) * nn);
  ps.wk = alloc(actx, rs * nn * plan.geom.C);
  ps.wabs = (float*)alloc(actx, sizeof(float) * nn);
  ps.bin_start = (int*)alloc(actx, sizeof(int) * (ps.nbins_total + 1));
  unsigned long long hbad = 0;
  if (e == cudaSuccess) {
    chk(cudaMemsetAsync(bad, 0, sizeof(unsigned long long), st));
    if (n > 0) k_cells<<<blocks_for(n, 256), 256, 0, st>>>(x_dev, n, ca, l0_tmp, xi_tmp, keys, idx, bad);
    chk(cudaGetLastError());
    int end_bit = 1;
    while ((1ll << end_bit) <= ps.nbins_total) ++end_bit;
    if (n > 0) {
      chk(cub::DeviceRadixSort::SortPairs(nullptr, cub_bytes, keys, keys_sorted, idx, ps.perm, (int)n, 0, end_bit, st));
      chk(cudaMalloc(&cub_tmp, std::max<size_t>(cub_bytes, 16)));
      chk(cub::DeviceRadixSort::SortPairs(cub_tmp, cub_bytes, keys, keys_sorted, idx, ps.perm, (int)n, 0, end_bit,
                                          st));
    }
    k_bin_start<<<blocks_for(ps.nbins_total + 1, 256), 256, 0, st>>>(keys_sorted, n, ps.nbins_total, ps.bin_start);
    chk(cudaGetLastError());
    ChebArgs cb{};
    cb.C = plan.geom.C;
    cb.d = d;
    for (int k = 0; k < cb.C; ++k) {
      cb.nodes[k] = plan.tb.nodes[k];
      cb.bary[k] = plan.tb.bary[k];
    }
    if (n > 0) {
      if (plan.precision == GP_FP32)
        k_gather_points<float><<<blocks_for(n, 256), 256, 0, st>>>(
            ps.perm, n, d, l0_tmp, xi_tmp, ps.cell0[0], ps.cell0[1], ps.cell0[2], (float*)ps.xi[0], (float*)ps.xi[1],
            (float*)ps.xi[2], w_dev, sig_dev, cb, (float*)ps.wk, ps.wabs);
      else if (plan.precision == GP_DF64)
        k_gather_points<dd><<<blocks_for(n, 256), 256, 0, st>>>(
            ps.perm, n, d, l0_tmp, xi_tmp, ps.cell0[0], ps.cell0[1], ps.cell0[2], (dd*)ps.xi[0], (dd*)ps.xi[1],
            (dd*)ps.xi[2], w_dev, sig_dev, cb, (dd*)ps.wk, ps.wabs);
      else
        k_gather_points<double><<<blocks_for(n, 256), 256, 0, st>>>(
            ps.perm, n, d, l0_tmp, xi_tmp, ps.cell0[0], ps.cell0[1], ps.cell0[2], (double*)ps.xi[0],
            (double*)ps.xi[1], (double*)ps.xi[2], w_dev, sig_dev, cb, (double*)ps.wk, ps.wabs);
    }
    chk(cudaGetLastError());
    if (n > 0 && psi_tabulated(plan) && e == cudaSuccess) {
      const int W = h.width;
      for (int a = 0; a < d; ++a) ps.psi[a] = alloc(actx, rs * nn * W);
      if (plan.precision == GP_DF64)
        k_psi_tables<dd><<<blocks_for(n * W, 256), 256, 0, st>>>(
            n, d, W, (const dd*)ps.xi[0], (const dd*)ps.xi[1], (const dd*)ps.xi[2], es_beta_arg<dd>(h.beta),
            dd(2.0 / h.width), (dd*)ps.psi[0], (dd*)ps.psi[1], (dd*)ps.psi[2]);
      else
        k_psi_tables<double><<<blocks_for(n * W, 256), 256, 0, st>>>(
            n, d, W, (const double*)ps.xi[0], (const double*)ps.xi[1], (const double*)ps.xi[2],
            es_beta_arg<double>(h.beta), 2.0 / h.width, (double*)ps.psi[0], (double*)ps.psi[1],
            (double*)ps.psi[2]);
      chk(cudaGetLastError());
    }
    chk(cudaMemcpyAsync(&hbad, bad, sizeof(hbad), cudaMemcpyDeviceToHost, st));
    chk(cudaStreamSynchronize(st));
  }
  cudaFree(l0_tmp);
  cudaFree(xi_tmp);
  cudaFree(keys);
  cudaFree(keys_sorted);
  cudaFree(idx);
  cudaFree(bad);
  cudaFree(cub_tmp);
  GPN_CUDA(e);
  GPN_CHECK(hbad == 0, GP_EINVAL, std::to_string(hbad) + " points outside the plan box");
  // list of non-empty bins (the interp launch set)
  std::vector<int> hs(ps.nbins_total + 1);
  GPN_CUDA(cudaMemcpy(hs.data(), ps.bin_start, sizeof(int) * hs.size(), cudaMemcpyDeviceToHost));
  std::vector<int> act;
  for (long long b = 0; b < ps.nbins_total; ++b)
    if (hs[b + 1] > hs[b]) act.push_back((int)b);
  ps.n_active_bins = (long long)act.size();
  ps.active_bins = (int*)alloc(actx, sizeof(int) * std::max<size_t>(act.size(), 1));
  if (!act.empty())
    GPN_CUDA(cudaMemcpy(ps.active_bins, act.data(), sizeof(int) * act.size(), cudaMemcpyHostToDevice));
  if (bin_start_host) bin_start_host->swap(hs);
}

// Exact diagonal correction (an extension for small nu): defect_i = K_ii - K~_ii with
//   K_ii = w_i^2 (4 pi sigma_i^2)^(-d/2)                    Eq. (nonstat2) at x = y
//   K~_ii = sum_kl w_k(x_i) w_l(x_i) S_kl,  S = sum_{n in {-M..M}^d} A[n]   Eq. (Ktilde) at x = y
// A[n] = sum_j v~_j G^_kj[n] G^_lj[n] (Remark rem:step3, without the NUFFT deconvolution)
// is a product over dimensions, so S_kl = sum_j v~_j (sum_{|m|<=M} e_kj(m) e_lj(m))^d with
// e_kj(m) = sqrt(2 pi) sigma_k chi_j exp(-2 pi^2 (sigma_k chi_j dw m)^2).  The defect is
// stored in sorted order (float64) and added to the matvec's shift term.
void build_diag_correction(Plan& plan, const double* w_dev, const double* sig_dev, cudaStream_t st) {
  const Hyper& h = plan.h;
  const Tables& tb = plan.tb;
  const int C = plan.geom.C, J = (int)tb.vt.size(), d = h.d;
  std::vector<double> S((size_t)C * C, 0.0);
  for (int j = 0; j < J; ++j)
    for (int k = 0; k < C; ++k)
      for (int l = k; l < C; ++l) {
        double s1 = 0.0;
        for (long long m = h.M; m >= 0; --m) {   // small terms first
          const double ak = tb.nodes[k] * tb.chi[j] * h.dw * (double)m;
          const double al = tb.nodes[l] * tb.chi[j] * h.dw * (double)m;
          const double pk = std::sqrt(2.0 * kPi) * tb.nodes[k] * tb.chi[j] * std::exp(-2.0 * kPi * kPi * ak * ak);
          const double pl = std::sqrt(2.0 * kPi) * tb.nodes[l] * tb.chi[j] * std::exp(-2.0 * kPi * kPi * al * al);
          s1 += (m == 0 ? 1.0 : 2.0) * pk * pl;
        }
        const double v = tb.vt[j] * std::pow(s1, d);
        S[(size_t)k * C + l] += v;
        if (l != k) S[(size_t)l * C + k] += v;
      }
  plan.dcorr = (double*)plan.alloc(sizeof(double) * (size_t)std::max<long long>(plan.N, 1));
  double* Sd = nullptr;
  GPN_CUDA(cudaMalloc(&Sd, sizeof(double) * S.size()));
  cudaError_t e = cudaMemcpyAsync(Sd, S.data(), sizeof(double) * S.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && plan.N > 0) {
    ChebArgs cb{};
    cb.C = C;
    cb.d = d;
    for (int k = 0; k < C; ++k) {
      cb.nodes[k] = tb.nodes[k];
      cb.bary[k] = tb.bary[k];
    }
    k_diag_defect<<<blocks_for(plan.N, 256), 256, 0, st>>>(plan.pts.perm, plan.N, w_dev, sig_dev, cb, Sd, plan.dcorr);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(Sd);
  GPN_CUDA(e);
}

}  // namespace gpn
