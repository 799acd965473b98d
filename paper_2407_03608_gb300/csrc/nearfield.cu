// Near-field correction (an extension for small nu, not in the paper).
//
// For the Matern family with small nu, phi has a cusp at r = 0, and the Fourier modes
// {-M..M}^d on the grid leave out the slowly decaying tail of its transform: K~ (Eq.
// Ktilde) falls short of K (Eq. nonstat2) over a neighbourhood of the diagonal.  With
// gp_plan_opts.near_radius = r_c > 0 the plan stores, for every pair of distinct points
// closer than r_c, the exact defect K_ij - K~_ij (CSR in sorted order, float64), and every
// matvec on the plan's points adds
//   out_i += sum_{j != i, |x_i - x_j| < r_c} (K_ij - K~_ij) alpha_j.
//
// K_ij: Eq. (nonstat2) with the closed forms of phi (nu = 1/2, 3/2, 5/2; squared exponential).
// K~_ij: Eq. (Ktilde) with the multiplier of Lemma stage3warmup,
//   G^_kj[n] = prod_a e_kj(n_a),  e_kj(m) = sqrt(2 pi) sigma_k chi_j exp(-2 pi^2 (sigma_k chi_j dw m)^2);
// the grid {-M..M}^d is a product of symmetric ranges and the summand is even in each n_a,
// so the sum over the grid factors by dimension:
//   K~(x, y) = sum_j v~_j sum_{k,l} w_k(x) w_l(y) prod_a t_klj(x_a - y_a),
//   t_klj(rho) = sum_{|m|<=M} e_kj(m) e_lj(m) cos(2 pi m dw rho)
//             = 2 pi sigma_k sigma_l chi_j^2 (1 + 2 sum_{m=1}^{M} exp(-a m^2) cos(m theta)),
//   a = 2 pi^2 (sigma_k^2 + sigma_l^2) chi_j^2 dw^2,  theta = 2 pi dw rho.
// The factors are tabulated once per plan on a uniform grid of rho in [0, r_c] (spacing
// h = 0.08 / (2 pi M dw), so that 8-point Lagrange interpolation of a function with
// frequencies up to M dw is exact to about 2e-12 of its size), then read per pair.
#include <cub/cub.cuh>

#include <climits>
#include <cmath>
#include <vector>

#include "kernels.h"

namespace gpn {

namespace {

constexpr double kPiNF = 3.14159265358979323846;
constexpr int kLagrange = 8;    // interpolation points
constexpr int kTabPad = 4;      // table entry q holds rho = (q - kTabPad) h (mirrored below 0)

struct NearTabArgs {
  const double* nodes;   // sigma_k, C of them
  const double* chi;     // chi_j, J of them
  double* tab;           // [pair (k <= l)][j][nq]
  int C, J, nq;
  long long M;
  double dw, h;
};

// t_klj at rho = (q - kTabPad) h for one (pair, j, q): the sum over m by recurrences (the
// Gaussian factor through its ratio exp(-a (2m + 1)), the cosine by cos((m+1) th) =
// 2 cos(th) cos(m th) - cos((m-1) th)), stopped once the Gaussian is below 1e-30.
__global__ void k_near_tables(NearTabArgs a) {
  const long long id = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long npair = (long long)a.C * (a.C + 1) / 2;
  if (id >= npair * a.J * a.nq) return;
  const int q = (int)(id % a.nq);
  const long long pj = id / a.nq;
  const int j = (int)(pj % a.J);
  int p = (int)(pj / a.J), k = 0;
  while (p >= a.C - k) {     // pair index -> (k, l), k <= l, packed row by row
    p -= a.C - k;
    ++k;
  }
  const int l = k + p;
  const double sk = a.nodes[k] * a.chi[j], sl = a.nodes[l] * a.chi[j];
  const double aa = 2.0 * kPiNF * kPiNF * (sk * sk + sl * sl) * a.dw * a.dw;
  const double rho = (double)(q - kTabPad) * a.h;
  const double th = 2.0 * kPiNF * a.dw * rho;
  const double c1 = cos(th);
  double cm = c1, cprev = 1.0;          // cos(m th), cos((m-1) th) at m = 1
  double g = exp(-aa), ratio = exp(-3.0 * aa);
  const double step = exp(-2.0 * aa);
  double sum = 0.0;
  for (long long m = 1; m <= a.M && g > 1e-30; ++m) {
    sum += g * cm;
    const double cn = 2.0 * c1 * cm - cprev;
    cprev = cm;
    cm = cn;
    g *= ratio;
    ratio *= step;
  }
  a.tab[id] = 2.0 * kPiNF * sk * sl * (1.0 + 2.0 * sum);
}

// phi of Eq. (matern) in closed form (nu = 1/2, 3/2, 5/2) or Eq. (squaredexp)
__device__ __forceinline__ double phi_closed(int family, double nu, double r) {
  if (family == GP_SE) return exp(-0.5 * r * r);
  if (nu == 0.5) return exp(-r);
  if (nu == 1.5) {
    const double z = 1.7320508075688772935 * r;
    return (1.0 + z) * exp(-z);
  }
  const double z = 2.2360679774997896964 * r;   // nu = 5/2
  return (1.0 + z + z * z / 3.0) * exp(-z);
}

struct NearPairArgs {
  const double* x;       // caller order, n x d
  const double* w;       // paper fields, caller order
  const double* sig;
  const int* perm;       // sorted -> caller
  const int* cell0[kMaxDim];
  const int* bin_start;
  int nbins[kMaxDim];
  int tile;
  int reach;             // neighbour bins each way
  long long n;
  int d;
  double r2;             // r_c^2
  int family;
  double nu;
  ChebArgs cb;
  const double* vt;      // v~_j
  const double* tab;     // t_klj tables
  int J, nq;
  double inv_h;          // 1 / table spacing
  const int* row_ptr;    // fill pass: CSR offsets (null in the count pass)
  int* count;            // count pass: pairs per row
  int* col;              // fill pass
  double* val;
};

// K~ of one pair by the separable form (tables interpolated per dimension)
__device__ double ktilde_pair(const NearPairArgs& a, const double* wi, const double* wj, const double* dx) {
  // Lagrange weights and first table entry per dimension
  double lw[kMaxDim][kLagrange];
  int q0[kMaxDim];
  for (int ax = 0; ax < a.d; ++ax) {
    const double u = fabs(dx[ax]) * a.inv_h;
    const int base = (int)floor(u) - (kLagrange / 2 - 1);     // nodes base .. base + 7
    const double s = u - base;                                 // in [3, 4)
    q0[ax] = base + kTabPad;
    for (int i = 0; i < kLagrange; ++i) {
      double num = 1.0, den = 1.0;
      for (int t = 0; t < kLagrange; ++t)
        if (t != i) {
          num *= s - t;
          den *= (double)(i - t);
        }
      lw[ax][i] = num / den;
    }
  }
  const int C = a.cb.C;
  double total = 0.0;
  int p = 0;
  for (int k = 0; k < C; ++k)
    for (int l = k; l < C; ++l, ++p) {
      const double wkl = (k == l) ? wi[k] * wj[k] : wi[k] * wj[l] + wi[l] * wj[k];
      if (wkl == 0.0) continue;
      double s = 0.0;
      for (int j = 0; j < a.J; ++j) {
        const double* t = a.tab + ((size_t)p * a.J + j) * a.nq;
        double prod = a.vt[j];
        for (int ax = 0; ax < a.d; ++ax) {
          const double* tq = t + q0[ax];
          double f = 0.0;
#pragma unroll
          for (int i = 0; i < kLagrange; ++i) f += lw[ax][i] * tq[i];
          prod *= f;
        }
        s += prod;
      }
      total += wkl * s;
    }
  return total;
}

// One thread per sorted point i: visits the bins within `reach` of its own, and for every
// other point j closer than r_c counts the pair (count pass) or writes j and K_ij - K~_ij
// (fill pass, in visiting order).
__global__ void k_near_pairs(NearPairArgs a) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  const long long ci = a.perm[i];
  double xi[kMaxDim], wi[kMaxChannels], wj[kMaxChannels];
  for (int ax = 0; ax < a.d; ++ax) xi[ax] = a.x[ci * a.d + ax];
  const double si = a.sig[ci], wpi = a.w[ci];
  cheb_weights(wpi, si, a.cb, wi);
  int bi[kMaxDim] = {0, 0, 0}, lo[kMaxDim] = {0, 0, 0}, hi[kMaxDim] = {0, 0, 0};
  for (int ax = 0; ax < a.d; ++ax) {
    bi[ax] = min(a.cell0[ax][i] / a.tile, a.nbins[ax] - 1);
    lo[ax] = max(0, bi[ax] - a.reach);
    hi[ax] = min(a.nbins[ax] - 1, bi[ax] + a.reach);
  }
  int cnt = 0;
  const long long off = a.row_ptr ? a.row_ptr[i] : 0;
  int b[kMaxDim];
  for (b[0] = lo[0]; b[0] <= hi[0]; ++b[0])
    for (b[1] = (a.d > 1 ? lo[1] : 0); b[1] <= (a.d > 1 ? hi[1] : 0); ++b[1])
      for (b[2] = (a.d > 2 ? lo[2] : 0); b[2] <= (a.d > 2 ? hi[2] : 0); ++b[2]) {
        long long lin = 0;
        for (int ax = 0; ax < a.d; ++ax) lin = lin * a.nbins[ax] + b[ax];
        const int s0 = a.bin_start[lin], s1 = a.bin_start[lin + 1];
        for (int jj = s0; jj < s1; ++jj) {
          if (jj == i) continue;
          const long long cj = a.perm[jj];
          double dx[kMaxDim], r2 = 0.0;
          for (int ax = 0; ax < a.d; ++ax) {
            dx[ax] = xi[ax] - a.x[cj * a.d + ax];
            r2 += dx[ax] * dx[ax];
          }
          if (r2 >= a.r2) continue;
          if (a.row_ptr) {
            const double sj = a.sig[cj], wpj = a.w[cj];
            cheb_weights(wpj, sj, a.cb, wj);
            const double ss = si * si + sj * sj;
            const double kij = wpi * wpj * pow(2.0 * kPiNF * ss, -0.5 * a.d) * phi_closed(a.family, a.nu, sqrt(r2 / ss));
            a.col[off + cnt] = jj;
            a.val[off + cnt] = kij - ktilde_pair(a, wi, wj, dx);
          }
          ++cnt;
        }
      }
  if (!a.row_ptr) a.count[i] = cnt;
}

// out[r n + i] += sum_e val[e] alpha[r n + col[e]] over row i's pairs (sorted order)
__global__ void k_near_apply(const int* __restrict__ row_ptr, const int* __restrict__ col,
                             const double* __restrict__ val, const double* __restrict__ alpha,
                             double* __restrict__ out, long long n, int R) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int e0 = row_ptr[i], e1 = row_ptr[i + 1];
  for (int r = 0; r < R; ++r) {
    const double* ar = alpha + (size_t)r * n;
    double s = 0.0;
    for (int e = e0; e < e1; ++e) s += val[e] * ar[col[e]];
    out[(size_t)r * n + i] += s;
  }
}

}  // namespace

bool near_field_supported(int family, double nu) {
  return family == GP_SE || nu == 0.5 || nu == 1.5 || nu == 2.5;
}

void build_near_field(Plan& plan, double radius, const double* x_dev, const double* w_dev, const double* sig_dev,
                      cudaStream_t st) {
  const Hyper& h = plan.h;
  const Tables& tb = plan.tb;
  const int C = plan.geom.C, d = h.d, J = (int)tb.vt.size();
  GPN_CHECK(near_field_supported(h.family, h.nu), GP_EUNSUPPORTED,
            "the near-field correction needs nu = 1/2, 3/2, 5/2 or the squared exponential");
  GPN_CHECK(radius > 0.0 && std::isfinite(radius), GP_EINVAL, "near_radius must be > 0");
  const long long n = plan.N;
  const double spacing = 0.08 / (2.0 * kPiNF * (double)std::max<long long>(h.M, 1) * h.dw);
  const double nq_d = std::ceil(radius / spacing) + 10.0;
  const long long npair = (long long)C * (C + 1) / 2;
  const double tab_bytes = 8.0 * (double)npair * J * nq_d;
  GPN_CHECK(tab_bytes <= 16e9, GP_ENOMEM,
            "near-field tables of " + std::to_string((long long)tab_bytes) + " bytes: take a smaller near_radius");
  const int nq = (int)nq_d;
  // tables of t_klj
  std::vector<double> host(C + J + J);
  for (int k = 0; k < C; ++k) host[k] = tb.nodes[k];
  for (int j = 0; j < J; ++j) host[C + j] = tb.chi[j];
  for (int j = 0; j < J; ++j) host[C + J + j] = tb.vt[j];
  double* small = (double*)plan.alloc(sizeof(double) * host.size());
  GPN_CUDA(cudaMemcpyAsync(small, host.data(), sizeof(double) * host.size(), cudaMemcpyHostToDevice, st));
  double* tab = (double*)plan.alloc((size_t)tab_bytes);
  NearTabArgs ta{small, small + C, tab, C, J, nq, h.M, h.dw, spacing};
  const long long ntab = npair * J * nq;
  k_near_tables<<<(unsigned)((ntab + 255) / 256), 256, 0, st>>>(ta);
  GPN_CUDA(cudaGetLastError());
  // pairs: count, offsets, fill
  const PointSet& ps = plan.pts;
  NearPairArgs a{};
  a.x = x_dev;
  a.w = w_dev;
  a.sig = sig_dev;
  a.perm = ps.perm;
  for (int ax = 0; ax < kMaxDim; ++ax) {
    a.cell0[ax] = ps.cell0[ax];
    a.nbins[ax] = ps.nbins[ax];
  }
  a.bin_start = ps.bin_start;
  a.tile = h.tile;
  const double cell = 1.0 / (h.dw * (double)h.nf);    // fine-grid spacing in x units
  a.reach = (int)std::ceil(radius / (cell * h.tile)) + 1;
  a.n = n;
  a.d = d;
  a.r2 = radius * radius;
  a.family = h.family;
  a.nu = h.nu;
  a.cb.C = C;
  a.cb.d = d;
  for (int k = 0; k < C; ++k) {
    a.cb.nodes[k] = tb.nodes[k];
    a.cb.bary[k] = tb.bary[k];
  }
  a.vt = small + C + J;
  a.tab = tab;
  a.J = J;
  a.nq = nq;
  a.inv_h = 1.0 / spacing;
  int* ptr = (int*)plan.alloc(sizeof(int) * (size_t)(n + 1));
  a.count = ptr;
  const unsigned nb = (unsigned)((n + 127) / 128);
  k_near_pairs<<<nb, 128, 0, st>>>(a);
  GPN_CUDA(cudaGetLastError());
  // the total in 64 bits first: the row offsets are ints
  {
    std::vector<int> counts((size_t)n);
    GPN_CUDA(cudaMemcpyAsync(counts.data(), ptr, sizeof(int) * (size_t)n, cudaMemcpyDeviceToHost, st));
    GPN_CUDA(cudaStreamSynchronize(st));
    long long sum = 0;
    for (int c : counts) sum += c;
    GPN_CHECK(sum <= (long long)INT_MAX, GP_ENOMEM,
              std::to_string(sum) + " near-field pairs: more than the int row offsets hold; take a smaller near_radius");
  }
  // exclusive scan of the counts into the row offsets (the last entry is the total)
  GPN_CUDA(cudaMemsetAsync(ptr + n, 0, sizeof(int), st));
  size_t tmp_bytes = 0;
  GPN_CUDA(cub::DeviceScan::ExclusiveSum(nullptr, tmp_bytes, ptr, ptr, (int)(n + 1), st));
  void* tmp = nullptr;
  GPN_CUDA(cudaMalloc(&tmp, std::max<size_t>(tmp_bytes, 16)));
  cudaError_t e = cub::DeviceScan::ExclusiveSum(tmp, tmp_bytes, ptr, ptr, (int)(n + 1), st);
  int total = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&total, ptr + n, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(tmp);
  GPN_CUDA(e);
  plan.near_ptr = ptr;
  plan.near_nnz = total;
  plan.near_col = (int*)plan.alloc(sizeof(int) * (size_t)std::max(total, 1));
  plan.near_val = (double*)plan.alloc(sizeof(double) * (size_t)std::max(total, 1));
  a.row_ptr = ptr;
  a.col = plan.near_col;
  a.val = plan.near_val;
  if (total > 0) k_near_pairs<<<nb, 128, 0, st>>>(a);
  GPN_CUDA(cudaGetLastError());
  GPN_CUDA(cudaStreamSynchronize(st));
  plan.near_radius = radius;
}

void launch_near_apply(Plan& plan, const double* alpha_sorted, double* out_sorted, int R, cudaStream_t st) {
  if (!plan.near_ptr || plan.near_nnz == 0 || plan.N == 0) return;
  k_near_apply<<<(unsigned)((plan.N + 127) / 128), 128, 0, st>>>(plan.near_ptr, plan.near_col, plan.near_val,
                                                                 alpha_sorted, out_sorted, plan.N, R);
  GPN_CUDA(cudaGetLastError());
}

}  // namespace gpn
