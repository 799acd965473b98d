// Conjugate gradients for (K~ + eta^2 I) alpha = y (Eq. gprsolve; Sec. 6.2 wraps the
// matvec in CG without a preconditioner).  All vectors are float64 in the plan's
// sorted point order; each of the R columns runs its own CG and all columns share
// every matvec launch.  Inner products are two-stage block reductions in a fixed
// order, so results do not depend on scheduling.
//
// Device scalars (plan.scal), per column r of R:
//   [0] rr = ||r||^2   [1] pAp   [2] rr_new   [3] yy = ||y||^2   [4] active (1/0)
// Convergence and breakdown are decided on the device at the end of every iteration
// (k_cg_check), so the host runs blocks of iterations and looks at the flags once per
// block; a full block is replayed from a CUDA graph captured once per solve.
#include <cmath>
#include <vector>

#include "plan.h"

namespace gpn {

namespace {

constexpr int kRedBlocks = 512;
constexpr int kRedThreads = 256;

__device__ __forceinline__ double block_sum(double v) {
  __shared__ double sh[kRedThreads / 32];
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x < 32) {
    s = (lane < kRedThreads / 32) ? sh[lane] : 0.0;
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  }
  __syncthreads();
  return s;
}

// partial[r * kRedBlocks + b] = sum over block b's chunk of u[:, r] . v[:, r]
__global__ void __launch_bounds__(kRedThreads) k_dot_partial(const double* __restrict__ u,
                                                              const double* __restrict__ v, long long n,
                                                              double* __restrict__ partial) {
  int r = blockIdx.y;
  const double* ur = u + (size_t)r * n;
  const double* vr = v + (size_t)r * n;
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    acc += ur[i] * vr[i];
  double s = block_sum(acc);
  if (threadIdx.x == 0) partial[(size_t)r * kRedBlocks + blockIdx.x] = s;
}

// out[slot * R + r] = sum_b partial[r][b]
__global__ void __launch_bounds__(kRedThreads) k_dot_final(const double* __restrict__ partial, int nblk,
                                                            double* __restrict__ scal, int slot, int R) {
  int r = blockIdx.x;
  double acc = 0.0;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) acc += partial[(size_t)r * kRedBlocks + b];
  double s = block_sum(acc);
  if (threadIdx.x == 0) scal[slot * R + r] = s;
}

// x += a p, r -= a Ap for active columns (a = rr / pAp), and partial sums of r.r.
__global__ void __launch_bounds__(kRedThreads) k_update_xr(double* __restrict__ x, double* __restrict__ res,
                                                            const double* __restrict__ p,
                                                            const double* __restrict__ ap, long long n,
                                                            const double* __restrict__ scal, int R,
                                                            double* __restrict__ partial) {
  int r = blockIdx.y;
  bool active = scal[4 * R + r] != 0.0;
  double a = active ? scal[0 * R + r] / scal[1 * R + r] : 0.0;
  double* xr = x + (size_t)r * n;
  double* rr = res + (size_t)r * n;
  const double* pr = p + (size_t)r * n;
  const double* apr = ap + (size_t)r * n;
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    double ri = rr[i];
    if (active) {
      xr[i] += a * pr[i];
      ri -= a * apr[i];
      rr[i] = ri;
    }
    acc += ri * ri;
  }
  double s = block_sum(acc);
  if (threadIdx.x == 0) partial[(size_t)r * kRedBlocks + blockIdx.x] = s;
}

// p = r + (rr_new / rr) p for active columns; then rr = rr_new.
__global__ void __launch_bounds__(kRedThreads) k_update_p(double* __restrict__ p, const double* __restrict__ res,
                                                           long long n, const double* __restrict__ scal, int R) {
  int r = blockIdx.y;
  if (scal[4 * R + r] == 0.0) return;
  double b = scal[2 * R + r] / scal[0 * R + r];
  double* pr = p + (size_t)r * n;
  const double* rr = res + (size_t)r * n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    pr[i] = rr[i] + b * pr[i];
}

__global__ void k_roll_scalars(double* scal, int R) {
  int r = threadIdx.x;
  if (r < R && scal[4 * R + r] != 0.0) scal[0 * R + r] = scal[2 * R + r];
}

// End of an iteration: count it for every column that was active, and stop the columns
// that converged (rr_new <= rtol^2 yy) or broke down (pAp <= 0 or not finite).
// cnt[R] is set to 1 on a breakdown.
__global__ void k_cg_check(double* scal, int R, double rtol2, int* cnt) {
  const int r = threadIdx.x;
  if (r >= R || scal[4 * R + r] == 0.0) return;
  cnt[r] += 1;
  const double pap = scal[1 * R + r], rrn = scal[2 * R + r];
  if (!(pap > 0.0) || !isfinite(pap) || !isfinite(rrn)) {
    scal[4 * R + r] = 0.0;
    cnt[R] = 1;
  } else if (rrn <= rtol2 * scal[3 * R + r]) {
    scal[4 * R + r] = 0.0;
  }
}

__global__ void k_axpy_cols(double* __restrict__ y, const double* __restrict__ x, double a, long long total) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x)
    y[i] += a * x[i];
}

// num_i += sum_r z_ri x_ri, den_i += sum_r z_ri^2 (probe estimate of a diagonal)
__global__ void k_probe_accum(const double* __restrict__ z, const double* __restrict__ x, long long n, int R,
                              double* __restrict__ num, double* __restrict__ den) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    double a = 0.0, b = 0.0;
    for (int r = 0; r < R; ++r) {
      const double zi = z[(size_t)r * n + i];
      a += zi * x[(size_t)r * n + i];
      b += zi * zi;
    }
    num[i] += a;
    den[i] += b;
  }
}

// var_i = eta2 - eta2^2 num_i / den_i
__global__ void k_variance_finish(const double* __restrict__ num, const double* __restrict__ den, long long n,
                                  double eta2, double* __restrict__ var) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    var[i] = den[i] > 0.0 ? eta2 - eta2 * eta2 * (num[i] / den[i]) : eta2;
}

int red_blocks(long long n) { return (int)std::max<long long>(1, std::min<long long>(kRedBlocks, (n + kRedThreads - 1) / kRedThreads)); }

void dot(const double* u, const double* v, long long n, int R, double* partial, double* scal, int slot,
         cudaStream_t st) {
  int nb = red_blocks(n);
  k_dot_partial<<<dim3(nb, R), kRedThreads, 0, st>>>(u, v, n, partial);
  k_dot_final<<<R, kRedThreads, 0, st>>>(partial, nb, scal, slot, R);
}

void read_scalars(Plan& plan, int R, cudaStream_t st) {
  GPN_CUDA(cudaGetLastError());
  GPN_CUDA(cudaMemcpyAsync(plan.host_scal, plan.scal, sizeof(double) * 5 * R, cudaMemcpyDeviceToHost, st));
  check_device_status(plan, st);
}

}  // namespace

// iterations per host check (and per captured graph)
constexpr int kCgBlock = 16;

void cg_iteration(Plan& plan, double* xr, int R, double eta2, double rtol, cudaStream_t st) {
  const long long n = plan.N;
  const int nb = red_blocks(n);
  double* r = plan.cg_r;
  double* p = plan.cg_p;
  double* ap = plan.cg_ap;
  matvec_sorted(plan, p, ap, R, eta2, st);
  dot(p, ap, n, R, plan.partials, plan.scal, 1, st);
  k_update_xr<<<dim3(nb, R), kRedThreads, 0, st>>>(xr, r, p, ap, n, plan.scal, R, plan.partials);
  k_dot_final<<<R, kRedThreads, 0, st>>>(plan.partials, nb, plan.scal, 2, R);
  k_update_p<<<dim3(nb, R), kRedThreads, 0, st>>>(p, r, n, plan.scal, R);
  k_roll_scalars<<<1, ((R + 31) / 32) * 32, 0, st>>>(plan.scal, R);
  k_cg_check<<<1, ((R + 31) / 32) * 32, 0, st>>>(plan.scal, R, rtol * rtol, plan.cg_cnt);
}

// A graph of kCgBlock iterations for (x, R, eta2, rtol); false when it cannot be made
// (the caller then launches the iterations directly).
bool cg_graph(Plan& plan, double* xr, int R, double eta2, double rtol) {
  CgGraph& g = plan.cg_graph;
  if (g.exec && g.x == xr && g.R == R && g.eta2 == eta2 && g.rtol == rtol) return true;
  if (g.exec) {
    cudaGraphExecDestroy(g.exec);
    g.exec = nullptr;
  }
  if (!plan.cap_stream && cudaStreamCreateWithFlags(&plan.cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    plan.cap_stream = nullptr;
    return false;
  }
  if (cudaStreamBeginCapture(plan.cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  bool ok = true;
  try {
    for (int i = 0; i < kCgBlock; ++i) cg_iteration(plan, xr, R, eta2, rtol, plan.cap_stream);
  } catch (const Error&) {
    ok = false;
  }
  cudaGraph_t graph = nullptr;
  const cudaError_t e = cudaStreamEndCapture(plan.cap_stream, &graph);
  ok = ok && e == cudaSuccess && graph != nullptr;
  if (ok) ok = cudaGraphInstantiate(&g.exec, graph, 0) == cudaSuccess;
  if (graph) cudaGraphDestroy(graph);
  if (!ok) {
    cudaGetLastError();
    g.exec = nullptr;
    return false;
  }
  g.x = xr;
  g.R = R;
  g.eta2 = eta2;
  g.rtol = rtol;
  return true;
}

int cg_solve_sorted(Plan& plan, const double* y_sorted, double* x_sorted, int R, double eta2, double rtol, int maxit,
                    int* iters, double* relres, cudaStream_t st) {
  const long long n = plan.N;
  const size_t bytes = sizeof(double) * n * R;
  double* xr = x_sorted;
  GPN_CUDA(cudaMemsetAsync(xr, 0, bytes, st));
  GPN_CUDA(cudaMemcpyAsync(plan.cg_r, y_sorted, bytes, cudaMemcpyDeviceToDevice, st));
  GPN_CUDA(cudaMemcpyAsync(plan.cg_p, y_sorted, bytes, cudaMemcpyDeviceToDevice, st));
  GPN_CUDA(cudaMemsetAsync(plan.cg_cnt, 0, sizeof(int) * (R + 1), st));
  dot(plan.cg_r, plan.cg_r, n, R, plan.partials, plan.scal, 0, st);
  dot(y_sorted, y_sorted, n, R, plan.partials, plan.scal, 3, st);
  read_scalars(plan, R, st);
  std::vector<double> hs(plan.host_scal, plan.host_scal + 5 * R);
  bool any = false;
  for (int c = 0; c < R; ++c) {
    const double yy = hs[3 * R + c];
    const bool active = !(yy == 0.0 || std::sqrt(hs[0 * R + c] / yy) <= rtol);
    hs[4 * R + c] = active ? 1.0 : 0.0;
    any = any || active;
  }
  GPN_CUDA(cudaMemcpyAsync(plan.scal + 4 * R, &hs[4 * R], sizeof(double) * R, cudaMemcpyHostToDevice, st));
  // graphs need no profiling events inside, and the first iterations create any lazy
  // transform plans outside a capture
  const bool use_graph = !plan.prof.on;
  bool captured = false;
  int done = 0;
  while (any && done < maxit) {
    const int k = std::min(kCgBlock, maxit - done);
    if (use_graph && k == kCgBlock && done > 0 && (captured || cg_graph(plan, xr, R, eta2, rtol))) {
      captured = true;
      GPN_CUDA(cudaGraphLaunch(plan.cg_graph.exec, st));
    } else {
      for (int i = 0; i < k; ++i) cg_iteration(plan, xr, R, eta2, rtol, st);
    }
    done += k;
    read_scalars(plan, R, st);
    any = false;
    for (int c = 0; c < R; ++c) any = any || plan.host_scal[4 * R + c] != 0.0;
  }
  std::vector<int> cnt(R + 1, 0);
  GPN_CUDA(cudaMemcpyAsync(cnt.data(), plan.cg_cnt, sizeof(int) * (R + 1), cudaMemcpyDeviceToHost, st));
  read_scalars(plan, R, st);
  bool unconverged = false;
  for (int c = 0; c < R; ++c) {
    const double yy = plan.host_scal[3 * R + c];
    const double rel = yy > 0.0 ? std::sqrt(plan.host_scal[0 * R + c] / yy) : 0.0;
    if (iters) iters[c] = cnt[c];
    if (relres) relres[c] = rel;
    if (plan.host_scal[4 * R + c] != 0.0) unconverged = true;
  }
  if (cnt[R]) return GP_EBREAKDOWN;
  return unconverged ? GP_ENOTCONV : GP_OK;
}

void probe_accumulate(const double* z_sorted, const double* x_sorted, long long n, int R, double* num, double* den,
                      cudaStream_t st) {
  k_probe_accum<<<(int)std::min<long long>(4096, (n + 255) / 256), 256, 0, st>>>(z_sorted, x_sorted, n, R, num, den);
  GPN_CUDA(cudaGetLastError());
}

void variance_finish(const double* num, const double* den, long long n, double eta2, double* var, cudaStream_t st) {
  k_variance_finish<<<(int)std::min<long long>(4096, (n + 255) / 256), 256, 0, st>>>(num, den, n, eta2, var);
  GPN_CUDA(cudaGetLastError());
}

int cg_refined_sorted(Plan& lo, Plan& hi, const double* y_hi_sorted, double* x_hi_sorted, int R, double eta2,
                      double rtol, double inner_rtol, int outer_max, int maxit, int* iters, double* relres,
                      cudaStream_t st) {
  // Outer iterative refinement in hi's sorted order; inner CG in lo's sorted order.
  const long long n = hi.N;
  const size_t bytes = sizeof(double) * n * R;
  double* x = x_hi_sorted;
  double* res = hi.vec_a;       // residual (hi order)
  double* tmp = hi.vec_b;       // K x (hi order)
  double* orig = hi.cg_r;       // caller-order scratch
  double* rhs_lo = lo.vec_a;    // residual in lo order
  double* d_lo = lo.cg_x;       // correction in lo order
  GPN_CUDA(cudaMemsetAsync(x, 0, bytes, st));
  std::vector<int> total(R, 0);
  std::vector<int> inner_it(R, 0);
  std::vector<double> inner_rel(R, 0.0);
  dot(y_hi_sorted, y_hi_sorted, n, R, hi.partials, hi.scal, 3, st);
  read_scalars(hi, R, st);
  std::vector<double> yy(R);
  for (int c = 0; c < R; ++c) yy[c] = hi.host_scal[3 * R + c];
  int status = GP_ENOTCONV;
  std::vector<double> rel(R, 1.0);
  for (int outer = 0; outer <= outer_max; ++outer) {
    // res = y - (K~_hi + eta2 I) x
    if (outer == 0) {
      GPN_CUDA(cudaMemcpyAsync(res, y_hi_sorted, bytes, cudaMemcpyDeviceToDevice, st));
    } else {
      matvec_sorted(hi, x, tmp, R, eta2, st);
      GPN_CUDA(cudaMemcpyAsync(res, y_hi_sorted, bytes, cudaMemcpyDeviceToDevice, st));
      k_axpy_cols<<<1024, 256, 0, st>>>(res, tmp, -1.0, (long long)n * R);
    }
    dot(res, res, n, R, hi.partials, hi.scal, 0, st);
    read_scalars(hi, R, st);
    bool done = true;
    for (int c = 0; c < R; ++c) {
      rel[c] = yy[c] > 0.0 ? std::sqrt(hi.host_scal[c] / yy[c]) : 0.0;
      if (rel[c] > rtol) done = false;
    }
    if (done) {
      status = GP_OK;
      break;
    }
    if (outer == outer_max) break;
    // move the residual to lo's order, solve, and add the correction back
    scatter_sorted(hi.pts, res, orig, R, st);
    gather_sorted(lo.pts, orig, rhs_lo, R, st);
    int s = cg_solve_sorted(lo, rhs_lo, d_lo, R, eta2, inner_rtol, maxit, inner_it.data(), inner_rel.data(), st);
    if (s == GP_EBREAKDOWN) return s;
    for (int c = 0; c < R; ++c) total[c] += inner_it[c];
    scatter_sorted(lo.pts, d_lo, orig, R, st);
    gather_sorted(hi.pts, orig, tmp, R, st);
    k_axpy_cols<<<1024, 256, 0, st>>>(x, tmp, 1.0, (long long)n * R);
    GPN_CUDA(cudaGetLastError());
  }
  for (int c = 0; c < R; ++c) {
    if (iters) iters[c] = total[c];
    if (relres) relres[c] = rel[c];
  }
  return status;
}

}  // namespace gpn
