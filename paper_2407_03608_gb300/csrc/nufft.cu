// Matvec driver for K~ (Sec. 4.2 steps (1)-(5)), the cuFFT stages, and the
// plan-time build of the step-3 tensor A' (Remark rem:step3).
//
// Fine-grid convention: grid coordinate g = (x - centre)/h + nf/2 with h = 1/(dw nf);
// the points never come within width/2 cells of the grid edge, so no wrap-around
// is needed.  Type 1: U = FFT(u) with u[l] = sum_i c_i psi(l - g_i) gives
// b[n] = (-1)^n U[n]/psihat(n); type 2 mirrors it, so the (-1)^n phases cancel in
// the composition and step 3 only needs the real factor 1/psihat(n)^2, which is
// folded into A' = A / psihat^2.
#include <cufft.h>

#include <algorithm>
#include <cmath>

#include "ff64.h"
#include "plan.h"

namespace gpn {

namespace {

template <typename T>
struct ATensorArgs {
  const double* etab;   // [k][j][m]
  const double* vt;     // [j]
  T* A;
  long long n_freq;
  long long M;
  int C;
  int J;
  int d;
  int quad;             // 1: d = 2 quadrant layout [pair][m_1][m_0], m_a = 0..M
};

__global__ void k_build_a_f32(ATensorArgs<float> a);
__global__ void k_build_a_f64(ATensorArgs<double> a);

template <typename T>
__device__ void build_a_body(const ATensorArgs<T>& a) {
  long long f = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (f >= a.n_freq) return;
  long long m[kMaxDim];
  long long rest = f;
  if (a.quad) {
    m[0] = rest % (a.M + 1);
    m[1] = rest / (a.M + 1);
  } else {
    m[a.d - 1] = rest % (a.M + 1);
    rest /= (a.M + 1);
    for (int q = a.d - 2; q >= 0; --q) {
      long long v = rest % (2 * a.M + 1) - a.M;
      rest /= (2 * a.M + 1);
      m[q] = v < 0 ? -v : v;
    }
  }
  const long long Mp = a.M + 1;
  int p = 0;
  for (int k1 = 0; k1 < a.C; ++k1)
    for (int k2 = k1; k2 < a.C; ++k2, ++p) {
      double acc = 0.0;
      for (int j = 0; j < a.J; ++j) {
        const double* e1 = a.etab + ((size_t)k1 * a.J + j) * Mp;
        const double* e2 = a.etab + ((size_t)k2 * a.J + j) * Mp;
        double g = a.vt[j];
        for (int q = 0; q < a.d; ++q) g *= e1[m[q]] * e2[m[q]];
        acc += g;
      }
      a.A[(size_t)p * a.n_freq + f] = (T)acc;
    }
}

__global__ void k_build_a_f32(ATensorArgs<float> a) { build_a_body<float>(a); }
__global__ void k_build_a_f64(ATensorArgs<double> a) { build_a_body<double>(a); }
__global__ void k_build_a_dd(ATensorArgs<dd> a) { build_a_body<dd>(a); }

inline int blocks_for(long long n, int t) { return (int)((n + t - 1) / t); }

}  // namespace

void build_a_tensor(Plan& plan, cudaStream_t st) {
  const Hyper& h = plan.h;
  const int C = plan.geom.C;
  const int J = (int)plan.tb.vt.size();
  double *etab = nullptr, *vt = nullptr;
  cudaError_t e = cudaMalloc(&etab, sizeof(double) * plan.tb.etab.size());
  if (e == cudaSuccess) e = cudaMalloc(&vt, sizeof(double) * J);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(etab, plan.tb.etab.data(), sizeof(double) * plan.tb.etab.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(vt, plan.tb.vt.data(), sizeof(double) * J, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) {
    int nb = blocks_for(plan.n_freq, 128);
    if (plan.precision == GP_FP32) {
      ATensorArgs<float> a{etab, vt, (float*)plan.a_tensor, plan.n_freq, h.M, C, J, h.d, plan.tr3 ? 1 : 0};
      k_build_a_f32<<<nb, 128, 0, st>>>(a);
    } else if (plan.precision == GP_DF64) {
      ATensorArgs<dd> a{etab, vt, (dd*)plan.a_tensor, plan.n_freq, h.M, C, J, h.d, plan.tr3 ? 1 : 0};
      k_build_a_dd<<<nb, 128, 0, st>>>(a);
    } else {
      ATensorArgs<double> a{etab, vt, (double*)plan.a_tensor, plan.n_freq, h.M, C, J, h.d, plan.tr3 ? 1 : 0};
      k_build_a_f64<<<nb, 128, 0, st>>>(a);
    }
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(etab);
  cudaFree(vt);
  GPN_CUDA(e);
}

#define GPN_CUFFT(call)                                                                                 \
  do {                                                                                                  \
    cufftResult r_ = (call);                                                                            \
    if (r_ != CUFFT_SUCCESS) ::gpn::fail(GP_ECUFFT, std::string(#call " failed: code ") + std::to_string((int)r_)); \
  } while (0)

namespace {
// A full-grid R2C or C2R plan over C * R grids.  Its cuFFT work area: for the forward
// transform the interpolation grid (idle until the inverse rewrites every cell of it);
// for the inverse, with the memory-lean step 3, the spreading grid (idle after the forward
// transform; run_fft_inverse zeroes it again), else the plan's shared work allocation,
// grown, with every inverse plan pointed at the larger one, when a plan needs more.
cufftHandle make_full_plan(Plan& p, int R, bool forward) {
  int n[3] = {(int)p.geom.nf, (int)p.geom.nf, (int)p.geom.nf};
  const cufftType t = p.precision == GP_FP32 ? (forward ? CUFFT_R2C : CUFFT_C2R) : (forward ? CUFFT_D2Z : CUFFT_Z2D);
  cufftHandle hdl;
  GPN_CUFFT(cufftCreate(&hdl));
  size_t ws = 0;
  cufftResult r = cufftSetAutoAllocation(hdl, 0);
  if (r == CUFFT_SUCCESS) r = cufftMakePlanMany(hdl, p.geom.d, n, nullptr, 1, 0, nullptr, 1, 0, t, p.geom.C * R, &ws);
  if (r != CUFFT_SUCCESS) {
    cufftDestroy(hdl);
    GPN_CUFFT(r);
  }
  try {
    if (ws > 0 && forward && ws <= p.grid_bytes) {
      GPN_CUFFT(cufftSetWorkArea(hdl, p.grid_out));
    } else if (ws > 0 && !forward && p.lean && ws <= p.grid_bytes) {
      GPN_CUFFT(cufftSetWorkArea(hdl, p.grid));
      p.inv_in_grid[R] = ws;
    } else if (ws > 0) {
      if (ws > p.fft_work_bytes) {
        p.fft_work = p.alloc(ws);
        p.fft_work_bytes = ws;
        for (auto& kv : p.fft_inv)
          if (!p.inv_in_grid.count(kv.first)) GPN_CUFFT(cufftSetWorkArea(kv.second, p.fft_work));
        for (auto& kv : p.fft_fwd) {
          size_t w = 0;
          GPN_CUFFT(cufftGetSize(kv.second, &w));
          if (w > p.grid_bytes) GPN_CUFFT(cufftSetWorkArea(kv.second, p.fft_work));
        }
      }
      GPN_CUFFT(cufftSetWorkArea(hdl, p.fft_work));
    }
  } catch (...) {
    cufftDestroy(hdl);
    throw;
  }
  return hdl;
}
}  // namespace

cufftHandle Plan::fwd_plan(int R) {
  auto it = fft_fwd.find(R);
  if (it != fft_fwd.end()) return it->second;
  const cufftHandle hdl = make_full_plan(*this, R, true);
  fft_fwd[R] = hdl;
  return hdl;
}

cufftHandle Plan::inv_plan(int R) {
  auto it = fft_inv.find(R);
  if (it != fft_inv.end()) return it->second;
  const cufftHandle hdl = make_full_plan(*this, R, false);
  fft_inv[R] = hdl;
  return hdl;
}

void run_fft_forward(Plan& plan, int R, cudaStream_t st) {
  // the row-kernel paths mark between their rows and cuFFT's columns themselves
  if (plan.tr3) return tr3_forward(plan, R, st);
  if (plan.rowfft) return rowfft_forward(plan, R, st);
  prof_mark(plan, 0, st);                          // all of the phase is cuFFT
  cufftHandle h = plan.fwd_plan(R);
  GPN_CUFFT(cufftSetStream(h, st));
  if (plan.precision == GP_FP32)
    GPN_CUFFT(cufftExecR2C(h, (cufftReal*)plan.grid, (cufftComplex*)plan.spec));
  else
    GPN_CUFFT(cufftExecD2Z(h, (cufftDoubleReal*)plan.grid, (cufftDoubleComplex*)plan.spec));
}

void run_fft_inverse(Plan& plan, int R, cudaStream_t st) {
  if (plan.tr3) return tr3_inverse(plan, R, st);
  if (plan.rowfft) return rowfft_inverse(plan, R, st);
  cufftHandle h = plan.inv_plan(R);
  GPN_CUFFT(cufftSetStream(h, st));
  if (plan.precision == GP_FP32)
    GPN_CUFFT(cufftExecC2R(h, (cufftComplex*)plan.spec, (cufftReal*)plan.grid_out));
  else
    GPN_CUFFT(cufftExecZ2D(h, (cufftDoubleComplex*)plan.spec, (cufftDoubleReal*)plan.grid_out));
  const auto in_grid = plan.inv_in_grid.find(R);
  if (in_grid != plan.inv_in_grid.end()) GPN_CUDA(cudaMemsetAsync(plan.grid, 0, in_grid->second, st));
  prof_mark(plan, 1, st);
}

void prof_mark(Plan& plan, int which, cudaStream_t st) {
  if (plan.prof.in_matvec) GPN_CUDA(cudaEventRecord(plan.prof.mid[which], st));
}

void PhaseProfile::harvest() {
  if (!pending) return;
  GPN_CUDA(cudaEventSynchronize(ev[5]));
  for (int q = 0; q < 5; ++q) {
    float ms = 0.f;
    GPN_CUDA(cudaEventElapsedTime(&ms, ev[q], ev[q + 1]));
    acc[q] += ms;
  }
  float ms = 0.f;
  GPN_CUDA(cudaEventElapsedTime(&ms, ev[1], mid[0]));
  acc_rows[0] += ms;
  GPN_CUDA(cudaEventElapsedTime(&ms, mid[1], ev[4]));
  acc_rows[1] += ms;
  ++count;
  pending = false;
}

void PhaseProfile::destroy() {
  if (!created) return;
  for (auto& e : ev) cudaEventDestroy(e);
  for (auto& e : mid) cudaEventDestroy(e);
  created = false;
}

namespace {
// steps (1)-(5) for R <= grid_rhs right-hand sides (one pass through the grids)
void matvec_block(Plan& plan, const double* alpha_sorted, double* out_sorted, int R, double shift, cudaStream_t st) {
  PhaseProfile& pf = plan.prof;
  const bool rec = pf.on;
  if (rec) {
    pf.harvest();
    if (!pf.created) {
      for (auto& e : pf.ev) GPN_CUDA(cudaEventCreate(&e));
      for (auto& e : pf.mid) GPN_CUDA(cudaEventCreate(&e));
      pf.created = true;
    }
    GPN_CUDA(cudaEventRecord(pf.ev[0], st));
    pf.in_matvec = true;
  }
  launch_spread(plan, alpha_sorted, R, st);
  if (rec) GPN_CUDA(cudaEventRecord(pf.ev[1], st));
  run_fft_forward(plan, R, st);
  if (rec) GPN_CUDA(cudaEventRecord(pf.ev[2], st));
  launch_diag(plan, R, st);
  if (rec) GPN_CUDA(cudaEventRecord(pf.ev[3], st));
  run_fft_inverse(plan, R, st);
  if (rec) GPN_CUDA(cudaEventRecord(pf.ev[4], st));
  launch_interp(plan, plan.pts, alpha_sorted, shift, out_sorted, R, st);
  launch_near_apply(plan, alpha_sorted, out_sorted, R, st);
  if (rec) {
    pf.in_matvec = false;
    GPN_CUDA(cudaEventRecord(pf.ev[5], st));
    pf.pending = true;
  }
}
}  // namespace

// Columns beyond the grids' rhs_block run in blocks, one after the other on the stream
// (each block is one recorded pass when the phases are profiled).
void matvec_sorted(Plan& plan, const double* alpha_sorted, double* out_sorted, int R, double shift, cudaStream_t st) {
  const size_t n = (size_t)plan.N;
  for (int r0 = 0; r0 < R; r0 += plan.grid_rhs) {
    const int rc = std::min(plan.grid_rhs, R - r0);
    matvec_block(plan, alpha_sorted + (size_t)r0 * n, out_sorted + (size_t)r0 * n, rc, shift, st);
  }
}

double time_matvecs(Plan& plan, cudaStream_t st) {
  // every byte 0x3F: each alpha_i is the same finite double (about 4.8e-4); the kernels'
  // work does not depend on the values
  GPN_CUDA(cudaMemsetAsync(plan.vec_a, 0x3F, sizeof(double) * (size_t)plan.N, st));
  for (int i = 0; i < 2; ++i) matvec_sorted(plan, plan.vec_a, plan.vec_b, 1, 0.0, st);
  cudaEvent_t e0, e1;
  GPN_CUDA(cudaEventCreate(&e0));
  GPN_CUDA(cudaEventCreate(&e1));
  constexpr int kReps = 3;
  cudaError_t e = cudaEventRecord(e0, st);
  for (int i = 0; i < kReps && e == cudaSuccess; ++i) {
    matvec_sorted(plan, plan.vec_a, plan.vec_b, 1, 0.0, st);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1, st);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  GPN_CUDA(e);
  check_device_status(plan, st);
  return ms / kReps;
}

}  // namespace gpn
