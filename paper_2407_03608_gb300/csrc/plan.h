// Plan object: hyperparameters, device-resident point data, tables, grids and cuFFT plans.
#pragma once

#include <map>
#include <vector>

#include <cuda.h>
#include <cufft.h>

#include "common.h"
#include "params.h"

namespace gpn {

// Points binned into fine-grid tiles and sorted by tile (device memory).
// A point's spreading support is the cells l0_a .. l0_a + width - 1 in each
// dimension a; its bin is floor(l0_a / tile).  xi_a = g_a - l0_a where g_a is
// the point's fine-grid coordinate.
struct PointSet {
  long long n = 0;
  int nbins[kMaxDim] = {1, 1, 1};
  long long nbins_total = 0;
  int* cell0[kMaxDim] = {nullptr, nullptr, nullptr};   // l0_a, sorted order
  void* xi[kMaxDim] = {nullptr, nullptr, nullptr};     // xi_a (real_t), sorted order
  void* wk = nullptr;                                  // w_k(x_i) (real_t) [n][C]
  float* wabs = nullptr;                               // max_k |w_k(x_i)| [n]
  int* perm = nullptr;                                 // sorted position -> caller index
  int* bin_start = nullptr;                            // nbins_total + 1 offsets
  int* active_bins = nullptr;                          // bins holding at least one point
  long long n_active_bins = 0;
  // kernel values psi(j - xi_a), j < width, per axis [n][width] (real_t, sorted order):
  // tabulated once for the 2-D float64 and float-float plans, whose kernel values cost
  // a float64 or float-float exponential each; null otherwise (the kernels evaluate psi)
  void* psi[kMaxDim] = {nullptr, nullptr, nullptr};
};

// Launch parameters shared by the kernels.
struct GridGeom {
  int d;
  long long nf;          // fine grid per dimension
  int width;
  float beta_f;
  double beta;
  int tile;
  int C;                 // channels = n_sigma + 1
  long long M;
};

// Per-phase event timing of matvecs (diagnostic, off by default).
struct PhaseProfile {
  bool on = false;
  bool created = false;
  bool pending = false;
  bool in_matvec = false;   // between the first and last event of a recorded matvec
  cudaEvent_t ev[6];
  // mid[0]: the forward phase's own row kernels end and its cuFFT part begins;
  // mid[1]: the inverse phase's cuFFT part ends and its own row kernels begin
  cudaEvent_t mid[2];
  double acc[5] = {0, 0, 0, 0, 0};
  double acc_rows[2] = {0, 0};   // ms in the transform phases' own row kernels
  long long count = 0;
  void harvest();   // fold the pending event set into acc (waits for it)
  void destroy();
};

// A CUDA graph of a block of CG iterations, valid for one (x, R, eta2, rtol).
struct CgGraph {
  cudaGraphExec_t exec = nullptr;
  double* x = nullptr;
  int R = 0;
  double eta2 = 0.0, rtol = 0.0;
};

struct Plan {
  int device = 0;
  PhaseProfile prof;
  int precision = GP_FP64;
  int param_mode = GP_PARAMS_SCALES;
  long long N = 0;
  int max_rhs = 1;
  int grid_rhs = 1;                     // right-hand sides the grids and spectra hold (rhs_block)
  long long max_bytes = 0;
  Hyper h;
  Tables tb;
  GridGeom geom;
  PointSet pts;
  size_t real_size = 8;                 // sizeof(real_t)
  // device buffers
  void* a_tensor = nullptr;             // packed A'[p][f] (real_t), p < C(C+1)/2, f over the half box
  // memory-lean step 3 (no A'): per-dimension factors tab[j][m][lean_cp] and sqrt(v~_j)
  bool lean = false;
  void* lean_tab = nullptr;
  void* lean_sqv = nullptr;
  int lean_cp = 0;                      // channel pitch of tab (16-byte multiple)
  int lean_J = 0;                       // quadrature nodes N_t + 1
  double* dcorr = nullptr;              // diagonal defect K_ii - K~_ii (sorted order), null when off
  // near-field correction: K_ij - K~_ij for pairs closer than near_radius (CSR, sorted order)
  double near_radius = 0.0;
  int* near_ptr = nullptr;
  int* near_col = nullptr;
  double* near_val = nullptr;
  long long near_nnz = 0;
  int tuned = 0;                        // plans timed by the tile autotuner (0: not tuned)
  double tune_ms = 0.0;                 // this plan's matvec time in the autotuner
  long long n_freq = 0;                 // frequencies in the half box
  void* grid = nullptr;                 // spreading grids (R2C input), C * max_rhs * nf^d; cells no
                                        // active tile covers stay zero from plan creation on
  void* grid_out = nullptr;             // C2R output read by interp, same shape
  int* active_tiles = nullptr;          // tiles some point's support reaches
  long long n_active_tiles = 0;
  int* sp2_tiles = nullptr;             // 2-D register-accumulating spread: active 16 x TY tiles
  long long n_sp2_tiles = 0;
  int interp_cc = 1;                    // channels per interp staging chunk
  CUtensorMap tmap_out;                 // TMA descriptor of grid_out (d >= 2)
  int* dev_status = nullptr;            // set by kernels whose bounded waits ran out
  int* host_status = nullptr;           // pinned mirror
  void* spec = nullptr;                 // half spectra, C * max_rhs * nf^(d-1) * (nf/2+1) complex
  long long grid_elems = 0, spec_elems = 0;   // per channel
  double* vec_a = nullptr;              // sorted-order work vectors, N * max_rhs each
  double* vec_b = nullptr;
  double* cg_x = nullptr;               // CG state (sorted order)
  double* cg_r = nullptr;
  double* cg_p = nullptr;
  double* cg_ap = nullptr;
  double* cg_y = nullptr;
  double* scal = nullptr;               // device scalars (see cg.cu)
  int* cg_cnt = nullptr;                // CG iterations per column, then a breakdown flag
  CgGraph cg_graph;                     // captured block of CG iterations
  cudaStream_t cap_stream = nullptr;    // stream the graph is captured on
  double* partials = nullptr;           // reduction partials
  double* host_scal = nullptr;          // pinned mirror
  double* stage_in = nullptr;           // staging for host-pointer calls, N * max_rhs
  double* stage_out = nullptr;
  std::map<int, cufftHandle> fft_fwd, fft_inv;  // keyed by R (full-grid path)
  // cuFFT work areas of the full-grid plans (cuFFT's own allocation would give every
  // plan one, as large as a spectrum when nf is not a power of two): the forward
  // transforms work in grid_out, which the inverse rewrites whole afterwards; the inverse
  // ones in one shared allocation, or, with the memory-lean step 3, in the spreading grid,
  // zeroed again after the transform (the spread writes only the tiles points reach)
  size_t grid_bytes = 0;                // allocation of grid and of grid_out
  void* fft_work = nullptr;
  size_t fft_work_bytes = 0;
  std::map<int, size_t> inv_in_grid;    // R -> bytes of the spreading grid an inverse plan works in
  // pruned transform path (d <= 2, power-of-two nf): compact spectra
  // [rows][C*R][M+1] and the data extent of the fine grid
  bool rowfft = false;
  void* fx = nullptr;                   // row-transform output (rows without data stay zero)
  void* fy = nullptr;                   // column-transform output / inverse-column output
  void* fz = nullptr;                   // step-3 output (rows |m0| > M stay zero)
  void* twiddle = nullptr;              // exp(-2 pi i k / nf), k < nf
  void* stage_twiddle = nullptr;        // per-stage twiddles of the length-nf/2 FFT
  int fft_log2h = 0;                    // log2(nf / 2)
  int row_lo = 0, row_hi = 0;           // grid rows holding data (first axis, d = 2)
  int col_lo = 0, col_hi = 0;           // grid columns holding data or read by interp (last axis)
  std::map<int, cufftHandle> fft_col;   // first-axis C2C plans keyed by R
  cufftHandle col_plan(int R);
  // transposed pruned path (transform 3, d = 2): fx, fy, fz hold [cr][M+1][nf] columns,
  // the A' tensor is stored on the quadrant [pair][m][|n1|]
  bool tr3 = false;
  int t3_rb = 1;                        // grid rows per CTA of the row kernels
  void* tw_half = nullptr;              // two-level twiddle tables of the row kernels
  void* col_tw = nullptr;               // pass tables of the float-float column transforms
  std::map<int, cufftHandle> fft_t3;    // contiguous column C2C plans keyed by R
  cufftHandle t3_plan(int R);
  long long bytes = 0;
  std::vector<void*> owned;             // every cudaMalloc of the plan

  ~Plan();
  void* alloc(size_t bytes);
  cufftHandle fwd_plan(int R);
  cufftHandle inv_plan(int R);
};

// Kernel values tabulated per point (PointSet::psi): the 2-D float64 and float-float plans
inline bool psi_tabulated(int d, int precision) { return d == 2 && precision != GP_FP32; }
inline bool psi_tabulated(const Plan& p) { return psi_tabulated(p.geom.d, p.precision); }

// Hyperparameters, layout and device footprint of a plan (host only; abi.cpp).
struct PlanShape {
  Hyper h;
  int C = 0;
  bool tr3 = false, rowfft = false, lean = false;
  long long G = 0, S = 0, nfreq = 0;
  long long a_bytes = 0, lean_bytes = 0, est_rest = 0, est = 0;
};
PlanShape plan_shape(int d, long long N, double nu, double eps, const gp_plan_opts& o, double smin, double smax,
                     const double* lo, const double* hi, long long free_b, Tables* tb);

// ---- launchers (defined in the .cu files) ---------------------------------------

// Bin and sort points given in caller order (device, row-major N x d), compute xi,
// l0, bins, permutation, and the Chebyshev weights from the paper-native (w, sigma)
// fields (device, caller order).  Allocates into ps through plan.alloc.
// alloc(bytes) returns device memory owned by the caller of build_pointset.
// The host copy of bin_start is returned in *bin_start_host when not null.
using DevAlloc = void* (*)(void* ctx, size_t bytes);
void build_pointset(Plan& plan, PointSet& ps, const double* x_dev, const double* w_dev, const double* sig_dev,
                    long long n, cudaStream_t st, DevAlloc alloc, void* alloc_ctx,
                    std::vector<int>* bin_start_host = nullptr);

// Read and clear the device status word; fails with GP_ETIMEOUT when a kernel's
// bounded wait ran out.  Synchronises the stream.
void check_device_status(Plan& plan, cudaStream_t st);

// Convert (s, l) to (w, sigma) in place (device, n entries), or validate (w, sigma).
void fields_to_paper(const double* a, const double* b, double* w_out, double* sig_out, long long n, int d, int mode,
                     cudaStream_t st);

// min / max of sigma and of each coordinate, and the count of invalid entries.
void field_stats(const double* x, const double* w, const double* sig, long long n, int d, double* host_out,
                 cudaStream_t st);

// Build the packed A' tensor on the device from the E' tables.
void build_a_tensor(Plan& plan, cudaStream_t st);

// Shared-memory layout helpers of the spread / interp kernels.
constexpr size_t kInterpSmemBudget = size_t(96) << 10;   // target when sizing channel chunks
constexpr size_t kInterpSmemMax = size_t(200) << 10;      // one staged channel must fit
constexpr size_t kSpreadSmemMax = size_t(160) << 10;      // shared tile of one spreading channel chunk
constexpr double kHostTableMax = 32e9;                     // bytes of plan-time host tables
int spread_pitch(int d, int tile);
size_t spread_smem_bytes(int d, int tile, int C, size_t rs, int width);
int interp_pitch(int d, int tile, int width, size_t rs);
size_t interp_stage_bytes(int d, int tile, int width, size_t rs);

// Steps (1)+(2a): spread sorted-order coefficients alpha (N x R, float64) onto the
// fine grids (C * R channels).
void launch_spread(Plan& plan, const double* alpha_sorted, int R, cudaStream_t st);
// 2-D spreading with register accumulators (used when supported for the plan)
bool spread2d_supported(const Plan& plan);
int spread2d_rows(const Plan& plan);
void build_spread2d_tiles(Plan& plan, const std::vector<int>& bstart);
void launch_spread2d(Plan& plan, const double* alpha_sorted, int R, cudaStream_t st);
// Steps (2b)+(3)+(4a): deconvolve, apply A', zero outside the mode box (in spec).
void launch_diag(Plan& plan, int R, cudaStream_t st);
// Exact diagonal correction: plan.dcorr[p] = K_pp - K~_pp (points.cu).
void build_diag_correction(Plan& plan, const double* w_dev, const double* sig_dev, cudaStream_t st);
// Near-field correction (nearfield.cu): tables of the separable K~ factors and the pairs
// closer than `radius` with their defect K_ij - K~_ij, from the caller-order coordinates
// and paper-native fields; the apply adds them to a matvec on the plan's points.
bool near_field_supported(int family, double nu);
void build_near_field(Plan& plan, double radius, const double* x_dev, const double* w_dev, const double* sig_dev,
                      cudaStream_t st);
void launch_near_apply(Plan& plan, const double* alpha_sorted, double* out_sorted, int R, cudaStream_t st);
// Memory-lean step 3 (step3_lean.cu): the same map from the per-dimension factors,
// for the transposed (tr3) and the full-grid layouts.
int lean_channel_pitch(int C, size_t rs);
size_t lean_smem_bytes(const Plan& plan);
void build_lean_tables(Plan& plan);
void launch_step3_lean(Plan& plan, int R, cudaStream_t st);
// Steps (4b)+(5): interpolate at the points of ps and combine channels:
// out[i] = sum_k w_k(x_i) beta_k(x_i) + (shift + dcorr_i) * alpha_sorted[i] (alpha may be
// null; dcorr_i, the plan's diagonal defect, only for the plan's own points when on).
void launch_interp(Plan& plan, const PointSet& ps, const double* alpha_sorted, double shift, double* out_sorted,
                   int R, cudaStream_t st);

// Static scratch of gp_posterior_mean_noalloc (one array per device): a rejected-
// query counter in the first kNoAllocHeaderBytes, then float64 staging for host
// queries (x: Nq*d, the two fields: 2*Nq) and for a host output (Nq).
constexpr size_t kNoAllocHeaderBytes = 256;
constexpr size_t kNoAllocScratchBytes =
    kNoAllocHeaderBytes + sizeof(double) * (kMaxDim + 3) * (size_t)GP_NOALLOC_MAX_QUERIES;
// Device address of the scratch on `device` (must be current) and the device's SM
// count; looked up on the first call per device (again after the device's context
// was reset).
struct NoAllocScratch {
  void* ptr;
  int sms;
};
NoAllocScratch noalloc_scratch(int device);
// mu_q = sum_k w_k(x_q) beta_k(x_q) from plan.grid_out (right-hand side 0), one warp
// per query; *bad counts queries outside the box or sigma range (mu is NaN there).
// sms: the device's SM count (sizes the grid).
void launch_query_interp(Plan& plan, const double* x, const double* fa, const double* fb, long long nq, double* mu,
                         unsigned* bad, int sms, cudaStream_t st);
// FFTs of the fine grids (forward R2C, inverse C2R), batched over C * R.
void run_fft_forward(Plan& plan, int R, cudaStream_t st);
void run_fft_inverse(Plan& plan, int R, cudaStream_t st);

// Pruned transforms (fft_rows.cu).
bool rowfft_supported(int d, long long nf, size_t rs);
void build_twiddles(Plan& plan);
// Record the transform-phase boundary `which` (0 forward, 1 inverse) of the matvec
// being profiled; nothing when no matvec is being recorded.
void prof_mark(Plan& plan, int which, cudaStream_t st);
void rowfft_forward(Plan& plan, int R, cudaStream_t st);
void rowfft_diag(Plan& plan, int R, cudaStream_t st);
void rowfft_inverse(Plan& plan, int R, cudaStream_t st);
// transposed pruned transforms (d = 2, nf = 2^a)
bool tr3_supported(int d, long long nf, int precision);
void tr3_setup(Plan& plan);
void tr3_forward(Plan& plan, int R, cudaStream_t st);
void tr3_diag(Plan& plan, int R, cudaStream_t st);
void tr3_inverse(Plan& plan, int R, cudaStream_t st);

// Full matvec in sorted order: out = (K~ + shift I) alpha.
void matvec_sorted(Plan& plan, const double* alpha_sorted, double* out_sorted, int R, double shift, cudaStream_t st);
// Milliseconds per matvec (R = 1, CUDA events, after two untimed ones) on a fixed input.
double time_matvecs(Plan& plan, cudaStream_t st);

// Permutations between caller order and sorted order (N x R column-major).
void gather_sorted(const PointSet& ps, const double* src, double* dst, int R, cudaStream_t st);
void scatter_sorted(const PointSet& ps, const double* src, double* dst, int R, cudaStream_t st);

// CG in sorted order (cg.cu).
// Probe estimate of a diagonal: num += sum_r z_r * x_r, den += sum_r z_r^2 (sorted
// order, n entries); then var = eta2 - eta2^2 num / den.
void probe_accumulate(const double* z_sorted, const double* x_sorted, long long n, int R, double* num, double* den,
                      cudaStream_t st);
void variance_finish(const double* num, const double* den, long long n, double eta2, double* var, cudaStream_t st);
int cg_solve_sorted(Plan& plan, const double* y_sorted, double* x_sorted, int R, double eta2, double rtol,
                    int maxit, int* iters, double* relres, cudaStream_t st);
int cg_refined_sorted(Plan& lo, Plan& hi, const double* y_sorted, double* x_sorted, int R, double eta2,
                      double rtol, double inner_rtol, int outer_max, int maxit, int* iters, double* relres,
                      cudaStream_t st);

}  // namespace gpn
