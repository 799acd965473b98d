// The C ABI of include/gpnufft.h: argument checks, host/device pointer handling,
// plan construction, and the entry points.  No exception crosses the ABI.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include <cudaTypedefs.h>

#include "plan.h"

namespace gpn {

namespace {
thread_local std::string g_last_error;

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at{};
  cudaError_t e = cudaPointerGetAttributes(&at, p);
  if (e != cudaSuccess) {
    cudaGetLastError();  // clear: plain host memory on some drivers
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Temporary device buffer freed at scope exit.
struct DevTmp {
  void* p = nullptr;
  explicit DevTmp(size_t bytes) {
    if (bytes && cudaMalloc(&p, bytes) != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
      fail(GP_ENOMEM, "cudaMalloc of " + std::to_string(bytes) + " temporary bytes failed");
    }
  }
  ~DevTmp() {
    if (p) cudaFree(p);
  }
  DevTmp(const DevTmp&) = delete;
  DevTmp& operator=(const DevTmp&) = delete;
};

// A device view of caller data: used in place when already on the device.
struct DevIn {
  const double* ptr = nullptr;
  std::unique_ptr<DevTmp> tmp;
  DevIn(const double* src, size_t count, cudaStream_t st) {
    if (is_device_ptr(src)) {
      ptr = src;
      return;
    }
    tmp.reset(new DevTmp(sizeof(double) * std::max<size_t>(count, 1)));
    GPN_CUDA(cudaMemcpyAsync(tmp->p, src, sizeof(double) * count, cudaMemcpyHostToDevice, st));
    ptr = (const double*)tmp->p;
  }
};

void* plan_alloc_cb(void* ctx, size_t bytes) { return static_cast<Plan*>(ctx)->alloc(bytes); }

struct TmpList {
  std::vector<void*> ptrs;
  ~TmpList() {
    for (void* p : ptrs) cudaFree(p);
  }
};
void* tmp_alloc_cb(void* ctx, size_t bytes) {
  void* p = nullptr;
  if (cudaMalloc(&p, std::max<size_t>(bytes, 16)) != cudaSuccess) {
    cudaGetLastError();
    fail(GP_ENOMEM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed");
  }
  static_cast<TmpList*>(ctx)->ptrs.push_back(p);
  return p;
}

// Spread/interp tile edge (with d >= 2, a multiple of 16 bytes of grid values): the
// largest candidate whose shared tile fits the budget
// (64 KB keeps several CTAs per SM, then the spreading maximum) with all channels, and
// that covers a point's support in two bins (tile >= width - 1).  When no tile holds
// every channel, the largest holding one channel: the spreading then runs in channel
// chunks.
const int kTiles1[] = {4096, 2048, 1024, 512, 256, 128, 64, 32, 16};
const int kTiles2[] = {64, 48, 32, 24, 16, 12, 8};
const int kTiles3[] = {16, 12, 10, 8, 6, 4};

// A tile the kernels accept: no smaller than the support, 16-byte TMA boxes along x for
// d >= 2 (staged from x = bin * tile), a staged interp block that fits, and a spreading
// tile of `chans` channels within `budget` bytes of shared memory.
bool tile_ok(int d, int t, int chans, size_t rs, int width, size_t budget) {
  if (t < width - 1) return false;
  if (d >= 2 && (t * rs) % 16 != 0) return false;
  return spread_smem_bytes(d, t, chans, rs, width) <= budget && interp_stage_bytes(d, t, width, rs) <= kInterpSmemMax;
}

int choose_tile(int d, int C, size_t rs, int width) {
  const int* c = d == 1 ? kTiles1 : (d == 2 ? kTiles2 : kTiles3);
  int nc = d == 1 ? 9 : (d == 2 ? 7 : 6);
  for (int chans : {C, 1}) {
    for (size_t budget : {size_t(64) << 10, kSpreadSmemMax}) {
      for (int i = 0; i < nc; ++i)
        if (tile_ok(d, c[i], chans, rs, width, budget)) return c[i];
    }
  }
  fail(GP_EUNSUPPORTED, "no spreading tile fits in shared memory for this kernel width");
}

// The autotuner's search space: every tile the kernels accept for (d, C, rs, width),
// largest first (channel chunks allowed, as for the heuristic's last resort).
std::vector<int> tile_candidates(int d, int C, size_t rs, int width) {
  const int* c = d == 1 ? kTiles1 : (d == 2 ? kTiles2 : kTiles3);
  int nc = d == 1 ? 9 : (d == 2 ? 7 : 6);
  std::vector<int> out;
  for (int i = 0; i < nc; ++i)
    if (tile_ok(d, c[i], C, rs, width, kSpreadSmemMax) || tile_ok(d, c[i], 1, rs, width, kSpreadSmemMax))
      out.push_back(c[i]);
  return out;
}

// The autotuner's trial order around the heuristic's tile t0: t0's neighbours in the
// candidate list, nearest first, at most `max_trials` of them.
std::vector<int> tile_trials(const std::vector<int>& cands, int t0, int max_trials) {
  std::vector<int> rest;
  for (int t : cands)
    if (t != t0) rest.push_back(t);
  std::stable_sort(rest.begin(), rest.end(), [t0](int a, int b) {
    return std::fabs(std::log((double)a / t0)) < std::fabs(std::log((double)b / t0));
  });
  if ((int)rest.size() > max_trials) rest.resize(max_trials);
  return rest;
}

int set_error(const Error& e) {
  g_last_error = e.what();
  return e.status;
}

template <class F>
int guarded(F f) {
  try {
    g_last_error.clear();
    return f();
  } catch (const Error& e) {
    return set_error(e);
  } catch (const std::bad_alloc&) {
    g_last_error = "host allocation failed";
    return GP_ENOMEM;
  } catch (const std::exception& e) {
    g_last_error = e.what();
    return GP_ECUDA;
  } catch (...) {
    g_last_error = "unknown internal error";
    return GP_ECUDA;
  }
}

Plan* as_plan(gp_plan_t p) {
  GPN_CHECK(p != nullptr, GP_EINVAL, "null plan");
  return reinterpret_cast<Plan*>(p);
}

void bind_device(const Plan& p) { GPN_CUDA(cudaSetDevice(p.device)); }

}  // namespace

void fail(int status, const std::string& msg) { throw Error(status, msg); }

Plan::~Plan() {
  prof.destroy();
  for (auto& kv : fft_fwd) cufftDestroy(kv.second);
  for (auto& kv : fft_inv) cufftDestroy(kv.second);
  for (auto& kv : fft_col) cufftDestroy(kv.second);
  for (auto& kv : fft_t3) cufftDestroy(kv.second);
  if (cg_graph.exec) cudaGraphExecDestroy(cg_graph.exec);
  if (cap_stream) cudaStreamDestroy(cap_stream);
  for (void* p : owned) cudaFree(p);
  if (host_scal) cudaFreeHost(host_scal);
  if (host_status) cudaFreeHost(host_status);
}

void* Plan::alloc(size_t nbytes) {
  void* p = nullptr;
  size_t b = std::max<size_t>(nbytes, 16);
  if (cudaMalloc(&p, b) != cudaSuccess) {
    cudaGetLastError();
    fail(GP_ENOMEM, "cudaMalloc of " + std::to_string(nbytes) + " bytes failed (plan holds " + std::to_string(bytes) +
                        ")");
  }
  owned.push_back(p);
  bytes += (long long)b;
  return p;
}

void check_device_status(Plan& plan, cudaStream_t st) {
  GPN_CUDA(cudaMemcpyAsync(plan.host_status, plan.dev_status, sizeof(int), cudaMemcpyDeviceToHost, st));
  GPN_CUDA(cudaStreamSynchronize(st));
  if (*plan.host_status != 0) {
    *plan.host_status = 0;
    GPN_CUDA(cudaMemsetAsync(plan.dev_status, 0, sizeof(int), st));
    GPN_CUDA(cudaStreamSynchronize(st));
    fail(GP_ETIMEOUT, "a device wait ran out (TMA copy did not complete); results of the call are invalid");
  }
}

namespace {

// Tiles that some point's support reaches: tile t gets the points of the bins at
// offsets {0,-1}^d from it.
void build_active_tiles(Plan& plan, const std::vector<int>& bstart) {
  const PointSet& ps = plan.pts;
  const int d = plan.h.d;
  std::vector<int> act;
  for (long long t = 0; t < ps.nbins_total; ++t) {
    int tc[kMaxDim] = {0, 0, 0};
    long long rest = t;
    for (int q = d - 1; q >= 0; --q) {
      tc[q] = (int)(rest % ps.nbins[q]);
      rest /= ps.nbins[q];
    }
    bool any = false;
    for (int o = 0; o < (1 << d) && !any; ++o) {
      long long lin = 0;
      bool valid = true;
      for (int q = 0; q < d; ++q) {
        int b = tc[q] - ((o >> q) & 1);
        valid = valid && b >= 0;
        lin = lin * ps.nbins[q] + (b < 0 ? 0 : b);
      }
      if (valid && bstart[lin + 1] > bstart[lin]) any = true;
    }
    if (any) act.push_back((int)t);
  }
  plan.n_active_tiles = (long long)act.size();
  plan.active_tiles = (int*)plan.alloc(sizeof(int) * std::max<size_t>(act.size(), 1));
  if (!act.empty())
    GPN_CUDA(cudaMemcpy(plan.active_tiles, act.data(), sizeof(int) * act.size(), cudaMemcpyHostToDevice));
}

// Rows (first axis) and columns (last axis) of the fine grid that hold spread data
// or that the interpolation reads: the active tiles' extent plus one kernel width.
void set_data_extent(Plan& plan) {
  const int d = plan.h.d, TS = plan.h.tile;
  const long long nf = plan.h.nf;
  std::vector<int> t(plan.n_active_tiles);
  if (plan.n_active_tiles)
    GPN_CUDA(cudaMemcpy(t.data(), plan.active_tiles, sizeof(int) * t.size(), cudaMemcpyDeviceToHost));
  long long lo[kMaxDim] = {nf, nf, nf}, hi[kMaxDim] = {0, 0, 0};
  for (int id : t) {
    long long rest = id;
    for (int q = d - 1; q >= 0; --q) {
      long long c = rest % plan.pts.nbins[q];
      rest /= plan.pts.nbins[q];
      lo[q] = std::min(lo[q], c * TS);
      hi[q] = std::max(hi[q], std::min(nf, (c + 1) * TS + plan.h.width));
    }
  }
  if (t.empty())
    for (int q = 0; q < d; ++q) lo[q] = hi[q] = 0;
  plan.col_lo = (int)lo[d - 1];
  plan.col_hi = (int)hi[d - 1];
  plan.row_lo = d == 2 ? (int)lo[0] : 0;
  plan.row_hi = d == 2 ? (int)hi[0] : 1;
}

// TMA descriptor of the interp input grid: dims (nf, ..., nf, C * max_rhs), box =
// (pitch, ext, ..., ext, interp_cc) so one copy stages a bin's block of cc channels.
void make_tensor_map(Plan& plan) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    GPN_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q));
    GPN_CHECK(q == cudaDriverEntryPointSuccess && fn, GP_ECUDA, "cuTensorMapEncodeTiled unavailable");
    encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
  }
  const Hyper& h = plan.h;
  const int d = h.d;
  const size_t rs = plan.real_size;
  const int ext = h.tile + h.width - 1;
  cuuint64_t dims[4], strides[3];
  cuuint32_t box[4], es[4] = {1, 1, 1, 1};
  for (int q = 0; q < d; ++q) dims[q] = (cuuint64_t)h.nf;
  dims[d] = (cuuint64_t)plan.geom.C * plan.grid_rhs;
  cuuint64_t st = rs;
  for (int q = 0; q < d; ++q) {
    st *= (cuuint64_t)h.nf;
    strides[q] = st;
  }
  box[0] = (cuuint32_t)interp_pitch(d, h.tile, h.width, rs);
  for (int q = 1; q < d; ++q) box[q] = (cuuint32_t)ext;
  box[d] = (cuuint32_t)plan.interp_cc;
  for (int q = 0; q <= d; ++q)
    GPN_CHECK(box[q] >= 1 && box[q] <= 256, GP_EUNSUPPORTED, "TMA box dimension out of range");
  CUresult r = encode(&plan.tmap_out, rs == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64,
                      (cuuint32_t)(d + 1), plan.grid_out, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                      CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  GPN_CHECK(r == CUDA_SUCCESS, GP_ECUDA, "cuTensorMapEncodeTiled failed: " + std::to_string((int)r));
}

}  // namespace

// The hyperparameters, layout and device footprint of a plan, from the data's ranges
// (sigma in [smin, smax], points in the box [lo, hi]); host only.  free_b: device memory
// available to the plan (-1: unknown, then the memory-lean step 3 is chosen only by
// max_bytes or explicitly).  tb, when given, receives the plan's tables.
PlanShape plan_shape(int d, long long N, double nu, double eps, const gp_plan_opts& o, double smin, double smax,
                     const double* lo_in, const double* hi_in, long long free_b, Tables* tb) {
  PlanShape ps;
  Hyper& h = ps.h;
  const int max_rhs = o.max_rhs > 0 ? o.max_rhs : 1;
  const size_t rs = o.precision == GP_FP32 ? 4 : 8;
  h.d = d;
  h.family = o.family;
  h.nu = o.family == GP_SE ? INFINITY : nu;
  h.eps = eps;
  if (o.set & GP_SET_SIGMA_RANGE) {
    GPN_CHECK(o.sigma_lo > 0.0 && o.sigma_hi >= o.sigma_lo, GP_EINVAL, "need 0 < sigma_lo <= sigma_hi");
    GPN_CHECK(smin >= o.sigma_lo * (1 - 1e-12) && smax <= o.sigma_hi * (1 + 1e-12), GP_EINVAL,
              "data sigma outside [sigma_lo, sigma_hi]");
    h.sig_lo = o.sigma_lo;
    h.sig_hi = o.sigma_hi;
  } else if (smax - smin <= 1e-12 * smax) {
    h.sig_lo = h.sig_hi = smax;
  } else {
    double pad = 0.01 * smax;
    h.sig_lo = std::max(smin - pad, 0.5 * smin);
    h.sig_hi = smax + pad;
  }
  for (int q = 0; q < d; ++q) {
    double lo = lo_in[q], hi = hi_in[q];
    if (o.set & GP_SET_BOX) {
      GPN_CHECK(o.box_hi[q] > o.box_lo[q], GP_EINVAL, "box_hi must exceed box_lo");
      GPN_CHECK(lo >= o.box_lo[q] && hi <= o.box_hi[q], GP_EINVAL, "points outside the given box");
      h.box_lo[q] = o.box_lo[q];
      h.box_hi[q] = o.box_hi[q];
    } else {
      double m = 1e-9 * std::max(hi - lo, 1e-3) + 1e-12;
      h.box_lo[q] = lo - m;
      h.box_hi[q] = hi + m;
    }
  }
  select_hyper(h, o, o.precision, N);
  GPN_CHECK(d == 1 || (h.nf * (long long)rs) % 16 == 0, GP_EINVAL,
            "nf must be a multiple of 4 (FP32) or 2 (FP64) for d >= 2: the interpolation's TMA copies need "
            "16-byte row strides");
  const int C = h.n_sigma + 1;
  ps.C = C;
  h.tile = (o.set & GP_SET_TILE) ? o.tile : choose_tile(d, C, rs, h.width);
  if (!(o.set & GP_SET_TILE) && o.precision == GP_DF64 && d == 2) {
    // float-float plans spread with the register kernel (its tiles do not depend on this
    // edge), so the edge sizes the interpolation's staged blocks and the spread's candidate
    // bins: 24 cells measured best (22.9 ms a CG iteration on the 2-D benchmark workload,
    // against 23.7 at 16 and 25.2 at 32)
    for (int t : {24, 16, 32, 12, 8})
      if (tile_ok(d, t, C, rs, h.width, kSpreadSmemMax) || tile_ok(d, t, 1, rs, h.width, kSpreadSmemMax)) {
        h.tile = t;
        break;
      }
  }
  GPN_CHECK(d == 1 || (h.tile * rs) % 16 == 0, GP_EINVAL,
            "tile must be a multiple of 16 bytes of grid values (4 in FP32, 2 in FP64) for d >= 2");
  GPN_CHECK(h.tile >= h.width - 1 && h.tile >= 1, GP_EINVAL, "tile must be >= kernel width - 1");
  // the host tables hold C (N_t + 1) (M + 1) doubles of per-dimension factors (and
  // M + 1 values of psi^); refuse them before allocating when M is out of reach (nu = 1/2
  // at tight eps), and build them only for a plan, not for a parameter query
  const long long J = h.family == GP_SE ? 1 : (long long)h.n_t + 1;
  const double table_bytes = 8.0 * (double)C * (double)J * (double)(h.M + 1);
  GPN_CHECK(table_bytes <= kHostTableMax, GP_ENOMEM,
            "host tables of " + std::to_string((long long)table_bytes) + " bytes for M = " + std::to_string(h.M) +
                " exceed the limit of " + std::to_string((long long)kHostTableMax));
  if (tb) build_tables(h, *tb);

  long long G = 1;
  for (int q = 0; q < d; ++q) G *= h.nf;
  const long long S = G / h.nf * (h.nf / 2 + 1);
  long long nfreq = 1;
  for (int q = 0; q < d - 1; ++q) nfreq *= (2 * h.M + 1);
  nfreq *= (h.M + 1);
  GPN_CHECK(o.transform >= 0 && o.transform <= 3, GP_EINVAL, "transform must be 0, 1, 2 or 3");
  const bool ddp = o.precision == GP_DF64;
  const bool row_ok = !ddp && rowfft_supported(d, h.nf, rs);
  const bool t3_ok = tr3_supported(d, h.nf, o.precision);
  GPN_CHECK(!ddp || (d == 2 && t3_ok && (o.transform == 0 || o.transform == 3)), GP_EUNSUPPORTED,
            "GP_DF64 needs d = 2 with the transposed pruned transforms (transform 3, nf = 2^a <= 8192)");
  GPN_CHECK(o.transform != 2 || row_ok, GP_EUNSUPPORTED, "pruned row transforms need d <= 2 and power-of-two nf");
  GPN_CHECK(o.transform != 3 || t3_ok, GP_EUNSUPPORTED, "transposed pruned transforms need d = 2 and nf = 2^a");
  // auto: the transposed pruned transforms for d = 2; the pruned row transforms for
  // d = 1 in FP64 (FP64 FFT arithmetic is ALU-bound on GB300); else full-grid cuFFT
  ps.tr3 = o.transform == 3 || (o.transform == 0 && t3_ok);
  ps.rowfft = o.transform == 2 || (o.transform == 0 && !ps.tr3 && row_ok && o.precision == GP_FP64);
  if (ps.tr3) nfreq = (h.M + 1) * (h.M + 1);
  ps.G = G;
  ps.S = S;
  ps.nfreq = nfreq;
  ps.a_bytes = (long long)(C * (C + 1) / 2) * nfreq * (long long)rs;
  ps.lean_bytes = J * (h.M + 1) * lean_channel_pitch(C, rs) * (long long)rs;
  // the large allocations: spreading and interpolation grids, spectra or the pruned
  // transforms' column buffers (for a block of rhs_block right-hand sides), per-point data
  // and the nine work vectors (for max_rhs)
  GPN_CHECK(o.rhs_block >= 0, GP_EINVAL, "rhs_block must be >= 0");
  const int grid_rhs = (o.rhs_block > 0 && o.rhs_block < max_rhs) ? o.rhs_block : max_rhs;
  const long long CR = (long long)C * grid_rhs;
  const long long spectra = (ps.tr3 || ps.rowfft) ? 3 * (d == 2 ? h.nf : 1) * CR * (h.M + 1) * 2 * (long long)rs
                                                  : CR * S * 2 * (long long)rs;
  // full-grid transforms: each grid buffer holds a whole spectrum as well (cuFFT's work
  // area of one transform direction lives in the buffer that direction leaves idle);
  // cuFFT needs a work area as large as the spectrum unless nf is a power of two, and the
  // inverse one gets its own allocation unless step 3 is memory-lean
  const bool full = !ps.tr3 && !ps.rowfft;
  const long long grid_pitch = full ? std::max(G, 2 * S) : G;
  const bool pow2 = (h.nf & (h.nf - 1)) == 0;
  const long long inv_work = (full && !pow2) ? CR * S * 2 * (long long)rs : 0;
  ps.est_rest = 2 * CR * grid_pitch * (long long)rs + spectra + N * (long long)(d * (4 + rs) + 8 + C * rs) +
                (long long)N * max_rhs * 8 * 9 +
                (psi_tabulated(d, o.precision) ? N * (long long)d * h.width * (long long)rs : 0);
  // step 3: the stored tensor A' (1) or the memory-lean form from per-dimension
  // factors (2); auto takes the tensor unless it alone breaks max_bytes or the free
  // device memory
  GPN_CHECK(o.step3 >= 0 && o.step3 <= 2, GP_EINVAL, "step3 must be 0, 1 or 2");
  GPN_CHECK(o.step3 != 2 || !ps.rowfft, GP_EUNSUPPORTED,
            "the memory-lean step 3 runs with transform 1 or 3, not the pruned row transforms");
  GPN_CHECK(o.step3 != 2 || !ddp, GP_EUNSUPPORTED, "GP_DF64 plans use the stored step-3 tensor (step3 = 1)");
  if (ddp) {
    ps.lean = false;
  } else if (o.step3 == 2) {
    ps.lean = true;
  } else if (o.step3 == 0 && !ps.rowfft) {
    const long long with_a = ps.est_rest + ps.a_bytes + inv_work, with_f = ps.est_rest + ps.lean_bytes;
    const bool over_budget = o.max_bytes > 0 && with_a > o.max_bytes && with_f <= o.max_bytes;
    const bool over_free = free_b >= 0 && with_a > free_b && with_f <= free_b;
    ps.lean = over_budget || over_free;
  }
  ps.est = ps.est_rest + (ps.lean ? ps.lean_bytes : ps.a_bytes + inv_work);
  return ps;
}

namespace {

Plan* make_plan(const double* points, long long N, int d, const double* fa, const double* fb, double nu, double eps,
                const gp_plan_opts& o, cudaStream_t st) {
  GPN_CHECK(d >= 1 && d <= 3, GP_EINVAL, "d must be 1, 2 or 3");
  GPN_CHECK(N >= 1, GP_EINVAL, "N must be >= 1");
  GPN_CHECK(points && fa && fb, GP_EINVAL, "null points or fields");
  GPN_CHECK(o.family == GP_MATERN || o.family == GP_SE, GP_EINVAL, "family must be GP_MATERN or GP_SE");
  GPN_CHECK(o.family == GP_SE || (nu > 0.0 && std::isfinite(nu)), GP_EINVAL, "nu must be > 0");
  GPN_CHECK(eps > 0.0 && eps <= 0.1, GP_EINVAL, "eps must be in (0, 0.1]");
  GPN_CHECK(o.precision == GP_FP64 || o.precision == GP_FP32 || o.precision == GP_DF64, GP_EINVAL,
            "precision must be GP_FP64, GP_FP32 or GP_DF64");
  GPN_CHECK(o.param_mode == GP_PARAMS_SCALES || o.param_mode == GP_PARAMS_PAPER, GP_EINVAL, "bad param_mode");
  int max_rhs = o.max_rhs > 0 ? o.max_rhs : 1;
  GPN_CHECK(max_rhs <= 1024, GP_EINVAL, "max_rhs must be <= 1024");

  std::unique_ptr<Plan> plan(new Plan());
  GPN_CUDA(cudaGetDevice(&plan->device));
  plan->precision = o.precision;
  plan->param_mode = o.param_mode;
  plan->N = N;
  plan->max_rhs = max_rhs;
  plan->grid_rhs = (o.rhs_block > 0 && o.rhs_block < max_rhs) ? o.rhs_block : max_rhs;
  const int grid_rhs = plan->grid_rhs;
  plan->max_bytes = o.max_bytes;
  plan->real_size = o.precision == GP_FP32 ? 4 : 8;

  DevIn x(points, (size_t)N * d, st), a(fa, N, st), b(fb, N, st);
  DevTmp wbuf(sizeof(double) * N), sbuf(sizeof(double) * N);
  double* w = (double*)wbuf.p;
  double* sig = (double*)sbuf.p;
  fields_to_paper(a.ptr, b.ptr, w, sig, N, d, o.param_mode, st);
  double stats[9];
  field_stats(x.ptr, w, sig, N, d, stats, st);
  GPN_CHECK(stats[8] == 0.0, GP_EINVAL,
            std::to_string((long long)stats[8]) + " invalid entries (non-finite point, scale <= 0 or weight < 0)");

  size_t free_b = 0, total_b = 0;
  GPN_CUDA(cudaMemGetInfo(&free_b, &total_b));
  const PlanShape ps = plan_shape(d, N, nu, eps, o, stats[0], stats[1], stats + 2, stats + 5, (long long)free_b,
                                  &plan->tb);
  Hyper& h = plan->h;
  h = ps.h;
  const int C = ps.C;
  const size_t rs = plan->real_size;
  GridGeom& g = plan->geom;
  g.d = d;
  g.nf = h.nf;
  g.width = h.width;
  g.beta = h.beta;
  g.beta_f = (float)h.beta;
  g.tile = h.tile;
  g.C = C;
  g.M = h.M;
  const long long G = ps.G, S = ps.S;
  plan->grid_elems = ps.G;
  plan->spec_elems = ps.S;
  plan->n_freq = ps.nfreq;
  plan->tr3 = ps.tr3;
  plan->rowfft = ps.rowfft;
  plan->lean = ps.lean;
  const long long a_bytes = ps.a_bytes;
  GPN_CHECK(o.max_bytes <= 0 || ps.est <= o.max_bytes, GP_ENOMEM,
            "plan needs about " + std::to_string(ps.est) + " device bytes, above max_bytes");

  std::vector<int> bstart;
  build_pointset(*plan, plan->pts, x.ptr, w, sig, N, st, plan_alloc_cb, plan.get(), &bstart);
  GPN_CHECK(o.diag_correct == 0 || o.diag_correct == 1, GP_EINVAL, "diag_correct must be 0 or 1");
  if (o.diag_correct) build_diag_correction(*plan, w, sig, st);
  GPN_CHECK(o.near_radius >= 0.0 && std::isfinite(o.near_radius), GP_EINVAL, "near_radius must be >= 0");
  if (o.near_radius > 0.0) build_near_field(*plan, o.near_radius, x.ptr, w, sig, st);
  build_active_tiles(*plan, bstart);
  if (spread2d_supported(*plan)) build_spread2d_tiles(*plan, bstart);
  GPN_CHECK(o.precision != GP_DF64 || plan->sp2_tiles, GP_EUNSUPPORTED,
            "GP_DF64 needs the two-dimensional register spread (kernel width <= 16, channels <= 32)");
  if (plan->lean) {
    build_lean_tables(*plan);
    GPN_CHECK(lean_smem_bytes(*plan) <= (size_t(200) << 10), GP_EUNSUPPORTED,
              "memory-lean step 3: the per-block factor table does not fit in shared memory");
  } else {
    plan->a_tensor = plan->alloc((size_t)a_bytes);
    build_a_tensor(*plan, st);
  }
  // full-grid transforms: room for a spectrum in each grid buffer (cuFFT work areas)
  const long long grid_pitch = (!plan->tr3 && !plan->rowfft) ? std::max(G, 2 * S) : G;
  plan->grid_bytes = (size_t)C * grid_rhs * grid_pitch * rs;
  plan->grid = plan->alloc(plan->grid_bytes);
  GPN_CUDA(cudaMemsetAsync(plan->grid, 0, plan->grid_bytes, st));
  plan->grid_out = plan->alloc(plan->grid_bytes);
  GPN_CUDA(cudaMemsetAsync(plan->grid_out, 0, plan->grid_bytes, st));
  if (plan->rowfft || plan->tr3) {
    set_data_extent(*plan);
    const size_t rows = d == 2 ? (size_t)h.nf : 1;
    const size_t fbytes = rows * C * (size_t)grid_rhs * (h.M + 1) * 2 * rs;
    plan->fx = plan->alloc(fbytes);
    plan->fy = plan->alloc(fbytes);
    plan->fz = plan->alloc(fbytes);
    GPN_CUDA(cudaMemsetAsync(plan->fx, 0, fbytes, st));
    GPN_CUDA(cudaMemsetAsync(plan->fz, 0, fbytes, st));
    if (plan->tr3)
      tr3_setup(*plan);
    else
      build_twiddles(*plan);
  } else {
    plan->spec = plan->alloc((size_t)C * grid_rhs * S * 2 * rs);
  }
  plan->interp_cc = (int)std::max<size_t>(
      1, std::min<size_t>((size_t)C, kInterpSmemBudget / interp_stage_bytes(d, h.tile, h.width, rs)));
  if (d >= 2) make_tensor_map(*plan);
  plan->dev_status = (int*)plan->alloc(sizeof(int));
  GPN_CUDA(cudaMemsetAsync(plan->dev_status, 0, sizeof(int), st));
  GPN_CUDA(cudaMallocHost(&plan->host_status, sizeof(int)));
  const size_t vb = sizeof(double) * (size_t)N * max_rhs;
  plan->vec_a = (double*)plan->alloc(vb);
  plan->vec_b = (double*)plan->alloc(vb);
  plan->cg_x = (double*)plan->alloc(vb);
  plan->cg_r = (double*)plan->alloc(vb);
  plan->cg_p = (double*)plan->alloc(vb);
  plan->cg_ap = (double*)plan->alloc(vb);
  plan->cg_y = (double*)plan->alloc(vb);
  plan->stage_in = (double*)plan->alloc(vb);
  plan->stage_out = (double*)plan->alloc(vb);
  plan->scal = (double*)plan->alloc(sizeof(double) * 8 * max_rhs);
  plan->cg_cnt = (int*)plan->alloc(sizeof(int) * (max_rhs + 1));
  plan->partials = (double*)plan->alloc(sizeof(double) * 512 * max_rhs);
  GPN_CUDA(cudaMallocHost(&plan->host_scal, sizeof(double) * 8 * max_rhs));
  if (plan->tr3) {
    if (o.precision != GP_DF64) plan->t3_plan(1);   // float-float columns are the library's own kernel
  } else if (plan->rowfft) {
    if (d == 2) plan->col_plan(1);
  } else {
    // the widest batch first, so that the shared cuFFT work area is sized once
    plan->fwd_plan(plan->grid_rhs);
    plan->inv_plan(plan->grid_rhs);
    plan->fwd_plan(1);
    plan->inv_plan(1);
  }
  GPN_CUDA(cudaStreamSynchronize(st));
  GPN_CHECK(plan->max_bytes <= 0 || plan->bytes <= plan->max_bytes, GP_ENOMEM, "plan exceeds max_bytes");
  return plan.release();
}

// Resolve an output pointer: device pointers are written in place; host pointers go
// through the plan's staging buffer and are copied back by finish().
struct DevOut {
  double* dev;
  double* host = nullptr;
  size_t count;
  DevOut(double* dst, double* stage, size_t n) : dev(dst), count(n) {
    if (!is_device_ptr(dst)) {
      host = dst;
      dev = stage;
    }
  }
  void finish(Plan& plan, cudaStream_t st) {
    if (host) {
      GPN_CUDA(cudaMemcpyAsync(host, dev, sizeof(double) * count, cudaMemcpyDeviceToHost, st));
      check_device_status(plan, st);
    }
  }
};

// Input through the plan staging buffer when on the host.
const double* dev_input(const double* src, double* stage, size_t count, cudaStream_t st) {
  if (is_device_ptr(src)) return src;
  GPN_CUDA(cudaMemcpyAsync(stage, src, sizeof(double) * count, cudaMemcpyHostToDevice, st));
  return stage;
}

void check_same_hyper(const Plan& a, const Plan& b) {
  const Hyper &x = a.h, &y = b.h;
  bool same = a.N == b.N && x.d == y.d && x.family == y.family && x.n_t == y.n_t && x.t_min == y.t_min &&
              x.t_max == y.t_max && x.n_sigma == y.n_sigma && x.sig_lo == y.sig_lo && x.sig_hi == y.sig_hi &&
              x.M == y.M && x.dw == y.dw && (x.family == GP_SE || x.nu == y.nu) &&
              (a.dcorr != nullptr) == (b.dcorr != nullptr) && a.near_radius == b.near_radius;
  GPN_CHECK(same, GP_EINVAL, "plan_lo and plan_hi must share points and hyperparameters");
}

}  // namespace
}  // namespace gpn

using namespace gpn;

namespace gpn {
namespace {
// the hyperparameter fields of gp_plan_info
void fill_hyper_info(const Hyper& h, gp_plan_info* info) {
  info->d = h.d;
  info->family = h.family;
  info->nu = h.nu;
  info->eps = h.eps;
  info->n_t = h.n_t;
  info->t_min = h.t_min;
  info->t_max = h.t_max;
  info->n_sigma = h.n_sigma;
  info->sigma_lo = h.sig_lo;
  info->sigma_hi = h.sig_hi;
  info->M = h.M;
  info->dw = h.dw;
  info->nf = h.nf;
  info->kernel_width = h.width;
  info->kernel_beta = h.beta;
  info->upsampfac = h.upsamp;
  info->nufft_tol = h.nufft_tol;
  info->tile = h.tile;
  for (int q = 0; q < 3; ++q) {
    info->box_lo[q] = h.box_lo[q];
    info->box_hi[q] = h.box_hi[q];
  }
  info->est_err_t = h.est_t;
  info->est_err_sigma = h.est_sigma;
  info->est_err_trunc = h.est_trunc;
  info->est_err_alias = h.est_alias;
}
}  // namespace
}  // namespace gpn

extern "C" {

void gp_plan_opts_default(gp_plan_opts* opts) {
  if (!opts) return;
  std::memset(opts, 0, sizeof(*opts));
  opts->max_rhs = 1;
}

int gp_plan(gp_plan_t* out, const double* points, long long N, int d, const double* field_a, const double* field_b,
            double nu, double eps, const gp_plan_opts* opts, void* cuda_stream) {
  if (out) *out = nullptr;
  return guarded([&]() {
    GPN_CHECK(out != nullptr, GP_EINVAL, "null output handle");
    gp_plan_opts o;
    gp_plan_opts_default(&o);
    if (opts) o = *opts;
    GPN_CHECK(o.autotune >= 0 && o.autotune <= 8, GP_EINVAL, "autotune must be in 0..8");
    const cudaStream_t st = (cudaStream_t)cuda_stream;
    std::unique_ptr<Plan> best(make_plan(points, N, d, field_a, field_b, nu, eps, o, st));
    if (o.autotune > 0 && !(o.set & GP_SET_TILE)) {
      // time the heuristic's plan and up to `autotune` alternatives with other tiles;
      // keep the fastest (two plans are held at a time)
      const Hyper& h = best->h;
      const auto trials = tile_trials(tile_candidates(h.d, best->geom.C, best->real_size, h.width), h.tile, o.autotune);
      best->tune_ms = time_matvecs(*best, st);
      for (int t : trials) {
        gp_plan_opts o2 = o;
        o2.set |= GP_SET_TILE;
        o2.tile = t;
        o2.autotune = 0;
        std::unique_ptr<Plan> cand;
        try {
          cand.reset(make_plan(points, N, d, field_a, field_b, nu, eps, o2, st));
        } catch (const Error&) {
          cudaGetLastError();   // clear a failed allocation's error state
          continue;             // this tile does not fit (memory, shared memory): not a candidate
        }
        cand->tune_ms = time_matvecs(*cand, st);
        if (cand->tune_ms < best->tune_ms) best.swap(cand);
      }
      best->tuned = (int)trials.size() + 1;
    }
    *out = reinterpret_cast<gp_plan_t>(best.release());
    return GP_OK;
  });
}

int gp_tile_candidates(int d, int n_channels, int precision, int width, int* tiles, int max_tiles) {
  return guarded([&]() {
    GPN_CHECK(d >= 1 && d <= 3 && n_channels >= 1 && n_channels <= kMaxChannels && width >= 2 && width <= kMaxWidth,
              GP_EINVAL, "bad d, n_channels or width");
    GPN_CHECK(precision == GP_FP64 || precision == GP_FP32 || precision == GP_DF64, GP_EINVAL, "bad precision");
    GPN_CHECK(tiles != nullptr || max_tiles == 0, GP_EINVAL, "null output");
    const auto c = tile_candidates(d, n_channels, precision == GP_FP32 ? 4 : 8, width);
    const int n = std::min<int>((int)c.size(), max_tiles);
    for (int i = 0; i < n; ++i) tiles[i] = c[i];
    return (int)c.size();
  });
}

int gp_matvec(gp_plan_t plan, const double* alpha, double* out, int R, double shift, void* cuda_stream) {
  return guarded([&]() {
    Plan* p = as_plan(plan);
    bind_device(*p);
    cudaStream_t st = (cudaStream_t)cuda_stream;
    GPN_CHECK(alpha && out, GP_EINVAL, "null alpha or out");
    GPN_CHECK(R >= 1 && R <= p->max_rhs, GP_EINVAL, "R must be in [1, max_rhs]");
    GPN_CHECK(std::isfinite(shift), GP_EINVAL, "shift must be finite");
    const size_t cnt = (size_t)p->N * R;
    const double* a = dev_input(alpha, p->stage_in, cnt, st);
    DevOut o(out, p->stage_out, cnt);
    gather_sorted(p->pts, a, p->vec_a, R, st);
    matvec_sorted(*p, p->vec_a, p->vec_b, R, shift, st);
    scatter_sorted(p->pts, p->vec_b, o.dev, R, st);
    GPN_CUDA(cudaGetLastError());
    o.finish(*p, st);
    return GP_OK;
  });
}

int gp_cg_solve(gp_plan_t plan, const double* y, double* alpha, int R, double eta2, double rtol, int maxit,
                int* iters_out, double* relres_out, void* cuda_stream) {
  return guarded([&]() {
    Plan* p = as_plan(plan);
    bind_device(*p);
    cudaStream_t st = (cudaStream_t)cuda_stream;
    GPN_CHECK(y && alpha, GP_EINVAL, "null y or alpha");
    GPN_CHECK(R >= 1 && R <= p->max_rhs, GP_EINVAL, "R must be in [1, max_rhs]");
    GPN_CHECK(eta2 >= 0.0 && std::isfinite(eta2), GP_EINVAL, "eta2 must be >= 0");
    GPN_CHECK(rtol > 0.0 && maxit >= 1, GP_EINVAL, "rtol > 0 and maxit >= 1 required");
    const size_t cnt = (size_t)p->N * R;
    const double* yd = dev_input(y, p->stage_in, cnt, st);
    DevOut o(alpha, p->stage_out, cnt);
    gather_sorted(p->pts, yd, p->cg_y, R, st);
    int s = cg_solve_sorted(*p, p->cg_y, p->cg_x, R, eta2, rtol, maxit, iters_out, relres_out, st);
    scatter_sorted(p->pts, p->cg_x, o.dev, R, st);
    o.finish(*p, st);
    if (s == GP_ENOTCONV) g_last_error = "CG reached maxit before rtol";
    if (s == GP_EBREAKDOWN) g_last_error = "CG breakdown (p^T A p <= 0 or not finite)";
    return s;
  });
}

int gp_cg_solve_refined(gp_plan_t plan_lo, gp_plan_t plan_hi, const double* y, double* alpha, int R, double eta2,
                        double rtol, double inner_rtol, int outer_max, int maxit, int* iters_out, double* relres_out,
                        void* cuda_stream) {
  return guarded([&]() {
    Plan* lo = as_plan(plan_lo);
    Plan* hi = as_plan(plan_hi);
    GPN_CHECK(lo != hi, GP_EINVAL, "plan_lo and plan_hi must differ");
    GPN_CHECK(lo->device == hi->device, GP_EINVAL, "plans on different devices");
    bind_device(*hi);
    check_same_hyper(*lo, *hi);
    cudaStream_t st = (cudaStream_t)cuda_stream;
    GPN_CHECK(y && alpha, GP_EINVAL, "null y or alpha");
    GPN_CHECK(R >= 1 && R <= lo->max_rhs && R <= hi->max_rhs, GP_EINVAL, "R must be in [1, max_rhs] of both plans");
    GPN_CHECK(eta2 >= 0.0 && rtol > 0.0 && inner_rtol > 0.0 && inner_rtol < 1.0 && outer_max >= 1 && maxit >= 1,
              GP_EINVAL, "bad solver parameters");
    const size_t cnt = (size_t)hi->N * R;
    const double* yd = dev_input(y, hi->stage_in, cnt, st);
    DevOut o(alpha, hi->stage_out, cnt);
    gather_sorted(hi->pts, yd, hi->cg_y, R, st);
    int s = cg_refined_sorted(*lo, *hi, hi->cg_y, hi->cg_x, R, eta2, rtol, inner_rtol, outer_max, maxit, iters_out,
                              relres_out, st);
    scatter_sorted(hi->pts, hi->cg_x, o.dev, R, st);
    o.finish(*hi, st);
    if (s == GP_ENOTCONV) g_last_error = "refinement reached outer_max before rtol";
    return s;
  });
}

int gp_posterior_mean(gp_plan_t plan, const double* alpha, const double* xq, long long Nq, const double* field_aq,
                      const double* field_bq, double* mu, void* cuda_stream) {
  return guarded([&]() {
    Plan* p = as_plan(plan);
    bind_device(*p);
    cudaStream_t st = (cudaStream_t)cuda_stream;
    GPN_CHECK(alpha && xq && field_aq && field_bq && mu, GP_EINVAL, "null argument");
    GPN_CHECK(Nq >= 1, GP_EINVAL, "Nq must be >= 1");
    const int d = p->h.d;
    DevIn x(xq, (size_t)Nq * d, st), a(field_aq, Nq, st), b(field_bq, Nq, st);
    DevTmp wbuf(sizeof(double) * Nq), sbuf(sizeof(double) * Nq), outs(sizeof(double) * Nq), outo(sizeof(double) * Nq);
    fields_to_paper(a.ptr, b.ptr, (double*)wbuf.p, (double*)sbuf.p, Nq, d, p->param_mode, st);
    double stats[9];
    field_stats(x.ptr, (double*)wbuf.p, (double*)sbuf.p, Nq, d, stats, st);
    GPN_CHECK(stats[8] == 0.0, GP_EINVAL, "invalid query entries");
    GPN_CHECK(stats[0] >= p->h.sig_lo * (1 - 1e-12) && stats[1] <= p->h.sig_hi * (1 + 1e-12), GP_EINVAL,
              "query sigma outside the plan's [sigma_lo, sigma_hi]");
    for (int q = 0; q < d; ++q)
      GPN_CHECK(stats[2 + q] >= p->h.box_lo[q] && stats[5 + q] <= p->h.box_hi[q], GP_EINVAL,
                "query points outside the plan box");
    TmpList tl;
    PointSet qs;
    build_pointset(*p, qs, x.ptr, (double*)wbuf.p, (double*)sbuf.p, Nq, st, tmp_alloc_cb, &tl);
    const double* al = dev_input(alpha, p->stage_in, (size_t)p->N, st);
    gather_sorted(p->pts, al, p->vec_a, 1, st);
    launch_spread(*p, p->vec_a, 1, st);
    run_fft_forward(*p, 1, st);
    launch_diag(*p, 1, st);
    run_fft_inverse(*p, 1, st);
    launch_interp(*p, qs, nullptr, 0.0, (double*)outs.p, 1, st);
    DevOut o(mu, (double*)outo.p, (size_t)Nq);
    scatter_sorted(qs, (double*)outs.p, o.dev, 1, st);
    GPN_CUDA(cudaGetLastError());
    o.finish(*p, st);
    check_device_status(*p, st);  // temporaries are freed on return
    return GP_OK;
  });
}

int gp_posterior_variance(gp_plan_t plan, const double* probes, int R, double eta2, double rtol, int maxit,
                          double* var, int* iters_out, void* cuda_stream) {
  return guarded([&]() {
    Plan* p = as_plan(plan);
    bind_device(*p);
    cudaStream_t st = (cudaStream_t)cuda_stream;
    GPN_CHECK(probes && var, GP_EINVAL, "null probes or var");
    GPN_CHECK(R >= 1, GP_EINVAL, "R must be >= 1");
    GPN_CHECK(eta2 > 0.0 && std::isfinite(eta2), GP_EINVAL, "eta2 must be > 0");
    GPN_CHECK(rtol > 0.0 && maxit >= 1, GP_EINVAL, "rtol > 0 and maxit >= 1 required");
    const long long n = p->N;
    const bool dev_probes = is_device_ptr(probes);
    double* num = p->vec_a;
    double* den = p->vec_b;
    GPN_CUDA(cudaMemsetAsync(num, 0, sizeof(double) * n, st));
    GPN_CUDA(cudaMemsetAsync(den, 0, sizeof(double) * n, st));
    int status = GP_OK;
    std::vector<int> it(p->max_rhs);
    for (int r0 = 0; r0 < R; r0 += p->max_rhs) {
      const int rc = std::min(p->max_rhs, R - r0);
      const double* z = probes + (size_t)r0 * n;
      if (!dev_probes) {
        GPN_CUDA(cudaMemcpyAsync(p->stage_in, z, sizeof(double) * n * rc, cudaMemcpyHostToDevice, st));
        z = p->stage_in;
      }
      gather_sorted(p->pts, z, p->cg_y, rc, st);
      const int s = cg_solve_sorted(*p, p->cg_y, p->cg_x, rc, eta2, rtol, maxit, it.data(), nullptr, st);
      if (s == GP_EBREAKDOWN) fail(GP_EBREAKDOWN, "CG breakdown on a probe");
      if (s == GP_ENOTCONV) status = GP_ENOTCONV;
      if (iters_out)
        for (int c = 0; c < rc; ++c) iters_out[r0 + c] = it[c];
      probe_accumulate(p->cg_y, p->cg_x, n, rc, num, den, st);
    }
    DevOut o(var, p->stage_out, (size_t)n);
    variance_finish(num, den, n, eta2, p->cg_r, st);
    scatter_sorted(p->pts, p->cg_r, o.dev, 1, st);
    GPN_CUDA(cudaGetLastError());
    o.finish(*p, st);
    if (status == GP_ENOTCONV) g_last_error = "CG reached maxit before rtol on some probe";
    return status;
  });
}

int gp_posterior_mean_noalloc(gp_plan_t plan, const double* alpha, const double* xq, long long Nq,
                              const double* field_aq, const double* field_bq, double* mu, void* cuda_stream) {
  return guarded([&]() {
    Plan* p = as_plan(plan);
    bind_device(*p);
    cudaStream_t st = (cudaStream_t)cuda_stream;
    GPN_CHECK(alpha && xq && field_aq && field_bq && mu, GP_EINVAL, "null argument");
    GPN_CHECK(Nq >= 1 && Nq <= GP_NOALLOC_MAX_QUERIES, GP_EINVAL,
              "Nq must be in [1, " + std::to_string(GP_NOALLOC_MAX_QUERIES) +
                  "]: the static scratch of gp_posterior_mean_noalloc holds that many queries");
    const int d = p->h.d;
    const NoAllocScratch ns = noalloc_scratch(p->device);
    unsigned char* scratch = static_cast<unsigned char*>(ns.ptr);
    unsigned* bad = reinterpret_cast<unsigned*>(scratch);
    double* stage = reinterpret_cast<double*>(scratch + kNoAllocHeaderBytes);
    double* sx = stage;
    double* sa = sx + (size_t)Nq * d;
    double* sb = sa + Nq;
    double* smu = sb + Nq;
    GPN_CUDA(cudaMemsetAsync(bad, 0, sizeof(unsigned), st));  // the counter starts at zero every call
    const double* x = dev_input(xq, sx, (size_t)Nq * d, st);
    const double* fa = dev_input(field_aq, sa, (size_t)Nq, st);
    const double* fb = dev_input(field_bq, sb, (size_t)Nq, st);
    DevOut o(mu, smu, (size_t)Nq);
    const double* al = dev_input(alpha, p->stage_in, (size_t)p->N, st);
    gather_sorted(p->pts, al, p->vec_a, 1, st);
    launch_spread(*p, p->vec_a, 1, st);
    run_fft_forward(*p, 1, st);
    launch_diag(*p, 1, st);
    run_fft_inverse(*p, 1, st);
    launch_query_interp(*p, x, fa, fb, Nq, o.dev, bad, ns.sms, st);
    if (o.host) GPN_CUDA(cudaMemcpyAsync(o.host, o.dev, sizeof(double) * Nq, cudaMemcpyDeviceToHost, st));
    check_device_status(*p, st);  // also waits for the stream
    GPN_CUDA(cudaMemcpyAsync(p->host_status, bad, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    GPN_CUDA(cudaStreamSynchronize(st));
    const int nbad = *p->host_status;
    *p->host_status = 0;
    GPN_CHECK(nbad == 0, GP_EINVAL,
              std::to_string((unsigned)nbad) + " queries outside the plan box or sigma range (mu is NaN there)");
    return GP_OK;
  });
}

int gp_profile_enable(gp_plan_t plan, int on) {
  return guarded([&]() {
    Plan* p = as_plan(plan);
    bind_device(*p);
    if (on) {
      p->prof.harvest();
      for (double& a : p->prof.acc) a = 0.0;
      for (double& a : p->prof.acc_rows) a = 0.0;
      p->prof.count = 0;
    }
    p->prof.on = on != 0;
    return GP_OK;
  });
}

int gp_profile_read(gp_plan_t plan, double* ms_avg, long long* count) {
  return guarded([&]() {
    Plan* p = as_plan(plan);
    bind_device(*p);
    GPN_CHECK(ms_avg != nullptr, GP_EINVAL, "null ms_avg");
    p->prof.harvest();
    check_device_status(*p, nullptr);
    long long n = p->prof.count;
    for (int q = 0; q < 5; ++q) ms_avg[q] = n ? p->prof.acc[q] / n : 0.0;
    if (count) *count = n;
    return GP_OK;
  });
}

int gp_profile_read_rows(gp_plan_t plan, double* ms_avg) {
  return guarded([&]() {
    Plan* p = as_plan(plan);
    bind_device(*p);
    GPN_CHECK(ms_avg != nullptr, GP_EINVAL, "null ms_avg");
    p->prof.harvest();
    check_device_status(*p, nullptr);
    long long n = p->prof.count;
    for (int q = 0; q < 2; ++q) ms_avg[q] = n ? p->prof.acc_rows[q] / n : 0.0;
    return GP_OK;
  });
}

int gp_plan_params(int d, long long N, double nu, double eps, double scale_min, double scale_max,
                   const double* box_lo, const double* box_hi, const gp_plan_opts* opts, gp_plan_info* info) {
  return guarded([&]() {
    GPN_CHECK(info != nullptr && box_lo != nullptr && box_hi != nullptr, GP_EINVAL, "null info or box");
    GPN_CHECK(d >= 1 && d <= 3, GP_EINVAL, "d must be 1, 2 or 3");
    GPN_CHECK(N >= 1, GP_EINVAL, "N must be >= 1");
    GPN_CHECK(scale_min > 0.0 && scale_max >= scale_min && std::isfinite(scale_max), GP_EINVAL,
              "need 0 < scale_min <= scale_max");
    for (int q = 0; q < d; ++q)
      GPN_CHECK(std::isfinite(box_lo[q]) && std::isfinite(box_hi[q]) && box_hi[q] >= box_lo[q], GP_EINVAL,
                "bad point box");
    gp_plan_opts o;
    gp_plan_opts_default(&o);
    if (opts) o = *opts;
    GPN_CHECK(o.param_mode == GP_PARAMS_SCALES || o.param_mode == GP_PARAMS_PAPER, GP_EINVAL,
              "param_mode must be GP_PARAMS_SCALES or GP_PARAMS_PAPER");
    // the range of the second field in the plan's parametrisation: the length l (sigma =
    // l / sqrt(2), the same product gp_plan applies to every point) or sigma itself
    const double kInvSqrt2 = 0.70710678118654752440;
    const double sigma_min = o.param_mode == GP_PARAMS_SCALES ? scale_min * kInvSqrt2 : scale_min;
    const double sigma_max = o.param_mode == GP_PARAMS_SCALES ? scale_max * kInvSqrt2 : scale_max;
    GPN_CHECK(o.family == GP_MATERN || o.family == GP_SE, GP_EINVAL, "family must be GP_MATERN or GP_SE");
    GPN_CHECK(o.family == GP_SE || (nu > 0.0 && std::isfinite(nu)), GP_EINVAL, "nu must be > 0");
    GPN_CHECK(eps > 0.0 && eps <= 0.1, GP_EINVAL, "eps must be in (0, 0.1]");
    GPN_CHECK(o.precision == GP_FP64 || o.precision == GP_FP32 || o.precision == GP_DF64, GP_EINVAL,
              "precision must be GP_FP64, GP_FP32 or GP_DF64");
    const PlanShape ps = plan_shape(d, N, nu, eps, o, sigma_min, sigma_max, box_lo, box_hi, -1, nullptr);
    std::memset(info, 0, sizeof(*info));
    fill_hyper_info(ps.h, info);
    info->N = N;
    info->precision = o.precision;
    info->transform = ps.tr3 ? 3 : (ps.rowfft ? 2 : 1);
    info->bytes_resident = ps.est;
    info->max_rhs = o.max_rhs > 0 ? o.max_rhs : 1;
    info->rhs_block = (o.rhs_block > 0 && o.rhs_block < info->max_rhs) ? o.rhs_block : info->max_rhs;
    info->step3 = ps.lean ? 2 : 1;
    info->diag_correct = o.diag_correct ? 1 : 0;
    return GP_OK;
  });
}

int gp_plan_info_get(gp_plan_t plan, gp_plan_info* info) {
  return guarded([&]() {
    Plan* p = as_plan(plan);
    GPN_CHECK(info != nullptr, GP_EINVAL, "null info");
    const Hyper& h = p->h;
    std::memset(info, 0, sizeof(*info));
    info->d = h.d;
    info->N = p->N;
    info->family = h.family;
    info->precision = p->precision;
    info->nu = h.nu;
    info->eps = h.eps;
    info->n_t = h.n_t;
    info->t_min = h.t_min;
    info->t_max = h.t_max;
    info->n_sigma = h.n_sigma;
    info->sigma_lo = h.sig_lo;
    info->sigma_hi = h.sig_hi;
    info->M = h.M;
    info->dw = h.dw;
    info->nf = h.nf;
    info->kernel_width = h.width;
    info->kernel_beta = h.beta;
    info->upsampfac = h.upsamp;
    info->nufft_tol = h.nufft_tol;
    info->tile = h.tile;
    info->transform = p->tr3 ? 3 : (p->rowfft ? 2 : 1);
    for (int q = 0; q < 3; ++q) {
      info->box_lo[q] = h.box_lo[q];
      info->box_hi[q] = h.box_hi[q];
    }
    info->est_err_t = h.est_t;
    info->est_err_sigma = h.est_sigma;
    info->est_err_trunc = h.est_trunc;
    info->est_err_alias = h.est_alias;
    info->bytes_resident = p->bytes;
    info->max_rhs = p->max_rhs;
    info->rhs_block = p->grid_rhs;
    info->near_radius = p->near_radius;
    info->near_pairs = p->near_nnz;
    info->step3 = p->lean ? 2 : 1;
    info->diag_correct = p->dcorr ? 1 : 0;
    info->tuned = p->tuned;
    info->tune_ms = p->tune_ms;
    return GP_OK;
  });
}

void gp_destroy(gp_plan_t plan) {
  if (!plan) return;
  Plan* p = reinterpret_cast<Plan*>(plan);
  cudaSetDevice(p->device);
  delete p;
}

const char* gp_last_error(void) { return g_last_error.c_str(); }

const char* gp_version(void) { return "gpnufft 0.1.0 (sm_103a)"; }

}  // extern "C"
