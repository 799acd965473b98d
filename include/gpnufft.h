/* gpnufft.h -- C ABI of the GB300 (sm_103a) NUFFT-based GP matvec and solve.
 *
 * Method: Kielstra & Lindsey, "Gaussian process regression with log-linear
 * scaling for common non-stationary kernels" (arXiv 2407.03608).
 *
 * The library applies the approximate kernel matrix K~ of Eq. (Ktilde) (Sec. 3.5)
 * to vectors through the five steps of Sec. 4.2:
 *   (1) per-point Chebyshev weights c_k = w_k(x_i) alpha_i        (Eq. c, Eq. Wk)
 *   (2) N_sigma+1 type-1 NUFFTs onto the Fourier grid            (App. D)
 *   (3) a_k' = sum_j v~_j G^_k',j sum_k G^_k,j b_k  (precomputed A, Remark rem:step3)
 *   (4) N_sigma+1 type-2 NUFFTs back to the points                (App. D)
 *   (5) sum_k w_k(x_i) beta_k
 * and wraps it in conjugate gradients for (K + eta^2 I) alpha = y (Eq. gprsolve).
 *
 * Kernel (Sec. 3, Eq. nonstat2):
 *   K(x,y) = w(x) w(y) (2 pi [sigma^2(x)+sigma^2(y)])^(-d/2) phi(|x-y| / sqrt(sigma^2(x)+sigma^2(y)))
 * with phi the Matern function of Eq. (matern) or the squared exponential of
 * Eq. (squaredexp).  By default the two per-point fields are the vertical scale
 * s(x) and the Matern length l(x); the library converts them with
 *   sigma(x) = l(x)/sqrt(2),  w(x) = s(x) (2 pi)^(d/4) l(x)^(d/2),
 * which makes Eq. (nonstat2) the Paciorek non-stationary Matern with
 * K(x,x) = s(x)^2.  GP_PARAMS_PAPER passes w(x) and sigma(x) directly.
 *
 * Conventions for every entry point:
 *  - Return value is a gp_status; 0 is success.  No C++ exception and no exit()
 *    crosses the ABI.  gp_last_error() returns a message for the calling thread.
 *  - Pointers may be device pointers (cudaMalloc / torch CUDA tensors, on the
 *    plan's device) or host pointers (pageable or pinned).  The library detects
 *    which with cudaPointerGetAttributes.  Device pointers are used in place and
 *    the call is stream ordered: it returns before the work is done, and the
 *    inputs must stay valid until the stream passes the call.  For host
 *    pointers the library copies through its own device staging buffers and
 *    synchronises the stream before returning, so results are ready on return.
 *  - Floating-point data crosses the ABI in float64 whatever the plan's
 *    internal precision.
 *  - Vectors with R right-hand sides are N x R column-major (column r starts at
 *    element r*N), in the caller's original point order.
 *  - cuda_stream is a cudaStream_t (NULL = the legacy default stream).
 *  - A plan owns all device memory it allocates and frees it in gp_destroy.
 *    Calls on one plan must not overlap on different streams or threads.
 */
#ifndef GPNUFFT_H
#define GPNUFFT_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gp_plan_s* gp_plan_t;

typedef enum {
  GP_OK = 0,
  GP_EINVAL = -1,        /* invalid argument (message in gp_last_error)            */
  GP_ENOMEM = -2,        /* device allocation failed or plan exceeds opts.max_bytes */
  GP_ECUDA = -3,         /* CUDA runtime error                                       */
  GP_ECUFFT = -4,        /* cuFFT error                                              */
  GP_ENOTCONV = -5,      /* CG reached maxit before rtol; alpha holds the last iterate */
  GP_EBREAKDOWN = -6,    /* CG breakdown: p^T A p <= 0 or not finite                 */
  GP_ETIMEOUT = -7,      /* a bounded device wait ran out                            */
  GP_EUNSUPPORTED = -8   /* a configuration the kernels do not support               */
} gp_status;

/* Arithmetic of spread/FFT/step 3/interp: float64; float32; or float-float (each value
 * the unevaluated sum of two float32 words, about 48 significant bits, run on the FP32
 * pipe: FP64-grade results without the FP64 pipe, whose rate on GB300 is a small
 * fraction of the FP32 rate).  GP_DF64 is available for d = 2 with the transposed
 * pruned transforms (transform 3, nf = 2^a <= 8192) and the stored step-3 tensor;
 * other configurations get GP_EUNSUPPORTED. */
enum { GP_FP64 = 0, GP_FP32 = 1, GP_DF64 = 2 };
enum { GP_MATERN = 0, GP_SE = 1 };                 /* phi: Eq. (matern) or Eq. (squaredexp)   */
enum { GP_PARAMS_SCALES = 0, GP_PARAMS_PAPER = 1 };/* fields are (s, l) or (w, sigma)         */

/* Bits of gp_plan_opts.set: which override fields are valid.  Zero = all
 * hyperparameters chosen from eps (Sec. 5.4 recipe with numeric stage estimates). */
enum {
  GP_SET_NT = 1u << 0,        /* n_t, t_min, t_max           (Eq. dtscheme)          */
  GP_SET_NSIGMA = 1u << 1,    /* n_sigma                     (Eq. chebscheme)        */
  GP_SET_SIGMA_RANGE = 1u << 2,/* sigma_lo, sigma_hi (paper sigma, not l)            */
  GP_SET_M = 1u << 3,         /* M: Fourier grid {-M..M}^d   (Sec. 3.4)              */
  GP_SET_DW = 1u << 4,        /* dw: Fourier grid spacing    (Sec. 3.4)              */
  GP_SET_NUFFT = 1u << 5,     /* nufft_tol, upsampfac        (App. D)                */
  GP_SET_BOX = 1u << 6,       /* box_lo, box_hi: region all points and queries lie in */
  GP_SET_NF = 1u << 7,        /* nf: fine-grid size per dimension (FFT length)        */
  GP_SET_TILE = 1u << 8       /* tile: spread/interp tile edge in fine-grid cells; for d >= 2 a multiple of 4 (FP32) or 2 (FP64) */
};

typedef struct gp_plan_opts {
  int precision;          /* GP_FP64 (default) or GP_FP32                               */
  int family;             /* GP_MATERN (default) or GP_SE (nu ignored)                  */
  int param_mode;         /* GP_PARAMS_SCALES (default) or GP_PARAMS_PAPER              */
  unsigned set;           /* GP_SET_* bits                                              */
  int n_t; double t_min, t_max;
  int n_sigma; double sigma_lo, sigma_hi;
  long long M; double dw;
  double nufft_tol; double upsampfac;
  double box_lo[3], box_hi[3];
  long long nf;
  int tile;
  int transform;          /* 0 auto (3 for d = 2 when nf = 2^a; 2 for d = 1 in FP64;
                               else 1);
                             1 full-grid cuFFT R2C/C2R;
                             2 pruned: custom shared-memory row FFTs keeping modes 0..M,
                               cuFFT along the first axis (d <= 2, nf = 2^a);
                             3 pruned, transposed (d = 2, nf = 2^a): custom row FFTs
                               write columns of modes 0..M, cuFFT transforms each
                               contiguous column, step 3 on the mode box only    */
  int max_rhs;            /* largest R the plan will be called with (default 1)         */
  long long max_bytes;    /* refuse plans whose resident device bytes exceed this (0 = no limit) */
  int step3;              /* step (3) of Sec. 4.2:
                             0 auto: 1 unless the tensor alone would break max_bytes or
                               the free device memory, then 2;
                             1 the stored tensor A[n] of Remark rem:step3 (deconvolutions
                               folded in; C(C+1)/2 reals per frequency of the half box);
                             2 memory-lean: a_k = sum_j v~_j G^_kj sum_l G^_lj b_l formed
                               per frequency from the separable per-dimension factors of
                               G^ (C (N_t+1) (M+1) reals in total), the sequential
                               processing over j and k the paper gives as the
                               alternative to storing A; about 4.5 C (N_t+1)
                               multiply-adds per frequency.  Not with transform 2
                               (GP_EUNSUPPORTED).                                        */
  int diag_correct;       /* 1: add the exact diagonal defect, out_i += (K_ii - K~_ii) alpha_i
                             with K_ii = w_i^2 (4 pi sigma_i^2)^(-d/2) (Eq. nonstat2 at x = y)
                             and K~_ii = sum_kl w_k(x_i) w_l(x_i) sum_n A_kl[n] (Eq. Ktilde at
                             x = y).  An extension, not in the paper: it removes the part of
                             the truncation error that sits on the diagonal, the largest for
                             small nu (the cusp of phi at r = 0).  Off-diagonal entries are
                             K~'s.  Applies to matvecs and solves on the plan's own points,
                             not to posterior means.  0 (default): K~ as in the paper.  */
  int autotune;           /* 0 (default): the spread/interp tile from the shared-memory
                             heuristic.  k in 1..8: also build plans with up to k other
                             tiles the kernels accept (gp_tile_candidates, nearest to the
                             heuristic's first), time R = 1 matvecs of each with CUDA events
                             on the caller's stream, keep the fastest.  Tiles and bins are
                             the same size, so this tunes both.  Holds two plans at a time;
                             ignored when GP_SET_TILE is set.                            */
  int rhs_block;          /* right-hand sides per pass through the fine grids and spectra
                             (0 = max_rhs): the plan holds grids, spectra and transform
                             buffers for rhs_block right-hand sides and the CG vectors for
                             max_rhs; a matvec or CG iteration with R > rhs_block runs steps
                             (1)-(5) over the columns in blocks of rhs_block, one after the
                             other on the caller's stream, so R up to max_rhs fits where
                             max_rhs sets of grids would not.                             */
  double near_radius;     /* > 0: add the exact defect of every pair of distinct plan points
                             closer than near_radius (in x units), out_i += sum_{0 < |x_i - x_j|
                             < near_radius} (K_ij - K~_ij) alpha_j, K_ij of Eq. (nonstat2),
                             K~_ij of Eq. (Ktilde) through its per-dimension factors.  An
                             extension, not in the paper: for small nu the truncation error of
                             K~ sits on a neighbourhood of the diagonal (the cusp of phi at
                             r = 0), not on the diagonal alone; with diag_correct the plan
                             equals K on every pair within the radius.  nu = 1/2, 3/2, 5/2 or
                             GP_SE only (else GP_EUNSUPPORTED).  The pairs are built at plan
                             time (float64, about 12 bytes each, not in the footprint
                             estimate) and applied in every matvec and solve on the plan's
                             points, not to posterior means.  Meant for sparse point sets: the
                             cost grows with the number of pairs.  GP_ENOMEM when the factor
                             tables would pass 16 GB or the pairs 2^31 - 1; GP_EINVAL when
                             negative or not finite.  0 (default): off.                  */
} gp_plan_opts;

typedef struct gp_plan_info {
  int d; long long N; int family; int precision; double nu; double eps;
  int n_t; double t_min, t_max;            /* trapezoid rule in t (Eq. dtscheme)          */
  int n_sigma; double sigma_lo, sigma_hi;  /* Chebyshev-Lobatto interval (Eq. chebscheme) */
  long long M; double dw;                  /* Fourier grid n dw, n in {-M..M}^d           */
  long long nf;                            /* fine grid per dimension (FFT length)        */
  int kernel_width; double kernel_beta;    /* exponential-of-semicircle spreading kernel  */
  double upsampfac; double nufft_tol;
  int tile;                                /* spread/interp tile edge (cells)             */
  int transform;                           /* transform mode in use (1, 2 or 3)           */
  double box_lo[3], box_hi[3];             /* region points and queries must lie in       */
  double est_err_t, est_err_sigma, est_err_trunc, est_err_alias; /* stage estimates, relative entrywise */
  long long bytes_resident;                /* device bytes the plan holds                 */
  int max_rhs;
  int step3;                               /* step-3 form in use: 1 tensor, 2 memory-lean */
  int diag_correct;                        /* 1 when the diagonal defect is added         */
  int tuned;                               /* plans the autotuner timed (0: not tuned)    */
  double tune_ms;                          /* this plan's matvec time in the autotuner    */
  int rhs_block;                           /* right-hand sides per pass through the grids */
  double near_radius;                      /* near-field radius (0: off)                  */
  long long near_pairs;                    /* pairs with their defect stored              */
} gp_plan_info;

/* The autotuner's search space (host only, no GPU needed): every spread/interp tile
 * edge the kernels accept for d, n_channels = N_sigma + 1, precision (GP_FP32 or
 * GP_FP64) and the spreading kernel width, largest first.  Writes at most max_tiles
 * of them to tiles and returns how many there are (or a negative gp_status). */
int gp_tile_candidates(int d, int n_channels, int precision, int width, int* tiles, int max_tiles);

/* The parameters a plan would get, and its device footprint, without building it and
 * without a GPU (host only).  The data enter through their ranges: scale_min..scale_max,
 * the range of the second per-point field in opts->param_mode (the length l(x_i) for
 * GP_PARAMS_SCALES, the default; the paper's horizontal scale sigma(x_i) for
 * GP_PARAMS_PAPER; the library maps l to sigma = l / sqrt(2) as gp_plan does), and the
 * box box_lo[q] <= x_iq <= box_hi[q] (d entries each).  The hyperparameters are
 * chosen as gp_plan chooses them (Sec. 5.4 recipe, fine grid, tile, transform mode,
 * step-3 form).  info->bytes_resident is the estimate of the large allocations that
 * gp_plan checks against max_bytes.  The free device memory is not known here, so the
 * memory-lean step 3 is predicted only from max_bytes or an explicit opts->step3.
 * Errors: GP_EINVAL, GP_EUNSUPPORTED as for gp_plan; GP_ENOMEM when the host-side
 * tables of the chosen parameters (C (N_t+1) (M+1) doubles) do not fit in host memory,
 * as for nu = 1/2 at tight eps, where M grows like eps^(-1/(2 nu)) (Sec. 5.4). */
int gp_plan_params(int d, long long N, double nu, double eps, double scale_min, double scale_max,
                   const double* box_lo, const double* box_hi, const gp_plan_opts* opts, gp_plan_info* info);

/* Fill opts with the defaults (all zero except max_rhs = 1). */
void gp_plan_opts_default(gp_plan_opts* opts);

/* Build a plan for the N points x_i in R^d.
 *   points : N x d row-major float64 (host or device).
 *   field_a, field_b : N float64 each. GP_PARAMS_SCALES: s(x_i) > 0 and l(x_i) > 0.
 *                      GP_PARAMS_PAPER: w(x_i) >= 0 and sigma(x_i) > 0 (Eq. nonstat2).
 *   nu  : Matern smoothness > 0 (Eq. matern); ignored for GP_SE.
 *   eps : target entrywise error of K~ relative to sqrt(K_ii K_jj) (Theorem main),
 *         in (0, 0.1].  It drives every hyperparameter that opts does not set.
 * Builds the quadrature in t (Sec. 3.2), the Chebyshev nodes (Sec. 3.3), the Fourier
 * grid (Sec. 3.4), sorts the points into fine-grid tiles, and precomputes the
 * per-point weights w_k(x_i) (Eq. Wk) and either the tensor A[n] (Remark rem:step3) or,
 * with opts->step3 (see there), the per-dimension factors of the memory-lean step 3.
 * The fine grid: a power of two for d <= 2; for d = 3 the 7-smooth multiple of 4 that
 * minimises a measured FFT + spreading cost for this N (gp_plan_params shows the
 * choice without a GPU).  opts->autotune times alternative tiles; opts->diag_correct
 * adds the exact diagonal defect.  Device memory: about info.bytes_resident, checked
 * against opts->max_bytes before the large allocations.
 * Errors: GP_EINVAL (d not 1..3, N < 1, nu <= 0, eps out of range, non-positive
 * scale, inconsistent overrides), GP_EUNSUPPORTED (no kernel configuration for these
 * sizes, e.g. no spreading tile fits in shared memory for the kernel width, or the
 * memory-lean step 3 with transform 2), GP_ENOMEM, GP_ECUDA, GP_ECUFFT.
 * On error *out is NULL. */
int gp_plan(gp_plan_t* out, const double* points, long long N, int d, const double* field_a,
            const double* field_b, double nu, double eps, const gp_plan_opts* opts, void* cuda_stream);

/* out = (K~ + shift I) alpha for R right-hand sides (steps (1)-(5) of Sec. 4.2).
 *   alpha, out : N x R column-major float64 (host or device; may not alias).
 *   R : 1 <= R <= opts.max_rhs of the plan.
 * Errors: GP_EINVAL, GP_ECUDA, GP_ECUFFT. */
int gp_matvec(gp_plan_t plan, const double* alpha, double* out, int R, double shift, void* cuda_stream);

/* Solve (K~ + eta2 I) alpha = y (Eq. gprsolve) by conjugate gradients, each column
 * independently, all columns sharing each matvec launch.  x0 = 0; column r stops
 * when ||r_k|| / ||y_r|| <= rtol (recurrence residual).
 *   y, alpha : N x R column-major float64 (host or device).
 *   iters_out, relres_out : R entries each (host pointers, may be NULL): iterations
 *              taken and final recurrence relative residual per column.
 * CG scalars and reductions are float64 whatever the plan precision.
 * Errors: GP_EINVAL, GP_ENOTCONV (alpha holds the last iterate), GP_EBREAKDOWN,
 * GP_ECUDA, GP_ECUFFT. */
int gp_cg_solve(gp_plan_t plan, const double* y, double* alpha, int R, double eta2, double rtol, int maxit,
                int* iters_out, double* relres_out, void* cuda_stream);

/* Mixed-precision solve: CG with the matvec of plan_lo (normally GP_FP32) inside an
 * outer iterative-refinement loop whose residual y - (K~ + eta2 I) alpha is
 * recomputed with plan_hi (normally GP_FP64).  Both plans must have been built
 * on the same points and fields with identical hyperparameters (pass plan_hi's
 * gp_plan_info values as overrides when building plan_lo).  Stops when the
 * plan_hi relative residual is <= rtol.  inner_rtol is the relative reduction each
 * inner CG asks for; outer_max bounds the refinement steps.
 *   iters_out : total inner CG iterations per column; relres_out : final plan_hi
 *   relative residual per column.  Errors as gp_cg_solve. */
int gp_cg_solve_refined(gp_plan_t plan_lo, gp_plan_t plan_hi, const double* y, double* alpha, int R, double eta2,
                        double rtol, double inner_rtol, int outer_max, int maxit, int* iters_out,
                        double* relres_out, void* cuda_stream);

/* Posterior mean mu(x_q) = sum_n alpha_n K~(x_q, x_n) (Eq. postmean) at Nq query points.
 *   alpha : N float64 (training coefficients, original order).
 *   xq : Nq x d row-major; field_aq, field_bq : the two scale fields at the queries, in
 *        the plan's param_mode.  Queries must lie in the plan box and their sigma in
 *        [sigma_lo, sigma_hi] (gp_plan_info), else GP_EINVAL.
 *   mu : Nq float64. */
int gp_posterior_mean(gp_plan_t plan, const double* alpha, const double* xq, long long Nq, const double* field_aq,
                      const double* field_bq, double* mu, void* cuda_stream);

/* Posterior variance of the latent function at the training points: the diagonal of
 * Eq. (postcov) with K~, which equals eta2 - eta2^2 [(K~ + eta2 I)^{-1}]_ii.  The
 * diagonal of the inverse is estimated from R probe vectors z_r (entries +-1 give the
 * Hutchinson-type estimator; the estimator is an extension, the paper has none):
 *   d_i = (sum_r z_ri x_ri) / (sum_r z_ri^2),  x_r = (K~ + eta2 I)^{-1} z_r by CG
 * (gp_cg_solve's iteration, max_rhs probes per batch).
 *   probes : N x R column-major float64, original point order (host or device).
 *   eta2 > 0; rtol, maxit as gp_cg_solve.
 *   var : N float64.   iters_out : R ints (host, may be NULL).
 * Errors: GP_EINVAL, GP_ENOTCONV (some probe stopped at maxit; var is still written),
 * GP_EBREAKDOWN, GP_ECUDA, GP_ECUFFT. */
int gp_posterior_variance(gp_plan_t plan, const double* probes, int R, double eta2, double rtol, int maxit,
                          double* var, int* iters_out, void* cuda_stream);

/* Largest query batch of gp_posterior_mean_noalloc (sizes its static scratch). */
#define GP_NOALLOC_MAX_QUERIES 32768

/* gp_posterior_mean without any device allocation.  The paper has no counterpart:
 * it computes the same result as gp_posterior_mean, for callers that must not
 * allocate while they run, such as a serving loop that shares the device with
 * other streams (cudaFree synchronises the whole device) or a process that has
 * committed the device memory up front.
 *   Arguments as gp_posterior_mean, with 1 <= Nq <= GP_NOALLOC_MAX_QUERIES (else
 *   GP_EINVAL, nothing launched).  Host or device pointers; host inputs and a host
 *   mu are staged through a static device array of 256 + 48 * GP_NOALLOC_MAX_QUERIES
 *   bytes (about 1.5 MB) per device, and the rest of the work uses buffers the
 *   plan already holds.  Each query is evaluated straight from the fine grid
 *   (no binning), so large batches are better served by gp_posterior_mean.
 *   Queries outside the plan box or sigma range get mu = NaN and the call
 *   returns GP_EINVAL after the others are written.
 * The first call on each device does a one-time set-up (it looks up the device
 * address of the static array and the SM count, with the plan's device current;
 * again after the device's context has been reset); make that first call before
 * any stream capture begins.  The static array is shared by all calls
 * on a device: calls whose GPU work overlaps (other streams, other host threads,
 * other plans) race on it.  The call waits for its stream before returning.
 * Errors: GP_EINVAL, GP_ECUDA, GP_ECUFFT, GP_ETIMEOUT. */
int gp_posterior_mean_noalloc(gp_plan_t plan, const double* alpha, const double* xq, long long Nq,
                              const double* field_aq, const double* field_bq, double* mu, void* cuda_stream);

/* Per-phase timing of the matvec, with CUDA events recorded on the stream each
 * phase is launched on.  gp_profile_enable(plan, 1) clears the counters and starts
 * recording around every later matvec of this plan (gp_matvec, each CG iteration,
 * posterior mean); gp_profile_enable(plan, 0) stops.  While recording, a matvec
 * waits for the previous matvec's events before launching, so use it for
 * measurement, not in production.  gp_profile_read writes the average
 * milliseconds per launch into ms_avg[0..4]:
 *   [0] spread (steps 1+2a)  [1] forward FFT  [2] step 3 (diag)  [3] inverse FFT
 *   [4] interp (steps 4b+5)
 * and the number of matvecs recorded into *count (may be NULL); it waits for the
 * last recorded matvec.  Errors: GP_EINVAL, GP_ECUDA. */
int gp_profile_enable(gp_plan_t plan, int on);
int gp_profile_read(gp_plan_t plan, double* ms_avg, long long* count);

/* The library's own row kernels inside the two transform phases of the same
 * recording (App. D: the row half of each 2-D FFT), as average milliseconds per
 * matvec: ms_avg[0] of phase [1] (forward) and ms_avg[1] of phase [3] (inverse).
 * The rest of each phase is cuFFT (the column transforms in d = 2).  Plans whose
 * transforms are cuFFT alone give 0; the 1-D row transforms, which use no cuFFT,
 * give the whole phase.  It waits for the last recorded matvec.
 * Errors: GP_EINVAL, GP_ECUDA. */
int gp_profile_read_rows(gp_plan_t plan, double* ms_avg);

/* Copy the plan's chosen hyperparameters and sizes into *info. */
int gp_plan_info_get(gp_plan_t plan, gp_plan_info* info);

/* Free everything the plan owns.  NULL is ignored. */
void gp_destroy(gp_plan_t plan);

/* Message of the last failing call on this thread ("" if none). */
const char* gp_last_error(void);

/* Library version string. */
const char* gp_version(void);

#ifdef __cplusplus
}
#endif
#endif /* GPNUFFT_H */
