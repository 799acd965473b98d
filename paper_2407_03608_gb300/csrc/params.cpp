// Hyperparameter selection for K~ (Sec. 3, recipe of Sec. 5.4) and the host tables.
//
// The paper fixes the hyperparameters only up to big-O (Sec. 5.4: "we cannot make
// explicit choices").  This file turns each stage of Theorem main into a numeric
// estimate that is evaluated directly, and picks the smallest parameter meeting
// its share of eps:
//   stage 1 (Lemma dt):      sup_r |phi(r) - sum_j tau_j u(t_j) exp(-r^2/(2 chi_j^2))|   <= eps/4,
//                            tails P(nu, e^t_min) = Q(nu, e^t_max) = eps/12;
//   stage 2 (Lemma sigma):   sup over sigma_x, sigma_y, rho of the Chebyshev error of the
//                            normalised product B_t B_t* (independent of t at fixed r/chi) <= eps/4;
//   stage 3 (Lemma stage3):  truncation  d sum_j tau_j u_j erfc(2 pi sigma_lo chi_j M dw) <= eps/4,
//                            aliasing    d sum_j tau_j u_j exp(-(1/dw - L)^2/(4 sigma_hi^2 chi_j^2)) <= eps/8,
// with L the largest side of the point box.  Each estimate is relative to
// sqrt(K(x,x) K(y,y)).
#include "params.h"

#include <algorithm>
#include <cmath>
#include <utility>
#include <limits>

namespace gpn {

namespace {
constexpr double kPi = 3.14159265358979323846;

// Gauss-Legendre nodes and weights on [-1, 1]: the nodes are the roots of the Legendre
// polynomial P_n, found by Newton's method from the asymptotic first guess
// cos(pi (i + 3/4) / (n + 1/2)), with P_n and P_n' from the three-term (Bonnet) recurrence
// (k P_k = (2k - 1) z P_{k-1} - (k - 1) P_{k-2}); the weights are 2 / ((1 - z^2) P_n'(z)^2).
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < (n + 1) / 2; ++i) {
    double z = std::cos(kPi * (i + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      double pn = (n == 1) ? z : p1;
      double pnm1 = (n == 1) ? 1.0 : p0;
      dp = n * (z * pn - pnm1) / (z * z - 1.0);
      double dz = pn / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    x[i] = -z;
    x[n - 1 - i] = z;
    w[i] = w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

double matern_phi(double nu, double r) {
  r = std::fabs(r);
  if (nu == 0.5) return std::exp(-r);
  if (nu == 1.5) {
    double a = std::sqrt(3.0) * r;
    return (1.0 + a) * std::exp(-a);
  }
  if (nu == 2.5) {
    double a = std::sqrt(5.0) * r;
    return (1.0 + a + a * a / 3.0) * std::exp(-a);
  }
  double z = std::sqrt(2.0 * nu) * r;
  if (z == 0.0) return 1.0;
  if (z > 700.0) return 0.0;
  return std::exp((1.0 - nu) * std::log(2.0) - std::lgamma(nu) + nu * std::log(z)) * std::cyl_bessel_k(nu, z);
}

// u(t) of Eq. (maternpres), chi(t) of the same equation.
inline double u_of(double nu, double t) { return std::exp(nu * t - std::exp(t) - std::lgamma(nu)); }
inline double chi_of(double nu, double t) { return std::exp(0.5 * t) / std::sqrt(nu); }

struct TRule {
  std::vector<double> t, wu, chi;  // wu = tau_j u(t_j)
};

TRule trapezoid(const Hyper& h) {
  TRule r;
  if (h.family == GP_SE) {
    r.t = {0.0};
    r.wu = {1.0};
    r.chi = {1.0};
    return r;
  }
  int n = h.n_t;
  double dt = (h.t_max - h.t_min) / n;
  for (int j = 0; j <= n; ++j) {
    double t = h.t_min + (h.t_max - h.t_min) * j / n;
    double tau = (j == 0 || j == n) ? 0.5 * dt : dt;
    r.t.push_back(t);
    r.wu.push_back(tau * u_of(h.nu, t));
    r.chi.push_back(chi_of(h.nu, t));
  }
  return r;
}

// Stage 1: sup_r |phi - phi_quad| on a grid of r.
double stage1_error(const Hyper& h) {
  if (h.family == GP_SE) return 0.0;
  TRule q = trapezoid(h);
  double target_tail = 1e-3 * h.eps;
  double rmax = 1.0;
  while (matern_phi(h.nu, rmax) > target_tail && rmax < 1e4) rmax *= 1.5;
  const int nr = 1500;
  double worst = 0.0;
  for (int i = 0; i <= nr; ++i) {
    double r = rmax * i / nr;
    double s = 0.0;
    for (size_t j = 0; j < q.t.size(); ++j) s += q.wu[j] * std::exp(-r * r / (2.0 * q.chi[j] * q.chi[j]));
    worst = std::max(worst, std::fabs(s - matern_phi(h.nu, r)));
  }
  return worst;
}

std::vector<double> cheb_nodes(double lo, double hi, int n) {
  std::vector<double> s(n + 1);
  if (n == 0) {
    s[0] = hi;
    return s;
  }
  for (int k = 0; k <= n; ++k) s[k] = 0.5 * (std::cos(kPi * k / n) + 1.0) * (hi - lo) + lo;
  return s;
}

std::vector<double> cheb_bary(int n) {
  std::vector<double> b(n + 1);
  for (int k = 0; k <= n; ++k) {
    b[k] = (k % 2 == 0) ? 1.0 : -1.0;
    if (k == 0 || k == n) b[k] *= 0.5;
  }
  return b;
}

// Lagrange basis values at s by the barycentric formula (second kind).
void lagrange_bary(const std::vector<double>& nd, const std::vector<double>& b, double s, double* P) {
  int n = (int)nd.size();
  for (int k = 0; k < n; ++k)
    if (s == nd[k]) {
      for (int j = 0; j < n; ++j) P[j] = (j == k) ? 1.0 : 0.0;
      return;
    }
  double den = 0.0;
  for (int k = 0; k < n; ++k) {
    P[k] = b[k] / (s - nd[k]);
    den += P[k];
  }
  for (int k = 0; k < n; ++k) P[k] /= den;
}

// Stage 2: Chebyshev error of the normalised Gaussian product (see file header).
double stage2_error(int d, double lo, double hi, int n_sigma) {
  if (n_sigma == 0) return (hi - lo) <= 1e-14 * hi ? 0.0 : 1.0;
  std::vector<double> nd = cheb_nodes(lo, hi, n_sigma), b = cheb_bary(n_sigma);
  const int ns = 24, nr = 48;
  int C = n_sigma + 1;
  std::vector<double> P((size_t)ns * C), sv(ns);
  for (int a = 0; a < ns; ++a) {
    sv[a] = lo + (hi - lo) * a / (ns - 1);
    lagrange_bary(nd, b, sv[a], &P[(size_t)a * C]);
  }
  std::vector<double> ckl((size_t)C * C), skl((size_t)C * C);
  for (int k = 0; k < C; ++k)
    for (int l = 0; l < C; ++l) {
      double a2 = nd[k] * nd[k], b2 = nd[l] * nd[l];
      skl[k * C + l] = a2 + b2;
      ckl[k * C + l] = std::pow(a2 * b2 / (a2 + b2), 0.5 * d);
    }
  double worst = 0.0;
  std::vector<double> ekl((size_t)C * C);
  for (int ir = 0; ir < nr; ++ir) {
    double rho = 12.0 * hi * ir / (nr - 1);
    for (int k = 0; k < C * C; ++k) ekl[k] = ckl[k] * std::exp(-rho * rho / (2.0 * skl[k]));
    for (int a = 0; a < ns; ++a)
      for (int bb = 0; bb < ns; ++bb) {
        const double* Pa = &P[(size_t)a * C];
        const double* Pb = &P[(size_t)bb * C];
        double approx = 0.0;
        for (int k = 0; k < C; ++k) {
          double row = 0.0;
          for (int l = 0; l < C; ++l) row += ekl[k * C + l] * Pb[l];
          approx += Pa[k] * row;
        }
        double sx2 = sv[a] * sv[a], sy2 = sv[bb] * sv[bb];
        double exact = std::pow(sx2 * sy2 / (sx2 + sy2), 0.5 * d) * std::exp(-rho * rho / (2.0 * (sx2 + sy2)));
        double norm = std::pow(0.5 * sv[a] * sv[bb], 0.5 * d);
        worst = std::max(worst, std::fabs(approx - exact) / norm);
      }
  }
  return worst;
}

double trunc_error(const TRule& q, int d, double lo, double omega) {
  double s = 0.0;
  for (size_t j = 0; j < q.t.size(); ++j) s += q.wu[j] * std::erfc(2.0 * kPi * lo * q.chi[j] * omega);
  return d * s;
}

double alias_error(const TRule& q, int d, double hi, double P, double L) {
  double gap = std::max(P - L, 0.0);
  double s = 0.0;
  for (size_t j = 0; j < q.t.size(); ++j) s += q.wu[j] * std::exp(-gap * gap / (4.0 * hi * hi * q.chi[j] * q.chi[j]));
  return d * s;
}

template <class F>
double bisect_smallest(F ok, double lo, double hi) {
  // smallest x in [lo, hi] with ok(x) (ok monotone false -> true)
  for (int it = 0; it < 200; ++it) {
    double mid = 0.5 * (lo + hi);
    if (ok(mid))
      hi = mid;
    else
      lo = mid;
    if (hi - lo <= 1e-12 * hi) break;
  }
  return hi;
}

double inv_gamma_p(double a, double target) {
  // x with P(a, x) = target, bisection in log x
  double lo = -200.0, hi = std::log(std::max(1.0, a) * 100.0 + 100.0);
  for (int it = 0; it < 300; ++it) {
    double mid = 0.5 * (lo + hi);
    if (gamma_p(a, std::exp(mid)) > target)
      hi = mid;
    else
      lo = mid;
  }
  return std::exp(0.5 * (lo + hi));
}

double inv_gamma_q(double a, double target) {
  double lo = -200.0, hi = std::log(std::max(1.0, a) * 100.0 + 1000.0);
  for (int it = 0; it < 300; ++it) {
    double mid = 0.5 * (lo + hi);
    if (gamma_q(a, std::exp(mid)) > target)
      lo = mid;
    else
      hi = mid;
  }
  return std::exp(0.5 * (lo + hi));
}

// Fine-grid sizes: powers of two (the pruned row transforms of d <= 2 need them,
// and cuFFT is fastest there), and also 3 * 2^a in 3-D.
// Fine-grid sizes: powers of two for d <= 2 (the custom row transforms are radix 2^k);
// for d = 3 (cuFFT) any 7-smooth multiple of 4 (the interpolation's TMA copies need row
// strides of whole 16-byte units: nf * 4 bytes in FP32).
bool fft_friendly(long long n, int d) {
  if (d == 3 && n % 4 != 0) return false;
  while (n % 2 == 0) n /= 2;
  if (d != 3) return n == 1;
  for (long long p : {3ll, 5ll, 7ll})
    while (n % p == 0) n /= p;
  return n == 1;
}

// Spreading width for a NUFFT tolerance at upsampling sigma: the ES kernel's
// error behaves like c exp(-pi w sqrt(1 - 1/sigma)) with c between 3 and 6 for
// sigma in [1.25, 2] (checked against brute-force NUDFTs), so w is the smallest
// width with 6 exp(-pi w sqrt(1 - 1/sigma)) <= tol.
int width_for(double tol, double sigma) {
  double w = std::log(6.0 / tol) / (kPi * std::sqrt(1.0 - 1.0 / sigma));
  return std::max(2, (int)std::ceil(w - 1e-9));
}

}  // namespace

double phi_radial(int family, double nu, double r) {
  if (family == GP_SE) return std::exp(-0.5 * r * r);
  return matern_phi(nu, r);
}

// Regularised incomplete gamma functions P(a, x) and Q(a, x) = 1 - P(a, x), by the two
// textbook expansions: for x < a + 1 the power series
//   P(a, x) = e^{-x} x^a / Gamma(a) * sum_n x^n / (a (a+1) ... (a+n)),
// and for x >= a + 1 the continued fraction of Legendre for Q(a, x),
//   Q(a, x) = e^{-x} x^a / Gamma(a) * 1 / (x + 1 - a - 1 (1 - a) / (x + 3 - a - 2 (2 - a) / (x + 5 - a - ...))),
// evaluated from the front by the modified Lentz method (Lentz 1976, with Thompson and
// Barnett's guard against zero denominators).
double gamma_p(double a, double x) {
  if (x <= 0.0) return 0.0;
  if (x < a + 1.0) {
    double ap = a, sum = 1.0 / a, del = sum;
    for (int n = 0; n < 100000; ++n) {
      ap += 1.0;
      del *= x / ap;
      sum += del;
      if (std::fabs(del) < std::fabs(sum) * 1e-17) break;
    }
    return sum * std::exp(-x + a * std::log(x) - std::lgamma(a));
  }
  return 1.0 - gamma_q(a, x);
}

double gamma_q(double a, double x) {
  if (x <= 0.0) return 1.0;
  if (x < a + 1.0) return 1.0 - gamma_p(a, x);
  const double tiny = 1e-300;
  double b = x + 1.0 - a, c = 1.0 / tiny, dd = 1.0 / b, hh = dd;
  for (int i = 1; i < 100000; ++i) {
    double an = -i * (i - a);
    b += 2.0;
    dd = an * dd + b;
    if (std::fabs(dd) < tiny) dd = tiny;
    c = b + an / c;
    if (std::fabs(c) < tiny) c = tiny;
    dd = 1.0 / dd;
    double del = dd * c;
    hh *= del;
    if (std::fabs(del - 1.0) < 1e-16) break;
  }
  return std::exp(-x + a * std::log(x) - std::lgamma(a)) * hh;
}

double es_kernel(double s, int width, double beta) {
  double z = 2.0 * s / width;
  if (std::fabs(z) >= 1.0) return 0.0;
  return std::exp(beta * (std::sqrt(1.0 - z * z) - 1.0));
}

void select_hyper(Hyper& h, const gp_plan_opts& o, int precision, long long n_points) {
  const double eps = h.eps;
  const int d = h.d;
  // ---- stage 1: t quadrature -------------------------------------------------
  if (h.family == GP_SE) {
    h.n_t = 0;
    h.t_min = h.t_max = 0.0;
  } else if (o.set & GP_SET_NT) {
    GPN_CHECK(o.n_t >= 1 && o.t_max > o.t_min, GP_EINVAL, "n_t >= 1 and t_max > t_min required");
    h.n_t = o.n_t;
    h.t_min = o.t_min;
    h.t_max = o.t_max;
  } else {
    double e1 = eps / 4.0;
    h.t_min = std::log(inv_gamma_p(h.nu, e1 / 3.0));
    h.t_max = std::log(inv_gamma_q(h.nu, e1 / 3.0));
    int lo = 2, hi = 2;
    for (;;) {
      h.n_t = hi;
      if (stage1_error(h) <= e1 || hi >= 4096) break;
      lo = hi;
      hi *= 2;
    }
    while (hi - lo > 1) {
      int mid = (lo + hi) / 2;
      h.n_t = mid;
      if (stage1_error(h) <= e1)
        hi = mid;
      else
        lo = mid;
    }
    h.n_t = hi;
  }
  h.est_t = stage1_error(h);
  TRule q = trapezoid(h);
  // ---- stage 2: Chebyshev in sigma -------------------------------------------
  const bool flat = (h.sig_hi - h.sig_lo) <= 1e-14 * h.sig_hi;
  if (o.set & GP_SET_NSIGMA) {
    GPN_CHECK(o.n_sigma >= 0 && o.n_sigma < kMaxChannels, GP_EINVAL, "n_sigma out of range");
    GPN_CHECK(o.n_sigma > 0 || flat, GP_EINVAL, "n_sigma = 0 needs sigma_lo == sigma_hi");
    h.n_sigma = o.n_sigma;
  } else if (flat) {
    h.n_sigma = 0;
  } else {
    h.n_sigma = kMaxChannels - 1;
    for (int n = 1; n < kMaxChannels; ++n)
      if (stage2_error(d, h.sig_lo, h.sig_hi, n) <= eps / 4.0) {
        h.n_sigma = n;
        break;
      }
  }
  h.est_sigma = stage2_error(d, h.sig_lo, h.sig_hi, h.n_sigma);
  // ---- stage 3: Fourier grid -------------------------------------------------
  double L = 0.0;
  for (int a = 0; a < d; ++a) L = std::max(L, h.box_hi[a] - h.box_lo[a]);
  double P;
  if (o.set & GP_SET_DW) {
    GPN_CHECK(o.dw > 0.0, GP_EINVAL, "dw must be > 0");
    P = 1.0 / o.dw;
  } else {
    P = bisect_smallest([&](double p) { return alias_error(q, d, h.sig_hi, p, L) <= eps / 8.0; }, L, L + 1e3);
  }
  GPN_CHECK(P > L, GP_EINVAL, "Fourier period 1/dw must exceed the box side");
  h.dw = 1.0 / P;
  if (o.set & GP_SET_M) {
    GPN_CHECK(o.M >= 1, GP_EINVAL, "M must be >= 1");
    h.M = o.M;
  } else {
    double om = bisect_smallest([&](double w) { return trunc_error(q, d, h.sig_lo, w) <= eps / 4.0; }, 0.0, 1e9);
    h.M = (long long)std::ceil(om * P);
  }
  h.est_trunc = trunc_error(q, d, h.sig_lo, h.M * h.dw);
  h.est_alias = alias_error(q, d, h.sig_hi, P, L);
  // ---- NUFFT discretisation (App. D) -----------------------------------------
  if (o.set & GP_SET_NUFFT) {
    GPN_CHECK(o.nufft_tol > 0.0 && o.nufft_tol < 1.0, GP_EINVAL, "nufft_tol in (0,1)");
    h.nufft_tol = o.nufft_tol;
  } else {
    h.nufft_tol = precision == GP_FP32 ? std::max(eps / 10.0, 1e-6) : eps / 10.0;
  }
  const long long modes = 2 * h.M + 1;
  double min_up = (o.set & GP_SET_NUFFT) && o.upsampfac > 1.0 ? o.upsampfac : 1.25;
  long long nf;
  if (o.set & GP_SET_NF) {
    nf = o.nf;
    GPN_CHECK(nf > modes, GP_EINVAL, "nf must exceed 2M+1");
  } else {
    nf = 16;
    while (nf < (long long)std::ceil(min_up * modes) || !fft_friendly(nf, d)) ++nf;
  }
  for (;;) {
    h.nf = nf;
    h.upsamp = (double)nf / modes;
    h.width = width_for(h.nufft_tol, h.upsamp);
    // no wrap-around: the occupied cells plus the kernel support stay inside the grid
    double occ = L / P * nf + h.width + 4;
    bool fits = h.width <= kMaxWidth && occ <= nf;
    if (fits || (o.set & GP_SET_NF)) break;
    ++nf;
    while (!fft_friendly(nf, d)) ++nf;
  }
  // d = 3: pick nf by a cost model measured on the GB300 (FP32, 10 channels):
  //   FFTs:  rate(nf) s per cell and channel for the forward and inverse transform together
  //          (cuFFT batched 3-D R2C + C2R; the rate depends on the size's factors: 768 and
  //          840 run at 3.4e-11 and 5.2e-11, 864 and 1024 at 2.1e-11 and 1.8e-11);
  //   spreading + interpolation: 4.3e-12 s per point, channel and support cell (width^3),
  //          times 1.5 above width 9 (a bin tile of 8 cells no longer holds the support:
  //          channel chunks, fewer CTAs an SM).
  // Candidates are the measured sizes (below 240 any 7-smooth size at 2e-11, above 1024
  // powers of two at 1.8e-11) from the smallest admissible one up to 2.5 times the modes.
  // Measured on the 3-D N = 2e6 workload at eps = 1e-6: nf 768 (width 11) -> 864 (width 9)
  // took a CG iteration from 328 to 192 ms.
  if (d == 3 && !(o.set & GP_SET_NF)) {
    static const std::pair<int, double> kRate[] = {{240, 1.95e-11}, {250, 2.10e-11}, {252, 1.97e-11}, {256, 1.21e-11}, {270, 1.95e-11}, {280, 2.22e-11}, {288, 1.90e-11}, {294, 3.35e-11}, {300, 2.06e-11}, {320, 1.99e-11}, {336, 2.19e-11}, {350, 2.41e-11}, {360, 1.90e-11}, {378, 1.78e-11}, {384, 1.92e-11}, {392, 2.07e-11}, {400, 2.86e-11}, {420, 2.13e-11}, {432, 1.91e-11}, {448, 2.47e-11}, {450, 2.32e-11}, {480, 2.19e-11}, {486, 2.94e-11}, {490, 2.01e-11}, {500, 1.97e-11}, {504, 1.89e-11}, {512, 1.43e-11}, {540, 2.04e-11}, {560, 1.97e-11}, {576, 2.16e-11}, {588, 2.09e-11}, {600, 2.59e-11}, {630, 1.98e-11}, {640, 1.96e-11}, {648, 2.46e-11}, {672, 2.51e-11}, {686, 2.74e-11}, {700, 1.92e-11}, {720, 1.92e-11}, {750, 2.16e-11}, {756, 3.99e-11}, {768, 3.44e-11}, {784, 2.45e-11}, {800, 2.06e-11}, {810, 4.28e-11}, {840, 5.22e-11}, {864, 2.09e-11}, {882, 4.09e-11}, {896, 2.55e-11}, {900, 3.84e-11}, {960, 4.36e-11}, {972, 3.33e-11}, {980, 4.48e-11}, {1000, 2.06e-11}, {1008, 3.07e-11}, {1024, 1.80e-11}};
    auto rate = [&](long long c) -> double {
      if (!fft_friendly(c, 3)) return 0.0;
      if (c < 240) return 2.0e-11;
      if (c > 1024) return (c & (c - 1)) == 0 ? 1.8e-11 : 0.0;
      for (const auto& e : kRate)
        if (e.first == c) return e.second;
      return 0.0;
    };
    double best = -1.0;
    long long best_nf = nf;
    const double npts = (double)std::max<long long>(n_points, 1);
    for (long long c = nf; c <= (long long)(2.5 * modes) + 16; ++c) {
      const double rc = rate(c);
      if (rc <= 0.0) continue;
      const int w = width_for(h.nufft_tol, (double)c / modes);
      if (w > kMaxWidth || L / P * c + w + 4 > c) continue;
      const double cost = rc * (double)c * c * c + 4.3e-12 * npts * w * w * w * (w > 9 ? 1.5 : 1.0);
      if (best < 0.0 || cost < best) {
        best = cost;
        best_nf = c;
      }
    }
    nf = best_nf;
    h.nf = nf;
    h.upsamp = (double)nf / modes;
    h.width = width_for(h.nufft_tol, h.upsamp);
  }
  GPN_CHECK(h.width <= kMaxWidth, GP_EINVAL, "spreading kernel wider than 16 cells: raise nf or nufft_tol");
  GPN_CHECK(L / P * h.nf + h.width + 4 <= h.nf, GP_EINVAL, "points do not fit in the fine grid without wrap-around");
  h.beta = 0.97 * kPi * h.width * (1.0 - 1.0 / (2.0 * h.upsamp));
}

void build_tables(const Hyper& h, Tables& tb) {
  TRule q = trapezoid(h);
  const int J = (int)q.t.size();
  tb.t = q.t;
  tb.tau_u = q.wu;
  tb.chi = q.chi;
  tb.vt.resize(J);
  const double dwd = std::pow(h.dw, h.d);
  for (int j = 0; j < J; ++j) tb.vt[j] = dwd * q.wu[j] * std::pow(q.chi[j], -h.d);
  tb.nodes = cheb_nodes(h.sig_lo, h.sig_hi, h.n_sigma);
  tb.bary = cheb_bary(h.n_sigma);
  // 1-D transform of the spreading kernel in grid units:
  //   psihat(m) = int psi(s) cos(2 pi m s / nf) ds over |s| < width/2
  std::vector<double> gx, gw;
  gauss_legendre(4 * h.width + 40, gx, gw);
  tb.psihat.assign(h.M + 1, 0.0);
  for (long long m = 0; m <= h.M; ++m) {
    double acc = 0.0;
    for (size_t i = 0; i < gx.size(); ++i) {
      double s = 0.5 * h.width * gx[i];
      acc += gw[i] * es_kernel(s, h.width, h.beta) * std::cos(2.0 * kPi * m * s / h.nf);
    }
    tb.psihat[m] = 0.5 * h.width * acc;
  }
  const int C = h.n_sigma + 1;
  tb.etab.assign((size_t)C * J * (h.M + 1), 0.0);
  for (int k = 0; k < C; ++k)
    for (int j = 0; j < J; ++j) {
      double sc = tb.nodes[k] * tb.chi[j];
      double pre = std::sqrt(2.0 * kPi) * sc;
      double c = 2.0 * kPi * kPi * sc * sc * h.dw * h.dw;
      for (long long m = 0; m <= h.M; ++m)
        tb.etab[((size_t)k * J + j) * (h.M + 1) + m] = pre * std::exp(-c * (double)m * (double)m) / tb.psihat[m];
    }
}

}  // namespace gpn
