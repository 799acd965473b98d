// Hyperparameter selection and host tables of the approximation K~ (Sec. 3, Sec. 5.4).
#pragma once

#include <vector>

#include "common.h"

namespace gpn {

// Everything that defines K~ (Eq. Ktilde) plus the NUFFT discretisation of App. D.
struct Hyper {
  int d = 1;
  int family = GP_MATERN;
  double nu = 1.5;
  double eps = 1e-6;
  // Sec. 3.2: trapezoid rule in t
  int n_t = 0;
  double t_min = 0.0, t_max = 0.0;
  // Sec. 3.3: Chebyshev-Lobatto interpolation in sigma
  int n_sigma = 0;
  double sig_lo = 0.0, sig_hi = 0.0;
  // Sec. 3.4: Fourier grid n dw, n in {-M..M}^d
  long long M = 0;
  double dw = 0.0;
  // App. D: fine grid and spreading kernel
  long long nf = 0;
  int width = 0;
  double beta = 0.0;
  double upsamp = 0.0;
  double nufft_tol = 0.0;
  int tile = 0;
  // region the points (and queries) occupy; grid coordinate g = (x - centre)/h + nf/2
  double box_lo[kMaxDim] = {0, 0, 0}, box_hi[kMaxDim] = {0, 0, 0};
  // stage error estimates (relative, entrywise)
  double est_t = 0, est_sigma = 0, est_trunc = 0, est_alias = 0;
};

// Quadrature and interpolation tables, float64, host side.
struct Tables {
  std::vector<double> t, tau_u, chi, vt;   // vt_j = dw^d tau_j chi_j^-d u(t_j)
  std::vector<double> nodes, bary;         // sigma_k and barycentric weights
  std::vector<double> psihat;              // 1-D transform of the spreading kernel, m = 0..M
  std::vector<double> etab;                // E'[k][j][m] = sqrt(2 pi) sigma_k chi_j exp(-2 pi^2 (sigma_k chi_j dw m)^2) / psihat(m)
};

// phi of Eq. (matern) (family GP_MATERN) or Eq. (squaredexp) (GP_SE).
double phi_radial(int family, double nu, double r);

// Regularised incomplete gamma functions P(a, x) and Q(a, x) = 1 - P(a, x).
double gamma_p(double a, double x);
double gamma_q(double a, double x);

// Pick every hyperparameter not fixed by opts (opts->set bits).  sig_lo/sig_hi and
// box must already be set in h (from data or overrides).  Fills h.
void select_hyper(Hyper& h, const gp_plan_opts& o, int precision, long long n_points);

// Build the tables for h (h must be complete).
void build_tables(const Hyper& h, Tables& tb);

// Exponential-of-semicircle kernel value at offset s (grid cells) from the point.
double es_kernel(double s, int width, double beta);

}  // namespace gpn
