/* Exact sampled rows of K alpha by direct summation (TEST INFRASTRUCTURE).
 *
 * Part of the CPU oracle: only tests, the smoke check and the CPU-baseline leg
 * of the benchmark use it.  It shares no code with the CUDA library.
 *
 * For each requested row i:
 *   out[i] = sum_j K(x_i, x_j) alpha_j,
 *   K(x, y) = w(x) w(y) (2 pi [sigma^2(x) + sigma^2(y)])^(-d/2) phi(|x - y| / sqrt(sigma^2(x) + sigma^2(y)))
 * (Sec. 3, Eq. (nonstat2)) with phi the Matern function (Sec. 2, Eq. (matern)) in
 * its closed forms for nu = 1/2, 3/2, 5/2, or the squared exponential
 * (Eq. (squaredexp)) when nu is passed as a negative number.
 *
 * Arrays: X is N x d row-major; w, sigma are N; alpha is N x R column-major
 * (column r at alpha + r*N); rows has n_rows indices; out is n_rows x R
 * column-major.  Sums run in ascending j in double precision; each row is
 * independent and rows are spread over OpenMP threads.
 */
#include <math.h>
#include <stdint.h>

static double phi_eval(double r, double nu) {
  if (nu < 0.0) return exp(-0.5 * r * r);
  if (nu == 0.5) return exp(-r);
  if (nu == 1.5) {
    double a = sqrt(3.0) * r;
    return (1.0 + a) * exp(-a);
  }
  /* nu == 2.5 */
  double a = sqrt(5.0) * r;
  return (1.0 + a + a * a / 3.0) * exp(-a);
}

int oracle_rows_supported(double nu) { return nu < 0.0 || nu == 0.5 || nu == 1.5 || nu == 2.5; }

int oracle_rows(const double* X, const double* w, const double* sigma, int64_t N, int d, double nu,
                const double* alpha, int R, const int64_t* rows, int64_t n_rows, double* out) {
  if (!oracle_rows_supported(nu) || d < 1 || d > 3 || R < 1) return -1;
  const double two_pi = 6.283185307179586476925286766559;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t q = 0; q < n_rows; ++q) {
    int64_t i = rows[q];
    double acc[64];
    for (int r = 0; r < R && r < 64; ++r) acc[r] = 0.0;
    for (int64_t j = 0; j < N; ++j) {
      double r2 = 0.0;
      for (int a = 0; a < d; ++a) {
        double t = X[i * d + a] - X[j * d + a];
        r2 += t * t;
      }
      double ss = sigma[i] * sigma[i] + sigma[j] * sigma[j];
      double k = w[i] * w[j] * pow(two_pi * ss, -0.5 * d) * phi_eval(sqrt(r2 / ss), nu);
      for (int r = 0; r < R && r < 64; ++r) acc[r] += k * alpha[(int64_t)r * N + j];
    }
    for (int r = 0; r < R && r < 64; ++r) out[(int64_t)r * n_rows + q] = acc[r];
  }
  return 0;
}
