// Host-side chain diagnostics: effective sample size of the theta rows.
//
// The paper compares samplers by the time they need for an effective sample size of about
// 1000 in the population parameters after burn-in (Sec. 3, the normal-normal benchmark), and
// judges the luminosity-function chains by ESS and autocorrelation (Sec. 5.3). The estimator
// here is Geyer's (1992) initial monotone sequence: with the biased autocovariances
// gamma_k = (1/n) sum_t (x_t - xbar)(x_{t+k} - xbar) and rho_k = gamma_k / gamma_0, the pair
// sums Gamma_m = rho_2m + rho_2m+1 are summed while positive, each capped by the one before,
// tau = 2 sum Gamma_m - 1 (at least 1/n), ESS = n / tau.
#include <cmath>
#include <cstdint>
#include <vector>

#include "cudahm.h"
#include "internal.h"

namespace {

// gamma_k of one column (stride `cols`), by a direct sum: the estimator stops at the first
// non-positive pair, so only lags up to about twice the autocorrelation time are formed.
double autocov(const double* x, int64_t n, int32_t cols, double mean, int64_t k) {
  double s = 0.0;
  for (int64_t t = 0; t + k < n; ++t) s += (x[t * cols] - mean) * (x[(t + k) * cols] - mean);
  return s / static_cast<double>(n);
}

double ess_column(const double* x, int64_t n, int32_t cols) {
  if (n < 4) return static_cast<double>(n);
  double mean = 0.0;
  for (int64_t t = 0; t < n; ++t) mean += x[t * cols];
  mean /= static_cast<double>(n);
  const double g0 = autocov(x, n, cols, mean, 0);
  if (!(g0 > 0.0)) return static_cast<double>(n);
  double sum = 0.0, prev = INFINITY;
  for (int64_t m = 0; 2 * m + 1 < n; ++m) {
    const double r0 = (m == 0) ? 1.0 : autocov(x, n, cols, mean, 2 * m) / g0;
    const double g = r0 + autocov(x, n, cols, mean, 2 * m + 1) / g0;
    if (!(g > 0.0)) break;
    const double gm = g < prev ? g : prev;
    sum += gm;
    prev = gm;
  }
  double tau = 2.0 * sum - 1.0;
  if (tau < 1.0 / static_cast<double>(n)) tau = 1.0 / static_cast<double>(n);
  return static_cast<double>(n) / tau;
}

}  // namespace

extern "C" int cudahm_ess(const double* x_host, int64_t rows, int32_t cols, double* ess_out) {
  if (!x_host || !ess_out) return chm::record_error(CUDAHM_EINVAL, "cudahm_ess: NULL pointer");
  if (rows < 1 || cols < 1) return chm::record_error(CUDAHM_EINVAL, "cudahm_ess: rows and cols must be >= 1");
  for (int64_t q = 0; q < rows * static_cast<int64_t>(cols); ++q)
    if (!std::isfinite(x_host[q])) return chm::record_error(CUDAHM_ENUMERIC, "cudahm_ess: non-finite sample");
  for (int32_t c = 0; c < cols; ++c) ess_out[c] = ess_column(x_host + c, rows, cols);
  return CUDAHM_OK;
}
