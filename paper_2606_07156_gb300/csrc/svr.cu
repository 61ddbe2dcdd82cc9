// SVR-RBF precision model of Section 3.4: training on the host (a comparator
// to the MLP predictor; the sample count is small, 1280 in the paper). The
// model, the dual and the coordinate-descent solver are stated with
// anns_svr_fit in anns_amp.h. Host code only: no GPU is used.
#include <cmath>
#include <new>
#include <vector>

#include "internal.h"

using namespace anns;

extern "C" int anns_svr_fit(const double* X, const double* y, int64_t n, int32_t dim, double C, double gamma,
                            double eps, double tol, int64_t max_sweeps, double* beta_out, int64_t* sweeps_out) {
  if (!X || !y || !beta_out) return fail(ANNS_ERR_INVALID_ARG, "null pointer");
  if (n < 1 || n > ANNS_SVR_MAX_SAMPLES) return fail(ANNS_ERR_INVALID_ARG, "n must be in [1, ANNS_SVR_MAX_SAMPLES]");
  if (dim < 1) return fail(ANNS_ERR_INVALID_ARG, "dim must be >= 1");
  if (!(C > 0.0) || !(gamma > 0.0) || !(eps >= 0.0) || !(tol >= 0.0) || max_sweeps < 1)
    return fail(ANNS_ERR_INVALID_ARG, "need C > 0, gamma > 0, eps >= 0, tol >= 0, max_sweeps >= 1");
  std::vector<double> K1, f, beta;
  try {
    K1.assign((size_t)n * n, 0.0);
    f.assign(n, 0.0);
    beta.assign(n, 0.0);
  } catch (const std::bad_alloc&) {
    return fail(ANNS_ERR_OOM, "svr kernel matrix");
  }
  // K1[i][j] = exp(-gamma |x_i - x_j|^2) + 1, the squared distance summed over
  // features in ascending order
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = 0; j < n; ++j) {
      double d2 = 0.0;
      for (int32_t c = 0; c < dim; ++c) {
        const double e = X[i * dim + c] - X[j * dim + c];
        d2 += e * e;
      }
      K1[(size_t)i * n + j] = std::exp(-gamma * d2) + 1.0;
    }
  int64_t sweeps = 0;
  for (sweeps = 1; sweeps <= max_sweeps; ++sweeps) {
    double big = 0.0;
    for (int64_t i = 0; i < n; ++i) {
      const double a = K1[(size_t)i * n + i];
      // the objective in coordinate i: 1/2 a b^2 + c b + eps |b|
      const double c = f[i] - a * beta[i] - y[i];
      double b = 0.0;
      if (c < -eps) b = (-c - eps) / a;
      else if (c > eps) b = (-c + eps) / a;
      b = std::fmin(std::fmax(b, -C), C);
      const double d = b - beta[i];
      if (d != 0.0) {
        for (int64_t j = 0; j < n; ++j) f[j] += d * K1[(size_t)j * n + i];
        beta[i] = b;
        big = std::fmax(big, std::fabs(d));
      }
    }
    if (big <= tol) break;
  }
  if (sweeps > max_sweeps) sweeps = max_sweeps;
  for (int64_t i = 0; i < n; ++i) beta_out[i] = beta[i];
  if (sweeps_out) *sweeps_out = sweeps;
  return ANNS_OK;
}
