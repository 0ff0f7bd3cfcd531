// Host post-processing of the paper's Sec. 4.4-4.6 results, behind the C ABI:
// Delta+- of Eqs. diff1, diff2 over bond strengths that the lattice makes
// equivalent, the polynomial extrapolation of e_g (or any observable) to
// eps -> 0 (Eq. tru and the quadratic fit of the energy against the
// truncation error), and the exponential fit of a correlation function that
// gives the correlation length.  Least squares by Householder QR of the
// design matrix (no normal equations), standard deviations from the residual
// variance: sd(c_i)^2 = s^2 [(A^T A)^-1]_ii = s^2 |row i of R^-1|^2,
// s^2 = RSS / (N - p).
#include <math.h>

#include <vector>

#include "idmrg.h"

namespace {

// min |A c - y| for A (n x p, row-major), p <= 8; returns false when A is
// rank deficient.  rinv_row2[i] = |row i of R^-1|^2, rss = residual sum.
bool lsq_qr(std::vector<double> A, std::vector<double> y, int n, int p, double *c, double *rinv_row2,
            double *rss) {
  if (n < p || p < 1 || p > 8) return false;
  double scale = 0.0;
  for (double v : A) scale = fmax(scale, fabs(v));
  for (int k = 0; k < p; ++k) {
    double nrm = 0.0;
    for (int i = k; i < n; ++i) nrm += A[(size_t)i * p + k] * A[(size_t)i * p + k];
    nrm = sqrt(nrm);
    if (!(nrm > 1e-14 * scale)) return false;
    const double alpha = A[(size_t)k * p + k] > 0 ? -nrm : nrm;
    // v = x - alpha e_k, H = I - 2 v v^T / v^T v
    std::vector<double> v(n - k);
    for (int i = k; i < n; ++i) v[i - k] = A[(size_t)i * p + k];
    v[0] -= alpha;
    double vv = 0.0;
    for (double t : v) vv += t * t;
    for (int j = k; j < p; ++j) {
      double d = 0.0;
      for (int i = k; i < n; ++i) d += v[i - k] * A[(size_t)i * p + j];
      const double f = 2.0 * d / vv;
      for (int i = k; i < n; ++i) A[(size_t)i * p + j] -= f * v[i - k];
    }
    double d = 0.0;
    for (int i = k; i < n; ++i) d += v[i - k] * y[i];
    const double f = 2.0 * d / vv;
    for (int i = k; i < n; ++i) y[i] -= f * v[i - k];
  }
  // back substitution R c = (Q^T y)[0..p)
  for (int i = p - 1; i >= 0; --i) {
    double s = y[i];
    for (int j = i + 1; j < p; ++j) s -= A[(size_t)i * p + j] * c[j];
    c[i] = s / A[(size_t)i * p + i];
  }
  double r = 0.0;
  for (int i = p; i < n; ++i) r += y[i] * y[i];
  *rss = r;
  // R^-1 (upper triangular), column by column
  std::vector<double> Ri((size_t)p * p, 0.0);
  for (int j = 0; j < p; ++j) {
    Ri[(size_t)j * p + j] = 1.0 / A[(size_t)j * p + j];
    for (int i = j - 1; i >= 0; --i) {
      double s = 0.0;
      for (int k = i + 1; k <= j; ++k) s += A[(size_t)i * p + k] * Ri[(size_t)k * p + j];
      Ri[(size_t)i * p + j] = -s / A[(size_t)i * p + i];
    }
  }
  for (int i = 0; i < p; ++i) {
    double s = 0.0;
    for (int j = 0; j < p; ++j) s += Ri[(size_t)i * p + j] * Ri[(size_t)i * p + j];
    rinv_row2[i] = s;
  }
  return true;
}

}  // namespace

extern "C" {

idmrg_status idmrg_delta_pm(const double *values, int n, double *avg, double *dplus, double *dminus) {
  if (!values || n < 1) return IDMRG_EINVAL;
  double s = 0.0, mx = values[0], mn = values[0];
  for (int i = 0; i < n; ++i) {
    if (!isfinite(values[i])) return IDMRG_EINVAL;
    s += values[i];
    mx = fmax(mx, values[i]);
    mn = fmin(mn, values[i]);
  }
  const double a = s / n;
  if (avg) *avg = a;
  if (dplus) *dplus = mx - a;
  if (dminus) *dminus = mn - a;
  return IDMRG_OK;
}

idmrg_status idmrg_extrapolate(const double *eps, const double *value, int n, int degree, double *v0, double *sd) {
  if (!eps || !value || degree < 0 || degree > 6 || n < degree + 1) return IDMRG_EINVAL;
  const int p = degree + 1;
  std::vector<double> A((size_t)n * p), y(value, value + n);
  for (int i = 0; i < n; ++i) {
    double x = 1.0;
    for (int j = 0; j < p; ++j) {
      A[(size_t)i * p + j] = x;
      x *= eps[i];
    }
  }
  double c[8], r2[8], rss = 0.0;
  if (!lsq_qr(A, y, n, p, c, r2, &rss)) return IDMRG_EINVAL;
  if (v0) *v0 = c[0];
  if (sd) *sd = n > p ? sqrt(fmax(rss / (n - p) * r2[0], 0.0)) : 0.0;
  return IDMRG_OK;
}

idmrg_status idmrg_fit_correlation_length(const double *r, const double *c, int n, double r_min, double *xi,
                                          double *sd) {
  if (!r || !c || n < 0) return IDMRG_EINVAL;
  std::vector<double> A, y;
  for (int i = 0; i < n; ++i)
    if (r[i] > r_min && c[i] != 0.0 && isfinite(c[i])) {
      A.push_back(1.0);
      A.push_back(r[i]);
      y.push_back(log(fabs(c[i])));
    }
  const int m = (int)y.size();
  if (m < 2) return IDMRG_EINVAL;
  double co[2], r2[2], rss = 0.0;
  if (!lsq_qr(A, y, m, 2, co, r2, &rss)) return IDMRG_EINVAL;
  const double b = co[1];
  if (!(b != 0.0)) return IDMRG_EINVAL;
  if (xi) *xi = -1.0 / b;
  if (sd) *sd = m > 2 ? sqrt(fmax(rss / (m - 2) * r2[1], 0.0)) / (b * b) : 0.0;
  return IDMRG_OK;
}

}  // extern "C"
