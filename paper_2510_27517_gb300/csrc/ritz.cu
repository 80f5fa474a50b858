// Condition-number estimates from PCG's own coefficients (host code).
//
// Sec. 4.5 judges a preconditioner by kappa and Kaporin's condition number of
// A M^-1.  The step lengths alpha_j and ratios beta_j of k PCG iterations
// define the symmetric tridiagonal Lanczos matrix T_k of M^-1 A
// (diagonal 1/alpha_j + beta_{j-1}/alpha_{j-1}, off-diagonal
// sqrt(beta_j)/alpha_j), whose eigenvalues (Ritz values) approximate the
// spectrum from inside.  Eigenvalues are found by bisection on Sturm-sequence
// counts (the LDL^T pivots of T - x I: the number of negative pivots is the
// number of eigenvalues below x); the first components of the eigenvectors
// come from the ratio of characteristic polynomials
//   w_i^2 = prod_j (theta_i - mu_j) / prod_{j != i} (theta_i - theta_j),
// mu_j the eigenvalues of T with its first row and column removed.
#include <cfloat>
#include <cmath>
#include <vector>

#include "internal.cuh"

namespace {

struct Tri {
  std::vector<double> a;   // diagonal
  std::vector<double> e2;  // squared off-diagonal
  double pivmin = DBL_MIN;
  double lo = 0.0, hi = 0.0;  // Gershgorin bounds
};

bool make_tri(const double* alpha, const double* beta, int64_t k, int64_t first, int64_t m, Tri& t) {
  t.a.assign(m, 0.0);
  t.e2.assign(m > 0 ? m - 1 : 0, 0.0);
  for (int64_t j = 0; j < k; ++j)
    if (!(alpha[j] > 0.0) || !std::isfinite(alpha[j])) return false;
  for (int64_t j = 0; j + 1 < k; ++j)
    if (!(beta[j] > 0.0) || !std::isfinite(beta[j])) return false;
  double emax = 0.0;
  for (int64_t i = 0; i < m; ++i) {
    const int64_t j = first + i;
    t.a[i] = 1.0 / alpha[j] + (j > 0 ? beta[j - 1] / alpha[j - 1] : 0.0);
    if (i + 1 < m) {
      const double e = std::sqrt(beta[j]) / alpha[j];
      t.e2[i] = e * e;
      emax = std::fmax(emax, e * e);
    }
  }
  t.pivmin = DBL_MIN * std::fmax(1.0, emax);
  t.lo = HUGE_VAL;
  t.hi = -HUGE_VAL;
  for (int64_t i = 0; i < m; ++i) {
    const double r = (i > 0 ? std::sqrt(t.e2[i - 1]) : 0.0) + (i + 1 < m ? std::sqrt(t.e2[i]) : 0.0);
    t.lo = std::fmin(t.lo, t.a[i] - r);
    t.hi = std::fmax(t.hi, t.a[i] + r);
  }
  return true;
}

// eigenvalues of t below x
int64_t count_below(const Tri& t, double x) {
  int64_t c = 0;
  double q = 1.0;
  for (size_t i = 0; i < t.a.size(); ++i) {
    q = (t.a[i] - x) - (i > 0 ? t.e2[i - 1] / q : 0.0);
    if (std::fabs(q) < t.pivmin) q = -t.pivmin;
    if (q < 0.0) ++c;
  }
  return c;
}

// the i-th smallest eigenvalue (0-based)
double kth_eigenvalue(const Tri& t, int64_t i) {
  double lo = t.lo, hi = t.hi;
  const double span = std::fmax(std::fabs(lo), std::fabs(hi));
  lo -= 2 * DBL_EPSILON * span + t.pivmin;
  hi += 2 * DBL_EPSILON * span + t.pivmin;
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    if (hi - lo <= 4 * DBL_EPSILON * std::fmax(std::fabs(lo), std::fabs(hi)) + t.pivmin) break;
    if (count_below(t, mid) > i) hi = mid;
    else lo = mid;
  }
  return 0.5 * (lo + hi);
}

}  // namespace

using namespace spai;

extern "C" int spai_ritz_extremes(const double* alpha, const double* beta, int64_t k, double* lam_min,
                                  double* lam_max) {
  if (!alpha || (k > 1 && !beta) || k < 1 || !lam_min || !lam_max)
    return set_error(SPAI_ERR_INVALID, "ritz: need k >= 1 coefficients and outputs");
  Tri t;
  if (!make_tri(alpha, beta, k, 0, k, t)) return set_error(SPAI_ERR_INVALID, "ritz: coefficients must be positive");
  *lam_min = kth_eigenvalue(t, 0);
  *lam_max = kth_eigenvalue(t, k - 1);
  return SPAI_OK;
}

extern "C" int spai_ritz_kaporin(const double* alpha, const double* beta, int64_t k, double* kaporin) {
  if (!alpha || (k > 1 && !beta) || k < 1 || !kaporin)
    return set_error(SPAI_ERR_INVALID, "ritz: need k >= 1 coefficients and an output");
  const int64_t m = k < 400 ? k : 400;
  Tri t, tt;
  if (!make_tri(alpha, beta, k, 0, m, t)) return set_error(SPAI_ERR_INVALID, "ritz: coefficients must be positive");
  std::vector<double> theta(m), mu(m > 1 ? m - 1 : 0);
  for (int64_t i = 0; i < m; ++i) theta[i] = kth_eigenvalue(t, i);
  if (m > 1) {
    tt.a.assign(t.a.begin() + 1, t.a.end());
    tt.e2.assign(t.e2.begin() + 1, t.e2.end());
    tt.pivmin = t.pivmin;
    tt.lo = t.lo;
    tt.hi = t.hi;
    for (int64_t j = 0; j + 1 < m; ++j) mu[j] = kth_eigenvalue(tt, j);
  }
  if (!(theta[0] > 0.0)) return set_error(SPAI_ERR_INVALID, "ritz: T is not positive definite");
  std::vector<double> lw(m, 0.0);
  double lmax = -HUGE_VAL;
  for (int64_t i = 0; i < m; ++i) {
    double s = 0.0;
    for (int64_t j = 0; j + 1 < m; ++j) s += std::log(std::fmax(std::fabs(theta[i] - mu[j]), DBL_MIN));
    for (int64_t j = 0; j < m; ++j)
      if (j != i) s -= std::log(std::fmax(std::fabs(theta[i] - theta[j]), DBL_MIN));
    lw[i] = s;
    lmax = std::fmax(lmax, s);
  }
  double wsum = 0.0, am = 0.0, lg = 0.0;
  for (int64_t i = 0; i < m; ++i) wsum += std::exp(lw[i] - lmax);
  for (int64_t i = 0; i < m; ++i) {
    const double w = std::exp(lw[i] - lmax) / wsum;
    am += w * theta[i];
    lg += w * std::log(theta[i]);
  }
  *kaporin = am / std::exp(lg);
  return SPAI_OK;
}
