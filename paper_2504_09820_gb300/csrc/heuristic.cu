// Precision selection of Sections III-B and IV-B (eq. heuristic / heuristic_bj) and a
// condition-number estimate from CG step sizes.  Host code only.
#include <math.h>

#include <vector>

#include "../../include/fpcg.h"

namespace {

// Unit roundoffs of Table I (round to nearest): 2^-8, 2^-11, 2^-24, 2^-53.
struct Fmt {
  int code;
  double u;
};
const Fmt kTableI[] = {{FPCG_BF16, 0.00390625}, {FPCG_FP16, 0.00048828125},
                       {FPCG_FP32, 5.9604644775390625e-08}, {FPCG_FP64, 1.1102230246251565e-16}};

// Number of eigenvalues of the symmetric tridiagonal (d, e) smaller than x
// (Sturm sequence count of negative pivots of T - x I).
int count_below(const std::vector<double>& d, const std::vector<double>& e, double x) {
  int c = 0;
  double q = 1.0;
  for (size_t i = 0; i < d.size(); ++i) {
    const double off = i ? e[i - 1] * e[i - 1] : 0.0;
    q = d[i] - x - (i ? off / q : 0.0);
    if (q == 0.0) q = -1e-300;  // a zero pivot counts as negative
    if (q < 0.0) ++c;
  }
  return c;
}

// The j-th smallest eigenvalue (0-based) by bisection in the Gershgorin interval.
double eig(const std::vector<double>& d, const std::vector<double>& e, int j) {
  double lo = INFINITY, hi = -INFINITY;
  for (size_t i = 0; i < d.size(); ++i) {
    const double r = (i ? fabs(e[i - 1]) : 0.0) + (i + 1 < d.size() ? fabs(e[i]) : 0.0);
    lo = fmin(lo, d[i] - r);
    hi = fmax(hi, d[i] + r);
  }
  for (int it = 0; it < 200 && hi - lo > 1e-15 * fmax(fabs(lo), fabs(hi)); ++it) {
    const double mid = 0.5 * (lo + hi);
    if (count_below(d, e, mid) > j) hi = mid;
    else lo = mid;
  }
  return 0.5 * (lo + hi);
}

// Multiplication weights of the cost model (Section V-A.1): 16-bit 1, fp32 2, fp64 4.
double weight(int32_t fmt) {
  switch (fmt) {
    case FPCG_BF16:
    case FPCG_FP16: return 1.0;
    case FPCG_FP32: return 2.0;
    case FPCG_FP64: return 4.0;
    default: return 0.0;
  }
}

// Iterations the CG bound 2 q^k <= tol asks for, q = (sqrt(kappa) - 1) / (sqrt(kappa) + 1).
int cg_iterations(double kappa, double tol) {
  const double sk = sqrt(kappa);
  const double q = (sk - 1.0) / (sk + 1.0);
  if (q <= 0.0) return 1;
  return (int)ceil(log(tol / 2.0) / log(q));
}

}  // namespace

extern "C" {

int fpcg_choose_precision(int32_t k, double kappa, double* u_bound) {
  if (k < 1 || !(kappa >= 1.0) || !isfinite(kappa)) return -FPCG_EINVAL;
  const double bound = 1.0 / (pow((double)k, 1.5) * sqrt(kappa));
  if (u_bound) *u_bound = bound;
  for (const Fmt& f : kTableI)
    if (f.u < bound) return f.code;
  return FPCG_FP64;
}

int fpcg_kappa_cg(const double* alpha, const double* beta, int32_t m, double* kappa_hat) {
  if (!alpha || !kappa_hat || m < 1 || (m > 1 && !beta)) return FPCG_EINVAL;
  std::vector<double> d((size_t)m), e((size_t)(m > 1 ? m - 1 : 0));
  for (int j = 0; j < m; ++j) {
    if (!(alpha[j] > 0.0) || (j < m - 1 && !(beta[j] >= 0.0))) return FPCG_EINVAL;
    d[(size_t)j] = 1.0 / alpha[j] + (j ? beta[j - 1] / alpha[j - 1] : 0.0);
    if (j < m - 1) e[(size_t)j] = sqrt(beta[j]) / alpha[j];
  }
  const double lmin = eig(d, e, 0), lmax = eig(d, e, m - 1);
  if (!(lmin > 0.0)) return FPCG_EINVAL;
  *kappa_hat = lmax / lmin;
  return FPCG_OK;
}

int fpcg_kappa_cg_batch(const float* coeffs, int32_t iters, int32_t m, int64_t batch, double* kappa_hat) {
  if (!coeffs || !kappa_hat || m < 1 || m > iters || batch < 0) return FPCG_EINVAL;
  std::vector<double> a((size_t)m), b((size_t)m);
  for (int64_t s = 0; s < batch; ++s) {
    const float* c = coeffs + (size_t)s * 2 * iters;
    for (int j = 0; j < m; ++j) {
      a[(size_t)j] = c[j];
      b[(size_t)j] = c[iters + j];
    }
    double k = NAN;
    if (fpcg_kappa_cg(a.data(), b.data(), m, &k) != FPCG_OK) k = NAN;
    kappa_hat[s] = k;
  }
  return FPCG_OK;
}

int fpcg_choose_method(int32_t k, int32_t block_L, double kappa, double kappa_bar, double tol, int32_t mv_cg,
                       int32_t mv_bj, int32_t w, int32_t* k_cg, int32_t* k_pcg) {
  const double wc = weight(mv_cg), wb = weight(mv_bj), ww = weight(w);
  if (k < 1 || block_L < 1 || k % block_L || !(kappa >= 1.0) || !isfinite(kappa) || !(kappa_bar >= 1.0) ||
      !isfinite(kappa_bar) || !(tol > 0.0 && tol < 1.0) || wc <= 0.0 || wb <= 0.0 || ww <= 0.0)
    return -FPCG_EINVAL;
  const int kc = cg_iterations(kappa, tol), kp = cg_iterations(kappa_bar, tol);
  if (k_cg) *k_cg = kc;
  if (k_pcg) *k_pcg = kp;
  const double K = k, L = block_L;
  const double c_it = K * K * wc, p_it = K * K * wb + K * L * ww, c_bj = (K / L) * L * L * L * ww;
  return (double)(kc - kp) > c_bj / c_it + kp * (p_it / c_it - 1.0) ? block_L : 0;
}

}  // extern "C"
