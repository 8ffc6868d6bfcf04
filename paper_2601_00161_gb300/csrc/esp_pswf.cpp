// Host-side FP64 numerics for plan construction: the order-zero prolate psi_0^c, the
// split constants, Gauss-Legendre rules and the piecewise Horner tables.
//
// psi_0^c (Appendix A.1, eqs. (formula)/(psidefinit)) is found as the lowest
// eigenfunction of the prolate differential operator L_c u = -((1-x^2)u')' + c^2 x^2 u,
// which commutes with the integral operator of eq. (formula).  In the Legendre basis
// sqrt(k+1/2) P_k the even part of L_c is a symmetric tridiagonal matrix; its smallest
// eigenvalue is bracketed by Sturm-sequence bisection and the eigenvector obtained by
// inverse iteration with a shift just below it (the shifted matrix is then positive
// definite, so the tridiagonal solve needs no pivoting).

#include "esp_pswf.h"

#include <algorithm>
#include <cmath>
#include <vector>

namespace esp {

namespace {

// number of eigenvalues of the symmetric tridiagonal (d, e) below x
int sturm_count(const std::vector<double>& d, const std::vector<double>& e, double x) {
  int count = 0;
  double piv = d[0] - x;
  if (piv < 0) ++count;
  for (size_t i = 1; i < d.size(); ++i) {
    double prev = (piv == 0.0) ? 1e-300 : piv;
    piv = d[i] - x - e[i - 1] * e[i - 1] / prev;
    if (piv < 0) ++count;
  }
  return count;
}

// solve (T - s I) y = b for symmetric tridiagonal T (positive definite after the shift)
void tridiag_solve(const std::vector<double>& d, const std::vector<double>& e, double s,
                   std::vector<double>& b) {
  const size_t n = d.size();
  std::vector<double> cp(n), dp(n);
  double den = d[0] - s;
  cp[0] = (n > 1) ? e[0] / den : 0.0;
  dp[0] = b[0] / den;
  for (size_t i = 1; i < n; ++i) {
    den = (d[i] - s) - e[i - 1] * cp[i - 1];
    if (den == 0.0) den = 1e-300;
    cp[i] = (i + 1 < n) ? e[i] / den : 0.0;
    dp[i] = (b[i] - e[i - 1] * dp[i - 1]) / den;
  }
  b[n - 1] = dp[n - 1];
  for (size_t i = n - 1; i-- > 0;) b[i] = dp[i] - cp[i] * b[i + 1];
}

}  // namespace

bool Prolate::solve(double c_in) {
  if (!(c_in > 0.0) || !std::isfinite(c_in)) return false;
  c = c_in;
  const int n = static_cast<int>(std::ceil(c)) + 40;  // even degrees 0, 2, ..., 2(n-1)
  std::vector<double> d(n), e(std::max(n - 1, 1));
  const double c2 = c * c;
  for (int i = 0; i < n; ++i) {
    const double k = 2.0 * i;
    d[i] = k * (k + 1.0) + c2 * (2.0 * k * k + 2.0 * k - 1.0) / ((2.0 * k - 1.0) * (2.0 * k + 3.0));
    if (i + 1 < n)
      e[i] = c2 * (k + 1.0) * (k + 2.0) / ((2.0 * k + 3.0) * std::sqrt((2.0 * k + 1.0) * (2.0 * k + 5.0)));
  }
  // Gershgorin bracket, then bisection to the smallest eigenvalue
  double lo = d[0] - std::fabs(e[0]), hi = d[0] + std::fabs(e[0]);
  for (int i = 0; i < n; ++i) {
    const double r = (i > 0 ? std::fabs(e[i - 1]) : 0.0) + (i + 1 < n ? std::fabs(e[i]) : 0.0);
    lo = std::min(lo, d[i] - r);
    hi = std::max(hi, d[i] + r);
  }
  for (int it = 0; it < 400; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (mid == lo || mid == hi) break;
    if (sturm_count(d, e, mid) >= 1)
      hi = mid;
    else
      lo = mid;
  }
  chi0 = hi;
  // inverse iteration with the shift just below chi0
  const double shift = lo - 1e-12 * std::max(1.0, std::fabs(lo));
  std::vector<double> v(n, 1.0);
  for (int it = 0; it < 6; ++it) {
    tridiag_solve(d, e, shift, v);
    double nrm = 0.0;
    for (double x : v) nrm += x * x;
    nrm = std::sqrt(nrm);
    for (double& x : v) x /= nrm;
  }
  // Legendre coefficients a_k of psi_0 = sum_k a_k P_k (odd k vanish)
  deg = 2 * (n - 1);
  a.assign(deg + 1, 0.0);
  for (int i = 0; i < n; ++i) a[2 * i] = v[i] * std::sqrt(2.0 * i + 0.5);
  if (eval(0.0) < 0.0)
    for (double& x : a) x = -x;
  psi_at_0 = eval(0.0);
  C0 = a[0];  // int_0^1 P_k = 1 for k = 0 and 0 for even k >= 2
  lambda0 = 2.0 * C0 / psi_at_0;  // (psidefinit) at x = 0: lambda_0 psi_0(0) = int psi_0
  return std::isfinite(psi_at_0) && psi_at_0 > 0.0 && C0 > 0.0;
}

double Prolate::eval(double x) const {
  // Legendre recurrence (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1}
  double p0 = 1.0, p1 = x, s = a[0];
  if (deg >= 1) s += a[1] * p1;
  for (int k = 1; k < deg; ++k) {
    const double p2 = ((2.0 * k + 1.0) * x * p1 - k * p0) / (k + 1.0);
    s += a[k + 1] * p2;
    p0 = p1;
    p1 = p2;
  }
  return s;
}

double Prolate::deriv(double x) const {
  // P'_{k+1} = P'_{k-1} + (2k+1) P_k
  double p0 = 1.0, p1 = x, dp0 = 0.0, dp1 = 1.0, s = 0.0;
  if (deg >= 1) s += a[1] * dp1;
  for (int k = 1; k < deg; ++k) {
    const double p2 = ((2.0 * k + 1.0) * x * p1 - k * p0) / (k + 1.0);
    const double dp2 = dp0 + (2.0 * k + 1.0) * p1;
    s += a[k + 1] * dp2;
    p0 = p1;
    p1 = p2;
    dp0 = dp1;
    dp1 = dp2;
  }
  return s;
}

double Prolate::integral(double u) const {
  // Legendre values P_0..P_{deg+1} at u and at 0
  std::vector<double> pu(deg + 2), pz(deg + 2);
  pu[0] = 1.0;
  pz[0] = 1.0;
  pu[1] = u;
  pz[1] = 0.0;
  for (int k = 1; k <= deg; ++k) {
    pu[k + 1] = ((2.0 * k + 1.0) * u * pu[k] - k * pu[k - 1]) / (k + 1.0);
    pz[k + 1] = (-k * pz[k - 1]) / (k + 1.0);
  }
  double s = a[0] * u;
  for (int k = 1; k <= deg; ++k)
    s += a[k] * ((pu[k + 1] - pu[k - 1]) - (pz[k + 1] - pz[k - 1])) / (2.0 * k + 1.0);
  return s;
}

void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < (n + 1) / 2; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    double dp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 1; k < n; ++k) {
        const double p2 = ((2.0 * k + 1.0) * z * p1 - k * p0) / (k + 1.0);
        p0 = p1;
        p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      const double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    double p0 = 1.0, p1 = z;
    for (int k = 1; k < n; ++k) {
      const double p2 = ((2.0 * k + 1.0) * z * p1 - k * p0) / (k + 1.0);
      p0 = p1;
      p1 = p2;
    }
    dp = n * (z * p1 - p0) / (z * z - 1.0);
    x[i] = -z;
    x[n - 1 - i] = z;
    w[i] = w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

// psi_0(1) / psi_0(0) without summing the Legendre series at x = 1 (that sum cancels
// down to the size of the ratio).  psi_0 is the solution of the prolate equation
// (1 - x^2) u'' - 2 x u' + (chi_0 - c^2 x^2) u = 0 that stays regular at the singular
// point x = 1: in y = 1 - x a power series sum_j b_j y^j with b_0 = 1 and
//   2 (j+1)^2 b_{j+1} = (j (j+1) + c^2 - chi_0) b_j - 2 c^2 b_{j-1} + c^2 b_{j-2},
// convergent for |y| < 2.  At x = 0 (y = 1) it sums to psi_0(0) / psi_0(1).
double Prolate::edge_ratio() const {
  const double c2 = c * c;
  double b0 = 1.0, bm1 = 0.0, bm2 = 0.0, sum = 1.0;
  for (int j = 0; j < 100000; ++j) {
    const double b1 = ((j * (j + 1.0) + c2 - chi0) * b0 - 2.0 * c2 * bm1 + c2 * bm2) /
                      (2.0 * (j + 1.0) * (j + 1.0));
    sum += b1;
    bm2 = bm1;
    bm1 = b0;
    b0 = b1;
    if (j >= 20 && std::fabs(b1) < 1e-18 * std::fabs(sum)) break;
  }
  return 1.0 / sum;
}

double c_from_tolerance(double delta) {
  if (!(delta > 0.0 && delta < 1.0)) return -1.0;
  auto ratio = [](double c) {
    Prolate p;
    if (!p.solve(c)) return -1.0;
    return p.edge_ratio();
  };
  double lo = 1e-3, hi = 4.0;
  while (ratio(hi) > delta) {
    hi *= 2.0;
    if (hi > 400.0) return -1.0;
  }
  for (int it = 0; it < 200 && hi - lo > 1e-14 * hi; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (ratio(mid) > delta)
      lo = mid;
    else
      hi = mid;
  }
  return 0.5 * (lo + hi);
}

double fit_piece(const std::function<double(double)>& f, double lo, double hi, int degree,
                 double* coef_out) {
  // Chebyshev interpolation in y in [-1, 1] (t = mid + half*y), then conversion to
  // monomials in tau = t - mid: b_k = (Chebyshev -> monomial in y)_k / half^k
  const int n = degree + 1;
  const double mid = 0.5 * (lo + hi), half = 0.5 * (hi - lo);
  std::vector<double> fy(n), cheb(n, 0.0);
  for (int i = 0; i < n; ++i) fy[i] = f(mid + half * std::cos(M_PI * (i + 0.5) / n));
  for (int k = 0; k < n; ++k) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += fy[i] * std::cos(M_PI * k * (i + 0.5) / n);
    cheb[k] = (k == 0 ? 1.0 : 2.0) * s / n;
  }
  // monomial coefficients of T_k via T_{k+1} = 2y T_k - T_{k-1}
  std::vector<double> mono(n, 0.0), tkm1(n, 0.0), tk(n, 0.0), tkp1(n, 0.0);
  tkm1[0] = 1.0;
  if (n > 1) tk[1] = 1.0;
  for (int j = 0; j < n; ++j) mono[j] += cheb[0] * tkm1[j];
  if (n > 1)
    for (int j = 0; j < n; ++j) mono[j] += cheb[1] * tk[j];
  for (int k = 1; k + 1 < n; ++k) {
    for (int j = 0; j < n; ++j) tkp1[j] = (j > 0 ? 2.0 * tk[j - 1] : 0.0) - tkm1[j];
    for (int j = 0; j < n; ++j) mono[j] += cheb[k + 1] * tkp1[j];
    tkm1.swap(tk);
    tk.swap(tkp1);
  }
  double scale = 1.0;
  for (int j = 0; j < n; ++j) {
    coef_out[j] = mono[j] / scale;
    scale *= half;
  }
  // verify against f on a fine set of points
  double err = 0.0;
  for (int i = 0; i <= 64; ++i) {
    const double t = lo + (hi - lo) * i / 64.0;
    const double tau = t - mid;
    double v = coef_out[degree];
    for (int j = degree - 1; j >= 0; --j) v = v * tau + coef_out[j];
    err = std::max(err, std::fabs(v - f(t)));
  }
  return err;
}

}  // namespace esp
