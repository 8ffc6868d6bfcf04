// Host-side FP64 numerics used at plan time (see esp_pswf.cpp).
#pragma once

#include <functional>
#include <vector>

namespace esp {

// psi_0^c on [-1, 1] as a Legendre series (Appendix A.1), unit L2 norm, psi_0(0) > 0.
struct Prolate {
  double c = 0.0;
  double chi0 = 0.0;      // smallest eigenvalue of the prolate differential operator
  double psi_at_0 = 0.0;  // psi_0(0)
  double C0 = 0.0;        // int_0^1 psi_0 (Sec. 3.1)
  double lambda0 = 0.0;   // eigenvalue of eq. (formula), from eq. (psidefinit) at x = 0
  int deg = 0;
  std::vector<double> a;  // coefficients of P_k, k = 0..deg

  bool solve(double c);
  double eval(double x) const;   // psi_0(x), |x| <= 1
  double deriv(double x) const;  // psi_0'(x), |x| <= 1
  // int_0^u psi_0, |u| <= 1, term by term: int P_k = (P_{k+1} - P_{k-1}) / (2k + 1), k >= 1
  double integral(double u) const;
  // psi_0(1) / psi_0(0) from the regular series of the prolate equation at x = 1 (no
  // cancellation, unlike eval(1.0) for small ratios)
  double edge_ratio() const;
};

void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w);

// c with psi_0^c(1) / psi_0^c(0) = delta; negative on failure.
double c_from_tolerance(double delta);

// Polynomial of the given degree interpolating f on [lo, hi] at Chebyshev points, as
// monomial coefficients in tau = t - (lo+hi)/2 (for Horner).  Returns max |error| on a
// uniform check grid.
double fit_piece(const std::function<double(double)>& f, double lo, double hi, int degree,
                 double* coef_out);

}  // namespace esp
