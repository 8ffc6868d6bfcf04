"""O-PSWF: the order-zero prolate spheroidal wave function (test infrastructure).

Part of the FP64 CPU oracle; only tests, the smoke check and the benchmark's CPU legs
may import it.

Definition followed (Appendix A.1, eqs. (formula) and (psidefinit)): psi_0^c is the
eigenfunction of F_c[phi](x) = int_{-1}^{1} phi(t) exp(i c x t) dt with the largest
eigenvalue lambda_0, normalised to unit L2 norm on [-1, 1] and taken positive at 0.

Method.  F_c commutes with the prolate differential operator
    L_c u = -((1 - x^2) u')' + c^2 x^2 u,
so psi_0^c is also the eigenfunction of L_c with the SMALLEST eigenvalue.  In the
orthonormal Legendre basis  Pbar_k = sqrt(k + 1/2) P_k  the matrix of L_c is symmetric
and couples only k and k +/- 2 (use x^2 P_k from the three-term recurrence twice), so
the even part is a small symmetric tridiagonal eigenproblem, solved here with a library
symmetric eigensolver.  This is the standard Legendre-Galerkin route to prolates
(Xiao, Rokhlin and Yarvin, Inverse Problems 17 (2001)); the paper itself only cites
Osipov-Rokhlin-Xiao for the function.

lambda_0 follows from (psidefinit) at x = 0:  lambda_0 psi_0(0) = int psi_0.
C_0 = int_0^1 psi_0 (Sec. 3.1, eq. (decomposition)).

For |x| > 1 the Legendre series is numerically unusable (P_k grows like
(x + sqrt(x^2-1))^k); there psi_0 means the entire extension defined by (psidefinit)
itself, lambda_0 psi_0(x) = int_{-1}^{1} psi_0(t) cos(c x t) dt, evaluated by
Gauss-Legendre quadrature.
"""

from __future__ import annotations

import math
from functools import lru_cache

import numpy as np
from numpy.polynomial import legendre as npleg


class Prolate0:
    """psi_0^c and its constants for one bandwidth parameter c > 0."""

    def __init__(self, c: float, n_even: int | None = None):
        if not (c > 0.0):
            raise ValueError("c must be positive")
        self.c = float(c)
        n = n_even if n_even is not None else int(math.ceil(c)) + 40
        k = 2.0 * np.arange(n)  # even Legendre degrees 0, 2, 4, ...
        c2 = self.c * self.c
        # L_c P_k = k(k+1) P_k + c^2 x^2 P_k, with
        # x^2 P_k = (k+1)(k+2)/((2k+1)(2k+3)) P_{k+2}
        #         + (2k^2+2k-1)/((2k-1)(2k+3)) P_k + k(k-1)/((2k+1)(2k-1)) P_{k-2}
        diag = k * (k + 1.0) + c2 * (2.0 * k * k + 2.0 * k - 1.0) / ((2.0 * k - 1.0) * (2.0 * k + 3.0))
        kk = k[:-1]
        off = c2 * (kk + 1.0) * (kk + 2.0) / ((2.0 * kk + 3.0) * np.sqrt((2.0 * kk + 1.0) * (2.0 * kk + 5.0)))
        A = np.diag(diag) + np.diag(off, 1) + np.diag(off, -1)
        w, v = np.linalg.eigh(A)
        beta = v[:, 0].copy()  # smallest eigenvalue of L_c  <->  largest |lambda| of F_c
        # coefficients in the (unnormalised) Legendre basis P_k, all degrees
        coef = np.zeros(2 * n - 1)
        coef[0::2] = beta * np.sqrt(k + 0.5)
        if npleg.legval(0.0, coef) < 0.0:
            coef = -coef
            beta = -beta
        self.chi0 = float(w[0])
        self.beta = beta  # orthonormal-basis coefficients: sum beta^2 = 1 <=> ||psi_0||_2 = 1
        self.coef = coef
        self.dcoef = npleg.legder(coef)
        self.icoef = npleg.legint(coef, lbnd=0.0)  # antiderivative vanishing at 0
        self.psi_at_0 = float(npleg.legval(0.0, coef))
        integral = math.sqrt(2.0) * abs(float(beta[0]))  # int_{-1}^{1} Pbar_0 = sqrt(2)
        self.lam0 = integral / self.psi_at_0  # (psidefinit) at x = 0
        self.C0 = 0.5 * integral  # int_0^1 psi_0, psi_0 even

    # -- evaluation -------------------------------------------------------------
    def psi(self, x):
        """psi_0^c(x); Legendre series on [-1, 1], the integral extension outside."""
        x = np.asarray(x, dtype=np.float64)
        out = np.empty_like(x)
        inside = np.abs(x) <= 1.0
        out[inside] = npleg.legval(x[inside], self.coef)
        if np.any(~inside):
            out[~inside] = self.psi_ext(x[~inside])
        return out if out.ndim else float(out)

    def dpsi(self, x):
        """d/dx psi_0^c(x); Legendre series on [-1, 1], the integral extension outside."""
        x = np.asarray(x, dtype=np.float64)
        out = np.empty_like(x)
        inside = np.abs(x) <= 1.0
        out[inside] = npleg.legval(x[inside], self.dcoef)
        if np.any(~inside):
            out[~inside] = self.dpsi_ext(x[~inside])
        return out if out.ndim else float(out)

    def int_psi(self, x):
        """int_0^x psi_0^c(t) dt for |x| <= 1."""
        x = np.asarray(x, dtype=np.float64)
        if np.any(np.abs(x) > 1.0 + 1e-15):
            raise ValueError("int_psi is defined here only on [-1, 1]")
        return npleg.legval(x, self.icoef)

    def psi_ext(self, x):
        """(psidefinit): psi_0(x) = (1/lambda_0) int_{-1}^{1} psi_0(t) cos(c x t) dt, any x."""
        t, wt = _gauss_legendre(_quad_nodes(self.c, x))
        f = npleg.legval(t, self.coef) * wt
        x = np.atleast_1d(np.asarray(x, dtype=np.float64))
        return (np.cos(self.c * np.outer(x, t)) @ f) / self.lam0

    def dpsi_ext(self, x):
        """Derivative of (psidefinit) in x: -(c/lambda_0) int psi_0(t) t sin(c x t) dt."""
        t, wt = _gauss_legendre(_quad_nodes(self.c, x))
        f = npleg.legval(t, self.coef) * wt * t
        x = np.atleast_1d(np.asarray(x, dtype=np.float64))
        return -self.c * (np.sin(self.c * np.outer(x, t)) @ f) / self.lam0


def _quad_nodes(c, x) -> int:
    xm = float(np.max(np.abs(np.atleast_1d(x)))) if np.size(x) else 1.0
    return int(80 + 1.5 * c * max(1.0, xm))


@lru_cache(maxsize=64)
def _gauss_legendre(n: int):
    return npleg.leggauss(n)


@lru_cache(maxsize=64)
def prolate(c: float) -> Prolate0:
    return Prolate0(c)


def edge_ratio(p: Prolate0) -> float:
    """psi_0^c(1) / psi_0^c(0) from the prolate differential equation at its end point.

    At x = 1 the Legendre series sums terms of order one to a value of order Delta, so it
    keeps only about 16 + log10(Delta) digits.  Instead: psi_0 solves
        (1 - x^2) u'' - 2 x u' + (chi_0 - c^2 x^2) u = 0,
    chi_0 the eigenvalue of L_c found above, and is the solution regular at the singular
    point x = 1.  With y = 1 - x that solution is the power series u = sum_j b_j y^j,
    b_0 = 1, whose coefficients follow from collecting powers of y in
        y (2 - y) u_yy + 2 (1 - y) u_y + (chi_0 - c^2 (1 - y)^2) u = 0:
        2 (j + 1)^2 b_{j+1} = (j (j + 1) + c^2 - chi_0) b_j - 2 c^2 b_{j-1} + c^2 b_{j-2}.
    The series converges for |y| < 2 (the other singular point is x = -1), so at x = 0
    (y = 1) psi_0(0) / psi_0(1) = sum_j b_j; the terms are positive for the most part and
    no cancellation to the size of Delta occurs.
    """
    c2 = p.c * p.c
    b = [1.0]
    total = 1.0
    j = 0
    while True:
        bj = b[j]
        bj1 = b[j - 1] if j >= 1 else 0.0
        bj2 = b[j - 2] if j >= 2 else 0.0
        nxt = ((j * (j + 1) + c2 - p.chi0) * bj - 2.0 * c2 * bj1 + c2 * bj2) / (2.0 * (j + 1) ** 2)
        b.append(nxt)
        total += nxt
        j += 1
        if j > 20 and abs(nxt) < 1e-18 * abs(total):
            break
        if j > 100000:
            raise RuntimeError("edge series did not converge")
    return 1.0 / total


def c_from_tolerance(delta: float) -> float:
    """Shape parameter c with psi_0^c(1) / psi_0^c(0) = delta (Sec. 5.1 tuning rule).

    The paper writes psi_0^c(1) = Delta without fixing the scale of psi_0 in that rule;
    the ratio to psi_0(0) is the reading used here (parity unpinned: the paper prints no
    value of c).  The ratio decreases monotonically in c, so plain bisection works; it is
    evaluated by ``edge_ratio`` (no cancellation at x = 1).
    """
    if not (0.0 < delta < 1.0):
        raise ValueError("delta must be in (0, 1)")

    def ratio(c):
        return edge_ratio(Prolate0(c))

    lo, hi = 1e-3, 4.0
    while ratio(hi) > delta:
        hi *= 2.0
        if hi > 400:
            raise ValueError("delta too small")
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if ratio(mid) > delta:
            lo = mid
        else:
            hi = mid
        if hi - lo < 1e-14 * hi:
            break
    return 0.5 * (lo + hi)
