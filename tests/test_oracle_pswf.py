"""Pins for O-PSWF against what the mathematics fixes (no GPU).

Each test checks the oracle's prolate against something it does not compute itself:
an independent Nystrom discretisation of the integral operator (Appendix A.1,
eq. (formula)), the defining eigen-equation (eq. (psidefinit)), its x-derivative
(eq. (derivative_psi)), the c -> 0 closed form, the closed-form window transform of
Sec. 4.2 and the 3D transform of the far kernel of eq. (UF).
"""

import math

import numpy as np
import pytest
from numpy.polynomial import legendre as npleg

from oracle.pswf import Prolate0, c_from_tolerance, edge_ratio, prolate

CS = [0.5, 2.0, 7.0, 13.36, 21.2, 30.0]


@pytest.mark.parametrize("c", CS)
def test_nystrom_eigenpair(c):
    # the even part of F_c is the cosine kernel; discretise it by Gauss-Legendre
    t, w = npleg.leggauss(160)
    K = np.sqrt(w)[:, None] * np.cos(c * np.outer(t, t)) * np.sqrt(w)[None, :]
    ev, vec = np.linalg.eigh(K)
    p = Prolate0(c)
    assert abs(ev[-1] - p.lam0) <= 1e-13 * p.lam0
    # eigenvector -> function values at the nodes, L2-normalised (sum w psi^2 = 1)
    psi_nodes = vec[:, -1] / np.sqrt(w)
    psi_nodes *= np.sign(psi_nodes[np.argmin(np.abs(t))])
    # The eigenvector is conditioned by the gap lambda_0 - lambda_2, which closes as c
    # grows (|lambda_n| -> sqrt(2 pi / c) for n < 2c/pi); there the eigen-equation test
    # below plus positivity on [-1, 1] (psi_2 has two zeros) single out psi_0 instead.
    gap = ev[-1] - ev[-2]
    if gap > 1e-4:
        assert np.max(np.abs(psi_nodes - p.psi(t))) <= 1e-15 / gap * 1e3 * np.max(np.abs(psi_nodes))


@pytest.mark.parametrize("c", CS)
def test_eigen_equation_and_norm(c):
    p = prolate(c)
    t, w = npleg.leggauss(200)
    x = np.linspace(-1.0, 1.0, 41)
    lhs = p.lam0 * p.psi(x)
    rhs = (np.exp(1j * c * np.outer(x, t)) @ (w * p.psi(t)))
    assert np.max(np.abs(rhs.imag)) < 1e-13
    assert np.max(np.abs(lhs - rhs.real)) < 1e-13 * p.lam0 * p.psi_at_0
    assert abs(np.sum(w * p.psi(t) ** 2) - 1.0) < 1e-13
    assert p.psi_at_0 > 0 and np.all(p.psi(x) > 0)  # psi_0 has no zero in [-1, 1]
    assert abs(p.C0 - 0.5 * np.sum(w * p.psi(t))) < 1e-14


@pytest.mark.parametrize("c", CS)
def test_derivative_identity(c):
    # eq. (derivative_psi): lambda_0 psi_0'(x) = -c int_{-1}^{1} psi_0(u) sin(c x u) u du
    p = prolate(c)
    u, w = npleg.leggauss(200)
    x = np.linspace(-1.0, 1.0, 33)
    rhs = -c * (np.sin(c * np.outer(x, u)) @ (w * u * p.psi(u)))
    assert np.max(np.abs(p.lam0 * p.dpsi(x) - rhs)) < 1e-12 * max(1.0, c) * p.psi_at_0


def test_small_c_limit():
    # c -> 0: F_c -> the rank-one operator int phi, so psi_0 -> 1/sqrt(2) and lambda_0 -> 2
    p = Prolate0(1e-6)
    x = np.linspace(-1, 1, 11)
    assert np.max(np.abs(p.psi(x) - 1 / math.sqrt(2))) < 1e-10
    assert abs(p.lam0 - 2.0) < 1e-10


@pytest.mark.parametrize("c", [7.0, 14.08])
def test_extension_matches_series_at_the_edge(c):
    p = prolate(c)
    x = np.array([0.3, 0.9, 1.0])
    assert np.max(np.abs(p.psi_ext(x) - p.psi(x))) < 1e-13 * p.psi_at_0
    assert np.max(np.abs(p.dpsi_ext(x) - p.dpsi(x))) < 1e-12 * c * p.psi_at_0


@pytest.mark.parametrize("P,M", [(6, 24), (8, 64), (5, 40)])
def test_window_fourier_closed_form(P, M):
    # Sec. 4.2: the transform of w(u) = psi_0(u/omega) on |u| <= omega is omega lambda_0
    # psi_0(2 pi m omega / c), here compared with direct quadrature of the integral
    c = c_from_tolerance(1e-6)
    p = prolate(c)
    om = P / (2.0 * M)
    u, w = npleg.leggauss(400)
    for m in [0, 1, 3, M // 4, M // 2 - 1]:
        direct = om * np.sum(w * p.psi(u) * np.cos(2 * math.pi * m * om * u))
        closed = om * p.lam0 * p.psi(2 * math.pi * m * om / c)
        assert abs(direct - closed) < 1e-13 * om * p.lam0 * p.psi_at_0


@pytest.mark.parametrize("c,rc", [(13.36, 9.0), (21.2, 5.5)])
def test_far_kernel_transform(c, rc):
    # eq. (UF): the 3D transform of F^c(r) = phi_0(r)/r is (2 pi lambda_0/C_0) psi_0(k r_c/c)/k^2.
    # Independent route: F^c = 1/r - N^c with N^c compact, so its transform is
    # 4 pi/k^2 - 4 pi int_0^{r_c} (1 - phi_0(r)) sin(k r) / k dr  (radial transform, App. A.4)
    p = prolate(c)
    r, w = npleg.leggauss(300)
    r = 0.5 * rc * (r + 1.0)
    w = 0.5 * rc * w
    phi0 = p.int_psi(r / rc) / p.C0
    for k in [0.05, 0.5, 1.0, c / rc, 1.7 * c / rc]:
        direct = 4 * math.pi / k ** 2 - 4 * math.pi * np.sum(w * (1 - phi0) * np.sin(k * r)) / k
        closed = 2 * math.pi * p.lam0 / p.C0 * p.psi(k * rc / c) / k ** 2
        assert abs(direct - closed) < 1e-12 * 4 * math.pi / k ** 2


def test_split_kernel_facts():
    # Sec. 3.1: N^c(r_c) = 0 (phi_0(r_c) = 1) and F^c(0) = psi_0(0) / (C_0 r_c)
    c, rc = 13.36, 9.0
    p = prolate(c)
    assert abs(p.int_psi(1.0) / p.C0 - 1.0) < 1e-14
    r = 1e-7
    Fc0 = (p.int_psi(r / rc) / p.C0) / r
    assert abs(Fc0 - p.psi_at_0 / (p.C0 * rc)) < 1e-9 * Fc0


def test_tuning_rule_trend():
    # Sec. 5.1 rule psi_0(1)/psi_0(0) = Delta and the trend c ~ log(1/Delta) of eq. (c)
    prev = 0.0
    for d in [1e-3, 1e-5, 1e-7, 1e-10]:
        c = c_from_tolerance(d)
        p = Prolate0(c)
        # psi_0(1) is known to ~1e-16 absolute, so the ratio only to ~1e-8 relative at 1e-10
        assert abs(p.psi(1.0) / p.psi_at_0 - d) < 1e-15 + 1e-6 * d
        assert 0.0 < c - math.log(1 / d) < 4.0
        assert c > prev
        prev = c


@pytest.mark.parametrize("c", [0.5, 2.0, 7.0])
def test_edge_ratio_matches_legendre_series(c):
    # where psi_0(1) is not small the Legendre series at x = 1 loses nothing to
    # cancellation, and the regular series of the differential equation must agree
    p = Prolate0(c)
    assert abs(edge_ratio(p) / (p.psi(1.0) / p.psi_at_0) - 1.0) < 1e-13


def test_edge_ratio_small_c_limit():
    # c -> 0: psi_0 -> 1/sqrt(2), a constant, so the ratio tends to 1
    assert abs(edge_ratio(Prolate0(1e-4)) - 1.0) < 1e-8


@pytest.mark.parametrize("c", [14.08, 30.0])
def test_edge_ratio_against_extended_precision(c):
    # An independent 40-digit evaluation of the same ratio by the Legendre route (the
    # tridiagonal eigenproblem of L_c and the series at x = 1 and x = 0, with
    # P_k(1) = 1 and P_{2i}(0) = (-1)^i (2i-1)!!/(2i)!!), where FP64 would cancel.
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    n = int(math.ceil(c)) + 40
    c2 = mp.mpf(c) ** 2
    A = mp.matrix(n, n)
    for i in range(n):
        k = mp.mpf(2 * i)
        A[i, i] = k * (k + 1) + c2 * (2 * k * k + 2 * k - 1) / ((2 * k - 1) * (2 * k + 3))
        if i + 1 < n:
            A[i, i + 1] = A[i + 1, i] = c2 * (k + 1) * (k + 2) / ((2 * k + 3) * mp.sqrt((2 * k + 1) * (2 * k + 5)))
    E, Q = mp.eigsy(A)
    j = min(range(n), key=lambda i: E[i])
    at1 = mp.fsum(Q[i, j] * mp.sqrt(2 * i + mp.mpf(1) / 2) for i in range(n))
    at0, p0 = mp.mpf(0), mp.mpf(1)
    for i in range(n):
        if i > 0:
            p0 = -p0 * (2 * i - 1) / (2 * i)
        at0 += Q[i, j] * mp.sqrt(2 * i + mp.mpf(1) / 2) * p0
    ref = float(at1 / at0)
    assert abs(edge_ratio(Prolate0(c)) / ref - 1.0) < 1e-12
