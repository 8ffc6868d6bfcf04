"""Pressure for each cell coupling (Sec. 2.2) from the pressure tensor: esp_pressure_coupling
against finite differences of the Ewald energy in that coupling's own cell variables.

Sec. 2.2 defines each coupling's pressure as minus the derivative of the energy with
respect to its cell variables at fixed reduced coordinates s = h^{-1} r:
  isotropic        P = -dU/dV                       (V scaled, shape kept)
  semi-isotropic   P_A = -(1/L) dU/dA, P_L = -(1/A) dU/dL  (A = Lx Ly in the x-y plane)
  anisotropic      P_aa = -(L_a / V) dU/dL_a         (eq. (diagona))
The library forms these from the tensor P = W / V; here they are taken by central
differences of the oracle's Ewald energy (no GPU: a host-only entry point).
"""

import numpy as np
import pytest

from oracle.ewald import ewald

esp = pytest.importorskip("paper_2601_00161_gb300")

CELL = np.diag([9.0, 10.0, 11.5])


def system():
    rng = np.random.default_rng(77)
    n = 24
    pos = rng.uniform(0.0, 1.0, (n, 3)) @ CELL.T
    q = rng.normal(size=n)
    q -= q.mean()
    return pos, q


def energy(pos, q, cell):
    return ewald(pos, q, cell)["energy"]


def scaled(pos, cell, f):
    """Cell columns scaled by f[d], atoms kept at their reduced coordinates."""
    s = np.linalg.solve(cell, pos.T).T
    h = cell * np.asarray(f)[None, :]
    return s @ h.T, h


def tensor(pos, q):
    W = np.asarray(ewald(pos, q, CELL)["virial"]).reshape(3, 3)
    return W / np.linalg.det(CELL)


def test_isotropic_is_minus_dU_dV():
    pos, q = system()
    P = tensor(pos, q)
    V = np.linalg.det(CELL)
    eps = 1e-5
    up = scaled(pos, CELL, [(1 + eps) ** (1 / 3)] * 3)
    dn = scaled(pos, CELL, [(1 - eps) ** (1 / 3)] * 3)
    fd = -(energy(up[0], q, up[1]) - energy(dn[0], q, dn[1])) / (2 * eps * V)
    (p,) = esp.esp_pressure_coupling(P, esp.ESP_COUPLE_ISO)
    assert abs(p - fd) < 1e-6 * np.abs(P).max()


def test_semi_isotropic_area_and_height():
    pos, q = system()
    P = tensor(pos, q)
    Lx, Ly, L = np.diag(CELL)
    A = Lx * Ly
    eps = 1e-5
    sa_up, sa_dn = np.sqrt(1 + eps), np.sqrt(1 - eps)  # area A (1 +- eps), shape in-plane kept
    up = scaled(pos, CELL, [sa_up, sa_up, 1.0])
    dn = scaled(pos, CELL, [sa_dn, sa_dn, 1.0])
    PA = -(energy(up[0], q, up[1]) - energy(dn[0], q, dn[1])) / (2 * eps * A) / L
    up = scaled(pos, CELL, [1.0, 1.0, 1 + eps])
    dn = scaled(pos, CELL, [1.0, 1.0, 1 - eps])
    PL = -(energy(up[0], q, up[1]) - energy(dn[0], q, dn[1])) / (2 * eps * L) / A
    pa, pl = esp.esp_pressure_coupling(P, esp.ESP_COUPLE_SEMI)
    tol = 1e-6 * np.abs(P).max()
    assert abs(pa - PA) < tol and abs(pl - PL) < tol


def test_anisotropic_diagonal_and_flexible_tensor():
    pos, q = system()
    P = tensor(pos, q)
    V = np.linalg.det(CELL)
    eps = 1e-5
    out = esp.esp_pressure_coupling(P, esp.ESP_COUPLE_ANISO)
    for a in range(3):
        f_up, f_dn = np.ones(3), np.ones(3)
        f_up[a], f_dn[a] = 1 + eps, 1 - eps
        up, dn = scaled(pos, CELL, f_up), scaled(pos, CELL, f_dn)
        La = CELL[a, a]
        fd = -(La / V) * (energy(up[0], q, up[1]) - energy(dn[0], q, dn[1])) / (2 * eps * La)
        assert abs(out[a] - fd) < 1e-6 * np.abs(P).max()
    full = esp.esp_pressure_coupling(P, esp.ESP_COUPLE_FLEXIBLE)
    assert np.allclose(full, [P[0, 0], P[1, 1], P[2, 2], P[0, 1], P[0, 2], P[1, 2]], rtol=0, atol=0)
    # the tensor is symmetric, and the isotropic value is the mean of the anisotropic ones
    assert np.allclose(P, P.T, atol=1e-12 * np.abs(P).max())
    (iso,) = esp.esp_pressure_coupling(P, esp.ESP_COUPLE_ISO)
    assert abs(iso - out.mean()) < 1e-15 * np.abs(P).max() + 1e-300


def test_bad_mode_is_an_error():
    with pytest.raises(esp.ESPError) as ei:
        esp.esp_pressure_coupling(np.eye(3), 7)
    assert ei.value.code == esp.ESP_ERR_ARG
