"""Pins for O-SPLIT and O-GRID (no GPU).

O-SPLIT (Sec. 3) is pinned to O-EWALD (itself pinned by test_oracle_ewald) and to the
exact real-space identity behind eq. (UNS); O-GRID (Sec. 4, Appendix C) is pinned by
finite differences of its own energy (forces: the "no 1/2 in eq. (AD)" reading; cell:
the "+1/(2V^2)" reading of eq. (Far)), by a brute-force separable DFT of the spread
charge, by h-independence of the spectrum at fixed reduced coordinates (Sec. 3.2) and by
spectral convergence to O-SPLIT's explicit k-sum (Sec. 5.1).
"""

import itertools
import math

import numpy as np
import pytest

import synthetic as sy
from oracle import lattice
from oracle.esp_grid import esp_grid, modes, self_and_background, spread
from oracle.esp_split import esp_split, split_constants
from oracle.ewald import ewald
from oracle.pswf import c_from_tolerance, prolate

H = np.array([[9.0, 0.5, 0.3], [0.0, 10.0, 0.4], [0.0, 0.0, 8.5]])


def _system(n=20, seed=3, h=H):
    rng = np.random.default_rng(seed)
    pos = rng.random((n, 3)) @ h.T
    q = rng.normal(size=n)
    q -= q.mean()
    return pos, q


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


@pytest.mark.parametrize("delta", [1e-5, 1e-8, 1e-11])
def test_split_converges_to_ewald(delta):
    pos, q = _system(n=40, seed=1)
    E = ewald(pos, q, H)
    c = c_from_tolerance(delta)
    r = esp_split(pos, q, H, c, 4.2)
    assert rel(r["energy"], E["energy"]) < 10 * delta
    assert rel(r["virial"], E["virial"]) < 30 * delta
    assert rel(r["forces"], E["forces"]) < 30 * delta


def test_background_correction_matches_ewald_for_charged_cell():
    # eq. (Corr): with a uniform neutralising background ESP must reproduce Ewald's
    # charged-cell energy and virial; the background adds no force (Sec. 3.4)
    pos, q = _system(n=30, seed=2)
    q = q + 0.25
    E = ewald(pos, q, H)
    c = c_from_tolerance(1e-10)
    r = esp_split(pos, q, H, c, 4.2)
    assert abs(r["energy_bg"]) > 1e-2 * abs(r["energy"])  # the term matters here
    assert rel(r["energy"], E["energy"]) < 1e-8
    assert rel(r["virial"], E["virial"]) < 1e-8
    assert rel(r["forces"], E["forces"]) < 1e-8


def test_real_space_virial_defect_identity():
    # eq. (UNS), exact for any configuration:
    # (U_N + U_self) - tr W_N = -1/2 sum_i q_i xi(r_i),  xi = sum_{j,n} q_j psi_0(|r|/r_c)/(C_0 r_c)
    pos, q = _system()
    c, rc = c_from_tolerance(1e-6), 4.0
    p, _, _ = split_constants(c, rc)
    xi = q * p.psi_at_0 / (p.C0 * rc)
    for i, j, _, r in lattice.pair_images(pos, H, rc):
        np.add.at(xi, i, q[j] * p.psi(r / rc) / (p.C0 * rc))
    lhs = -0.5 * float(np.sum(q * xi))
    r = esp_split(pos, q, H, c, rc, forces=False)
    assert abs(r["energy_near"] + r["energy_self"] - np.trace(r["virial_near"]) - lhs) < 1e-12 * abs(lhs)
    # eq. (PSRela): the Fourier defect cancels it, up to the |k| <= c/r_c truncation
    assert abs(r["defect_far"] + lhs) < 10 * 1e-6 * abs(lhs)


def _dft_bruteforce(pos, q, h, M, P, c):
    """X(m) = sum_j q_j prod_d S_d(j, m_d), S_d = sum_p w_d(g_p/M_d - s) e^{-2 pi i m g_p/M_d}."""
    p = prolate(c)
    s = lattice.reduced(pos, h)
    X = np.zeros((M[0], M[1], M[2] // 2 + 1), dtype=complex)
    for j in range(len(q)):
        S = []
        for d in range(3):
            x = M[d] * s[j, d]
            b = math.floor(x) - P // 2 + 1 if P % 2 == 0 else math.floor(x + 0.5) - (P - 1) // 2
            g = b + np.arange(P)
            w = p.psi((g - x) / (0.5 * P))
            m = np.arange(M[d] if d < 2 else M[d] // 2 + 1)
            S.append(np.exp(-2j * math.pi * np.outer(m, g) / M[d]) @ w)
        X += q[j] * S[0][:, None, None] * S[1][None, :, None] * S[2][None, None, :]
    return X


@pytest.mark.parametrize("P,M", [(6, (12, 14, 16)), (5, (11, 13, 10)), (7, (16, 16, 15))])
def test_spread_plus_fft_equals_separable_dft(P, M):
    pos, q = _system(n=9, seed=11)
    c = c_from_tolerance(1e-6)
    X = np.fft.rfftn(spread(pos, q, H, M, P, c))
    Xb = _dft_bruteforce(pos, q, H, M, P, c)
    assert np.max(np.abs(X - Xb)) < 1e-12 * np.max(np.abs(Xb))


def test_spectrum_independent_of_cell_at_fixed_reduced_coordinates():
    # Sec. 3.2: rho(k) depends on the reduced coordinates only; with the window taken in
    # reduced coordinates the same holds for the gridded spectrum
    pos, q = _system(n=15, seed=4)
    s = lattice.reduced(pos, H)
    H2 = np.array([[12.0, -1.0, 2.0], [0.0, 8.0, 0.9], [0.0, 0.0, 11.0]])
    g1 = spread(s @ H.T, q, H, (12, 12, 12), 6, 13.0)
    g2 = spread(s @ H2.T, q, H2, (12, 12, 12), 6, 13.0)
    assert np.max(np.abs(g1 - g2)) < 1e-12 * np.max(np.abs(g1))


@pytest.mark.parametrize("P,M", [(7, (24, 26, 22)), (6, (20, 20, 20))])
def test_grid_forces_are_energy_gradients(P, M):
    pos, q = _system()
    c, rc = c_from_tolerance(1e-8), 4.0
    G = esp_grid(pos, q, H, M, P, c, rc)
    d = 1e-6
    for i, a in [(0, 0), (5, 1), (11, 2)]:
        p1, p2 = pos.copy(), pos.copy()
        p1[i, a] += d
        p2[i, a] -= d
        fd = -(esp_grid(p1, q, H, M, P, c, rc, forces=False)["energy"]
               - esp_grid(p2, q, H, M, P, c, rc, forces=False)["energy"]) / (2 * d)
        assert abs(fd - G["forces"][i, a]) < 1e-6 * np.max(np.abs(G["forces"]))


def test_grid_virial_is_cell_gradient():
    # W_F = -(dU_F/dh) h^T at fixed s (eq. (instheta)); exact on the grid because the
    # spectrum does not depend on h at fixed s (no mode crosses |k| = c/r_c for small dh)
    pos, q = _system()
    c, rc, M, P = c_from_tolerance(1e-8), 4.0, (22, 24, 20), 7
    G = esp_grid(pos, q, H, M, P, c, rc, forces=False)
    s = pos @ np.linalg.inv(H).T
    d = 1e-6
    dUdh = np.zeros((3, 3))
    n0 = modes(H, M, P, c, rc)["inside"].sum()
    for a, b in itertools.product(range(3), range(3)):
        h1, h2 = H.copy(), H.copy()
        h1[a, b] += d
        h2[a, b] -= d
        assert modes(h1, M, P, c, rc)["inside"].sum() == n0 == modes(h2, M, P, c, rc)["inside"].sum()
        dUdh[a, b] = (esp_grid(s @ h1.T, q, h1, M, P, c, rc, forces=False)["energy"]
                      - esp_grid(s @ h2.T, q, h2, M, P, c, rc, forces=False)["energy"]) / (2 * d)
    W = G["virial"]
    assert np.max(np.abs(-dUdh @ H.T - W)) < 1e-7 * np.max(np.abs(W))
    assert np.max(np.abs(W - W.T)) < 1e-13 * np.max(np.abs(W))


def test_grid_converges_to_exact_k_sum():
    # spectral convergence in the grid and stencil (Sec. 5.1, Figs. 1-3)
    pos, q = _system(n=40, seed=8)
    c, rc = c_from_tolerance(1e-10), 4.0
    S = esp_split(pos, q, H, c, rc, near=False)
    errs = []
    for M, P in [((24, 24, 24), 8), ((32, 32, 32), 10), ((40, 40, 40), 12)]:
        G = esp_grid(pos, q, H, M, P, c, rc)
        errs.append((rel(G["energy"], S["energy_far"]), rel(G["virial"], S["virial_far"]),
                     rel(G["forces"], S["forces_far"])))
    assert errs[-1][0] < 1e-10 and errs[-1][1] < 1e-9 and errs[-1][2] < 1e-7
    assert errs[0][1] > errs[-1][1]


def test_grid_rejects_too_coarse_grid():
    pos, q = _system()
    with pytest.raises(ValueError):
        esp_grid(pos, q, H, (8, 8, 8), 6, c_from_tolerance(1e-8), 2.0)


def test_water648_accuracy_against_ewald():
    # the configured Delta = 1e-6, P = 6, 24^3, r_c = 9 A meets the 1e-6 pressure target
    S = sy.water_cubic()
    E = ewald(S.pos, S.q, S.cell)
    c = c_from_tolerance(S.delta)
    sp = esp_split(S.pos, S.q, S.cell, c, S.rc, near=True)
    g = esp_grid(S.pos, S.q, S.cell, S.grid, S.P, c, S.rc)
    sb = self_and_background(S.q, S.cell, c, S.rc)
    W = sp["virial_near"] + g["virial"] + sb["energy_bg"] * np.eye(3)
    U = sp["energy_near"] + g["energy"] + sb["energy_self"] + sb["energy_bg"]
    F = sp["forces_near"] + g["forces"]
    assert rel(W, E["virial"]) < 1e-6
    assert rel(U, E["energy"]) < 1e-6
    assert rel(F, E["forces"]) < 1e-6
