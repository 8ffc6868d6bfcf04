"""O-SPLIT: ESP's PSWF kernel split with exact structure factors (test infrastructure).

Part of the FP64 CPU oracle; only tests, the smoke check and the benchmark's CPU legs
may import it.  No grid is involved: the Fourier part is an explicit sum over
reciprocal vectors, so this isolates the split (Sec. 3) from the gridding (Sec. 4).

Formulas followed (h: columns are cell vectors, V = det h, x = |k| r_c / c,
A = 2 pi lambda_0 / C_0):
* near kernel  N^c(r) = (1 - phi_0(r)) / r on r <= r_c, phi_0(r) = (1/C_0) int_0^{r/r_c}
  psi_0  (eq. (decomposition));
* U_N = 1/2 sum'_{n} sum_{ij} q_i q_j N^c(|r_ij + h n|)            (eq. (UN));
* U_F = 1/(2V) sum_{k != 0} Fhat(k) |rho(k)|^2, Fhat = A psi_0(x) / |k|^2   (eq. (UF));
* U_self = -psi_0(0) / (2 C_0 r_c) sum q^2                          (eq. (selfen));
* pair weight F_N(r) = 1 - phi_0(r) + r psi_0(r/r_c) / (C_0 r_c)    (eq. (mathFN));
* near virial  W_N = +1/2 sum' q_i q_j F_N(r) r (x) r / r^3.  The paper prints a minus
  sign in eq. (PinsN); the plus sign is what -(dU_N/dh) h^T gives and what its own
  eq. (UNS) needs (reading: sign of the real-space pressure);
* far virial   W_F = 1/(2V) sum_k |rho|^2 [Fhat I + (A x psi_0'(x)/|k|^4 - 2 Fhat/|k|^2) k k],
  i.e. V times eq. (UFPree)/(tensoraniso) with the +1/(2 V^2) prefactor (eq. (Far)
  prints -1/(2V), a typo by dimension);
* forces  F_N,i = sum_j q_i q_j F_N(r) r / r^3,
          F_F,i = (q_i / V) sum_k Fhat k Im[conj(rho) exp(i k.r_i)]   (eq. (Fc));
* neutralising background (eq. (Corr), Sec. 3.4): U_bg = -(2 pi Q^2 / V) X with
  X = r_c^2/2 - int_0^{r_c} r phi_0(r) dr = (r_c^2 / (2 C_0)) int_0^1 u^2 psi_0(u) du,
  W_bg = U_bg I (so P_bg = -(2 pi Q^2 / V^2) X I); no force.

The pressure tensor of eq. (tensoraniso) without the kinetic term is (W_N + W_F + W_bg)/V.
The Fourier sum is truncated at |k| <= c / r_c (Sec. 3.2, after eq. (Far)); with
``truncate=False`` it runs to ``kmax`` with psi_0's entire extension instead.
"""

from __future__ import annotations

import math

import numpy as np
from numpy.polynomial import legendre as npleg

from . import lattice
from .pswf import prolate


def split_constants(c: float, rc: float):
    p = prolate(c)
    A = 2.0 * math.pi * p.lam0 / p.C0
    u, wu = npleg.leggauss(120)
    u = 0.5 * (u + 1.0)
    X = rc * rc / (2.0 * p.C0) * 0.5 * float(np.sum(wu * u * u * p.psi(u)))
    return p, A, X


def fourier_kernel(k2, c, rc):
    """(Fhat, dterm) per mode: Fhat = A psi0(x)/k^2 and A x psi0'(x) / k^4."""
    p, A, _ = split_constants(c, rc)
    kk = np.sqrt(k2)
    x = kk * rc / c
    Fhat = A * p.psi(x) / k2
    dterm = A * x * p.dpsi(x) / (k2 * k2)
    return Fhat, dterm


def esp_split(pos, q, h, c, rc, truncate=True, kmax=None, forces=True, near=True, far=True,
              cell_list=False):
    h = lattice.check_cell(h)
    pos = np.asarray(pos, dtype=np.float64)
    q = np.asarray(q, dtype=np.float64)
    p, A, X = split_constants(c, rc)
    V = float(np.linalg.det(h))
    N = len(q)
    out = {}

    # -- near field ----------------------------------------------------------------
    U_N = 0.0
    W_N = np.zeros((3, 3))
    F_N = np.zeros((N, 3))
    if near:
        pairs = lattice.pair_cells if cell_list else lattice.pair_images
        for i, j, rv, r in pairs(pos, h, rc):
            qq = q[i] * q[j]
            u = r / rc
            phi0 = p.int_psi(u) / p.C0
            U_N += 0.5 * float(np.sum(qq * (1.0 - phi0) / r))
            FN = 1.0 - phi0 + u * p.psi(u) / p.C0
            f = qq * FN / r ** 3
            W_N += 0.5 * np.einsum("p,pa,pb->ab", f, rv, rv)
            if forces:
                np.add.at(F_N, i, f[:, None] * rv)

    # -- far field -------------------------------------------------------------------
    U_F, W_F, F_F, defect_F, n_modes = 0.0, np.zeros((3, 3)), np.zeros((N, 3)), 0.0, 0
    if far:
        K = c / rc
        m, k, wt = lattice.kvectors(h, K if truncate else (kmax or 2.0 * K), half=True)
        k2 = np.einsum("ij,ij->i", k, k)
        Fhat, dterm = fourier_kernel(k2, c, rc)
        S = lattice.structure_factor(k, pos, q)
        a = wt * np.abs(S) ** 2 / (2.0 * V)
        U_F = float(np.sum(a * Fhat))
        W_F = np.sum(a * Fhat) * np.eye(3) + np.einsum("p,pa,pb->ab", a * (dterm - 2.0 * Fhat / k2), k, k)
        F_F = np.zeros((N, 3))
        if forces:
            for s0 in range(0, len(k), 2048):
                kk = k[s0:s0 + 2048]
                ph = np.exp(1j * (pos @ kk.T))
                im = np.imag(np.conj(S[s0:s0 + 2048])[None, :] * ph)
                F_F += (q / V)[:, None] * ((im * (wt[s0:s0 + 2048] * Fhat[s0:s0 + 2048])[None, :]) @ kk)
        # the ξ-defect of eq. (UFS): U_F - tr W_F = -sum a A x psi0'(x) / k^2
        defect_F = -float(np.sum(a * dterm * k2))

        n_modes = len(k)

    U_self = -p.psi_at_0 / (2.0 * p.C0 * rc) * float(np.sum(q * q))
    Q = float(np.sum(q))
    U_bg = -2.0 * math.pi * Q * Q / V * X
    W_bg = U_bg * np.eye(3)

    out.update(
        energy=U_N + U_F + U_self + U_bg, energy_near=U_N, energy_far=U_F,
        energy_self=U_self, energy_bg=U_bg,
        virial_near=W_N, virial_far=W_F, virial_bg=W_bg, virial=W_N + W_F + W_bg,
        pressure=(W_N + W_F + W_bg) / V,
        forces_near=F_N if forces else None, forces_far=F_F if forces else None,
        forces=(F_N + F_F) if forces else None,
        defect_far=defect_F, n_modes=n_modes,
    )
    return out
