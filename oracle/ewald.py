"""O-EWALD: classical Ewald summation with an explicit k-sum (test infrastructure).

Part of the FP64 CPU oracle; only tests, the smoke check and the benchmark's CPU legs
may import it.

Splitting (Sec. 2.1): 1/r = erfc(beta r)/r + erf(beta r)/r.  The paper writes the
parameter as sqrt(alpha); ``beta`` here is that square root.  Tin-foil boundary
conditions (Sec. 3.2: the k = 0 mode is omitted).  A non-zero net charge Q gets the
usual uniform neutralising background, -pi Q^2 / (2 V beta^2).

Outputs, for the cell h (columns = cell vectors) and Cartesian positions:
* energies  U = U_real + U_recip + U_self (+ U_net);
* forces    F_i = -dU/dr_i;
* virial    W = -(dU/dh) h^T, so that the Coulomb part of the pressure tensor of
  eq. (instheta) is P = W / V.  Coulomb homogeneity (eq. (deth)) gives tr W = U.
"""

from __future__ import annotations

import math

import numpy as np
from scipy.special import erfc

from . import lattice


def default_params(h, tol: float = 1e-16, rcut: float | None = None):
    """(beta, rcut, kcut) with erfc(beta rcut) and exp(-kcut^2 / 4 beta^2) below ``tol``."""
    if rcut is None:
        rcut = 0.5 * float(np.min(lattice.widths(h)))
    x = math.sqrt(-math.log(tol))
    # erfc(x) ~ exp(-x^2) / (x sqrt(pi)); a slightly larger x keeps it below tol
    beta = (x + 0.1) / rcut
    kcut = 2.0 * beta * (x + 0.1)
    return beta, rcut, kcut


def ewald(pos, q, h, beta=None, rcut=None, kcut=None, forces=True, tol=1e-16, cell_list=False):
    h = lattice.check_cell(h)
    pos = np.asarray(pos, dtype=np.float64)
    q = np.asarray(q, dtype=np.float64)
    if beta is None:
        beta, rcut, kcut = default_params(h, tol=tol, rcut=rcut)
    V = float(np.linalg.det(h))
    N = len(q)
    F = np.zeros((N, 3))
    W = np.zeros((3, 3))

    # real space: u(r) = q_i q_j erfc(beta r) / r,  f(r) = -u'(r) / (r q_i q_j)
    U_real = 0.0
    pairs = lattice.pair_cells if cell_list else lattice.pair_images
    for i, j, rv, r in pairs(pos, h, rcut):
        qq = q[i] * q[j]
        e = erfc(beta * r) / r
        U_real += 0.5 * float(np.sum(qq * e))
        f = qq * (e + 2.0 * beta / math.sqrt(math.pi) * np.exp(-(beta * r) ** 2)) / (r * r)
        if forces:
            np.add.at(F, i, f[:, None] * rv)
        W += 0.5 * np.einsum("p,pa,pb->ab", f, rv, rv)

    # reciprocal space: U = (2 pi / V) sum_{k != 0} g(k) |S(k)|^2,  g = exp(-k^2/4b^2)/k^2
    m, k, wt = lattice.kvectors(h, kcut, half=True)
    k2 = np.einsum("ij,ij->i", k, k)
    g = np.exp(-k2 / (4.0 * beta * beta)) / k2
    S = lattice.structure_factor(k, pos, q)
    S2 = np.abs(S) ** 2
    pref = 2.0 * math.pi / V
    U_recip = pref * float(np.sum(wt * g * S2))
    # W = -(dU/dh) h^T with d|k|^2/dh h^T = -2 kk and d(1/V)/dh h^T = -I/V
    coef = wt * g * S2
    W += pref * (np.sum(coef) * np.eye(3)
                 - 2.0 * np.einsum("p,pa,pb->ab", coef * (1.0 / k2 + 1.0 / (4.0 * beta * beta)), k, k))
    if forces:
        # F_i = (4 pi q_i / V) sum_{all k} g k Im[conj(S) exp(i k.r_i)]; the summand is even
        # in k, so the half-space sum carries weight 2 (in wt) on top of 4 pi / V = 2 pref
        for a in range(0, len(k), 2048):
            kk = k[a:a + 2048]
            ph = np.exp(1j * (pos @ kk.T))  # [N, nk]
            im = np.imag(np.conj(S[a:a + 2048])[None, :] * ph)
            F += (2.0 * pref * q)[:, None] * ((im * (wt[a:a + 2048] * g[a:a + 2048])[None, :]) @ kk)

    U_self = -beta / math.sqrt(math.pi) * float(np.sum(q * q))
    Q = float(np.sum(q))
    U_net = -math.pi * Q * Q / (2.0 * V * beta * beta)
    W += U_net * np.eye(3)  # U_net is proportional to 1/V
    U = U_real + U_recip + U_self + U_net
    return {
        "energy": U, "energy_real": U_real, "energy_recip": U_recip, "energy_self": U_self,
        "energy_net": U_net, "forces": F if forces else None, "virial": W,
        "pressure": W / V, "params": (beta, rcut, kcut),
    }


def madelung_nacl(a: float = 2.0):
    """Rock-salt conventional cell (4 Na+ + 4 Cl-), lattice constant a: (pos, q, h)."""
    fcc = np.array([[0, 0, 0], [0, .5, .5], [.5, 0, .5], [.5, .5, 0]])
    pos = np.concatenate([fcc, fcc + np.array([.5, 0, 0])]) * a
    q = np.array([1.0] * 4 + [-1.0] * 4)
    return pos, q, np.eye(3) * a
