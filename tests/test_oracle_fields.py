"""Pins of the oracle's field variants (ik-differentiation, per-atom virial and energy).

* Per-atom virial and energy (Sec. 4.4, eqs. (rhodiag), (PinsFind)) sum to the global W_F
  and U_F (Plancherel; exact up to rounding).
* ik-differentiation forces (Appendix C, eq. (rhodiagforce)) conserve momentum exactly when
  the spreading window also interpolates: sum_i F_i = -sum_m i k G |X|^2 = 0, since k is odd
  and G |X|^2 even in m.
* They converge spectrally to the exact forces of the split (no grid), like the
  analytically differentiated ones.
"""

import numpy as np

import synthetic as sy
from oracle.esp_grid import esp_grid, esp_grid_fields
from oracle.esp_split import esp_split
from oracle.pswf import c_from_tolerance

TRI = np.array([[13.0, 1.3, -0.9], [0.0, 14.0, 1.1], [0.0, 0.0, 12.5]])


def system():
    return sy.small_random(120, TRI, seed=61, grid=(20, 22, 20), P=6, delta=1e-5, rc=4.5)


def test_per_atom_virial_and_energy_sum_to_the_global_ones():
    S = system()
    c = c_from_tolerance(S.delta)
    g = esp_grid(S.pos, S.q, S.cell, S.grid, S.P, c, S.rc, forces=False)
    Wi = esp_grid_fields(S.pos, S.q, S.cell, S.grid, S.P, c, S.rc, "virial").sum(axis=0)
    W = g["virial"]
    assert np.allclose(Wi, [W[0, 0], W[1, 1], W[2, 2], W[0, 1], W[0, 2], W[1, 2]], rtol=0,
                       atol=1e-12 * np.max(np.abs(W)))
    Ui = esp_grid_fields(S.pos, S.q, S.cell, S.grid, S.P, c, S.rc, "energy")
    assert abs(Ui.sum() - g["energy"]) < 1e-12 * abs(g["energy"])


def test_ik_forces_conserve_momentum():
    S = system()
    c = c_from_tolerance(S.delta)
    F = esp_grid_fields(S.pos, S.q, S.cell, S.grid, S.P, c, S.rc, "ik")
    assert np.max(np.abs(F.sum(axis=0))) < 1e-12 * np.sum(np.abs(F))
    # analytical differentiation does not (reading 16): its net force is not at rounding level
    Fa = esp_grid(S.pos, S.q, S.cell, S.grid, S.P, c, S.rc)["forces"]
    assert np.max(np.abs(Fa.sum(axis=0))) > 1e3 * np.max(np.abs(F.sum(axis=0)))


def test_ik_forces_converge_to_the_split_forces():
    S = system()
    c = c_from_tolerance(1e-8)
    ref = esp_split(S.pos, S.q, S.cell, c, S.rc, near=False)["forces_far"]
    errs = []
    for M, P in (((24, 26, 24), 8), ((36, 40, 36), 10)):
        F = esp_grid_fields(S.pos, S.q, S.cell, M, P, c, S.rc, "ik")
        errs.append(np.linalg.norm(F - ref) / np.linalg.norm(ref))
    assert errs[1] < 1e-7 and errs[1] < errs[0]
