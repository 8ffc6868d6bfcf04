"""The plain OpenMP ESP (oracle/esp_omp.c, the CPU baseline) against the numpy oracle.

The same discrete quantity (spread, transform, scaling, inverse transform, gather) in
FP64 by a different code: energy, virial and forces within 1e-12 (relative, normwise), for
cubic and triclinic cells, even and odd stencils, and a grid with a factor 7 (the plain
DFT branch of its transform).
"""

import numpy as np
import pytest

import synthetic as sy
from oracle.esp_grid import esp_grid
from oracle.esp_omp import esp_omp
from oracle.pswf import c_from_tolerance

TRI = np.array([[13.0, 1.3, -0.9], [0.0, 14.0, 1.1], [0.0, 0.0, 12.5]])
CASES = {
    "water648": lambda: sy.water_cubic(),
    "triclinic_P7_factor7": lambda: sy.small_random(300, TRI, seed=81, grid=(28, 30, 27), P=7, delta=1e-6, rc=4.0),
}


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


@pytest.mark.parametrize("case", list(CASES))
def test_openmp_esp_matches_the_oracle(case):
    S = CASES[case]()
    c = c_from_tolerance(S.delta)
    ref = esp_grid(S.pos, S.q, S.cell, S.grid, S.P, c, S.rc)
    got = esp_omp(S.pos, S.q, S.cell, S.grid, S.P, c, S.rc, threads=2)
    assert rel(got["energy"], ref["energy"]) < 1e-12
    assert rel(got["virial"], ref["virial"]) < 1e-12
    assert rel(got["forces"], ref["forces"]) < 1e-12
