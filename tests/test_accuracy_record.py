"""The membrane-slab workload meets its 1e-5 relative pressure error (Sec. 5.1).

``tests/golden/membrane_slab_accuracy.json`` is written by
``tests/golden/membrane_slab_accuracy.py`` from the FP64 oracle alone: the workload's
parameters (Delta = 1e-5, P = 6, r_c = 9 A, grid 128 x 128 x 160) against two ESP
references at Delta = 1e-11 and 1e-10 on a grid fine enough that no aliased mode reaches
the window's band.  The test checks the record against the workload definition so the
two cannot drift apart, and that the reference converged far below the error measured.
"""

import json
import os

import pytest

import synthetic as sy
from oracle.pswf import c_from_tolerance

HERE = os.path.dirname(os.path.abspath(__file__))
RECORD = os.path.join(HERE, "golden", "membrane_slab_accuracy.json")


@pytest.fixture(scope="module")
def record():
    with open(RECORD) as f:
        return json.load(f)


def test_record_matches_the_workload(record):
    S = sy.membrane_slab()
    cfg = record["configs"]["workload"]
    assert cfg["P"] == S.P and cfg["delta"] == S.delta and cfg["rc"] == S.rc
    assert tuple(cfg["grid"]) == tuple(S.grid)
    assert abs(cfg["c"] - c_from_tolerance(S.delta)) < 1e-9


def test_workload_pressure_error_below_1e5(record):
    e = record["workload_vs_reference_a"]
    # eq. (ref_pres): relative L2 error of the diagonal; also the full tensor
    assert e["pressure_diag"] < 1e-5
    assert e["pressure_frobenius"] < 1e-5
    assert e["forces_rms"] < 1e-5


def test_reference_converged(record):
    e = record["reference_b_vs_reference_a"]
    w = record["workload_vs_reference_a"]
    for k in ("pressure_diag", "pressure_offdiag", "pressure_frobenius", "forces_rms"):
        assert e[k] < 1e-3 * w[k]
