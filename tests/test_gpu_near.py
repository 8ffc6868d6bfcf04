"""GPU near (real-space) part of the split against the FP64 oracle (Sec. 3, eq. (UN)).

``esp_near`` against ``oracle.esp_split(..., far=False)``: energy, virial and forces, FP64
within 1e-12 and FP32 within 2e-6 (relative, normwise).  Cells wider and narrower than
the split radius (one bin with several periodic images per axis), triclinic cells, one
atom (only its own images), no atoms, forces added onto existing ones, a cell change,
and a 16,000-atom workload with sampled force rows.  With the long-range step the total
Coulomb energy and virial match classical Ewald to the split tolerance.
"""

import math

import numpy as np
import pytest

import synthetic as sy
from oracle.esp_split import esp_split
from oracle.ewald import ewald
from oracle.pswf import c_from_tolerance

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU containers
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2601_00161_gb300 as esp  # noqa: E402

TOL = {"fp64": 1e-12, "fp32": 2e-6}
TRI = np.array([[13.0, 1.3, -0.9], [0.0, 14.0, 1.1], [0.0, 0.0, 12.5]])


def rel(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / nb) if nb > 0 else float(np.linalg.norm(a))


def fitting_rc(cell, grid, delta, floor=3.0):
    c = c_from_tolerance(delta)
    lens = np.linalg.norm(np.asarray(cell), axis=0)
    return max(floor, max(lens[d] * c / (math.pi * (grid[d] - 2.5)) for d in range(3)))


def gpu_near(S, c, precision, rows=None):
    plan = esp.Plan(S.cell, S.n, S.grid, S.P, c, S.rc, precision=precision)
    dt = torch.float64 if precision == "fp64" else torch.float32
    pos = torch.tensor(S.pos, dtype=dt, device="cuda")
    q = torch.tensor(S.q, dtype=dt, device="cuda")
    U, W, F = plan.near(pos, q)
    torch.cuda.synchronize()
    return plan, U, W, F.double().cpu().numpy(), pos.double().cpu().numpy(), q.double().cpu().numpy()


def check(S, precision, cell_list=False):
    c = c_from_tolerance(S.delta)
    plan, U, W, F, pos, q = gpu_near(S, c, precision)
    ref = esp_split(pos, q, S.cell, c, S.rc, far=False, cell_list=cell_list)
    tol = TOL[precision]
    assert rel(U, ref["energy_near"]) < tol, (U, ref["energy_near"])
    assert rel(W, ref["virial_near"]) < tol
    assert rel(F, ref["forces_near"]) < tol
    plan.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_water648(precision):
    check(sy.water_cubic(), precision)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("rc", [3.4, 4.5, 6.9])
def test_triclinic_bins_and_images(precision, rc):
    # rc 3.4: three bins per axis; 4.5: two; 6.9: one bin with an image on each side
    S = sy.small_random(400, TRI, seed=51, grid=(24, 24, 24), P=6, delta=1e-6, rc=rc)
    check(S, precision)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_cell_narrower_than_the_cutoff(precision):
    # 6 A box, r_c = 9.5 A: every atom meets several images of every other atom, and its own
    cell = np.array([[6.0, 0.4, 0.0], [0.0, 6.5, -0.3], [0.0, 0.0, 7.0]])
    S = sy.small_random(40, cell, seed=52, grid=(64, 64, 64), P=6, delta=1e-5, rc=9.5)
    check(S, precision)


def test_one_atom_and_no_atoms():
    cell = np.diag([7.0, 8.0, 9.0])
    S = sy.small_random(1, cell, seed=53, grid=(40, 40, 40), P=6, delta=1e-5, rc=8.5)
    S.q[:] = 1.3
    check(S, "fp64")
    S0 = sy.small_random(0, cell, seed=53, grid=(16, 16, 16), P=6, delta=1e-5, rc=3.0)
    plan = esp.Plan(S0.cell, 0, S0.grid, S0.P, c_from_tolerance(S0.delta), S0.rc)
    U, W, F = plan.near(torch.zeros((0, 3), dtype=torch.float64, device="cuda"),
                        torch.zeros(0, dtype=torch.float64, device="cuda"))
    assert U == 0.0 and not W.any() and F.shape == (0, 3)
    plan.close()


def test_add_onto_existing_forces_and_cell_change():
    S = sy.small_random(300, TRI, seed=54, grid=(24, 24, 24), P=6, delta=1e-6, rc=4.2)
    c = c_from_tolerance(S.delta)
    plan = esp.Plan(S.cell, S.n, S.grid, S.P, c, S.rc)
    pos = torch.tensor(S.pos, dtype=torch.float64, device="cuda")
    q = torch.tensor(S.q, dtype=torch.float64, device="cuda")
    base = torch.full((S.n, 3), 0.75, dtype=torch.float64, device="cuda")
    _, _, F = plan.near(pos, q, forces=base.clone(), add=True)
    ref = esp_split(S.pos, S.q, S.cell, c, S.rc, far=False)
    assert rel(F.cpu().numpy() - 0.75, ref["forces_near"]) < 1e-12
    h2 = S.cell @ np.diag([1.05, 0.97, 1.02])  # NPT: the cell list follows the cell
    plan.set_cell(h2)
    U2, W2, F2 = plan.near(pos, q)
    ref2 = esp_split(S.pos, S.q, h2, c, S.rc, far=False)
    assert rel(U2, ref2["energy_near"]) < 1e-12 and rel(W2, ref2["virial_near"]) < 1e-12
    assert rel(F2.cpu().numpy(), ref2["forces_near"]) < 1e-12
    plan.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_litfsi16k(precision):
    S = sy.litfsi()
    c = c_from_tolerance(S.delta)
    plan, U, W, F, pos, q = gpu_near(S, c, precision)
    ref = esp_split(pos, q, S.cell, c, S.rc, far=False, cell_list=True)
    tol = TOL[precision]
    assert rel(U, ref["energy_near"]) < tol
    assert rel(W, ref["virial_near"]) < tol
    assert rel(F, ref["forces_near"]) < tol
    plan.close()


def test_total_coulomb_against_ewald():
    S = sy.water_cubic()
    c = c_from_tolerance(S.delta)
    plan = esp.Plan(S.cell, S.n, S.grid, S.P, c, S.rc)
    pos = torch.tensor(S.pos, dtype=torch.float64, device="cuda")
    q = torch.tensor(S.q, dtype=torch.float64, device="cuda")
    res, F = plan.compute(pos, q)
    U_N, W_N, F = plan.near(pos, q, forces=F, add=True)
    U = res["energy_recip"] + res["energy_self"] + res["energy_bg"] + U_N
    W = res["virial_recip"] + res["energy_bg"] * np.eye(3) + W_N
    E = ewald(S.pos, S.q, S.cell)
    assert rel(U, E["energy"]) < 1e-6
    assert rel(W, E["virial"]) < 1e-6
    assert rel(F.cpu().numpy(), E["forces"]) < 1e-6
    plan.close()
