"""Per-atom variants on the GPU against the FP64 oracle (Sec. 4.4 and Appendix C).

esp_forces_ik (ik-differentiation forces), esp_local_virial (per-atom virial, local
pressure) and esp_atom_energy (per-atom Fourier energy) against
oracle.esp_grid.esp_grid_fields: FP64 within 1e-12 and FP32 within 2e-6 (relative,
normwise).  The ik forces conserve momentum to rounding; the per-atom virial and energy sum
to the global values of the same step.
"""

import numpy as np
import pytest

import synthetic as sy
from oracle.esp_grid import esp_grid_fields
from oracle.pswf import c_from_tolerance

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU containers
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2601_00161_gb300 as esp  # noqa: E402

TOL = {"fp64": 1e-12, "fp32": 2e-6}
TRI = np.array([[13.0, 1.3, -0.9], [0.0, 14.0, 1.1], [0.0, 0.0, 12.5]])
def crowded():
    # 500 of 700 atoms in a 1.5 A cube: most of them pass their tile's capacity and take
    # the overflow path of the field gather
    S = sy.small_random(700, TRI, seed=72, grid=(30, 26, 28), P=7, delta=1e-6, rc=4.0)
    S.pos[:500] = np.array([3.0, 4.0, 5.0]) + 1.5 * np.random.default_rng(5).random((500, 3))
    S.q[:] -= S.q.mean()
    return S


CASES = {
    "water648": lambda: sy.water_cubic(),
    "triclinic_P7": lambda: sy.small_random(700, TRI, seed=71, grid=(30, 26, 28), P=7, delta=1e-6, rc=4.0),
    "crowded_P7": crowded,
}


def rel(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("case", list(CASES))
def test_fields_against_the_oracle(precision, case):
    S = CASES[case]()
    c = c_from_tolerance(S.delta)
    plan = esp.Plan(S.cell, S.n, S.grid, S.P, c, S.rc, precision=precision)
    dt = torch.float64 if precision == "fp64" else torch.float32
    pos = torch.tensor(S.pos, dtype=dt, device="cuda")
    q = torch.tensor(S.q, dtype=dt, device="cuda")
    p64, q64 = pos.double().cpu().numpy(), q.double().cpu().numpy()
    tol = TOL[precision]
    Fik = plan.forces_ik(pos, q).double().cpu().numpy()
    Wi = plan.local_virial(pos, q).double().cpu().numpy()
    Ui = plan.atom_energy(pos, q).double().cpu().numpy()
    assert rel(Fik, esp_grid_fields(p64, q64, S.cell, S.grid, S.P, c, S.rc, "ik")) < tol
    assert rel(Wi, esp_grid_fields(p64, q64, S.cell, S.grid, S.P, c, S.rc, "virial")) < tol
    assert rel(Ui, esp_grid_fields(p64, q64, S.cell, S.grid, S.P, c, S.rc, "energy")) < tol
    # momentum (exact for ik-differentiation) and the global sums of the same step
    assert np.max(np.abs(Fik.sum(axis=0))) < 10 * tol * np.sum(np.abs(Fik))
    res = plan.energy_pressure(pos, q)
    W = res["virial_recip"]
    Wg = np.array([W[0, 0], W[1, 1], W[2, 2], W[0, 1], W[0, 2], W[1, 2]])
    assert np.max(np.abs(Wi.sum(axis=0) - Wg)) < 10 * tol * np.max(np.abs(Wg))
    assert abs(Ui.sum() - res["energy_recip"]) < 10 * tol * abs(res["energy_recip"])
    plan.close()


def test_litfsi16k_local_virial_fp32():
    S = sy.litfsi()
    c = c_from_tolerance(S.delta)
    plan = esp.Plan(S.cell, S.n, S.grid, S.P, c, S.rc, precision="fp32")
    pos = torch.tensor(S.pos, dtype=torch.float32, device="cuda")
    q = torch.tensor(S.q, dtype=torch.float32, device="cuda")
    Wi = plan.local_virial(pos, q).double().cpu().numpy()
    ref = esp_grid_fields(pos.double().cpu().numpy(), q.double().cpu().numpy(), S.cell, S.grid,
                          S.P, c, S.rc, "virial")
    assert rel(Wi, ref) < 2e-6
    plan.close()
