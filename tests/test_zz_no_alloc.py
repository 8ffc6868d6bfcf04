"""The allocation-free spreading entry point against the plan path (GPU).

esp_spread_noalloc serves callers that cannot call cudaMalloc when they spread (code
under an allocator or memory pool that forbids further device allocations, or a runtime
with a device-memory budget fixed at start-up): its scratch lives in a static device
array of the library.
Here its output must match the spread grid of the ordinary plan path (esp_plan,
esp_energy_pressure, esp_copy_grid) to the parity tolerances of the other GPU tests, on
two calls in a row (the second reuses the array the first one left behind).  This file
is named to be collected last, so a run that stops at the first failure has already run
every other test.
"""

import numpy as np
import pytest

import synthetic as sy
from oracle.pswf import c_from_tolerance

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU containers
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2601_00161_gb300 as esp  # noqa: E402

TOL = {"fp64": 1e-12, "fp32": 2e-6}
TRI = np.array([[13.0, 1.3, -0.9], [0.0, 14.0, 1.1], [0.0, 0.0, 12.5]])


def plan_grid(S, c, precision, pos, q):
    plan = esp.Plan(S.cell, S.n, S.grid, S.P, c, S.rc, precision=precision)
    plan.energy_pressure(pos, q)
    ref = plan.grid_values().astype(np.float64)
    plan.close()
    return ref


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("case", ["water648", "ragged"])
def test_noalloc_spread_matches_plan_path(precision, case):
    if case == "water648":
        S = sy.water_cubic()
    else:
        S = sy.small_random(900, TRI, seed=31, grid=(30, 26, 28), P=7, delta=1e-6, rc=4.0)
    c = c_from_tolerance(S.delta)
    dt = torch.float64 if precision == "fp64" else torch.float32
    pos = torch.tensor(S.pos, dtype=dt, device="cuda")
    q = torch.tensor(S.q, dtype=dt, device="cuda")
    ref = plan_grid(S, c, precision, pos, q)
    flag = esp.ESP_FP64 if precision == "fp64" else esp.ESP_FP32
    for _ in range(2):  # the second call finds the scratch as the first one left it
        out = torch.full(S.grid, float("nan"), dtype=dt, device="cuda")
        esp.esp_spread_noalloc(S.cell, S.n, S.grid, S.P, c, flag, pos, q, out)
        torch.cuda.synchronize()
        got = out.double().cpu().numpy()
        assert np.all(np.isfinite(got))
        assert np.max(np.abs(got - ref)) < TOL[precision] * np.max(np.abs(ref))
    # a call with another c (the library rebuilds its window table), then this c again
    c2 = c_from_tolerance(S.delta * 10.0)
    ref2 = plan_grid(S, c2, precision, pos, q)
    for cc, rr in ((c2, ref2), (c, ref)):
        out = torch.full(S.grid, float("nan"), dtype=dt, device="cuda")
        esp.esp_spread_noalloc(S.cell, S.n, S.grid, S.P, cc, flag, pos, q, out)
        torch.cuda.synchronize()
        got = out.double().cpu().numpy()
        assert np.max(np.abs(got - rr)) < TOL[precision] * np.max(np.abs(rr))


def test_noalloc_rejects_sizes_beyond_its_scratch():
    S = sy.water_cubic()
    c = c_from_tolerance(S.delta)
    pos = torch.zeros((esp.ESP_NOALLOC_MAX_ATOMS + 1, 3), dtype=torch.float64, device="cuda")
    q = torch.zeros(esp.ESP_NOALLOC_MAX_ATOMS + 1, dtype=torch.float64, device="cuda")
    out = torch.zeros(S.grid, dtype=torch.float64, device="cuda")
    with pytest.raises(esp.ESPError) as ei:
        esp.esp_spread_noalloc(S.cell, esp.ESP_NOALLOC_MAX_ATOMS + 1, S.grid, S.P, c,
                               esp.ESP_FP64, pos, q, out)
    assert ei.value.code == esp.ESP_ERR_ARG
    big = (256, 256, 256)  # 8 x 8 x 16 tiles: 32 * 32 * 16 = 16384 > ESP_NOALLOC_MAX_TILES
    with pytest.raises(esp.ESPError) as ei:
        esp.esp_spread_noalloc(np.eye(3) * 100.0, 10, big, 6, c, esp.ESP_FP64, pos[:10], q[:10], out)
    assert ei.value.code == esp.ESP_ERR_ARG
