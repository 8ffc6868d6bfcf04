"""GPU parity: the CUDA path through the C ABI against the FP64 CPU oracle.

Bars: FP64 path within 1e-12 relative of the oracle (normwise for tensors and force
arrays), FP32 path within 2e-6 relative.  Sizes span several tiles and ragged tails;
odd and even stencils; cubic, orthorhombic and triclinic cells; empty and one-atom
inputs; atoms far outside the primary cell.
"""

import math

import numpy as np
import pytest

import synthetic as sy
from oracle.esp_grid import esp_grid, self_and_background, spread
from oracle.pswf import c_from_tolerance

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU containers
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2601_00161_gb300 as esp  # noqa: E402

TOL = {"fp64": 1e-12, "fp32": 2e-6}


def rel(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / nb) if nb > 0 else float(np.linalg.norm(a))


def fitting_rc(cell, grid, delta, floor=3.0):
    """Smallest split radius (>= floor) for which every in-sphere mode stays below Nyquist."""
    c = c_from_tolerance(delta)
    lens = np.linalg.norm(np.asarray(cell), axis=0)
    need = max(lens[d] * c / (math.pi * (grid[d] - 1.5)) for d in range(3))
    return max(floor, need)


def run_gpu(S, c, precision, forces=True):
    plan = esp.Plan(S.cell, S.n, S.grid, S.P, c, S.rc, precision=precision)
    dt = torch.float64 if precision == "fp64" else torch.float32
    pos = torch.tensor(S.pos, dtype=dt, device="cuda")
    q = torch.tensor(S.q, dtype=dt, device="cuda")
    if forces:
        res, F = plan.compute(pos, q)
        torch.cuda.synchronize()
        F = F.double().cpu().numpy()
    else:
        res, F = plan.energy_pressure(pos, q), None
    return plan, res, F, pos.double().cpu().numpy(), q.double().cpu().numpy()


def check(S, precision, c=None, forces=True, force_rows=None, ftol=None):
    c = c_from_tolerance(S.delta) if c is None else c
    plan, res, F, pos, q = run_gpu(S, c, precision, forces)
    # the oracle sees exactly the inputs the GPU saw (FP32 rounding included)
    ref = esp_grid(pos, q, S.cell, S.grid, S.P, c, S.rc, forces=forces, force_rows=force_rows)
    tol = TOL[precision]
    assert rel(res["energy_recip"], ref["energy"]) < tol, (res["energy_recip"], ref["energy"])
    assert rel(res["virial_recip"], ref["virial"]) < tol
    assert rel(res["pressure_recip"], ref["virial"] / np.linalg.det(S.cell)) < tol
    if forces:
        Fg = F if force_rows is None else F[force_rows]
        ft = tol if ftol is None else ftol
        assert rel(Fg, ref["forces"]) < ft
        assert np.max(np.abs(Fg - ref["forces"])) < 10 * ft * np.max(np.abs(ref["forces"]))
    plan.close()
    return res, F


# -- small and ragged cases ----------------------------------------------------------------
TRI = np.array([[13.0, 1.3, -0.9], [0.0, 14.0, 1.1], [0.0, 0.0, 12.5]])
ORTHO = np.diag([11.0, 13.0, 17.0])


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_water648(precision):
    check(sy.water_cubic(), precision)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("grid,cell,n", [
    # 1001 = 7 * 11 * 13: passes of radix 7 and of two larger primes, and a first axis long
    # enough that fewer columns share a CTA (4 in FP32, 2 in FP64).  The cross-section is
    # kept several r_c wide: a cell a few angstrom thin has transverse forces a hundred
    # times below the longitudinal ones, which FP32 cannot resolve to 2e-6 normwise.
    ((1001, 28, 30), np.diag([300.0, 12.0, 13.0]), 1200),
    # a prime first axis: one direct pass of length 127
    ((127, 16, 18), np.diag([60.0, 5.0, 5.5]), 150),
])
def test_first_axis_transform_sizes(precision, grid, cell, n):
    """The transform along the first axis (in shared memory, fused with the scaling) for
    lengths that the common grid sizes do not reach.  FP64 holds the 1e-12 bar.  FP32
    forces on the 1001-point axis come out 7.6e-6 from the oracle normwise, exactly as
    the full cuFFT 3D transform plus a separate scaling gave (measured on the same
    inputs), against 1.1e-6 on a 250-point axis at the same spacing: the loss is FP32
    arithmetic on the long axis, not this transform.  Those forces are held to the
    1e-5 accuracy bar of the method's target instead of 2e-6; energy and virial keep 2e-6."""
    rc = fitting_rc(cell, grid, 1e-5)
    S = sy.small_random(n, cell, seed=31, grid=grid, P=6, delta=1e-5, rc=rc)
    check(S, precision, ftol=1e-5 if (precision == "fp32" and grid[0] > 512) else None)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("P,grid,cell,n", [
    (6, (24, 26, 30), TRI, 300),     # ragged tiles in every dimension
    (5, (17, 23, 29), ORTHO, 211),   # odd P, prime grid sizes
    (7, (20, 21, 22), TRI, 97),
    (8, (33, 19, 41), ORTHO, 1000),
    (3, (12, 12, 12), ORTHO, 50),
    (12, (40, 36, 44), TRI, 400),    # widest stencil
    (4, (9, 10, 64), TRI, 123),      # grid smaller than a tile in two dimensions
])
def test_ragged_and_odd(precision, P, grid, cell, n):
    rc = fitting_rc(cell, grid, 1e-5)
    S = sy.small_random(n, cell, seed=7 + n, grid=grid, P=P, delta=1e-5, rc=rc)
    check(S, precision)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_empty_and_single_atom(precision):
    rc = fitting_rc(ORTHO, (16, 16, 16), 1e-6)
    S0 = sy.small_random(0, ORTHO, seed=1, grid=(16, 16, 16), P=6, rc=rc)
    c = c_from_tolerance(1e-6)
    plan = esp.Plan(S0.cell, 0, S0.grid, 6, c, rc, precision=precision)
    dt = torch.float64 if precision == "fp64" else torch.float32
    r = plan.energy_pressure(torch.zeros((0, 3), dtype=dt, device="cuda"), torch.zeros(0, dtype=dt, device="cuda"))
    assert r["energy_recip"] == 0.0 and np.all(r["virial_recip"] == 0.0) and r["q2sum"] == 0.0
    plan.close()
    S1 = sy.small_random(1, ORTHO, seed=2, grid=(16, 16, 16), P=6, rc=rc)
    S1.q[:] = 1.0  # a lone (non-neutral) charge: grid self-interaction plus background
    plan, res, F, pos, q = run_gpu(S1, c, precision)
    ref = esp_grid(pos, q, S1.cell, S1.grid, 6, c, rc)
    tol = TOL[precision]
    assert rel(res["energy_recip"], ref["energy"]) < tol
    assert rel(res["virial_recip"], ref["virial"]) < tol
    # the self-force of a lone charge is pure aliasing, ~1e-6 of the sums it cancels out
    # of; compare on the scale of the field of a unit charge at the split radius
    assert np.max(np.abs(F - ref["forces"])) < tol / rc ** 2
    assert res["energy_bg"] < 0.0
    plan.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("net", [1.0, -2.5])
def test_charged_cell_self_and_background(precision, net):
    """Host scalars of a non-neutral cell against the oracle: the self energy of eq.
    (selfen) from the device sum of q^2, and the background energy and pressure of eq.
    (Corr) from the device sum of q (FP64 sums on both paths)."""
    rc = fitting_rc(TRI, (24, 26, 30), 1e-6)
    S = sy.small_random(300, TRI, seed=13, grid=(24, 26, 30), P=6, delta=1e-6, rc=rc)
    S.q[:5] += net / 5.0
    c = c_from_tolerance(S.delta)
    for forces in (True, False):
        plan, res, F, pos, q = run_gpu(S, c, precision, forces)
        ref = self_and_background(q, S.cell, c, rc)
        assert abs(res["qsum"] - q.sum()) < 1e-12 * np.abs(q).sum()
        assert rel(res["q2sum"], (q * q).sum()) < 1e-12
        for key in ("energy_self", "energy_bg", "pressure_bg"):
            assert rel(res[key], ref[key]) < 1e-12, (key, res[key], ref[key])
        assert res["energy_bg"] < 0.0
        plan.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("case", ["water648", "odd_triclinic", "membrane_slab"])
def test_energy_pressure_only_path(precision, case):
    """esp_energy_pressure: the step without forces (Algorithm 1, Sec. 4.1; no inverse
    transform, no gather) runs its own transform sequence.  Energy, virial and pressure
    against the oracle, and the host scalars too."""
    if case == "water648":
        S = sy.water_cubic()
    elif case == "odd_triclinic":
        S = sy.small_random(411, TRI, seed=17, grid=(21, 25, 27), P=7, delta=1e-5,
                            rc=fitting_rc(TRI, (21, 25, 27), 1e-5))
    else:
        S = sy.membrane_slab()
    res, _ = check(S, precision, forces=False)
    q = torch.tensor(S.q, dtype=torch.float64 if precision == "fp64" else torch.float32).double().numpy()
    ref = self_and_background(q, S.cell, c_from_tolerance(S.delta), S.rc)
    assert rel(res["energy_self"], ref["energy_self"]) < 1e-12


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_crowded_tiles_overflow(precision):
    """Tiles hold about 2.5x the mean number of atoms; atoms past that go to an overflow
    list that spread and gather handle one atom at a time.  Here 700 of 1000 atoms sit in
    a 1.5 A cube (inside one or two tiles), so most of them overflow; the energy path and
    the kept-spectrum force path must still match the oracle."""
    rng = np.random.default_rng(77)
    cell = TRI
    grid = (24, 26, 28)
    n = 1000
    pos = rng.random((n, 3)) @ cell.T
    pos[:700] = np.array([4.0, 5.0, 6.0]) + 1.5 * rng.random((700, 3))
    q = rng.normal(size=n)
    q -= q.mean()
    S = sy.System("crowded", pos, q, cell, grid, 6, 1e-5, fitting_rc(cell, grid, 1e-5))
    check(S, precision)
    res, _ = check(S, precision, forces=False)
    # forces from the kept spectrum (the gather after an energy-only step)
    c = c_from_tolerance(S.delta)
    plan, r, _, pos_d, q_d = run_gpu(S, c, precision, forces=False)
    dt = torch.float64 if precision == "fp64" else torch.float32
    F = torch.empty((n, 3), dtype=dt, device="cuda")
    esp.esp_forces_from_spectrum(plan.handle, F)
    torch.cuda.synchronize()
    ref = esp_grid(pos_d, q_d, S.cell, S.grid, S.P, c, S.rc)
    assert rel(F.double().cpu().numpy(), ref["forces"]) < TOL[precision]
    plan.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_wrapping_of_far_images(precision):
    S = sy.small_random(200, TRI, seed=3, grid=(24, 24, 24), P=6, rc=3.5)
    shift = (np.array([5, -3, 2])[None, :] * 1.0) @ TRI.T  # integer combination of cell vectors
    S2 = sy.System(S.name, S.pos + shift, S.q, S.cell, S.grid, S.P, S.delta, S.rc)
    r1, F1 = check(S, precision)
    r2, F2 = check(S2, precision)
    assert rel(r2["virial_recip"], r1["virial_recip"]) < 10 * TOL[precision]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("P", [5, 6])
def test_stencil_ties(precision, P):
    # atoms exactly on grid points and on half points: the stencil base is a floor of an
    # exactly representable grid coordinate, decided identically by both sides (FP64)
    L, M = 16.0, 32
    cell = np.eye(3) * L
    rng = np.random.default_rng(P)
    g = rng.integers(0, 2 * M, size=(120, 3)) * 0.25  # multiples of L/(2M): points and half points
    q = rng.normal(size=120)
    q -= q.mean()
    S = sy.System("ties", g, q, cell, (M, M, M), P, 1e-5, fitting_rc(cell, (M, M, M), 1e-5))
    check(S, precision)


def test_spread_grid_and_spectrum_fp64():
    S = sy.water_cubic()
    c = c_from_tolerance(S.delta)
    plan, res, _, pos, q = run_gpu(S, c, "fp64", forces=False)
    rho = plan.grid_values()
    ref = spread(pos, q, S.cell, S.grid, S.P, c)
    assert np.max(np.abs(rho - ref)) < 1e-12 * np.max(np.abs(ref))
    X = plan.spectrum()
    Xr = np.fft.rfftn(ref)
    assert np.max(np.abs(X - Xr)) < 1e-12 * np.max(np.abs(Xr))
    plan.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_forces_from_kept_spectrum_and_host_entry(precision):
    S = sy.small_random(500, TRI, seed=11, grid=(28, 30, 26), P=7, rc=3.5)
    c = c_from_tolerance(S.delta)
    dt = torch.float64 if precision == "fp64" else torch.float32
    plan = esp.Plan(S.cell, S.n, S.grid, S.P, c, S.rc, precision=precision)
    pos = torch.tensor(S.pos, dtype=dt, device="cuda")
    q = torch.tensor(S.q, dtype=dt, device="cuda")
    r = plan.energy_pressure(pos, q)
    F1 = torch.empty((S.n, 3), dtype=dt, device="cuda")
    esp.esp_forces_from_spectrum(plan.handle, F1)
    F2 = plan.forces(pos, q)
    torch.cuda.synchronize()
    assert rel(F1.double().cpu().numpy(), F2.double().cpu().numpy()) < TOL[precision]
    with pytest.raises(esp.ESPError) as ei:
        esp.esp_forces_from_spectrum(plan.handle, F1)  # spectrum consumed by the force path
    assert ei.value.code == esp.ESP_ERR_STATE
    npdt = np.float64 if precision == "fp64" else np.float32
    Fh = np.empty((S.n, 3), dtype=npdt)
    rh = esp.esp_compute_host(plan.handle, S.pos.astype(npdt), S.q.astype(npdt), Fh)
    assert rel(rh.energy_recip, r["energy_recip"]) < TOL[precision]
    assert rel(Fh, F2.double().cpu().numpy()) < TOL[precision]
    # page-locked inputs are read in place by the binning kernel: same results, and a
    # second call with new contents of the same buffers sees the new positions
    pos_p = torch.tensor(S.pos.astype(npdt)).pin_memory().numpy()
    q_p = torch.tensor(S.q.astype(npdt)).pin_memory().numpy()
    Fp = torch.empty((S.n, 3), dtype=dt).pin_memory().numpy()
    rp = esp.esp_compute_host(plan.handle, pos_p, q_p, Fp)
    assert rel(rp.energy_recip, r["energy_recip"]) < TOL[precision]
    assert rel(Fp, F2.double().cpu().numpy()) < TOL[precision]
    shift = np.array([0.37, -0.21, 0.55])
    pos_p[:] = (S.pos + shift).astype(npdt)
    rp2 = esp.esp_compute_host(plan.handle, pos_p, q_p, Fp)
    r2 = plan.energy_pressure(torch.tensor(pos_p, device="cuda"), q)
    assert rel(rp2.energy_recip, r2["energy_recip"]) < TOL[precision]
    plan.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_set_cell_npt(precision):
    S = sy.small_random(400, TRI, seed=5, grid=(24, 24, 24), P=6, rc=3.5)
    c = c_from_tolerance(S.delta)
    dt = torch.float64 if precision == "fp64" else torch.float32
    plan = esp.Plan(S.cell, S.n, S.grid, S.P, c, S.rc, precision=precision)
    s = S.pos @ np.linalg.inv(S.cell).T
    for scale in [1.0, 1.02, 0.97]:
        cell = S.cell * np.array([scale, 1.0, 1.0 / scale])[:, None]
        pos = s @ cell.T
        plan.set_cell(cell)
        res, F = plan.compute(torch.tensor(pos, dtype=dt, device="cuda"), torch.tensor(S.q, dtype=dt, device="cuda"))
        posd = torch.tensor(pos, dtype=dt).double().numpy()
        qd = torch.tensor(S.q, dtype=dt).double().numpy()
        ref = esp_grid(posd, qd, cell, S.grid, S.P, c, S.rc)
        assert rel(res["virial_recip"], ref["virial"]) < TOL[precision]
        assert rel(F.double().cpu().numpy(), ref["forces"]) < TOL[precision]
    with pytest.raises(esp.ESPError) as ei:
        plan.set_cell(S.cell * 3.0)  # grid now too coarse
    assert ei.value.code == esp.ESP_ERR_GRID
    plan.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_graph_replay_on_own_stream(precision):
    # on a non-default stream esp_step captures its launches in a CUDA graph and replays
    # it; a new cell drops the graph
    S = sy.small_random(700, TRI, seed=21, grid=(28, 28, 28), P=6, rc=3.5)
    c = c_from_tolerance(S.delta)
    dt = torch.float64 if precision == "fp64" else torch.float32
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        plan = esp.Plan(S.cell, S.n, S.grid, S.P, c, S.rc, precision=precision, stream=st.cuda_stream)
        s = S.pos @ np.linalg.inv(S.cell).T
        for scale in [1.0, 1.0, 1.03, 1.03]:
            cell = S.cell * np.array([1.0, scale, 1.0])[:, None]
            plan.set_cell(cell)
            pos = torch.tensor(s @ cell.T, dtype=dt, device="cuda")
            q = torch.tensor(S.q, dtype=dt, device="cuda")
            F = torch.empty((S.n, 3), dtype=dt, device="cuda")
            acc = torch.zeros(esp.ESP_ACCUM_LEN, dtype=torch.float64, device="cuda")
            for _ in range(2):
                plan.step(pos, q, F, acc)
            st.synchronize()
            res = esp.esp_result_from_accum(plan.handle, acc.cpu().numpy()).as_dict()
            ref = esp_grid(pos.double().cpu().numpy(), q.double().cpu().numpy(), cell, S.grid, S.P, c, S.rc)
            assert rel(res["virial_recip"], ref["virial"]) < TOL[precision]
            assert rel(F.double().cpu().numpy(), ref["forces"]) < TOL[precision]
        plan.close()


def test_nonfinite_input_is_reported_not_faulted():
    S = sy.small_random(100, ORTHO, seed=9, grid=(16, 16, 16), P=6, rc=fitting_rc(ORTHO, (16, 16, 16), 1e-6))
    c = c_from_tolerance(S.delta)
    plan = esp.Plan(S.cell, S.n, S.grid, S.P, c, S.rc, precision="fp64")
    pos = torch.tensor(S.pos, device="cuda")
    pos[17, 1] = float("nan")
    with pytest.raises(esp.ESPError) as ei:
        plan.energy_pressure(pos, torch.tensor(S.q, device="cuda"))
    assert ei.value.code == esp.ESP_ERR_NONFINITE
    # the plan stays usable
    r = plan.energy_pressure(torch.tensor(S.pos, device="cuda"), torch.tensor(S.q, device="cuda"))
    assert math.isfinite(r["energy_recip"])
    plan.close()


def test_plan_tables_are_accurate():
    S = sy.water_cubic()
    for prec, tol in [("fp64", 1e-14), ("fp32", 5e-8)]:
        plan = esp.Plan(S.cell, S.n, S.grid, S.P, c_from_tolerance(S.delta), S.rc, precision=prec)
        info = plan.info()
        assert info["fit_err"] <= tol and info["rfit_err"] <= tol, info
        plan.close()


# -- full-size workloads ------------------------------------------------------------------
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("name", ["water30k_triclinic", "litfsi16k_ortho"])
def test_medium_workloads(name, precision):
    S = sy.WORKLOADS[name]()
    rows = np.random.default_rng(0).choice(S.n, 3000, replace=False)
    check(S, precision, force_rows=rows)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_membrane_slab_full_size(precision):
    S = sy.membrane_slab()
    rows = np.random.default_rng(1).choice(S.n, 2000, replace=False)
    check(S, precision, force_rows=rows)
