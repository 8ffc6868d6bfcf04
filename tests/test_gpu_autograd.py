"""Automatic differentiation of the long-range energy (GPU).

Checks of ``long_range_energy`` (forward: U = U_F + U_self + U_bg of one esp_step;
backward: the step's forces and ``esp_cell_gradient``):

* d U / d r against central finite differences of the energy;
* d U / d h at fixed Cartesian positions against central finite differences in each of
  the nine cell entries (only where no stencil base and no in-sphere mode changes between
  the two evaluations, so the discrete energy is smooth there);
* the chain rule through r = h s against the virial relation dU/dh|_s = -W h^{-T},
  W = W_F + U_bg I (Sec. 2.2 eq. (instheta)), for a charged cell too;
* the FP32 path against the FP64 one;
* the 16,000-atom LiTFSI-like box (60 x 64 x 72 grid, P = 8): energy, position gradient
  and cell gradient against the oracle's energy, forces and virial, and the position
  gradient against central finite differences at h = 1e-4 A.
"""

import math

import numpy as np
import pytest

import synthetic as sy
from oracle import lattice
from oracle.esp_grid import esp_grid, modes, self_and_background, stencil
from oracle.pswf import c_from_tolerance

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU containers
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2601_00161_gb300 as esp  # noqa: E402

TRI = np.array([[13.0, 1.3, -0.9], [0.0, 14.0, 1.1], [0.0, 0.0, 12.5]])
GRID, P, DELTA = (24, 24, 24), 6, 1e-6


def fitting_rc(cell, grid, delta, floor=3.0):
    c = c_from_tolerance(delta)
    lens = np.linalg.norm(np.asarray(cell), axis=0)
    return max(floor, max(lens[d] * c / (math.pi * (grid[d] - 2.5)) for d in range(3)))


def setup(precision="fp64", net=0.0):
    rc = fitting_rc(TRI, GRID, DELTA)
    S = sy.small_random(300, TRI, seed=41, grid=GRID, P=P, delta=DELTA, rc=rc)
    q = S.q.copy()
    q[0] += net
    c = c_from_tolerance(DELTA)
    plan = esp.Plan(S.cell, S.n, S.grid, S.P, c, S.rc, precision=precision)
    return S, q, c, plan


def energy(plan, pos, h, q):
    with torch.no_grad():
        return float(esp.long_range_energy(plan, pos, h, q))


def smooth_between(S, c, pos, h1, h2):
    """Same stencil bases and the same in-sphere modes for the two cells."""
    for d in range(3):
        b = [stencil(S.grid[d] * lattice.reduced(pos, h)[:, d], S.P)[0] for h in (h1, h2)]
        if not np.array_equal(b[0], b[1]):
            return False
    m1 = modes(h1, S.grid, S.P, c, S.rc)["inside"]
    m2 = modes(h2, S.grid, S.P, c, S.rc)["inside"]
    return np.array_equal(m1, m2)


def test_position_gradient_is_minus_forces_and_matches_fd():
    S, q_np, c, plan = setup()
    pos = torch.tensor(S.pos, dtype=torch.float64, device="cuda", requires_grad=True)
    h = torch.tensor(S.cell, dtype=torch.float64, device="cuda")
    q = torch.tensor(q_np, dtype=torch.float64, device="cuda")
    U = esp.long_range_energy(plan, pos, h, q)
    U.backward()
    g = pos.grad.cpu().numpy()
    res, F = plan.compute(pos.detach(), q)
    assert np.max(np.abs(g + F.cpu().numpy())) < 1e-13 * np.max(np.abs(g))
    u = float(U.detach())
    assert abs(u - (res["energy_recip"] + res["energy_self"] + res["energy_bg"])) < 1e-12 * abs(u)
    d = 1e-5
    rng = np.random.default_rng(5)
    checked = 0
    for i in rng.choice(S.n, 12, replace=False):
        for a in range(3):
            p1, p2 = S.pos.copy(), S.pos.copy()
            p1[i, a] += d
            p2[i, a] -= d
            if not smooth_between(S, c, p1, S.cell, S.cell) or not all(
                    np.array_equal(stencil(S.grid[e] * lattice.reduced(p1, S.cell)[:, e], S.P)[0],
                                   stencil(S.grid[e] * lattice.reduced(p2, S.cell)[:, e], S.P)[0])
                    for e in range(3)):
                continue
            t1 = torch.tensor(p1, dtype=torch.float64, device="cuda")
            t2 = torch.tensor(p2, dtype=torch.float64, device="cuda")
            fd = (energy(plan, t1, h, q) - energy(plan, t2, h, q)) / (2 * d)
            assert abs(fd - g[i, a]) < 1e-6 * np.max(np.abs(g)), (i, a, fd, g[i, a])
            checked += 1
    assert checked >= 30
    plan.close()


def test_cell_gradient_matches_fd_at_fixed_positions():
    S, q_np, c, plan = setup()
    pos = torch.tensor(S.pos, dtype=torch.float64, device="cuda")
    h = torch.tensor(S.cell, dtype=torch.float64, device="cuda", requires_grad=True)
    q = torch.tensor(q_np, dtype=torch.float64, device="cuda")
    U = esp.long_range_energy(plan, pos, h, q)
    U.backward()
    G = h.grad.cpu().numpy()
    d = 1e-5
    checked = 0
    for a in range(3):
        for b in range(3):
            h1, h2 = S.cell.copy(), S.cell.copy()
            h1[a, b] += d
            h2[a, b] -= d
            if np.linalg.det(h2) <= 0 or not smooth_between(S, c, S.pos, h1, h2):
                continue
            e1 = energy(plan, pos, torch.tensor(h1, device="cuda"), q)
            e2 = energy(plan, pos, torch.tensor(h2, device="cuda"), q)
            fd = (e1 - e2) / (2 * d)
            assert abs(fd - G[a, b]) < 1e-6 * np.max(np.abs(G)), (a, b, fd, G[a, b])
            checked += 1
    assert checked >= 7
    plan.close()


@pytest.mark.parametrize("net", [0.0, 0.37])
def test_chain_rule_through_reduced_coordinates_gives_the_virial(net):
    S, q_np, c, plan = setup(net=net)
    hinv = np.linalg.inv(S.cell)
    s = torch.tensor(S.pos @ hinv.T, dtype=torch.float64, device="cuda")
    h = torch.tensor(S.cell, dtype=torch.float64, device="cuda", requires_grad=True)
    q = torch.tensor(q_np, dtype=torch.float64, device="cuda")
    U = esp.long_range_energy(plan, s @ h.T, h, q)
    U.backward()
    res, _ = plan.compute(torch.tensor(S.pos, dtype=torch.float64, device="cuda"), q)
    W = res["virial_recip"] + res["energy_bg"] * np.eye(3)
    if net:
        assert abs(res["energy_bg"]) > 1e-6  # the background term takes part
    expect = -W @ hinv.T
    assert np.max(np.abs(h.grad.cpu().numpy() - expect)) < 1e-11 * np.max(np.abs(expect))
    plan.close()


def test_fp32_gradients_follow_fp64():
    out = {}
    for precision in ("fp64", "fp32"):
        S, q_np, c, plan = setup(precision)
        dt = torch.float64 if precision == "fp64" else torch.float32
        # both plans see the same FP32-rounded inputs; only the arithmetic differs
        pos = torch.tensor(S.pos.astype(np.float32), dtype=dt, device="cuda", requires_grad=True)
        h = torch.tensor(S.cell, dtype=dt, device="cuda", requires_grad=True)
        q = torch.tensor(q_np.astype(np.float32), dtype=dt, device="cuda")
        U = esp.long_range_energy(plan, pos, h, q)
        U.backward()
        res, _ = plan.compute(pos.detach(), q)
        scale = abs(res["energy_recip"]) + abs(res["energy_self"]) + abs(res["energy_bg"])
        out[precision] = (float(U.detach()), pos.grad.double().cpu().numpy(),
                          h.grad.double().cpu().numpy(), scale)
        plan.close()
    U64, g64, G64, scale = out["fp64"]
    U32, g32, G32, _ = out["fp32"]
    # U is a difference of larger terms: the FP32 bar applies to their magnitudes
    assert abs(U32 - U64) < 2e-6 * scale
    assert np.linalg.norm(g32 - g64) < 2e-5 * np.linalg.norm(g64)
    assert np.max(np.abs(G32 - G64)) < 2e-5 * np.max(np.abs(G64))


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_litfsi16k_gradients_against_the_oracle(precision):
    """The LiTFSI-like workload (16,000 atoms, orthorhombic 50 x 56 x 62 A).

    Forward: U = U_F + U_self + U_bg against the oracle.  Backward: -dU/dr against the
    oracle's forces (eq. (AD)) and dU/dh against -W h^{-T} + sum_i F_i s_i^T built from the
    oracle's virial W = W_F + U_bg I and forces (Sec. 2.2 eq. (instheta) with r = h s).
    Each side is held to the parity bar (1e-12 FP64, 2e-6 FP32) relative to the size of
    the terms it is made of: U against |U_F| + |U_self| + |U_bg|, the cell gradient
    against |W h^{-T}| + |F|^T |s|.  In FP64 the position gradient also meets central
    finite differences of the GPU energy at h = 1e-4 A, on coordinates whose +-h moves
    change no stencil base (the discrete energy jumps at a switch).
    """
    S = sy.litfsi()
    c = c_from_tolerance(S.delta)
    dt = torch.float64 if precision == "fp64" else torch.float32
    tol = 1e-12 if precision == "fp64" else 2e-6
    plan = esp.Plan(S.cell, S.n, S.grid, S.P, c, S.rc, precision=precision)
    pos = torch.tensor(S.pos, dtype=dt, device="cuda", requires_grad=True)
    h = torch.tensor(S.cell, dtype=torch.float64, device="cuda", requires_grad=True)
    q = torch.tensor(S.q, dtype=dt, device="cuda")
    U = esp.long_range_energy(plan, pos, h, q)
    U.backward()
    posd = pos.detach().double().cpu().numpy()
    qd = q.double().cpu().numpy()
    ref = esp_grid(posd, qd, S.cell, S.grid, S.P, c, S.rc)
    sb = self_and_background(qd, S.cell, c, S.rc)
    U_ref = ref["energy"] + sb["energy_self"] + sb["energy_bg"]
    scale = abs(ref["energy"]) + abs(sb["energy_self"]) + abs(sb["energy_bg"])
    assert abs(float(U.detach()) - U_ref) < tol * scale
    g = pos.grad.double().cpu().numpy()
    F = ref["forces"]
    assert np.linalg.norm(g + F) < tol * np.linalg.norm(F)
    hinv = np.linalg.inv(S.cell)
    s = posd @ hinv.T  # as given, not wrapped (the cell gradient's moment uses r = h s)
    W = ref["virial"] + sb["energy_bg"] * np.eye(3)
    G_ref = -W @ hinv.T + F.T @ s
    G = h.grad.double().cpu().numpy()
    size = np.linalg.norm(W @ hinv.T) + np.linalg.norm(np.abs(F).T @ np.abs(s))
    assert np.linalg.norm(G - G_ref) < tol * size, (np.linalg.norm(G - G_ref) / size)
    if precision == "fp64":
        d = 1e-4
        rng = np.random.default_rng(3)
        checked = 0
        hq = torch.tensor(S.cell, dtype=torch.float64, device="cuda")
        for i in rng.choice(S.n, 10, replace=False):
            for a in range(3):
                p1, p2 = S.pos.copy(), S.pos.copy()
                p1[i, a] += d
                p2[i, a] -= d
                s1 = lattice.reduced(p1[i:i + 1], S.cell)[0]
                s2 = lattice.reduced(p2[i:i + 1], S.cell)[0]
                if not all(np.array_equal(stencil(S.grid[e] * s1[e:e + 1], S.P)[0],
                                          stencil(S.grid[e] * s2[e:e + 1], S.P)[0]) for e in range(3)):
                    continue
                e1 = energy(plan, torch.tensor(p1, device="cuda"), hq, q)
                e2 = energy(plan, torch.tensor(p2, device="cuda"), hq, q)
                fd = (e1 - e2) / (2 * d)
                assert abs(fd - g[i, a]) < 1e-6 * np.max(np.abs(g)), (i, a, fd, g[i, a])
                checked += 1
        assert checked >= 20
    plan.close()
