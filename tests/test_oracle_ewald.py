"""Pins for O-EWALD (classical Ewald, Sec. 2.1) against what the mathematics fixes (no GPU)."""

import itertools
import math

import numpy as np
import pytest

from oracle.ewald import default_params, ewald, madelung_nacl

MADELUNG_NACL = 1.747564594633182190636212035544397403481  # rock salt, nearest-neighbour units


def _random_system(n=24, seed=5):
    rng = np.random.default_rng(seed)
    h = np.array([[10.0, 1.0, 0.5], [0.0, 11.0, 0.7], [0.0, 0.0, 9.0]])
    pos = rng.random((n, 3)) @ h.T
    q = rng.normal(size=n)
    q -= q.mean()
    return pos, q, h


def test_madelung_constant():
    a = 2.0  # nearest-neighbour distance a/2 = 1
    pos, q, h = madelung_nacl(a)
    r = ewald(pos, q, h)
    assert abs(r["energy"] - (-4 * MADELUNG_NACL / (a / 2))) < 1e-12 * 4 * MADELUNG_NACL
    W = r["virial"]
    # cubic symmetry: isotropic tensor, and tr W = U (Coulomb homogeneity, eq. (deth))
    assert np.max(np.abs(W - np.trace(W) / 3 * np.eye(3))) < 1e-12
    assert abs(np.trace(W) - r["energy"]) < 1e-11
    assert np.max(np.abs(r["forces"])) < 1e-12


def test_virial_identity_and_symmetry():
    pos, q, h = _random_system()
    r = ewald(pos, q, h)
    W = r["virial"]
    assert np.max(np.abs(W - W.T)) < 1e-12 * np.max(np.abs(W))
    # tr W = U; the reciprocal virial cancels terms of size ~beta sum q^2, hence the scale
    scale = r["params"][0] * np.sum(q * q)
    assert abs(np.trace(W) - r["energy"]) < 1e-12 * scale


def test_independent_of_splitting_parameter():
    pos, q, h = _random_system()
    a = ewald(pos, q, h)
    b = ewald(pos, q, h, *default_params(h, rcut=3.2))
    assert abs(a["energy"] - b["energy"]) < 1e-13 * abs(a["energy"]) + 1e-13
    assert np.max(np.abs(a["forces"] - b["forces"])) < 1e-12 * np.max(np.abs(a["forces"]))
    assert np.max(np.abs(a["virial"] - b["virial"])) < 1e-11 * np.max(np.abs(a["virial"]))


def test_translation_invariance_and_momentum():
    pos, q, h = _random_system()
    a = ewald(pos, q, h)
    b = ewald(pos + np.array([0.37, -1.3, 2.9]), q, h)
    assert abs(a["energy"] - b["energy"]) < 1e-13 * abs(a["energy"])
    assert np.max(np.abs(a["forces"] - b["forces"])) < 1e-12 * np.max(np.abs(a["forces"]))
    assert np.max(np.abs(a["forces"].sum(axis=0))) < 1e-12 * np.max(np.abs(a["forces"]))


def test_forces_and_virial_by_finite_differences():
    pos, q, h = _random_system(n=12, seed=9)
    r = ewald(pos, q, h)
    d = 1e-5
    for i, a in [(0, 0), (3, 1), (7, 2)]:
        p1, p2 = pos.copy(), pos.copy()
        p1[i, a] += d
        p2[i, a] -= d
        fd = -(ewald(p1, q, h, forces=False)["energy"] - ewald(p2, q, h, forces=False)["energy"]) / (2 * d)
        assert abs(fd - r["forces"][i, a]) < 1e-7 * max(1.0, abs(fd))
    # W = -(dU/dh) h^T at fixed reduced coordinates (eq. (instheta))
    s = pos @ np.linalg.inv(h).T
    dUdh = np.zeros((3, 3))
    for a, b in itertools.product(range(3), range(3)):
        h1, h2 = h.copy(), h.copy()
        h1[a, b] += d
        h2[a, b] -= d
        dUdh[a, b] = (ewald(s @ h1.T, q, h1, forces=False)["energy"]
                      - ewald(s @ h2.T, q, h2, forces=False)["energy"]) / (2 * d)
    assert np.max(np.abs(-dUdh @ h.T - r["virial"])) < 1e-7 * np.max(np.abs(r["virial"]))


def test_brute_force_spherical_image_sum():
    # eq. (1.1) summed over spherical shells of images converges, for a neutral cell with
    # zero dipole, to the tin-foil Ewald value (the surface term 2 pi |D|^2 / 3V vanishes)
    L = 5.0
    h = np.eye(3) * L
    pos = np.array([[1.3, 1.6, 1.7], [2.9, 1.6, 1.7], [1.3, 3.3, 1.7], [2.9, 3.3, 1.7],
                    [2.2, 3.1, 3.3], [2.2, 3.1, 4.4], [3.7, 1.1, 3.9], [3.7, 1.1, 2.8]])
    q = np.array([1, -1, -1, 1, 0.5, -0.5, 0.5, -0.5])
    assert np.max(np.abs(q @ pos)) < 1e-14
    E = ewald(pos, q, h)["energy"]
    errs = []
    for R in (10, 20, 40):
        n = np.array(list(itertools.product(range(-R, R + 1), repeat=3)), dtype=float)
        n = n[np.einsum("ij,ij->i", n, n) <= R * R] * L
        U = 0.0
        for i in range(len(q)):
            for j in range(len(q)):
                dd = pos[i] - pos[j] + n
                r = np.sqrt(np.einsum("ij,ij->i", dd, dd))
                if i == j:
                    r = r[r > 0]
                U += 0.5 * q[i] * q[j] * np.sum(1.0 / r)
        errs.append(abs(U - E))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 2e-8 * abs(E)


def test_net_charge_background():
    # a charged cell with its uniform background is again independent of beta
    pos, q, h = _random_system()
    q = q + 0.3
    a = ewald(pos, q, h)
    b = ewald(pos, q, h, *default_params(h, rcut=3.2))
    assert abs(a["energy"] - b["energy"]) < 1e-12 * abs(a["energy"])
    assert np.max(np.abs(a["virial"] - b["virial"])) < 1e-11 * np.max(np.abs(a["virial"]))
