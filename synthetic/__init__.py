"""Seeded synthetic systems for the ESP long-range step.

This module is the ONLY code shared by the CUDA path's callers (benchmark, tests) and
the CPU oracle.  It draws positions, charges and cells and holds none of the method's
arithmetic: no window, no kernel, no Fourier sum.

Recipes (numpy Generator(PCG64(seed)), seed = 1000 + workload index):

* ``water``   - rigid SPC/E-like water, O -0.8476 e and H +0.4238 e, O-H 1.0 A,
                H-O-H 109.47 deg; O at a uniform random point of the cell (uniform in
                reduced coordinates), orientation from a normalised 4D Gaussian quaternion.
* ``litfsi``  - Li+ (+1 e) and a rigid 15-site anion; the anion template has seeded
                sites within 3.5 A of its centre with pairwise separation >= 1.2 A and
                seeded charges N(0, 0.3 e) shifted to sum to -1 e; centres uniform,
                orientations uniform.
* ``slab``    - membrane-like slab: zwitterion pairs (+-0.7 e, 4 A apart) with centres
                uniform in the slab z-range and water (as above) filling the rest of
                the cell.

The cell is returned as the 3x3 matrix h whose COLUMNS are the cell vectors (triclinic
cells use the upper-triangular convention: a = (lx,0,0), b = (xy,ly,0), c = (xz,yz,lz)).
The stored workloads name the paper's systems they stand in for: equilibrated SPC/E
water, the LiTFSI ionic liquid and the bc1 membrane system, none of which ships here.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

Q_O = -0.8476
Q_H = 0.4238
R_OH = 1.0
THETA_HOH = math.radians(109.47)


@dataclass
class System:
    name: str
    pos: np.ndarray  # [N, 3] Cartesian, Angstrom, float64
    q: np.ndarray  # [N] charges, e, float64
    cell: np.ndarray  # [3, 3], columns are cell vectors
    grid: tuple  # (M1, M2, M3)
    P: int  # stencil width
    delta: float  # PSWF tolerance; c follows from psi_0(1)/psi_0(0) = delta
    rc: float  # split radius r_c, Angstrom
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return len(self.q)


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def random_rotations(rng: np.random.Generator, n: int) -> np.ndarray:
    """n rotation matrices, uniform on SO(3) (normalised Gaussian quaternions)."""
    qv = rng.normal(size=(n, 4))
    qv /= np.linalg.norm(qv, axis=1, keepdims=True)
    w, x, y, z = qv.T
    R = np.empty((n, 3, 3))
    R[:, 0, 0] = 1 - 2 * (y * y + z * z)
    R[:, 0, 1] = 2 * (x * y - z * w)
    R[:, 0, 2] = 2 * (x * z + y * w)
    R[:, 1, 0] = 2 * (x * y + z * w)
    R[:, 1, 1] = 1 - 2 * (x * x + z * z)
    R[:, 1, 2] = 2 * (y * z - x * w)
    R[:, 2, 0] = 2 * (x * z - y * w)
    R[:, 2, 1] = 2 * (y * z + x * w)
    R[:, 2, 2] = 1 - 2 * (x * x + y * y)
    return R


def water_template() -> tuple[np.ndarray, np.ndarray]:
    half = 0.5 * THETA_HOH
    sites = np.array([[0.0, 0.0, 0.0],
                      [R_OH * math.sin(half), 0.0, R_OH * math.cos(half)],
                      [-R_OH * math.sin(half), 0.0, R_OH * math.cos(half)]])
    return sites, np.array([Q_O, Q_H, Q_H])


def place(rng, template_xyz, template_q, centres):
    """Copies of a rigid template at ``centres`` with uniform random orientations."""
    R = random_rotations(rng, len(centres))
    xyz = centres[:, None, :] + np.einsum("nab,sb->nsa", R, template_xyz)
    q = np.broadcast_to(template_q, (len(centres), len(template_q)))
    return xyz.reshape(-1, 3), q.reshape(-1).copy()


def water(n_mol: int, cell: np.ndarray, rng) -> tuple[np.ndarray, np.ndarray]:
    s = rng.random((n_mol, 3))
    centres = s @ cell.T
    return place(rng, *water_template(), centres)


def anion_template(rng, n_sites=15, radius=3.5, min_sep=1.2, sigma=0.3, total=-1.0):
    pts = [np.zeros(3)]
    while len(pts) < n_sites:
        p = rng.uniform(-radius, radius, size=3)
        if np.linalg.norm(p) > radius:
            continue
        if min(np.linalg.norm(p - x) for x in pts) < min_sep:
            continue
        pts.append(p)
    xyz = np.array(pts)
    xyz -= xyz.mean(axis=0)
    q = rng.normal(0.0, sigma, size=n_sites)
    q += (total - q.sum()) / n_sites
    return xyz, q


def neutralise(q: np.ndarray) -> np.ndarray:
    """Remove the rounding residue of the net charge (spread evenly)."""
    return q - q.sum() / len(q)


def water_cubic() -> System:
    """216 rigid waters (648 atoms) in a cubic cell of 18.65 A; grid 24^3, P = 6."""
    rng = _rng(1000)
    cell = np.eye(3) * 18.65
    pos, q = water(216, cell, rng)
    return System("water648_cubic", pos, neutralise(q), cell, (24, 24, 24), 6, 1e-6, 9.0,
                  {"stands_for": "equilibrated SPC/E water (Sec. 5.1)"})


def water_triclinic() -> System:
    """10,000 waters (30,000 atoms), triclinic 67 A cell with tilts 0.1 L; grid 64^3, P = 8."""
    rng = _rng(1001)
    L = 67.0
    cell = np.array([[L, 0.1 * L, 0.1 * L], [0.0, L, 0.1 * L], [0.0, 0.0, L]])
    pos, q = water(10_000, cell, rng)
    return System("water30k_triclinic", pos, neutralise(q), cell, (64, 64, 64), 8, 1e-7, 9.0,
                  {"stands_for": "bulk SPC/E water, fully flexible cell"})


def litfsi() -> System:
    """1,000 Li+ and 1,000 15-site anions (16,000 atoms), 50x56x62 A; grid 60x64x72, P = 8."""
    rng = _rng(1002)
    cell = np.diag([50.0, 56.0, 62.0])
    axyz, aq = anion_template(rng)
    li = rng.random((1000, 3)) @ cell.T
    an_c = rng.random((1000, 3)) @ cell.T
    apos, aqq = place(rng, axyz, aq, an_c)
    pos = np.concatenate([li, apos])
    q = np.concatenate([np.ones(1000), aqq])
    return System("litfsi16k_ortho", pos, neutralise(q), cell, (60, 64, 72), 8, 1e-7, 9.0,
                  {"stands_for": "LiTFSI ionic liquid (Sec. 5.3)"})


def membrane_slab(P: int = 6, delta: float = 1e-5) -> System:
    """Slab of zwitterion pairs between water layers, 210,240 atoms, 120x120x150 A.

    Slab z in [55, 95) A: 25,920 pairs (+-0.7 e, 4 A apart), 0.09 atoms/A^3; water
    elsewhere, 52,800 molecules, 0.1 atoms/A^3.  Grid 128x128x160.
    """
    rng = _rng(1003)
    Lx, Ly, Lz = 120.0, 120.0, 150.0
    z0, z1 = 55.0, 95.0
    cell = np.diag([Lx, Ly, Lz])
    n_pair = 25_920
    cen = np.column_stack([rng.random(n_pair) * Lx, rng.random(n_pair) * Ly, z0 + rng.random(n_pair) * (z1 - z0)])
    zw_xyz = np.array([[0.0, 0.0, 2.0], [0.0, 0.0, -2.0]])
    zpos, zq = place(rng, zw_xyz, np.array([0.7, -0.7]), cen)
    n_w = 52_800
    zw = rng.random(n_w) * (Lz - (z1 - z0))
    zw = np.where(zw < z0, zw, zw + (z1 - z0))
    wcen = np.column_stack([rng.random(n_w) * Lx, rng.random(n_w) * Ly, zw])
    wpos, wq = place(rng, *water_template(), wcen)
    pos = np.concatenate([zpos, wpos])
    q = np.concatenate([zq, wq])
    return System("membrane_slab_210k", pos, neutralise(q), cell, (128, 128, 160), P, delta, 9.0,
                  {"stands_for": "bc1 transmembrane system (Sec. 5.4), semi-isotropic"})


def small_random(n: int, cell, seed: int, grid=(16, 18, 20), P=6, delta=1e-6, rc=4.0) -> System:
    """Uniform random charges N(0, 1), neutralised; for ragged and edge-case tests."""
    rng = _rng(seed)
    cell = np.asarray(cell, dtype=np.float64)
    pos = rng.random((n, 3)) @ cell.T
    q = neutralise(rng.normal(size=n)) if n else np.zeros(0)
    return System(f"random{n}", pos, q, cell, tuple(grid), P, delta, rc)


def selector_system(i: int) -> System:
    """System i (0..63) of the parameter selector's set.

    N log-uniform in [1e3, 1e6] (whole molecules or ion pairs), density 0.1 atoms/A^3,
    triclinic cell: diagonal lengths with aspect ratios in [0.8, 1.25] and upper-triangle
    tilts uniform in [0, 0.3] of the lengths; even i water, odd i the LiTFSI-like ionic
    composition.  Grid, P, Delta and r_c are placeholders: the selector chooses them.
    """
    rng = _rng(2000 + i)
    n_target = math.exp(rng.uniform(math.log(1e3), math.log(1e6)))
    ionic = i % 2 == 1
    per = 16 if ionic else 3
    units = max(2, int(round(n_target / per)))
    n = units * per
    vol = n / 0.1
    aspect = np.exp(rng.uniform(np.log(0.8), np.log(1.25), size=3))
    L = aspect * (vol / np.prod(aspect)) ** (1.0 / 3.0)
    cell = np.diag(L)
    cell[0, 1], cell[0, 2], cell[1, 2] = rng.uniform(0.0, 0.3, size=3) * np.array([L[0], L[0], L[1]])
    if ionic:
        axyz, aq = anion_template(rng)
        li = rng.random((units, 3)) @ cell.T
        apos, aqq = place(rng, axyz, aq, rng.random((units, 3)) @ cell.T)
        pos = np.concatenate([li, apos])
        q = np.concatenate([np.ones(units), aqq])
    else:
        pos, q = water(units, cell, rng)
    return System(f"selector{i:02d}", pos, neutralise(q), cell, (32, 32, 32), 6, 1e-5, 9.0,
                  {"composition": "ionic" if ionic else "water"})


N_SELECTOR_SYSTEMS = 64

WORKLOADS = {
    "water648_cubic": water_cubic,
    "water30k_triclinic": water_triclinic,
    "litfsi16k_ortho": litfsi,
    "membrane_slab_210k": membrane_slab,
}
