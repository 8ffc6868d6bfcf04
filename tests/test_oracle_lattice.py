"""Pins of the oracle's cell-list pair enumerator against the all-pairs image loop.

The cell list only finds pairs faster; it must yield exactly the ordered (i, j, image)
triples with the same displacement vectors as the brute-force loop over all atoms and
all periodic images, including for skewed cells, atoms on bin faces and cells that are
just wide enough for three bins.
"""

import numpy as np
import pytest

from oracle import lattice
from oracle.esp_split import esp_split
from oracle.pswf import c_from_tolerance


def triples(gen):
    """(i, j, rvec) rows sorted by i, j and the image (rvec rounded to 1e-4 for the key)."""
    rows = []
    for i, j, rv, r in gen:
        assert np.allclose(np.linalg.norm(rv, axis=1), r, rtol=0, atol=1e-12)
        rows.append(np.column_stack([i, j, rv]))
    t = np.concatenate(rows) if rows else np.zeros((0, 5))
    key = np.round(t[:, 2:], 4)
    order = np.lexsort((key[:, 2], key[:, 1], key[:, 0], t[:, 1], t[:, 0]))
    return t[order]


def same(a, b):
    return (a.shape == b.shape and np.array_equal(a[:, :2], b[:, :2])
            and np.allclose(a[:, 2:], b[:, 2:], rtol=0, atol=1e-12))


CELLS = {
    "triclinic": np.array([[19.0, 2.5, -3.1], [0.0, 21.0, 1.7], [0.0, 0.0, 23.5]]),
    # widths just above 3 rcut in one direction (exactly three bins there)
    "three_bins": np.array([[18.1, 0.0, 0.0], [0.0, 26.0, 0.0], [0.0, 0.0, 33.0]]),
    # too narrow for three bins: the enumerator falls back to the image loop
    "fallback": np.array([[14.0, 1.0, 0.0], [0.0, 15.0, 0.0], [0.0, 0.0, 30.0]]),
}


@pytest.mark.parametrize("name", list(CELLS))
def test_cell_list_yields_the_image_loop_pairs(name):
    h = CELLS[name]
    rng = np.random.default_rng(7)
    n = 260
    s = rng.random((n, 3))
    s[:5] = [[0.0, 0.0, 0.0], [1.0 / 3.0, 0.5, 0.25], [0.999999999, 0.0, 0.5],
             [0.5, 1.0 / 3.0, 2.0 / 3.0], [0.25, 0.75, 0.0]]  # on bin faces
    pos = (s - np.floor(s) + rng.integers(-2, 3, size=(n, 3))) @ h.T  # unwrapped inputs
    rcut = 6.0
    a = triples(lattice.pair_images(pos, h, rcut))
    b = triples(lattice.pair_cells(pos, h, rcut))
    assert len(a) > 1000
    assert same(a, b)


def test_cell_list_rows_subset():
    h = CELLS["triclinic"]
    rng = np.random.default_rng(3)
    pos = rng.random((200, 3)) @ h.T
    rows = np.array([0, 5, 17, 199])
    a = triples(lattice.pair_images(pos, h, 6.0, rows=rows))
    b = triples(lattice.pair_cells(pos, h, 6.0, rows=rows))
    assert same(a, b) and set(a[:, 0].astype(int).tolist()) <= set(rows.tolist())


def test_near_field_same_with_cell_list():
    h = CELLS["triclinic"]
    rng = np.random.default_rng(11)
    n = 300
    pos = rng.random((n, 3)) @ h.T
    q = rng.choice([-1.0, 1.0], n)
    c = c_from_tolerance(1e-5)
    a = esp_split(pos, q, h, c, 6.0, far=False)
    b = esp_split(pos, q, h, c, 6.0, far=False, cell_list=True)
    assert abs(a["energy_near"] - b["energy_near"]) < 1e-12 * abs(a["energy_near"])
    assert np.max(np.abs(a["virial_near"] - b["virial_near"])) < 1e-12 * np.max(np.abs(a["virial_near"]))
    assert np.max(np.abs(a["forces_near"] - b["forces_near"])) < 1e-12 * np.max(np.abs(a["forces_near"]))

