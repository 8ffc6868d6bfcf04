"""The stored Ewald references of the selector's systems (no GPU).

``tests/golden/selector_references.json`` is written by
``tests/golden/selector_references.py`` from the FP64 Ewald oracle, for the systems of at
most 20,000 atoms.  Each record must
belong to ``synthetic.selector_system(i)`` (same atom count and composition), and obey
Coulomb homogeneity, tr W = U (eq. (deth)), and the symmetry of the virial.
"""

import json
import os

import numpy as np

import synthetic as sy

HERE = os.path.dirname(os.path.abspath(__file__))


def test_selector_references_are_consistent():
    with open(os.path.join(HERE, "golden", "selector_references.json")) as f:
        refs = json.load(f)["systems"]
    # every system of at most 20,000 atoms has its oracle reference
    small = [i for i in range(sy.N_SELECTOR_SYSTEMS) if sy.selector_system(i).n <= 20000]
    assert [r["i"] for r in refs] == small and len(small) >= 20
    for r in refs:
        S = sy.selector_system(r["i"])
        assert r["n"] == S.n and r["composition"] == S.meta["composition"]
        W = np.array(r["virial"])
        assert np.max(np.abs(W - W.T)) < 1e-9 * np.max(np.abs(W))
        assert abs(np.trace(W) - r["energy"]) < 1e-8 * np.sum(np.abs(W))
