"""Classical Ewald references for the parameter selector's small systems (FP64 oracle only).

Writes ``selector_references.json`` beside this file: for each ``synthetic.selector_system(i)``
with at most MAX_ATOMS atoms, its Coulomb energy and virial tensor W = -(dU/dh) h^T (so the
pressure tensor of eq. (instheta) without the kinetic term is W / V), from ``oracle.ewald``
at splitting tolerance 1e-12 (tin-foil boundary, Sec. 3.2).  The selector's GPU test judges
the picks on these systems against these values, and validates there the tight-tolerance
method it uses as the reference of the larger systems (as the paper uses PPPM at 1e-12,
Sec. 5.1).

    python tests/golden/selector_references.py     # a few minutes on 8 cores
"""

from __future__ import annotations

import json
import multiprocessing as mp
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

TOL = 1e-12
MAX_ATOMS = 20000


def reference(i: int):
    import synthetic
    from oracle import lattice
    from oracle.ewald import ewald

    S = synthetic.selector_system(i)
    w = float(np.min(lattice.widths(S.cell)))
    # real-space cut-off: at most half the narrowest width, three cell-list bins when possible
    rcut = min(0.5 * w, max(8.0, w / 3.0))
    E = ewald(S.pos, S.q, S.cell, forces=False, tol=TOL, rcut=rcut, cell_list=True)
    return {"i": i, "n": S.n, "composition": S.meta["composition"], "energy": E["energy"],
            "virial": E["virial"].tolist(), "ewald_rcut": rcut, "ewald_beta": E["params"][0]}


def main():
    import synthetic

    small = [i for i in range(synthetic.N_SELECTOR_SYSTEMS)
             if synthetic.selector_system(i).n <= MAX_ATOMS]
    with mp.get_context("spawn").Pool(min(8, os.cpu_count() or 1)) as pool:
        refs = pool.map(reference, small)
    out = {"what": "Ewald energy and virial of synthetic.selector_system(i), oracle.ewald at "
                   f"splitting tolerance {TOL:g} (tin-foil)",
           "script": "tests/golden/selector_references.py (FP64 oracle only)",
           "systems": refs}
    with open(os.path.join(HERE, "selector_references.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(len(refs), "references")


if __name__ == "__main__":
    main()
