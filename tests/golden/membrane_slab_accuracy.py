"""Accuracy of the membrane-slab workload's ESP parameters against a converged reference.

Writes ``membrane_slab_accuracy.json`` beside this file.  Only the FP64 oracle is used.

The workload (210,240 atoms, 120 x 120 x 150 A, grid 128 x 128 x 160, P = 6,
Delta = 1e-5, r_c = 9 A) is evaluated in full: near field by the pair sum of eq. (UN)
(cell list), far field by the gridded ESP (spread, FFT, scaling, inverse FFT, gather),
self and background terms (eqs. (selfen), (Corr)).  The paper's own reference is PPPM
at tolerance 1e-12 (Sec. 5.1); here the reference is the same ESP evaluation at a much
tighter tolerance, on a grid fine enough that the first alias of every in-sphere mode
lies outside the window's band, M_d >= m_max,d / (1 - c / (pi P)).  Two such references
with different (Delta, P, r_c) show how far the reference itself has converged.  The
oracle tests tie ESP to classical Ewald on small systems.

Errors (Sec. 5.1, eq. (ref_pres)): relative L2 norms of the diagonal and off-diagonal
parts of the Coulomb pressure tensor (no kinetic term: there are no momenta here), the
Frobenius relative error, the energy error and the RMS relative force error.

    python tests/golden/membrane_slab_accuracy.py      # about 15 minutes on 3 cores
"""

from __future__ import annotations

import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

CONFIGS = {
    "workload": dict(delta=1e-5, P=6, rc=9.0, grid=(128, 128, 160)),
    "reference_a": dict(delta=1e-11, P=12, rc=12.0, grid=(180, 180, 225)),
    "reference_b": dict(delta=1e-10, P=11, rc=11.0, grid=(180, 180, 225)),
}


def evaluate(name: str):
    import synthetic
    from oracle.esp_grid import esp_grid, self_and_background
    from oracle.esp_split import esp_split
    from oracle.pswf import c_from_tolerance

    cfg = CONFIGS[name]
    S = synthetic.membrane_slab()
    c = c_from_tolerance(cfg["delta"])
    t0 = time.perf_counter()
    near = esp_split(S.pos, S.q, S.cell, c, cfg["rc"], far=False, cell_list=True)
    t1 = time.perf_counter()
    far = esp_grid(S.pos, S.q, S.cell, cfg["grid"], cfg["P"], c, cfg["rc"])
    t2 = time.perf_counter()
    sb = self_and_background(S.q, S.cell, c, cfg["rc"])
    U = near["energy_near"] + far["energy"] + sb["energy_self"] + sb["energy_bg"]
    W = near["virial_near"] + far["virial"] + sb["energy_bg"] * np.eye(3)
    F = near["forces_near"] + far["forces"]
    return name, dict(c=c, U=U, W=W, F=F, V=float(np.linalg.det(S.cell)),
                      seconds_near=t1 - t0, seconds_far=t2 - t1)


def errors(test, ref):
    e = test["W"] - ref["W"]
    iu = np.triu_indices(3, 1)
    diag = float(np.linalg.norm(np.diag(e)) / np.linalg.norm(np.diag(ref["W"])))
    off = float(np.linalg.norm(e[iu]) / np.linalg.norm(ref["W"][iu]))
    frob = float(np.linalg.norm(e) / np.linalg.norm(ref["W"]))
    dU = float(abs(test["U"] - ref["U"]) / abs(ref["U"]))
    dF = float(np.sqrt(np.sum((test["F"] - ref["F"]) ** 2) / np.sum(ref["F"] ** 2)))
    return {"pressure_diag": diag, "pressure_offdiag": off, "pressure_frobenius": frob,
            "energy": dU, "forces_rms": dF}


def main():
    ctx = mp.get_context("spawn")
    with ctx.Pool(len(CONFIGS)) as pool:
        res = dict(pool.map(evaluate, list(CONFIGS)))
    ref = res["reference_a"]
    out = {
        "what": "ESP accuracy of the membrane-slab workload (210,240 atoms) against a tight-"
                "tolerance ESP reference; metrics of Sec. 5.1 eq. (ref_pres) on the Coulomb "
                "pressure tensor (virial / V), energy and RMS relative forces",
        "script": "tests/golden/membrane_slab_accuracy.py (FP64 oracle only)",
        "configs": {k: dict(v, c=res[k]["c"], grid=list(v["grid"])) for k, v in CONFIGS.items()},
        "workload_vs_reference_a": errors(res["workload"], ref),
        "reference_b_vs_reference_a": errors(res["reference_b"], ref),
        "pressure_reference_a": (ref["W"] / ref["V"]).tolist(),
        "pressure_workload": (res["workload"]["W"] / ref["V"]).tolist(),
        "energy": {k: res[k]["U"] for k in res},
        "seconds": {k: [res[k]["seconds_near"], res[k]["seconds_far"]] for k in res},
    }
    with open(os.path.join(HERE, "membrane_slab_accuracy.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps({k: out[k] for k in ("workload_vs_reference_a", "reference_b_vs_reference_a")}, indent=1))


if __name__ == "__main__":
    main()
