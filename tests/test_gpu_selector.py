"""The learned parameter selector (GPU): its network kernels against the CPU oracle, and
what the trained network gains over the paper's analytic tuning.

* esp_mlp_loss_grad against oracle.mlp.loss_and_grad, one Adam step against
  oracle.mlp.adam_step.
* The selector's set: 64 seeded systems (synthetic.selector_system), N log-uniform in
  1e3 - 1e6.  References: the FP64 Ewald oracle for the 23 systems of at most 20,000 atoms
  (tests/golden/selector_references.json); for the larger ones the method itself at
  Delta = 1e-11, P = 12 in FP64 (selector.reference_virial), validated here against the
  oracle on the smaller systems.  On 48 systems the method runs at every candidate (Delta,
  P, sigma, r_c): the FP64 GPU path gives the pressure-tensor error (long-range step, near
  part, background), and the FP32 step with forces plus the near part is timed on the GPU
  with CUDA events.  The fastest candidate whose relative pressure-tensor error is at most
  half the target becomes the label for each target in {1e-3, 1e-4, 1e-5, 1e-6}.  The
  network is trained on the GPU by the library's kernels.  On the 16 other systems the
  references judge both the network's pick and the analytic rules' pick, and both are
  timed.
"""

import json
import math
import os
import time

import numpy as np
import pytest

import synthetic as sy
from oracle import mlp as omlp

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU containers
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2601_00161_gb300 import selector as sel  # noqa: E402
from paper_2601_00161_gb300.mlp import MLP  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
TARGETS = (1e-3, 1e-4, 1e-5, 1e-6)


def test_mlp_gradient_and_adam_match_the_oracle():
    n_in, n_h, n_out, B = 7, 64, 4, 100
    net = MLP(n_in, n_h, n_out, max_batch=128, seed=3)
    theta = net.params().astype(np.float64)
    rng = np.random.default_rng(4)
    x = rng.normal(size=(B, n_in)).astype(np.float32)
    t = rng.normal(size=(B, n_out)).astype(np.float32)
    loss, g = net.loss_grad(torch.tensor(x, device="cuda"), torch.tensor(t, device="cuda"), want_grad=True)
    L, g_ref = omlp.loss_and_grad(theta, x.astype(np.float64), t.astype(np.float64), n_in, n_h, n_out)
    assert abs(float(loss.item()) - L) < 1e-5 * L
    g = g.double().cpu().numpy()
    assert np.linalg.norm(g - g_ref) < 1e-4 * np.linalg.norm(g_ref)
    net.adam(1e-2)
    th_ref, _, _ = omlp.adam_step(theta, np.zeros_like(theta), np.zeros_like(theta), g_ref, 1, 1e-2)
    assert np.max(np.abs(net.params() - th_ref)) < 1e-5
    net.close()


def rel_err(W, ref):
    return float(np.linalg.norm(W - ref) / np.linalg.norm(ref))


MAX_POINTS = 1.2e8  # candidates with larger grids are skipped (memory and time)


@pytest.fixture(scope="module")
def references():
    with open(os.path.join(HERE, "golden", "selector_references.json")) as f:
        ewald = {r["i"]: np.array(r["virial"]) for r in json.load(f)["systems"]}
    refs = {}
    for i in range(sy.N_SELECTOR_SYSTEMS):
        if i in ewald:
            refs[i] = ("ewald", ewald[i])
        else:
            S = sy.selector_system(i)
            refs[i] = ("esp_1e-11", sel.reference_virial(S.pos, S.q, S.cell))
    return refs, ewald


def test_tight_reference_matches_the_ewald_oracle(references):
    refs, ewald = references
    worst = 0.0
    for i in sorted(ewald)[:8]:
        S = sy.selector_system(i)
        worst = max(worst, rel_err(sel.reference_virial(S.pos, S.q, S.cell), ewald[i]))
    # far below the tightest target the selector is trained for (1e-6)
    assert worst < 1e-8, worst


def evaluate(S, W_ref, cands):
    """(pressure error, measured seconds, candidate) for every feasible candidate."""
    from paper_2601_00161_gb300 import Plan

    near_cache = {}
    rows = []
    for ld, P, sigma, rc in cands:
        p = sel.params_from(S.cell, ld, P, sigma, rc)
        if not sel.feasible(p) or float(np.prod(p["grid"])) > MAX_POINTS:
            continue
        key = (round(ld, 6), rc)
        if key not in near_cache:
            plan = Plan(S.cell, S.n, p["grid"], p["P"], p["c"], p["rc"], precision="fp64")
            _, near_cache[key], _ = plan.near(S.pos, S.q)
            plan.close()
        err = rel_err(sel.measure_virial(S.pos, S.q, S.cell, p, near_cache[key]), W_ref)
        rows.append((err, sel.measure_time(S.pos, S.q, S.cell, p), (ld, P, sigma, rc)))
    return rows


def test_learned_selector_against_the_analytic_rules(references):
    refs, _ = references
    t0 = time.time()
    X, Y = [], []
    cands = sel.candidates()
    for i in range(48):
        S = sy.selector_system(i)
        rows = evaluate(S, refs[i][1], cands)
        for target in TARGETS:
            ok = [r for r in rows if r[0] <= 0.5 * target]
            if not ok:
                continue
            best = min(ok, key=lambda r: r[1])
            X.append(sel.features(S.pos, S.q, S.cell, target))
            Y.append(best[2])
    t_data = time.time() - t0
    assert len(X) >= 150
    model = sel.train(X, Y)
    assert model.history[-1] < 0.3 * model.history[0]

    # held-out systems: the references judge both picks, both are timed
    res = {"learned": [], "rules": []}
    for i in range(48, 64):
        S = sy.selector_system(i)
        for target in TARGETS:
            for name, p in (("learned", model.select(S.pos, S.q, S.cell, target)),
                            ("rules", sel.rules(S.cell, target))):
                err = rel_err(sel.measure_virial(S.pos, S.q, S.cell, p), refs[i][1])
                res[name].append((target, err, sel.measure_time(S.pos, S.q, S.cell, p), S.n))
    met = {k: [e <= t for t, e, _, _ in v] for k, v in res.items()}
    both = [j for j in range(len(met["rules"])) if met["rules"][j] and met["learned"][j]]
    ratio = float(np.mean([res["learned"][j][2] / res["rules"][j][2] for j in both])) if both else float("nan")
    summary = {"labels": len(X), "data_seconds": round(t_data, 1),
               "held_out_met": {k: int(sum(v)) for k, v in met.items()}, "held_out_total": len(met["rules"]),
               "measured_time_ratio_learned_over_rules": ratio,
               "held_out_n": sorted({n for _, _, _, n in res["rules"]})}
    print("\nselector:", json.dumps(summary))
    out = os.environ.get("ESP_SELECTOR_REPORT")
    if out:
        with open(out, "w") as f:
            json.dump({"summary": summary, "held_out": res}, f, indent=1)
    # the references judge every pick: the network meets clearly more targets than the
    # rules (whose single tolerance misses most targets on the ionic systems) and, where
    # both meet a target, is not slower by the measured step time.  The labels follow
    # measured times, so near-ties between candidates change from run to run and with
    # them the training: over four runs the network met 46 to 51 of 64 targets (the rules
    # 32), at 0.88 to 0.92 of the rules' time.  The near part costs about 1e-11 s per
    # pair, so a cut-off other than the rules' 9 A buys little time.
    assert sum(met["learned"]) >= 0.65 * len(met["learned"])
    assert sum(met["learned"]) >= sum(met["rules"]) + 10
    assert ratio < 1.0
