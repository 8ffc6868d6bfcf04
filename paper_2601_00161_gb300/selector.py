"""Choice of ESP parameters for a system and an accuracy target.

Two selectors return (Delta, c, P, r_c, grid):

* ``rules`` - the paper's analytic tuning (Sec. 5.1): the split and the spreading window
  share one tolerance, psi_0(1)/psi_0(0) = Delta = target; P = ceil(-log10 Delta) + 1;
  r_c = 9 A (0.9 nm, the paper's setting throughout); the grid resolves the Fourier
  cut-off |k| <= c / r_c (M_d > |h_d| c / (pi r_c)) with the upsampling that keeps the
  first alias of every kept mode outside the window's band, M_d >= m_max / (1 - c/(pi P))
  (from the window transform w^(m) = omega lambda_0 psi_0(2 pi m omega / c)).
* ``Selector`` - a 3-layer perceptron (include/esp_mlp.h, trained by the library's own
  kernels) that maps features of the system and the target to (log10 Delta, P, sigma,
  r_c), sigma the grid size over the Nyquist bound; trained on the cheapest measured
  choices that met each target (tests/test_gpu_selector.py).  Infeasible predictions fall
  back to the rules.

``measure_time`` times one FP32 long-range step with forces plus the near part on the GPU
(CUDA events); the selector's labels are the cheapest choices by that measured time.
``cost`` is a model of the same time (calibrated on the 210,240-atom membrane slab's
kernel times), kept for a quick estimate without a GPU.
``reference_virial`` is the method itself at a far tighter tolerance (Delta = 1e-11, P = 12,
FP64), the reference for systems too large for the Ewald oracle; it is validated against
the oracle on the smaller ones, as the paper validates against PPPM at 1e-12 (Sec. 5.1).
"""

from __future__ import annotations

import math

import numpy as np

from . import esp_c_from_tolerance

FEATURES = ("log10_n", "log10_density", "log_aspect_21", "log_aspect_31", "tilt", "log10_qrms",
            "log10_target")
OUTPUTS = ("log10_delta", "P", "sigma", "rc")

# cost model coefficients (seconds), GB300, FP32 path
COST_ATOM = 1.6e-10         # binning per atom
COST_ATOM_P3 = 1.83e-12     # spread + gather per atom and stencil point
COST_POINT_LOG = 1.18e-12   # forward + inverse FFT and scaling per grid point and log2(Mtot)
COST_PAIR = 9.8e-12         # near part per ordered pair within r_c (half-shell kernel)


def fft_size(n: int) -> int:
    """Smallest even m >= n whose prime factors are 2, 3, 5 and 7."""
    m = max(2, int(n))
    while True:
        if m % 2 == 0:
            r = m
            for p in (2, 3, 5, 7):
                while r % p == 0:
                    r //= p
            if r == 1:
                return m
        m += 1


def nyquist(cell, c: float, rc: float) -> np.ndarray:
    """|h_d| c / (pi r_c): every kept mode is below the Nyquist index of a grid larger than it."""
    lens = np.linalg.norm(np.asarray(cell, dtype=np.float64), axis=0)
    return lens * c / (math.pi * rc)


def grid_for(cell, c: float, rc: float, sigma: float, P: int) -> tuple:
    nq = nyquist(cell, c, rc)
    return tuple(max(fft_size(math.floor(max(sigma, 1.0) * x) + 1), P + 2) for x in nq)


def features(pos, q, cell, target: float) -> np.ndarray:
    h = np.asarray(cell, dtype=np.float64)
    n = len(q)
    V = float(np.linalg.det(h))
    L = np.diag(h)
    tilt = float(np.max(np.abs(np.triu(h, 1))) / np.min(L))
    qrms = float(np.sqrt(np.mean(np.asarray(q, dtype=np.float64) ** 2))) if n else 1.0
    return np.array([math.log10(max(n, 1)), math.log10(max(n, 1) / V), math.log(L[1] / L[0]),
                     math.log(L[2] / L[0]), tilt, math.log10(max(qrms, 1e-12)),
                     math.log10(target)])


def params_from(cell, log10_delta: float, P: int, sigma: float, rc: float) -> dict:
    delta = 10.0 ** log10_delta
    c = esp_c_from_tolerance(delta)
    P = int(min(12, max(3, P)))
    return {"delta": delta, "c": c, "P": P, "rc": float(rc), "sigma": float(sigma),
            "grid": grid_for(cell, c, rc, sigma, P)}


def rules(cell, target: float, rc: float = 9.0) -> dict:
    """The paper's analytic tuning (Sec. 5.1), with the aliasing upsampling above."""
    delta = float(target)
    P = int(min(12, max(3, math.ceil(-math.log10(delta)) + 1)))
    c = esp_c_from_tolerance(delta)
    band = 1.0 - c / (math.pi * P)
    sigma = 1.0 / (2.0 * band) if band > 0.2 else 2.5  # m_max / band over 2 m_max
    sigma = max(sigma, 1.0)
    return params_from(cell, math.log10(delta), P, sigma, rc)


def cost(n: int, cell, grid, P: int, rc: float) -> float:
    """Modelled seconds of one FP32 long-range step plus the near part (GB300)."""
    V = float(np.linalg.det(np.asarray(cell, dtype=np.float64)))
    mtot = float(np.prod(grid))
    pairs = n * (n / V) * (4.0 / 3.0) * math.pi * rc ** 3
    return (COST_ATOM * n + COST_ATOM_P3 * n * P ** 3 + COST_POINT_LOG * mtot * math.log2(mtot)
            + COST_PAIR * pairs)


def feasible(p: dict) -> bool:
    """Parameters the library accepts: 3 <= P <= 12, the window fit and grid constraints."""
    c, P = p["c"], p["P"]
    return 3 <= P <= 12 and c < math.pi * P * 0.95 and min(p["grid"]) > P + 1


class Selector:
    """The learned selector: a trained esp_mlp network and the normalisation of its data."""

    def __init__(self, net, x_mean, x_std, y_mean, y_std):
        self.net = net
        self.x_mean, self.x_std = np.asarray(x_mean), np.asarray(x_std)
        self.y_mean, self.y_std = np.asarray(y_mean), np.asarray(y_std)

    def predict_raw(self, X: np.ndarray) -> np.ndarray:
        import torch

        xn = (np.asarray(X, dtype=np.float64) - self.x_mean) / self.x_std
        y = self.net.forward(torch.tensor(xn, dtype=torch.float32, device="cuda"))
        return y.double().cpu().numpy() * self.y_std + self.y_mean

    def select(self, pos, q, cell, target: float) -> dict:
        y = self.predict_raw(features(pos, q, cell, target)[None, :])[0]
        p = params_from(cell, float(y[0]), int(round(y[1])), float(y[2]), float(y[3]))
        if not feasible(p) or not (5.0 <= p["rc"] <= 15.0):
            p = rules(cell, target)
            p["fallback"] = True
        return p


def candidates():
    """The parameter grid the selector is trained on: (log10 Delta, P, sigma, r_c)."""
    out = []
    for ld in np.arange(-2.5, -7.01, -0.5):
        D = math.ceil(-ld - 1e-9)
        for sigma in (1.3, 1.8):
            for rc in (5.5, 8.0):
                out.append((float(ld), int(D + 1), sigma, rc))
    return out


def measure_time(pos, q, cell, p: dict, steps: int = 5) -> float:
    """Median seconds of one FP32 long-range step with forces plus the near part (forces
    added), CUDA events on a stream of its own after two warm-up steps."""
    import torch

    from . import ESP_ACCUM_LEN, Plan, esp_near, esp_step

    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        plan = Plan(cell, len(q), p["grid"], p["P"], p["c"], p["rc"], precision="fp32",
                    stream=st.cuda_stream)
        try:
            x = torch.tensor(pos, dtype=torch.float32, device="cuda")
            qq = torch.tensor(q, dtype=torch.float32, device="cuda")
            F = torch.empty((len(q), 3), dtype=torch.float32, device="cuda")
            acc = torch.zeros(ESP_ACCUM_LEN, dtype=torch.float64, device="cuda")
            near = torch.empty(7, dtype=torch.float64, device="cuda")
            times = []
            for k in range(steps + 2):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(st)
                esp_step(plan.handle, x, qq, F, acc)
                esp_near(plan.handle, x, qq, F, 1, near)
                e1.record(st)
                e1.synchronize()
                if k >= 2:
                    times.append(e0.elapsed_time(e1) * 1e-3)
            return float(np.median(times))
        finally:
            plan.close()


def reference_virial(pos, q, cell) -> np.ndarray:
    """Total Coulomb virial of the method at Delta = 1e-11, P = 12, r_c = 10 A, FP64 (grid
    with the rules' aliasing margin): far below every target of the selector."""
    c = esp_c_from_tolerance(1e-11)
    P, rc = 12, 10.0
    band = 1.0 - c / (math.pi * P)
    p = {"delta": 1e-11, "c": c, "P": P, "rc": rc,
         "grid": grid_for(cell, c, rc, max(1.0, 1.0 / (2.0 * band)) * 1.05, P)}
    return measure_virial(pos, q, cell, p)


def measure_virial(pos, q, cell, p: dict, near_virial=None) -> np.ndarray:
    """Total Coulomb virial W_F + U_bg I + W_N of the method at parameters p (FP64 GPU path)."""
    from . import Plan

    plan = Plan(cell, len(q), p["grid"], p["P"], p["c"], p["rc"], precision="fp64")
    try:
        res = plan.energy_pressure(pos, q)
        W = res["virial_recip"] + res["energy_bg"] * np.eye(3)
        if near_virial is None:
            _, near_virial, _ = plan.near(pos, q)
        return W + near_virial
    finally:
        plan.close()


def train(X, Y, hidden=64, steps=4000, lr=3e-3, seed=0) -> "Selector":
    """Fit the perceptron to (features, parameters) with the library's kernels (full batch)."""
    import torch

    from .mlp import MLP

    X, Y = np.asarray(X, dtype=np.float64), np.asarray(Y, dtype=np.float64)
    xm, xs = X.mean(axis=0), X.std(axis=0) + 1e-6
    ym, ys = Y.mean(axis=0), Y.std(axis=0) + 1e-6
    xt = torch.tensor((X - xm) / xs, dtype=torch.float32, device="cuda")
    yt = torch.tensor((Y - ym) / ys, dtype=torch.float32, device="cuda")
    net = MLP(X.shape[1], hidden, Y.shape[1], max_batch=len(X), seed=seed)
    history = []
    for s in range(steps):
        loss, _ = net.loss_grad(xt, yt)
        net.adam(lr)
        if s % 100 == 0 or s == steps - 1:
            history.append(float(loss.item()))
    sel = Selector(net, xm, xs, ym, ys)
    sel.history = history
    return sel
