"""O-GRID: the gridded ESP long-range step, evaluated plainly (test infrastructure).

Part of the FP64 CPU oracle; only tests, the smoke check and the benchmark's CPU legs
may import it.  It computes the same discrete quantity as the CUDA path, in the paper's
order (Sec. 4.1, Algorithm 1, and Appendix C, analytical differentiation), with no
blocking, sorting or fusion:

1. reduced coordinates s = h^{-1} r wrapped into [0, 1) (Sec. 2.2);
2. spreading (eq. (gridding)) with the separable PSWF window of Sec. 4.2 taken in
   FRACTIONAL coordinates of the cell (reading: triclinic window):
       rho_s(g) = sum_j q_j prod_d w_d(g_d / M_d - s_jd),
       w_d(u) = psi_0^c(u / omega_d) for |u| <= omega_d,  omega_d = P / (2 M_d),
   on the P nearest grid points of Sec. 4.3 (P even: base floor(M s) - P/2 + 1; P odd:
   base floor(M s + 1/2) - (P-1)/2), indices taken mod M_d;
3. one forward FFT (library):  X(m) = sum_g rho_s(g) exp(-2 pi i m.g / M);
4. diagonal scaling and Fourier collection (eqs. (diag), (PFfinal)): for m != 0 with
   |k| <= c / r_c,  k = 2 pi h^{-T} m,
       a(m) = |X(m)|^2 / (2 V Mtot^2 what_1^2 what_2^2 what_3^2),
       what_d(m) = omega_d lambda_0 psi_0(2 pi m omega_d / c)   (Sec. 4.2),
       U_F = sum a Fhat,   W_F = sum a [Fhat I + (A x psi_0'(x)/|k|^4 - 2 Fhat/|k|^2) k k];
5. forces by analytical differentiation (eqs. (UFAnal), (AD)):
       phi(g) = sum_m G(m) X(m) exp(+2 pi i m.g / M),  G = Fhat / prod_d what_d^2,
       dU/ds_i = -(q_i / (V Mtot^2)) sum_g phi(g) grad_u W(g/M - s_i),
       F_i = -h^{-T} dU/ds_i.
   Eq. (AD) prints a factor 1/2 in front; U_F is quadratic in the charges and the
   derivative of eq. (UFAnal) has no 1/2 (reading: no 1/2; pinned by finite differences).
"""

from __future__ import annotations

import math

import numpy as np

from . import lattice
from .esp_split import split_constants


def stencil(x, P):
    """Base grid index and offsets (g - x) for the P nearest points, per Sec. 4.3."""
    if P % 2 == 0:
        base = np.floor(x) - (P // 2) + 1
    else:
        base = np.floor(x + 0.5) - (P - 1) // 2
    g = base[..., None] + np.arange(P)  # [..., P]
    return g.astype(np.int64), g - x[..., None]


def window_1d(p, x, P, M, deriv=False):
    """Window weights w_d (and d w_d / du) on the stencil of grid coordinate x = M s."""
    g, off = stencil(x, P)
    u = off / (0.5 * P)  # (g/M - s) / omega_d
    assert np.all(np.abs(u) <= 1.0 + 1e-12)
    w = p.psi(u)
    if not deriv:
        return g, w
    dw = p.dpsi(u) * (2.0 * M / P)
    return g, w, dw


def spread(pos, q, h, M, P, c, chunk=4096):
    """Step 1: the real grid rho_s, shape M (z fastest)."""
    p = split_constants(c, 1.0)[0]
    M = tuple(int(v) for v in M)
    s = lattice.reduced(pos, h)
    grid = np.zeros(int(np.prod(M)))
    for a in range(0, len(q), chunk):
        ws = []
        gs = []
        for d in range(3):
            g, w = window_1d(p, M[d] * s[a:a + chunk, d], P, M[d])
            gs.append(np.mod(g, M[d]))
            ws.append(w)
        idx = (gs[0][:, :, None, None] * M[1] + gs[1][:, None, :, None]) * M[2] + gs[2][:, None, None, :]
        val = q[a:a + chunk, None, None, None] * ws[0][:, :, None, None] * ws[1][:, None, :, None] * ws[2][:, None, None, :]
        grid += np.bincount(idx.ravel(), weights=val.ravel(), minlength=grid.size)
    return grid.reshape(M)


def modes(h, M, P, c, rc):
    """Per half-spectrum mode: weights, Fhat, derivative term, k, in-sphere mask, 1/what^2."""
    p, A, _ = split_constants(c, rc)
    M = tuple(int(v) for v in M)
    m1 = np.fft.fftfreq(M[0], 1.0 / M[0])
    m2 = np.fft.fftfreq(M[1], 1.0 / M[1])
    m3 = np.arange(M[2] // 2 + 1, dtype=np.float64)
    mm = np.stack(np.meshgrid(m1, m2, m3, indexing="ij"), axis=-1)
    k = 2.0 * math.pi * mm @ np.linalg.inv(h)  # k = 2 pi h^{-T} m  (row form)
    k2 = np.einsum("...i,...i->...", k, k)
    K = c / rc
    inside = (k2 <= K * K) & np.any(mm != 0, axis=-1)
    if np.any(inside):
        for d, Md in enumerate(M):
            if np.max(np.abs(mm[..., d][inside])) >= Md / 2.0:
                raise ValueError("grid too coarse: a mode with |k| <= c/r_c reaches the Nyquist index")
    # half-spectrum multiplicity of each stored mode
    wt = np.where((mm[..., 2] == 0) | ((M[2] % 2 == 0) & (mm[..., 2] == M[2] // 2)), 1.0, 2.0)
    inv_w2 = np.ones(mm.shape[:-1])
    for d, Md in enumerate(M):
        om = P / (2.0 * Md)
        what = om * p.lam0 * p.psi(2.0 * math.pi * mm[..., d] * om / c)
        inv_w2 = inv_w2 / (what * what)
    Fhat = np.zeros(k2.shape)
    dterm = np.zeros(k2.shape)
    ki = np.sqrt(k2[inside])
    x = ki * rc / c
    Fhat[inside] = A * p.psi(x) / k2[inside]
    dterm[inside] = A * x * p.dpsi(x) / (k2[inside] ** 2)
    return dict(wt=wt, k=k, k2=k2, inside=inside, inv_w2=inv_w2, Fhat=Fhat, dterm=dterm)


def esp_grid(pos, q, h, M, P, c, rc, forces=True, force_rows=None, return_fields=False):
    h = lattice.check_cell(h)
    pos = np.asarray(pos, dtype=np.float64)
    q = np.asarray(q, dtype=np.float64)
    M = tuple(int(v) for v in M)
    V = float(np.linalg.det(h))
    Mtot = float(np.prod(M))
    if min(M) <= P:
        raise ValueError("stencil wider than the grid")
    rho = spread(pos, q, h, M, P, c)
    X = np.fft.rfftn(rho)  # unnormalised forward transform
    md = modes(h, M, P, c, rc)
    a = np.where(md["inside"], md["wt"] * np.abs(X) ** 2 * md["inv_w2"], 0.0) / (2.0 * V * Mtot * Mtot)
    U_F = float(np.sum(a * md["Fhat"]))
    k = md["k"]
    coef = a * (md["dterm"] - np.where(md["inside"], 2.0 * md["Fhat"] / np.where(md["inside"], md["k2"], 1.0), 0.0))
    W_F = U_F * np.eye(3) + np.einsum("p,pa,pb->ab", coef.ravel(), k.reshape(-1, 3), k.reshape(-1, 3))
    out = dict(energy=U_F, virial=W_F, pressure=W_F / V)
    if return_fields:
        out["rho"] = rho
        out["X"] = X
    if forces:
        G = np.where(md["inside"], md["Fhat"] * md["inv_w2"], 0.0)
        phi = np.fft.irfftn(G * X, s=M, axes=(0, 1, 2)) * Mtot  # unnormalised inverse transform
        if return_fields:
            out["phi"] = phi
        out["forces"] = gather(pos, q, h, M, P, c, phi, rows=force_rows)
    return out


def gather(pos, q, h, M, P, c, phi, rows=None, chunk=2048):
    """Step 5: F_i = -h^{-T} dU/ds_i with dU/ds_i = -(q_i/(V Mtot^2)) sum_g phi grad W."""
    p = split_constants(c, 1.0)[0]
    V = float(np.linalg.det(h))
    Mtot = float(np.prod(M))
    s = lattice.reduced(pos, h)
    rows = np.arange(len(q)) if rows is None else np.asarray(rows)
    hinvT = np.linalg.inv(h).T
    F = np.zeros((len(rows), 3))
    flat = phi.ravel()
    for a in range(0, len(rows), chunk):
        ii = rows[a:a + chunk]
        g, w, dw = [], [], []
        for d in range(3):
            gd, wd, dwd = window_1d(p, M[d] * s[ii, d], P, M[d], deriv=True)
            g.append(np.mod(gd, M[d]))
            w.append(wd)
            dw.append(dwd)
        idx = (g[0][:, :, None, None] * M[1] + g[1][:, None, :, None]) * M[2] + g[2][:, None, None, :]
        ph = flat[idx]  # [n, P, P, P]
        gx = np.einsum("nijk,ni,nj,nk->n", ph, dw[0], w[1], w[2])
        gy = np.einsum("nijk,ni,nj,nk->n", ph, w[0], dw[1], w[2])
        gz = np.einsum("nijk,ni,nj,nk->n", ph, w[0], w[1], dw[2])
        dUds = -(q[ii] / (V * Mtot * Mtot))[:, None] * np.stack([gx, gy, gz], axis=1)
        F[a:a + chunk] = -dUds @ hinvT.T
    return F


def self_and_background(q, h, c, rc):
    """Host scalars: U_self (eq. (selfen)) and the background terms (eq. (Corr))."""
    p, A, X = split_constants(c, rc)
    q = np.asarray(q, dtype=np.float64)
    V = float(np.linalg.det(np.asarray(h, dtype=np.float64).reshape(3, 3)))
    U_self = -p.psi_at_0 / (2.0 * p.C0 * rc) * float(np.sum(q * q))
    Q = float(np.sum(q))
    U_bg = -2.0 * math.pi * Q * Q / V * X
    return dict(energy_self=U_self, energy_bg=U_bg, pressure_bg=U_bg / V)


def interpolate(pos, h, M, P, c, field, rows=None, chunk=2048):
    """sum_g field(g) w(g/M - s_i): a field on the grid read at the atoms with the window."""
    p = split_constants(c, 1.0)[0]
    s = lattice.reduced(pos, h)
    rows = np.arange(len(pos)) if rows is None else np.asarray(rows)
    out = np.zeros(len(rows))
    flat = field.ravel()
    for a in range(0, len(rows), chunk):
        ii = rows[a:a + chunk]
        g, w = [], []
        for d in range(3):
            gd, wd = window_1d(p, M[d] * s[ii, d], P, M[d])
            g.append(np.mod(gd, M[d]))
            w.append(wd)
        idx = (g[0][:, :, None, None] * M[1] + g[1][:, None, :, None]) * M[2] + g[2][:, None, None, :]
        out[a:a + chunk] = np.einsum("nijk,ni,nj,nk->n", flat[idx], w[0], w[1], w[2])
    return out


def esp_grid_fields(pos, q, h, M, P, c, rc, kind):
    """Per-atom quantities from fields on the grid (Sec. 4.4 and Appendix C).

    kind "ik":     forces by ik-differentiation, F_i = -(q_i / (V Mtot^2)) sum_g
                   E_d(g) w(g/M - s_i), E_d the inverse transform of i k_d G X (eq.
                   (rhodiagforce)); [N, 3].
    kind "virial": per-atom virial W^i_ab = (q_i / (2 V Mtot^2)) sum_g Pi_ab(g) w, Pi_ab the
                   inverse transform of K_ab X / w^2 with K the pressure kernel of eq.
                   (PFfinal) times V (eqs. (rhodiag), (PinsFind)); [N, 6] as xx yy zz xy xz yz.
    kind "energy": per-atom energy U^i = (q_i / (2 V Mtot^2)) sum_g phi(g) w, phi the inverse
                   transform of G X; [N].
    """
    h = lattice.check_cell(h)
    pos = np.asarray(pos, dtype=np.float64)
    q = np.asarray(q, dtype=np.float64)
    M = tuple(int(v) for v in M)
    V = float(np.linalg.det(h))
    Mtot = float(np.prod(M))
    X = np.fft.rfftn(spread(pos, q, h, M, P, c))
    md = modes(h, M, P, c, rc)
    ins = md["inside"]
    G = np.where(ins, md["Fhat"] * md["inv_w2"], 0.0)
    k = md["k"]

    def back(spec):
        return np.fft.irfftn(spec, s=M, axes=(0, 1, 2)) * Mtot

    if kind == "ik":
        out = np.empty((len(q), 3))
        for d in range(3):
            out[:, d] = -q / (V * Mtot * Mtot) * interpolate(pos, h, M, P, c, back(1j * k[..., d] * G * X))
        return out
    if kind == "energy":
        return q / (2.0 * V * Mtot * Mtot) * interpolate(pos, h, M, P, c, back(G * X))
    if kind == "virial":
        k2 = np.where(ins, md["k2"], 1.0)
        coef = np.where(ins, md["dterm"] - 2.0 * md["Fhat"] / k2, 0.0) * md["inv_w2"]
        Fw = np.where(ins, md["Fhat"] * md["inv_w2"], 0.0)
        out = np.empty((len(q), 6))
        for n, (a, b) in enumerate(((0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2))):
            K = coef * k[..., a] * k[..., b] + (Fw if a == b else 0.0)
            out[:, n] = q / (2.0 * V * Mtot * Mtot) * interpolate(pos, h, M, P, c, back(K * X))
        return out
    raise ValueError(kind)
