"""Cell geometry helpers for the oracle (test infrastructure; see ``oracle/__init__``).

Conventions (Sec. 2.2): the cell matrix h has the cell vectors h_1, h_2, h_3 as its
COLUMNS, V = det h, Cartesian r = h s with reduced coordinates s.  Reciprocal vectors
(eq. (vector)): k = 2 pi h^{-T} m, m integer.
"""

from __future__ import annotations

import itertools
import math

import numpy as np


def check_cell(h) -> np.ndarray:
    h = np.asarray(h, dtype=np.float64).reshape(3, 3)
    if not np.all(np.isfinite(h)) or np.linalg.det(h) <= 0.0:
        raise ValueError("cell must be finite with det h > 0")
    return h


def reduced(pos, h) -> np.ndarray:
    """s = h^{-1} r, wrapped into [0, 1) (an exact 1.0 after wrapping becomes 0.0)."""
    s = np.asarray(pos, dtype=np.float64) @ np.linalg.inv(h).T
    s = s - np.floor(s)
    s[s >= 1.0] = 0.0
    return s


def widths(h) -> np.ndarray:
    """Perpendicular widths of the cell: V / |h_e x h_f| for each direction d."""
    V = np.linalg.det(h)
    a, b, c = h[:, 0], h[:, 1], h[:, 2]
    return np.array([V / np.linalg.norm(np.cross(b, c)),
                     V / np.linalg.norm(np.cross(c, a)),
                     V / np.linalg.norm(np.cross(a, b))])


def kvectors(h, kmax: float, half: bool = True):
    """All m != 0 with |k| <= kmax, k = 2 pi h^{-T} m.

    With ``half`` only one of each +/- pair is returned together with weight 2 (the
    summands used here are even in k), else every mode with weight 1.
    Returns (m [n,3] int, k [n,3], weight [n]).
    """
    B = 2.0 * math.pi * np.linalg.inv(h).T  # columns b_1, b_2, b_3
    # |m_d| <= |h_d| kmax / (2 pi) since m_d = h_d . k / (2 pi)
    mmax = [int(math.floor(np.linalg.norm(h[:, d]) * kmax / (2.0 * math.pi))) + 1 for d in range(3)]
    r = [np.arange(-mm, mm + 1) for mm in mmax]
    m = np.stack(np.meshgrid(*r, indexing="ij"), axis=-1).reshape(-1, 3)
    k = m @ B.T
    k2 = np.einsum("ij,ij->i", k, k)
    keep = (k2 <= kmax * kmax) & np.any(m != 0, axis=1)
    if half:
        pos_half = (m[:, 2] > 0) | ((m[:, 2] == 0) & (m[:, 1] > 0)) | ((m[:, 2] == 0) & (m[:, 1] == 0) & (m[:, 0] > 0))
        keep &= pos_half
        w = 2.0
    else:
        w = 1.0
    m, k = m[keep], k[keep]
    return m, k, np.full(len(m), w)


def structure_factor(k, pos, q, chunk: int = 2048):
    """rho(k) = sum_i q_i exp(i k . r_i) (Sec. 3.2), for every row of k."""
    out = np.empty(len(k), dtype=np.complex128)
    for a in range(0, len(k), chunk):
        ph = pos @ k[a:a + chunk].T  # [N, nk]
        out[a:a + chunk] = q @ np.exp(1j * ph)
    return out


def pair_images(pos, h, rcut: float, rows=None, chunk: int = 64):
    """Yield (i, j, rvec, r) for all pairs/images with 0 < |r_i - r_j + h n| <= rcut.

    rvec = r_i - r_j + h n.  Pairs i == j are kept for n != 0 (self images).  ``rows``
    restricts i to a subset (every j is still visited).
    """
    pos = np.asarray(pos, dtype=np.float64)
    s = pos @ np.linalg.inv(h).T
    wd = widths(h)
    nmax = [int(math.ceil(rcut / wd[d] + 0.5)) for d in range(3)]
    images = np.array(list(itertools.product(*[range(-n, n + 1) for n in nmax])), dtype=np.float64)
    rows = np.arange(len(pos)) if rows is None else np.asarray(rows)
    for a in range(0, len(rows), chunk):
        ii = rows[a:a + chunk]
        d = s[ii, None, :] - s[None, :, :]
        d -= np.round(d)  # nearest fractional image; the image loop covers the rest
        for n in images:
            rv = (d + n) @ h.T
            r2 = np.einsum("ijk,ijk->ij", rv, rv)
            mask = (r2 <= rcut * rcut) & (r2 > 0.0)
            bi, bj = np.nonzero(mask)
            if len(bi):
                yield ii[bi], bj, rv[bi, bj], np.sqrt(r2[bi, bj])


def pair_cells(pos, h, rcut: float, rows=None):
    """The pairs of ``pair_images`` (each ordered (i, j, image) once, same rvec) found
    through a cell list, for systems too large for the all-pairs loop.

    The cell is cut into n_d = floor(width_d / rcut) slabs along each reduced axis, so a
    slab is at least rcut thick and two atoms closer than rcut lie in neighbouring bins
    (index difference -1, 0 or +1 per axis, with the periodic image given by the wrap of
    the index).  With n_d >= 3 the 27 neighbour bins of a bin are distinct, so no pair is
    visited twice; smaller cells fall back to ``pair_images``.
    """
    h = check_cell(h)
    wd = widths(h)
    nc = np.array([int(wd[d] // rcut) for d in range(3)])
    if np.any(nc < 3):
        yield from pair_images(pos, h, rcut, rows=rows)
        return
    s = reduced(pos, h)
    N = len(s)
    b = np.minimum((s * nc).astype(np.int64), nc - 1)
    bid = (b[:, 0] * nc[1] + b[:, 1]) * nc[2] + b[:, 2]
    order = np.argsort(bid, kind="stable")
    start = np.concatenate([[0], np.cumsum(np.bincount(bid, minlength=int(np.prod(nc))))])
    want = np.ones(N, dtype=bool) if rows is None else np.isin(np.arange(N), np.asarray(rows))
    offsets = np.array(list(itertools.product((-1, 0, 1), repeat=3)))
    r2max = rcut * rcut
    for b0 in range(nc[0]):
        for b1 in range(nc[1]):
            for b2 in range(nc[2]):
                home = (b0 * nc[1] + b1) * nc[2] + b2
                ii = order[start[home]:start[home + 1]]
                ii = ii[want[ii]]
                if len(ii) == 0:
                    continue
                nb = np.array([b0, b1, b2]) + offsets  # unwrapped neighbour bins
                shift = np.floor_divide(nb, nc)         # image of the neighbour bin
                nbw = nb - shift * nc
                nid = (nbw[:, 0] * nc[1] + nbw[:, 1]) * nc[2] + nbw[:, 2]
                jj = np.concatenate([order[start[x]:start[x + 1]] for x in nid])
                sh = np.concatenate([np.repeat(shift[o:o + 1], start[nid[o] + 1] - start[nid[o]], axis=0)
                                     for o in range(27)]).astype(np.float64)
                # rvec = r_i - (r_j + h shift) = h (s_i - s_j - shift)
                d = s[ii, None, :] - (s[None, jj, :] + sh[None, :, :])
                rv = d @ h.T
                r2 = np.einsum("ijk,ijk->ij", rv, rv)
                mask = (r2 <= r2max) & (r2 > 0.0)
                bi, bj = np.nonzero(mask)
                if len(bi):
                    yield ii[bi], jj[bj], rv[bi, bj], np.sqrt(r2[bi, bj])
