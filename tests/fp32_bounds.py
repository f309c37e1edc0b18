"""Forward error bounds for the FP32 sweeps of the mixed-precision path.

In mixed precision C is stored in FP32 and every 2x2 update of a sweep is
done in FP32: the coefficients (c, s of a rotation, -sigma_ij / 2 of a
combination) are FP64 values rounded to FP32, and an update is one product
and one fused multiply-add (rotation) or one fused multiply-add
(combination), followed by the truncation |x| < threshold -> 0 decided on the
FP32 value. The oracle does the same updates in FP64.

These helpers replay the oracle's schedule on the same inputs in FP64 and
carry, for every element, a bound on |FP32 result - FP64 result|:

* rotation  x' = c x + s y:  e' = (1 + 4u)(|c| e_x + |s| e_y) + 4u (|c x| + |s y|)
* combination x' = x - c y:  e' = (1 + 4u)(e_x + |c| e_y) + 3u (|x| + |c y|)
* normalisation x / d (FP32 division by the FP32-rounded d): e' = e / d + 3u |x / d|
* truncation at t: where t - e <= |x'| < t + e the two sides may decide
  differently, so e' = e + t there; where both truncate, e' = 0;

with u = 2^-24. Each rounding of an FP32 operation contributes at most u
times the magnitude it rounds, and the coefficient rounding u times the term
it scales; the factors 3 and 4 cover those sums with the second-order terms
folded into (1 + 4u). The replayed FP64 values are returned too, and the
tests check that they equal the oracle's own result bit for bit, so the
bound is attached to exactly the oracle's schedule.
"""
from __future__ import annotations

import numpy as np

from oracle import sparse

U = 2.0 ** -24


def _truncate(v: np.ndarray, e: np.ndarray, thr: float):
    a = np.abs(v)
    ambiguous = (a >= thr - e) & (a < thr + e)
    out = np.where(a < thr, 0.0, v)
    err = np.where(ambiguous, e + thr, np.where(a < thr, 0.0, e))
    return out, err


def rotations(C: np.ndarray, F_ov: np.ndarray, Fd: np.ndarray, st, sel: np.ndarray, thr: float):
    """Replays oracle B's rotation sweep (same schedule and angles); returns (values, bound)."""
    X = C.copy()
    E = np.zeros_like(C)
    for i, j in sparse.rotation_schedule(st, sel):
        c, s = sparse.rotation_angle(Fd[i], Fd[j], F_ov[i, j - st.n_occ])
        xi, xj = X[:, i].copy(), X[:, j].copy()
        ei, ej = E[:, i].copy(), E[:, j].copy()
        ni = c * xi + s * xj
        nj = -s * xi + c * xj
        bi = (1 + 4 * U) * (abs(c) * ei + abs(s) * ej) + 4 * U * (np.abs(c * xi) + np.abs(s * xj))
        bj = (1 + 4 * U) * (abs(s) * ei + abs(c) * ej) + 4 * U * (np.abs(s * xi) + np.abs(c * xj))
        X[:, i], E[:, i] = _truncate(ni, bi, thr)
        X[:, j], E[:, j] = _truncate(nj, bj, thr)
    return X, E


def combinations(C: np.ndarray, sigma: np.ndarray, st, which: str, tol: float, thr: float):
    """Replays oracle B's orthonormalisation pass on given overlaps; returns (values, bound)."""
    mos = np.arange(st.n_occ) if which == "occ" else np.arange(st.n_mo)
    sig = np.where(sparse.overlap_mask(st, mos), sigma, 0.0)
    d = np.sqrt(np.diag(sig))
    X = C.copy()
    E = np.zeros_like(C)
    sig_n = sig / np.outer(d, d)
    off = np.abs(sig_n - np.diag(np.diag(sig_n)))
    eta = float(off.max()) if off.size else 0.0
    if eta < tol:
        return X, E
    X[:, mos] = C[:, mos] / d[None, :]
    E[:, mos] = 3 * U * np.abs(X[:, mos])
    sel = sparse.overlap_mask(st, mos) & (np.abs(sig_n) >= 1e-3 * eta)
    np.fill_diagonal(sel, False)
    pa, pb = sparse.ortho_schedule(st, which, mos, sel)
    for a, b in zip(pa.tolist(), pb.tolist()):
        c = 0.5 * sig_n[a, b]
        i, j = mos[a], mos[b]
        xi, xj = X[:, i].copy(), X[:, j].copy()
        ei, ej = E[:, i].copy(), E[:, j].copy()
        bi = (1 + 4 * U) * (ei + abs(c) * ej) + 3 * U * (np.abs(xi) + np.abs(c * xj))
        bj = (1 + 4 * U) * (ej + abs(c) * ei) + 3 * U * (np.abs(xj) + np.abs(c * xi))
        X[:, i], E[:, i] = _truncate(xi - c * xj, bi, thr)
        X[:, j], E[:, j] = _truncate(xj - c * xi, bj, thr)
    return X, E
