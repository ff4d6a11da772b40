"""FP64 oracle of the regularizers of Table regularizers (refractive-index form) and their
gradients (test infrastructure only).  Added to the data term as in Eq. tikhonov.

Readings (the table prints the expressions without boundary or sign conventions):
* N_o = Lz * Ly * Lx; the TV weight gamma multiplies both the delta and the beta term;
* spatial gradient by forward differences C[i+1] - C[i] along x, y and z, with no term past the
  last index (no wrap-around);
* the subgradient of |u| at u = 0 is 0;
* reweighted l1: W = max(|C|) / (|C| + eps) from a snapshot of the object, treated as a constant.
"""
from __future__ import annotations

import numpy as np


def _diffs(c):
    """Forward differences along z, y, x (shapes shrink by one along their axis)."""
    return [np.diff(c, axis=a) for a in range(3)]


def regularize(delta, beta, alpha_delta=0.0, alpha_beta=0.0, w_delta=None, w_beta=None, gamma_tv=0.0):
    """Returns (R, dR/ddelta, dR/dbeta) for R = l1 (optionally reweighted) + TV."""
    d = np.asarray(delta, np.float64)
    b = np.asarray(beta, np.float64)
    No = d.size
    wd = np.ones_like(d) if w_delta is None else np.asarray(w_delta, np.float64)
    wb = np.ones_like(b) if w_beta is None else np.asarray(w_beta, np.float64)
    R = (alpha_delta * np.sum(wd * np.abs(d)) + alpha_beta * np.sum(wb * np.abs(b))) / No
    gd = alpha_delta * wd * np.sign(d) / No
    gb = alpha_beta * wb * np.sign(b) / No
    if gamma_tv:
        for c, g in ((d, gd), (b, gb)):
            for a, df in enumerate(_diffs(c)):
                R += gamma_tv * np.sum(np.abs(df)) / No
                s = np.sign(df) * gamma_tv / No
                lo = [slice(None)] * 3
                hi = [slice(None)] * 3
                lo[a] = slice(0, -1)
                hi[a] = slice(1, None)
                g[tuple(hi)] += s       # d|C[i+1] - C[i]| / dC[i+1]
                g[tuple(lo)] -= s       # d|C[i+1] - C[i]| / dC[i]
    return float(R), gd, gb


def l1_weights(c, eps):
    """Adaptive weights of the reweighted l1 norm: max(|C|) / (|C| + eps)."""
    a = np.abs(np.asarray(c, np.float64))
    return a.max() / (a + eps)
