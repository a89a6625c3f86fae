"""Exact dense sums for selected output rows (grids too large for the dense matrix).

For output node n and component l, row (l, n) of A = I - G X is
    y_(l,n) = u_(l,n) - sum_m sum_q G_lq(x_n - x_m) chi(x_m) u_(q,m)
(Eqs. (4.3)-(4.5)), an O(N) sum per row.  The regularised product A_R A u needs the
whole intermediate vector A u, so these rows are used for the plain product and
for A_R applied to a given intermediate.
"""
from __future__ import annotations

import math

import numpy as np

from .dense import node_positions
from .green import green_tensor


def rows_apply(chi: np.ndarray, u: np.ndarray, h: float, rows, k: float = 2 * math.pi):
    """Values of (I - G X(chi)) u at the given flat row indices (0 <= row < 2N)."""
    n2, n1 = chi.shape
    N = n1 * n2
    x1, x2 = node_positions(n1, n2, h)
    w = (chi.reshape(-1)[None, :] * u.reshape(2, N))
    out = np.empty(len(rows), dtype=np.complex128)
    for i, row in enumerate(rows):
        l, n = divmod(int(row), N)
        G11, G22, G12 = green_tensor(x1[n] - x1, x2[n] - x2, k, h)
        if l == 0:
            s = np.sum(G11 * w[0]) + np.sum(G12 * w[1])
        else:
            s = np.sum(G12 * w[0]) + np.sum(G22 * w[1])
        out[i] = u.reshape(-1)[row] - s
    return out
