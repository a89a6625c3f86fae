"""Dense 2N x 2N operators of the discretised TE problem (paper Sections 3-5).

Unknown ordering: u = [E1(x_1..x_N), E2(x_1..x_N)], node index m = i1 + n1 * i2
(x1 fastest), which is the (2, n2, n1) layout of the CUDA library flattened.

  A   = I - G X(chi),   chi  = eps_r - 1            (Eq. (2.11), Section 5: A = I - G X)
  A_R = I - G X(chi'),  chi' = 1/eps_r - 1          (Eq. (3.18): regulariser = same
                                                     operator with the contrast swapped)
"""
from __future__ import annotations

import math

import numpy as np

from .green import green_tensor


def centres(n: int, h: float) -> np.ndarray:
    return (np.arange(n, dtype=np.float64) + 0.5) * h - 0.5 * n * h


def node_positions(n1: int, n2: int, h: float):
    """(x1, x2) of every node, node m = i1 + n1 i2."""
    x1 = np.tile(centres(n1, h), n2)
    x2 = np.repeat(centres(n2, h), n1)
    return x1, x2


def dense_G(n1: int, n2: int, h: float, k: float) -> np.ndarray:
    """The 2N x 2N matrix G with [G]_{(l,n),(q,m)} = G_lq(x_n - x_m) (Eqs. (4.3)-(4.5))."""
    x1, x2 = node_positions(n1, n2, h)
    d1 = x1[:, None] - x1[None, :]
    d2 = x2[:, None] - x2[None, :]
    G11, G22, G12 = green_tensor(d1, d2, k, h)
    N = n1 * n2
    G = np.empty((2 * N, 2 * N), dtype=np.complex128)
    G[:N, :N] = G11
    G[:N, N:] = G12
    G[N:, :N] = G12
    G[N:, N:] = G22
    return G


def contrast(eps_r: np.ndarray) -> np.ndarray:
    """chi = eps_r - 1 (Eq. (2.11) with eps_b = 1)."""
    return np.asarray(eps_r, dtype=np.complex128) - 1.0


def reg_contrast(eps_r: np.ndarray) -> np.ndarray:
    """chi' = eps_b/eps - 1 = 1/eps_r - 1 (the regulariser's contrast, after Eq. (3.18))."""
    return 1.0 / np.asarray(eps_r, dtype=np.complex128) - 1.0


def dense_A_from_G(G: np.ndarray, chi: np.ndarray) -> np.ndarray:
    """A = I - G X for a contrast map chi of shape (n2, n1)."""
    c = np.asarray(chi, dtype=np.complex128).reshape(-1)
    X = np.concatenate([c, c])
    A = -G * X[None, :]
    A[np.diag_indices_from(A)] += 1.0
    return A


def dense_A(eps_r: np.ndarray, h: float, k: float = 2 * math.pi) -> np.ndarray:
    n2, n1 = eps_r.shape
    return dense_A_from_G(dense_G(n1, n2, h, k), contrast(eps_r))


def dense_AR(eps_r: np.ndarray, h: float, k: float = 2 * math.pi) -> np.ndarray:
    n2, n1 = eps_r.shape
    return dense_A_from_G(dense_G(n1, n2, h, k), reg_contrast(eps_r))


def plane_wave(n1: int, n2: int, h: float, psi: float, k: float = 2 * math.pi) -> np.ndarray:
    """Incident TE plane wave of unit |E| (Section 4, end; labels read as in the notes below).

    H3 = exp(i k (x1 cos psi + x2 sin psi)),  E1 = -sin(psi) H3,  E2 = cos(psi) H3.
    These follow from the source-free TE equations of Eq. (2.1) with eps = mu = 1,
    omega = k.  Returned as a (2, n2, n1) complex array.
    """
    x1 = centres(n1, h)[None, :]
    x2 = centres(n2, h)[:, None]
    H3 = np.exp(1j * k * (x1 * math.cos(psi) + x2 * math.sin(psi)))
    return np.stack([-math.sin(psi) * H3, math.cos(psi) * H3]).astype(np.complex128)


def matvec(A: np.ndarray, u: np.ndarray) -> np.ndarray:
    """y = A u for u of shape (2, n2, n1)."""
    return (A @ u.reshape(-1)).reshape(u.shape)
