"""The TE operator applied through a zero-padded 2-D FFT (scipy.fft, FP64).

Sections 1 and 5 of the paper rely on the block-Toeplitz structure of G: G
depends only on x_n - x_m, so G w is a 2-D linear convolution and can be done by
FFTs of size M1 x M2 >= (2 n1 - 1) x (2 n2 - 1).  This is the CPU throughput
baseline for grids where the dense matrix does not fit; it is pinned against
`dense.py` on small grids.

Kernel planes are indexed by offset (p, q) in cells, stored at (q mod M2, p mod M1);
offsets outside |p| < n1, |q| < n2 are zero.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.fft as sfft

from .dense import contrast, reg_contrast
from .green import green_tensor


class FFTOperator:
    """A = I - G X(chi) and A_R = I - G X(chi') with G applied by FFT convolution."""

    def __init__(self, eps_r: np.ndarray, h: float, k: float = 2 * math.pi,
                 M1: int | None = None, M2: int | None = None, workers: int = 1):
        self.eps_r = np.asarray(eps_r, dtype=np.complex128)
        n2, n1 = self.eps_r.shape
        self.n1, self.n2, self.h, self.k = n1, n2, h, k
        self.M1 = M1 or 2 * n1
        self.M2 = M2 or 2 * n2
        assert self.M1 >= 2 * n1 - 1 and self.M2 >= 2 * n2 - 1
        self.workers = workers
        self.chi = contrast(self.eps_r)
        self.chi_r = reg_contrast(self.eps_r)
        p = np.arange(-(n1 - 1), n1)
        q = np.arange(-(n2 - 1), n2)
        Q, P = np.meshgrid(q, p, indexing="ij")
        G11, G22, G12 = green_tensor(P * h, Q * h, k, h)
        self.Ghat = []
        for g in (G11, G22, G12):
            plane = np.zeros((self.M2, self.M1), dtype=np.complex128)
            plane[Q % self.M2, P % self.M1] = g
            self.Ghat.append(sfft.fft2(plane, workers=workers))

    def apply_G(self, w: np.ndarray) -> np.ndarray:
        """z = G w for w of shape (2, n2, n1) (linear convolution, exact up to rounding)."""
        n1, n2, M1, M2 = self.n1, self.n2, self.M1, self.M2
        W = sfft.fft2(w, s=(M2, M1), axes=(-2, -1), workers=self.workers)
        G11, G22, G12 = self.Ghat
        Z1 = G11 * W[0] + G12 * W[1]
        Z2 = G12 * W[0] + G22 * W[1]
        z = sfft.ifft2(np.stack([Z1, Z2]), axes=(-2, -1), workers=self.workers)
        return z[:, :n2, :n1]

    def apply(self, u: np.ndarray) -> np.ndarray:
        """y = A u = u - G (chi u)."""
        return u - self.apply_G(self.chi[None] * u)

    def apply_R(self, u: np.ndarray) -> np.ndarray:
        """y = A_R u = u - G (chi' u)."""
        return u - self.apply_G(self.chi_r[None] * u)

    def apply_regularized(self, u: np.ndarray) -> np.ndarray:
        """y = A_R A u (Section 5: the regularised product, two FFT applications)."""
        return self.apply_R(self.apply(u))
