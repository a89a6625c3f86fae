"""The TM (E-wave) scalar operator and its closed-form cylinder solution (paper Section 2).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Without magnetic contrast the third row of the TM system of Eq. (2.16) is scalar:
    E3_in = E3 - k_b^2 g * (chi E3),   g = (i/4) H0^(1)(k_b |x|)   (Eq. (2.14)).
Midpoint collocation on the grid of Section 4, with the diagonal integrated over the
equal-area disc of radius a = h / sqrt(pi) as Eq. (4.4) does for TE:
    off-diagonal  G(x_n - x_m) = k_b^2 h^2 (i/4) H0(k_b r_nm)
    diagonal      G(0) = k_b^2 int_{|y| < a} g(|y|) dy = (i pi / 2) k_b a H1(k_b a) - 1
(the integral: int_0^a H0(k r) r dr = a H1(k a) / k + 2 i / (pi k^2), from d/dr [r H1(k r)]
= k r H0(k r) and r H1(k r) -> -2 i / (pi k) at r = 0), and A = I - G X(chi) on the N
unknowns E3(x_n).  The regulariser is not needed in TM (the operator is identity plus
compact, Section 3); the deflation of Eq. (4.12) applies as in TE (Table 1).

Closed form for a homogeneous cylinder of radius R, m = sqrt(eps_r), incident
E3 = exp(i k (x1 cos psi + x2 sin psi)) (separation of variables; E3 and d E3 / d rho are
continuous at rho = R):
    outside: E3 = sum_n i^n [J_n(k rho) + b_n H_n(k rho)] e^{i n (phi - psi)}
    inside:  E3 = sum_n i^n  c_n J_n(m k rho)             e^{i n (phi - psi)}
    b_n = -[m J_n'(mkR) J_n(kR) - J_n(mkR) J_n'(kR)] / [m J_n'(mkR) H_n(kR) - J_n(mkR) H_n'(kR)]
    c_n = [J_n(kR) + b_n H_n(kR)] / J_n(mkR)
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import h1vp, hankel1, jv, jvp

from .dense import contrast, node_positions


def self_term(k: float, h: float) -> complex:
    """G(0): the integral of k^2 g over the disc of radius a = h / sqrt(pi)."""
    a = h / math.sqrt(math.pi)
    return complex(0.5j * math.pi * k * a * hankel1(1, k * a) - 1.0)


def kernel(d1, d2, k: float, h: float):
    """G at separation vectors (d1, d2); the self term where both are zero."""
    d1, d2 = np.broadcast_arrays(np.asarray(d1, dtype=np.float64), np.asarray(d2, dtype=np.float64))
    r = np.hypot(d1, d2)
    is_self = r == 0.0
    G = (k * h) ** 2 * 0.25j * hankel1(0, k * np.where(is_self, 1.0, r))
    return np.where(is_self, self_term(k, h), G)


def dense_A(eps_r: np.ndarray, h: float, k: float = 2 * math.pi) -> np.ndarray:
    """A = I - G X(chi), N x N, node m = i1 + n1 i2."""
    n2, n1 = eps_r.shape
    x1, x2 = node_positions(n1, n2, h)
    G = kernel(x1[:, None] - x1[None, :], x2[:, None] - x2[None, :], k, h)
    A = -G * contrast(eps_r).reshape(-1)[None, :]
    A[np.diag_indices_from(A)] += 1.0
    return A


def plane_wave(n1: int, n2: int, h: float, psi: float, k: float = 2 * math.pi) -> np.ndarray:
    """Incident E3 = exp(i k (x1 cos psi + x2 sin psi)), shape (n2, n1)."""
    x1 = ((np.arange(n1) + 0.5) * h - 0.5 * n1 * h)[None, :]
    x2 = ((np.arange(n2) + 0.5) * h - 0.5 * n2 * h)[:, None]
    return np.exp(1j * k * (x1 * math.cos(psi) + x2 * math.sin(psi))).astype(np.complex128)


def cylinder_field(eps: complex, R: float, X1, X2, psi: float = 0.0, k: float = 2 * math.pi,
                   nmax: int | None = None) -> np.ndarray:
    """Total E3 of the closed form above at points (X1, X2)."""
    X1 = np.asarray(X1, dtype=np.float64)
    X2 = np.asarray(X2, dtype=np.float64)
    rho = np.hypot(X1, X2)
    phi = np.arctan2(X2, X1)
    m = np.sqrt(complex(eps))
    if nmax is None:
        nmax = int(max(abs(m) * k * R, k * float(rho.max(initial=R))) + 20)
    n = np.arange(-nmax, nmax + 1)
    x, y = k * R, m * k * R
    b = -(m * jvp(n, y) * jv(n, x) - jv(n, y) * jvp(n, x)) / (m * jvp(n, y) * hankel1(n, x) - jv(n, y) * h1vp(n, x))
    c = (jv(n, x) + b * hankel1(n, x)) / jv(n, y)
    inside = rho < R
    E3 = np.zeros(X1.shape, dtype=np.complex128)
    for i, nn in enumerate(n):
        ang = (1j ** nn) * np.exp(1j * nn * (phi - psi))
        E3 += ang * np.where(inside, c[i] * jv(nn, m * k * rho), jv(nn, k * rho) + b[i] * hankel1(nn, k * rho))
    return E3
