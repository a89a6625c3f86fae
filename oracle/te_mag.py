"""The TE system with magnetic contrast: unknowns (E1, E2, H3), a 3N x 3N system
(paper Sections 2-4).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Normalised units as in the rest of the oracle: eps_b = mu_b = 1 and omega = k_b, so that
omega eps_b = omega mu_b = k_b.  The TE integro-differential equation of Eq. (2.15) reads
u_in = u - D [g*(chi_e E1), g*(chi_e E2), g*(chi_m H3)] with the differential matrix D of its
TE line and g = (i/4) H0^(1)(k_b |x|) (Eq. (2.14)).  With d/dx_l g = -(i k/4) H1(k r) theta_l,
midpoint collocation gives A = I - G X, X = diag(chi_e, chi_e, chi_m), where besides the
electric block of Eqs. (4.3)-(4.5) (oracle/green.py)

    G13 =  i omega mu_b  d2 g h^2 =  (k^2 h^2 / 4) H1(k r) theta_2
    G23 = -i omega mu_b  d1 g h^2 = -(k^2 h^2 / 4) H1(k r) theta_1
    G31 =  i omega eps_b d2 g h^2 =  G13
    G32 = -i omega eps_b d1 g h^2 =  G23
    G33 =  k^2 g h^2             =  (i/4) k^2 h^2 H0(k r)

(theta_l = (x_{l,n} - x_{l,m}) / r).  These are the compact kernels K13, K23, K31, K32, K33
of Section 3 times h^2 (A_lq = K_lq chi_q h^2 off the diagonal): K31 and K32 carry
omega eps_b and act on chi_e E, K13 and K23 carry omega mu_b and act on chi_m H3.  The
discrete relations printed in Section 4, A31 = -A13 and A23 = -A32, would give the H3 line
the magnetic contrast and the opposite sign; they are not used (a reading of the text).
Self terms: G13(0) = G23(0) = 0 (odd kernels integrate to zero over the disc of radius
a = h / sqrt(pi)); G33(0) = k^2 times the disc integral of g = (i pi / 2) k a H1(k a) - 1,
which is the [A33]_nn printed in Section 4; the electric block takes Eq. (4.4).

Regulariser (Section 3): the symbol of the 3 x 3 operator is I + chi_e Q with Q acting on
the electric components only, and its inverse is I + chi'_e Q, chi'_e = 1/eps_r - 1; the
same operator with the electric contrast replaced, A(chi'_e, chi_m), is the regulariser
(chi_m left unchanged: a reading; the symbol does not involve it).

Incident plane wave (the source-free TE equations with eps = mu = 1):
(E1, E2, H3) = (-sin psi, cos psi, 1) exp(i k (x1 cos psi + x2 sin psi)).

Closed form for a homogeneous cylinder of radius R with eps_r, mu_r (separation of
variables; H3 and E_phi ~ (1/eps) dH3/drho continuous at rho = R), m = sqrt(eps mu),
eta = m / eps:
    outside: H3 = sum_n i^n [J_n(k rho) + a_n H_n(k rho)] e^{i n (phi - psi)}
    inside:  H3 = sum_n i^n  c_n J_n(m k rho)             e^{i n (phi - psi)}
    a_n = -[eta J_n'(mkR) J_n(kR) - J_n(mkR) J_n'(kR)] / [eta J_n'(mkR) H_n(kR) - J_n(mkR) H_n'(kR)]
    c_n = [J_n(kR) + a_n H_n(kR)] / J_n(mkR)
(mu_r = 1 gives the coefficients of oracle/cylinder.py).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import h1vp, hankel1, jv, jvp

from .dense import centres, node_positions
from .green import green_tensor


def self_term_33(k: float, h: float) -> complex:
    """G33(0): k^2 times the integral of g over the disc of radius a = h / sqrt(pi)."""
    a = h / math.sqrt(math.pi)
    return complex(0.5j * math.pi * k * a * hankel1(1, k * a) - 1.0)


def coupling(d1, d2, k: float, h: float):
    """(G13, G23, G33) at separation vectors (d1, d2); self terms where both are zero."""
    d1, d2 = np.broadcast_arrays(np.asarray(d1, dtype=np.float64), np.asarray(d2, dtype=np.float64))
    r = np.hypot(d1, d2)
    is_self = r == 0.0
    rs = np.where(is_self, 1.0, r)
    H0 = hankel1(0, k * rs)
    H1 = hankel1(1, k * rs)
    c = (k * h) ** 2
    G13 = np.where(is_self, 0.0, 0.25 * c * H1 * d2 / rs)
    G23 = np.where(is_self, 0.0, -0.25 * c * H1 * d1 / rs)
    G33 = np.where(is_self, self_term_33(k, h), 0.25j * c * H0)
    return G13, G23, G33


def dense_G(n1: int, n2: int, h: float, k: float) -> np.ndarray:
    """The 3N x 3N matrix G, blocks [l][q] = G_lq(x_n - x_m), node m = i1 + n1 i2."""
    x1, x2 = node_positions(n1, n2, h)
    d1 = x1[:, None] - x1[None, :]
    d2 = x2[:, None] - x2[None, :]
    G11, G22, G12 = green_tensor(d1, d2, k, h)
    G13, G23, G33 = coupling(d1, d2, k, h)
    N = n1 * n2
    G = np.empty((3 * N, 3 * N), dtype=np.complex128)
    blocks = ((G11, G12, G13), (G12, G22, G23), (G13, G23, G33))
    for l in range(3):
        for q in range(3):
            G[l * N:(l + 1) * N, q * N:(q + 1) * N] = blocks[l][q]
    return G


def dense_A_from_G(G: np.ndarray, chi_e: np.ndarray, chi_m: np.ndarray) -> np.ndarray:
    """A = I - G X, X = diag(chi_e, chi_e, chi_m) (maps of shape (n2, n1))."""
    ce = np.asarray(chi_e, dtype=np.complex128).reshape(-1)
    cm = np.asarray(chi_m, dtype=np.complex128).reshape(-1)
    X = np.concatenate([ce, ce, cm])
    A = -G * X[None, :]
    A[np.diag_indices_from(A)] += 1.0
    return A


def dense_A(eps_r: np.ndarray, mu_r: np.ndarray, h: float, k: float = 2 * math.pi) -> np.ndarray:
    n2, n1 = eps_r.shape
    return dense_A_from_G(dense_G(n1, n2, h, k), np.asarray(eps_r) - 1.0, np.asarray(mu_r) - 1.0)


def dense_AR(eps_r: np.ndarray, mu_r: np.ndarray, h: float, k: float = 2 * math.pi) -> np.ndarray:
    """The regulariser A(chi'_e, chi_m), chi'_e = 1/eps_r - 1."""
    n2, n1 = eps_r.shape
    return dense_A_from_G(dense_G(n1, n2, h, k), 1.0 / np.asarray(eps_r, dtype=np.complex128) - 1.0,
                          np.asarray(mu_r) - 1.0)


def plane_wave(n1: int, n2: int, h: float, psi: float, k: float = 2 * math.pi) -> np.ndarray:
    """(E1, E2, H3) of the incident plane wave, shape (3, n2, n1)."""
    x1 = centres(n1, h)[None, :]
    x2 = centres(n2, h)[:, None]
    e = np.exp(1j * k * (x1 * math.cos(psi) + x2 * math.sin(psi)))
    return np.stack([-math.sin(psi) * e, math.cos(psi) * e, e]).astype(np.complex128)


def cylinder_field(eps: complex, mu: complex, R: float, X1, X2, psi: float = 0.0, k: float = 2 * math.pi,
                   nmax: int | None = None):
    """(E1, E2, H3) of the closed form above at points (X1, X2)."""
    X1 = np.asarray(X1, dtype=np.float64)
    X2 = np.asarray(X2, dtype=np.float64)
    rho = np.hypot(X1, X2)
    phi = np.arctan2(X2, X1)
    m = np.sqrt(complex(eps) * complex(mu))
    eta = m / complex(eps)
    if nmax is None:
        nmax = int(max(abs(m) * k * R, k * float(rho.max(initial=R))) + 20)
    n = np.arange(-nmax, nmax + 1)
    x, y = k * R, m * k * R
    a = -(eta * jvp(n, y) * jv(n, x) - jv(n, y) * jvp(n, x)) / (eta * jvp(n, y) * hankel1(n, x) - jv(n, y) * h1vp(n, x))
    c = (jv(n, x) + a * hankel1(n, x)) / jv(n, y)
    inside = rho < R
    H3 = np.zeros(X1.shape, dtype=np.complex128)
    dHr = np.zeros_like(H3)
    dHp = np.zeros_like(H3)
    for i, nn in enumerate(n):
        ang = (1j ** nn) * np.exp(1j * nn * (phi - psi))
        kin, kout = m * k * rho, k * rho
        F = np.where(inside, c[i] * jv(nn, kin), jv(nn, kout) + a[i] * hankel1(nn, kout))
        dF = np.where(inside, c[i] * m * k * jvp(nn, kin), k * (jvp(nn, kout) + a[i] * h1vp(nn, kout)))
        H3 += ang * F
        dHr += ang * dF
        dHp += 1j * nn * ang * F
    # Cartesian derivatives of H3, then E1 = -d2 H3 / (i omega eps), E2 = d1 H3 / (i omega eps)
    rs = np.where(rho == 0.0, 1.0, rho)
    d1H = np.cos(phi) * dHr - np.sin(phi) * dHp / rs
    d2H = np.sin(phi) * dHr + np.cos(phi) * dHp / rs
    eps_loc = np.where(inside, complex(eps), 1.0)
    E1 = -d2H / (1j * k * eps_loc)
    E2 = d1H / (1j * k * eps_loc)
    return E1, E2, H3
