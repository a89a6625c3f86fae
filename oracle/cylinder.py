"""Closed-form TE scattering by a homogeneous circular cylinder (a pin for Section 4).

Separation of variables in the TE system of Eq. (2.1) (time factor exp(-i omega t),
outgoing H^(1), eps_b = mu_b = 1, omega = k): with the incident wave
H3_in = exp(i k (x1 cos psi + x2 sin psi)), and m = sqrt(eps_r),

  outside (rho > R): H3 = sum_n i^n [J_n(k rho) + a_n H_n(k rho)] e^{i n (phi - psi)}
  inside  (rho < R): H3 = sum_n i^n  c_n J_n(m k rho)             e^{i n (phi - psi)}

H3 and the tangential E_phi ~ (1/eps) dH3/drho are continuous at rho = R, giving

  a_n = -[m J_n(mkR) J_n'(kR) - J_n'(mkR) J_n(kR)] / [m J_n(mkR) H_n'(kR) - J_n'(mkR) H_n(kR)]
  c_n = [J_n(kR) + a_n H_n(kR)] / J_n(mkR)

and the electric field follows from the first two lines of Eq. (2.1) with J = 0:
  E1 = -d2 H3 / (i omega eps),   E2 = d1 H3 / (i omega eps).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import h1vp, hankel1, jv, jvp


def coefficients(eps: complex, R: float, k: float, nmax: int):
    n = np.arange(-nmax, nmax + 1)
    m = np.sqrt(complex(eps))
    x, y = k * R, m * k * R
    Jm, dJm = jv(n, y), jvp(n, y)
    J, dJ = jv(n, x), jvp(n, x)
    H, dH = hankel1(n, x), h1vp(n, x)
    a = -(m * Jm * dJ - dJm * J) / (m * Jm * dH - dJm * H)
    c = (J + a * H) / Jm
    return n, a, c


def field(eps: complex, R: float, X1, X2, psi: float = 0.0, k: float = 2 * math.pi,
          nmax: int | None = None):
    """(E1, E2, H3) of the total field at points (X1, X2)."""
    X1 = np.asarray(X1, dtype=np.float64)
    X2 = np.asarray(X2, dtype=np.float64)
    rho = np.hypot(X1, X2)
    phi = np.arctan2(X2, X1)
    m = np.sqrt(complex(eps))
    if nmax is None:
        nmax = int(max(abs(m) * k * R, k * float(rho.max(initial=R))) + 20)
    n, a, c = coefficients(eps, R, k, nmax)
    inside = rho < R
    H3 = np.zeros(X1.shape, dtype=np.complex128)
    dHr = np.zeros_like(H3)    # d H3 / d rho
    dHp = np.zeros_like(H3)    # d H3 / d phi
    for i, nn in enumerate(n):
        ang = (1j ** nn) * np.exp(1j * nn * (phi - psi))
        kin = m * k * rho
        kout = k * rho
        F = np.where(inside, c[i] * jv(nn, kin), jv(nn, kout) + a[i] * hankel1(nn, kout))
        dF = np.where(inside, c[i] * m * k * jvp(nn, kin), k * (jvp(nn, kout) + a[i] * h1vp(nn, kout)))
        H3 += ang * F
        dHr += ang * dF
        dHp += 1j * nn * ang * F
    rs = np.where(rho == 0, 1.0, rho)
    d1 = np.cos(phi) * dHr - np.sin(phi) / rs * dHp
    d2 = np.sin(phi) * dHr + np.cos(phi) / rs * dHp
    eps_loc = np.where(inside, complex(eps), 1.0 + 0j)
    omega = k
    E1 = -d2 / (1j * omega * eps_loc)
    E2 = d1 / (1j * omega * eps_loc)
    return E1, E2, H3
