"""Matrix elements of the midpoint-collocation TE operator (paper Section 4).

The discretised system of Section 4 is A u = b with A = I - G X on the (E1, E2)
unknowns (no magnetic contrast, so the H3 rows/columns decouple; Eqs. (4.6)-(4.11)
are proportional to chi_m).  With r = |x_n - x_m|, theta_l = (x_{l,n} - x_{l,m})/r
and the scalar Green's function g = (i/4) H0^(1)(k_b r) of Eq. (2.14):

  off-diagonal, Eq. (4.3) and Eq. (4.5):
      G_ll(x) = k_b^2 h^2 [ P(r) theta_l theta_l + Q(r) ]
      G_lq(x) = k_b^2 h^2   P(r) theta_l theta_q               (l != q)
      P(r) = (i / (2 k_b r)) H1(k_b r) - (i/4) H0(k_b r)
      Q(r) = (i/4) H0(k_b r) - (i / (4 k_b r)) H1(k_b r)
  self term, Eq. (4.4), from an equal-area disc of radius a = h / sqrt(pi):
      G_ll(0) = -[ 1 - (i pi / 4) k_b a H1(k_b a) ],   G_12(0) = 0

so that [A_ll]_nm = delta_nm - G_ll(x_n - x_m) chi(x_m).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import hankel1


def self_term(k: float, h: float) -> complex:
    """G_ll(0) of Eq. (4.4): -(1 - (i pi/4) k a H1(k a)), a = h/sqrt(pi)."""
    a = h / math.sqrt(math.pi)
    return complex(-(1.0 - 0.25j * math.pi * k * a * hankel1(1, k * a)))


def green_tensor(d1, d2, k: float, h: float):
    """(G11, G22, G12) at separation vectors (d1, d2) (arrays, same shape).

    Entries with d1 = d2 = 0 take the self term of Eq. (4.4).
    """
    d1 = np.asarray(d1, dtype=np.float64)
    d2 = np.asarray(d2, dtype=np.float64)
    d1, d2 = np.broadcast_arrays(d1, d2)
    r = np.hypot(d1, d2)
    is_self = r == 0.0
    rs = np.where(is_self, 1.0, r)
    kr = k * rs
    H0 = hankel1(0, kr)
    H1 = hankel1(1, kr)
    P = 1j / (2.0 * kr) * H1 - 0.25j * H0
    Q = 0.25j * H0 - 1j / (4.0 * kr) * H1
    t1 = d1 / rs
    t2 = d2 / rs
    c = (k * h) ** 2
    G11 = c * (P * t1 * t1 + Q)
    G22 = c * (P * t2 * t2 + Q)
    G12 = c * P * t1 * t2
    if np.any(is_self):
        s = self_term(k, h)
        G11 = np.where(is_self, s, G11)
        G22 = np.where(is_self, s, G22)
        G12 = np.where(is_self, 0.0, G12)
    return G11, G22, G12
