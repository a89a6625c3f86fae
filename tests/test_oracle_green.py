"""Pins for the oracle's Green's-tensor entries and dense matrices (CPU only).

P2 (block-Toeplitz structure), P3 (static limit of the self term, Eq. (3.3) vs
Eq. (4.4)), and an independent finite-difference evaluation of
h^2 (k^2 delta + d_l d_q) g, g = (i/4) H0(k|x|) (Eq. (2.9) with Eq. (2.14)), which
fixes the P/Q formulas of Eqs. (4.3) and (4.5).  Each pin is also run against a
deliberately broken copy of the oracle to show it would catch that mistake.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy.special import hankel1

from oracle import dense, green

K = 2 * math.pi
GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def g_scalar(x1, x2, k=K):
    return 0.25j * hankel1(0, k * np.hypot(x1, x2))


def fd_green(x1, x2, h, k=K, d=2e-4):
    """h^2 (k^2 delta + d_l d_q) g by central differences of the scalar Green's function."""
    g0 = g_scalar(x1, x2, k)
    d11 = (g_scalar(x1 + d, x2, k) - 2 * g0 + g_scalar(x1 - d, x2, k)) / d**2
    d22 = (g_scalar(x1, x2 + d, k) - 2 * g0 + g_scalar(x1, x2 - d, k)) / d**2
    d12 = (g_scalar(x1 + d, x2 + d, k) - g_scalar(x1 + d, x2 - d, k)
           - g_scalar(x1 - d, x2 + d, k) + g_scalar(x1 - d, x2 - d, k)) / (4 * d * d)
    return h * h * (k * k * g0 + d11), h * h * (k * k * g0 + d22), h * h * d12


def check_fd(gt):
    h = 0.05
    pts = [(0.13, 0.0), (0.0, 0.21), (0.3, -0.17), (-0.55, 0.4), (1.3, 0.9), (-2.1, -0.05)]
    err = 0.0
    for x1, x2 in pts:
        a = np.array(gt(np.array(x1), np.array(x2), K, h), dtype=complex).ravel()
        b = np.array(fd_green(x1, x2, h), dtype=complex)
        err = max(err, float(np.max(np.abs(a - b)) / np.max(np.abs(b))))
    return err


def test_green_matches_finite_differences():
    assert check_fd(green.green_tensor) < 2e-5


def test_fd_pin_catches_dropped_term():
    def broken(d1, d2, k, h):            # Q term dropped from G_ll (a plausible slip)
        G11, G22, G12 = green.green_tensor(d1, d2, k, h)
        r = np.hypot(d1, d2)
        H0, H1 = hankel1(0, k * r), hankel1(1, k * r)
        Q = 0.25j * H0 - 1j / (4 * k * r) * H1
        return G11 - (k * h) ** 2 * Q, G22 - (k * h) ** 2 * Q, G12

    def sign(d1, d2, k, h):              # sign of G12 flipped
        G11, G22, G12 = green.green_tensor(d1, d2, k, h)
        return G11, G22, -G12

    assert check_fd(broken) > 1e-2
    assert check_fd(sign) > 1e-2


def test_self_term_static_limit():
    """Eq. (4.4) diagonal 1 - G_ll(0) chi -> 1 + chi/2 (free term s of Eq. (3.3)) as k h -> 0."""
    target = GOLDEN["free_term_coefficient"]["value"]
    vals = [-green.self_term(K, h) for h in (1e-3, 1e-4, 1e-5)]
    errs = [abs(v - target) for v in vals]
    assert errs[-1] < 1e-8
    assert errs[0] > errs[1] > errs[2]          # converges as the cell shrinks
    # the alternative reading -(1/2 - (i pi/4) k a H1) has limit 0, not 1/2
    a = 1e-5 / math.sqrt(math.pi)
    alt = -(0.5 - 0.25j * math.pi * K * a * hankel1(1, K * a))
    assert abs(-alt - target) > 0.4


@pytest.mark.parametrize("n1,n2", [(6, 6), (7, 5)])
def test_bttb_structure(n1, n2):
    """P2: G depends on x_n - x_m only; G = G^T; G11(p,q) = G22(q,p); G12 odd in p and q."""
    h = 0.1
    G = dense.dense_G(n1, n2, h, K)
    N = n1 * n2
    assert np.max(np.abs(G - G.T)) == 0.0
    idx = lambda i1, i2: i1 + n1 * i2
    for (a1, a2, b1, b2) in [(0, 0, 2, 3), (1, 1, 3, 4), (3, 0, 5, 3)]:
        if max(a1, b1) >= n1 or max(a2, b2) >= n2:
            continue
        # same separation, shifted pair
        s1, s2 = 1, 1
        if b1 + s1 < n1 and b2 + s2 < n2:
            for (l, q) in [(0, 0), (0, 1), (1, 1)]:
                v = G[l * N + idx(b1, b2), q * N + idx(a1, a2)]
                w = G[l * N + idx(b1 + s1, b2 + s2), q * N + idx(a1 + s1, a2 + s2)]
                assert v == pytest.approx(w, rel=1e-14, abs=1e-300)
    p, q = np.meshgrid(np.arange(-3, 4), np.arange(-3, 4), indexing="ij")
    G11, G22, G12 = green.green_tensor(p * h, q * h, K, h)
    G11t, G22t, _ = green.green_tensor(q * h, p * h, K, h)
    assert np.allclose(G11, G22t, rtol=1e-14, atol=0)
    _, _, G12m = green.green_tensor(-p * h, q * h, K, h)
    assert np.allclose(G12, -G12m, rtol=1e-14, atol=0)
    _, _, G12n = green.green_tensor(p * h, -q * h, K, h)
    assert np.allclose(G12, -G12n, rtol=1e-14, atol=0)


def test_zero_contrast_is_identity():
    eps = np.ones((4, 5), dtype=complex)
    A = dense.dense_A(eps, 0.1)
    assert np.array_equal(A, np.eye(A.shape[0]))
