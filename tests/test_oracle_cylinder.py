"""Pins for the closed-form cylinder series and, through it, the discretisation (P4)."""
import math

import numpy as np
import pytest

from oracle import cylinder, dense, fftmv, gmres, green
from paper_1104_4263_gb300 import workloads as W

K = 2 * math.pi


def test_unit_eps_is_plane_wave():
    """Jacobi-Anger: with eps_r = 1 the series must reproduce H3 = exp(i k x.d) exactly."""
    X1, X2 = np.meshgrid(np.linspace(-1.7, 1.7, 9), np.linspace(-1.3, 1.6, 8))
    for psi in (0.0, 1.1):
        E1, E2, H3 = cylinder.field(1.0, 0.8, X1, X2, psi)
        inc = np.exp(1j * K * (X1 * math.cos(psi) + X2 * math.sin(psi)))
        assert np.max(np.abs(H3 - inc)) < 1e-10
        assert np.max(np.abs(E1 + math.sin(psi) * inc)) < 1e-9
        assert np.max(np.abs(E2 - math.cos(psi) * inc)) < 1e-9


@pytest.mark.parametrize("eps", [4.0, 16.0 + 0j, -2.0 + 0.1j])
def test_series_satisfies_maxwell(eps):
    """Third TE equation of Eq. (2.1) (-d2 E1 + d1 E2 = i omega mu H3) by finite differences,
    inside and outside, and continuity of H3 and E_phi across rho = R."""
    R, d = 0.6, 1e-5
    pts = [(0.2, 0.1), (-0.3, 0.25), (0.9, -0.4), (-1.2, 1.0)]
    for (x1, x2) in pts:
        f = lambda a, b: cylinder.field(eps, R, np.array([a]), np.array([b]))
        E1p, _, _ = f(x1, x2 + d)
        E1m, _, _ = f(x1, x2 - d)
        _, E2p, _ = f(x1 + d, x2)
        _, E2m, _ = f(x1 - d, x2)
        _, _, H3 = f(x1, x2)
        lhs = -(E1p - E1m) / (2 * d) + (E2p - E2m) / (2 * d)
        rhs = 1j * K * H3
        assert abs(lhs[0] - rhs[0]) < 1e-5 * max(1.0, abs(rhs[0]))
    for phi in (0.3, 2.0, 4.0):
        c, s = math.cos(phi), math.sin(phi)
        fin = cylinder.field(eps, R, np.array([R * (1 - 1e-9) * c]), np.array([R * (1 - 1e-9) * s]))
        fout = cylinder.field(eps, R, np.array([R * (1 + 1e-9) * c]), np.array([R * (1 + 1e-9) * s]))
        assert abs(fin[2][0] - fout[2][0]) < 1e-6 * abs(fout[2][0]) + 1e-9
        ephi_in = -s * fin[0][0] + c * fin[1][0]
        ephi_out = -s * fout[0][0] + c * fout[1][0]
        assert abs(ephi_in - ephi_out) < 1e-6 * abs(ephi_out) + 1e-9


def solve_cylinder(n, tol=1e-7):
    p = W.config1(n)
    b = dense.plane_wave(n, n, p.h, 0.0)
    if n <= 32:
        u = np.linalg.solve(dense.dense_A(p.eps_r, p.h), b.reshape(-1)).reshape(b.shape)
    else:
        op = fftmv.FFTOperator(p.eps_r, p.h)
        u = gmres.gmres(op.apply, b, 20, tol, 20000).x
    X1, X2 = W.mesh(n, n, p.h)
    E1, E2, _ = cylinder.field(4.0, 1.0, X1, X2, 0.0)
    ref = np.stack([E1, E2])
    return np.linalg.norm(u - ref) / np.linalg.norm(ref)


def test_discretisation_converges_to_series():
    """P4: relative field error <= 0.35 on the 32^2 grid and first-order convergence."""
    e = [solve_cylinder(n) for n in (32, 48, 64)]
    assert e[0] <= 0.35
    assert e[0] > e[1] > e[2]
    order = math.log(e[0] / e[2]) / math.log(2.0)
    assert order >= 0.8, e


def test_series_pin_catches_wrong_self_term(monkeypatch):
    """Plant the alternative self-term reading in the oracle: P4 must fail loudly."""
    def alt(k, h):
        a = h / math.sqrt(math.pi)
        from scipy.special import hankel1
        return complex(-(0.5 - 0.25j * math.pi * k * a * hankel1(1, k * a)))
    monkeypatch.setattr(green, "self_term", alt)
    assert solve_cylinder(32) > 1.0
