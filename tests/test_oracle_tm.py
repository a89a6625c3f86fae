"""Pins of the TM oracle (oracle/tm.py): the self term against brute-force integration of
the kernel over the disc, its static limit, the plane wave against the series at eps = 1,
the series' boundary conditions, and convergence of the dense solve to the series."""
import math

import numpy as np
import pytest
from scipy import integrate
from scipy.special import hankel1

from oracle import tm
from paper_1104_4263_gb300 import workloads as W


@pytest.mark.parametrize("kh", [0.05, 0.4, 1.3])
def test_self_term_is_the_disc_integral(kh):
    """k^2 int_disc (i/4) H0(k |y|) dy by quadrature (log-singular integrand, split at a/10)."""
    k = 2 * math.pi
    h = kh / k
    a = h / math.sqrt(math.pi)
    f_re = lambda r: (0.25j * hankel1(0, k * r) * 2 * math.pi * r).real
    f_im = lambda r: (0.25j * hankel1(0, k * r) * 2 * math.pi * r).imag
    val = 0j
    for lo, hi in ((0.0, a / 10), (a / 10, a)):
        val += integrate.quad(f_re, lo, hi, limit=200, epsabs=1e-15)[0]
        val += 1j * integrate.quad(f_im, lo, hi, limit=200, epsabs=1e-15)[0]
    assert abs(k * k * val - tm.self_term(k, h)) < 1e-9


def test_self_term_static_limit():
    """The TM operator is identity plus compact (Section 3): the self term vanishes as ka -> 0."""
    k = 2 * math.pi
    assert abs(tm.self_term(k, 1e-6)) < 1e-9
    assert abs(tm.self_term(k, 1e-3)) < 1e-4


def test_plane_wave_is_series_at_eps_1():
    X1, X2 = W.mesh(9, 7, 0.13)
    for psi in (0.0, 0.7, -2.0):
        assert np.max(np.abs(tm.cylinder_field(1.0, 0.4, X1, X2, psi) - tm.plane_wave(9, 7, 0.13, psi))) < 1e-10


def test_series_continuity_at_the_interface():
    """E3 and d E3 / d rho continuous across rho = R (the matching conditions)."""
    eps, R = 4.0 + 0.5j, 0.8
    phi = np.linspace(0, 2 * math.pi, 7)
    for d in (1e-7,):
        fi = tm.cylinder_field(eps, R, (R - d) * np.cos(phi), (R - d) * np.sin(phi))
        fo = tm.cylinder_field(eps, R, (R + d) * np.cos(phi), (R + d) * np.sin(phi))
        assert np.max(np.abs(fi - fo)) < 1e-5
        gi = (tm.cylinder_field(eps, R, (R - d) * np.cos(phi), (R - d) * np.sin(phi)) -
              tm.cylinder_field(eps, R, (R - 3 * d) * np.cos(phi), (R - 3 * d) * np.sin(phi))) / (2 * d)
        go = (tm.cylinder_field(eps, R, (R + 3 * d) * np.cos(phi), (R + 3 * d) * np.sin(phi)) -
              tm.cylinder_field(eps, R, (R + d) * np.cos(phi), (R + d) * np.sin(phi))) / (2 * d)
        assert np.max(np.abs(gi - go)) < 1e-3 * np.max(np.abs(gi))


def test_dense_solve_converges_to_series():
    """Cylinder eps 4, R 1, side 2.5 (the config-1 geometry in TM): the relative error of the
    dense solve against the series falls with the grid (staircase boundary: about first
    order overall, not monotone step by step), at least like h^0.8 from 24^2 to 64^2."""
    errs = []
    for n in (24, 32, 64):
        p = W.config1(n)
        A = tm.dense_A(p.eps_r, p.h)
        b = tm.plane_wave(n, n, p.h, 0.0)
        u = np.linalg.solve(A, b.reshape(-1)).reshape(n, n)
        X1, X2 = W.mesh(n, n, p.h)
        ref = tm.cylinder_field(4.0, 1.0, X1, X2, 0.0)
        errs.append(np.linalg.norm(u - ref) / np.linalg.norm(ref))
    assert errs[0] > errs[1] > errs[2], errs
    order = math.log(errs[0] / errs[2]) / math.log(64 / 24)
    assert order > 0.8 and errs[2] < 0.05, (errs, order)
