"""Spectral pins of the oracle on tiny grids (P5-P9): Eqs. (3.20), (3.21), (4.12)-(4.13), (5.3)."""
import json
import math
import os

import numpy as np
import pytest

from oracle import deflation, dense
from paper_1104_4263_gb300 import workloads as W

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))
EPS = [complex(*v) for v in GOLDEN["homogeneous_map_test_eps"]["values"]]


@pytest.fixture(scope="module")
def homogeneous():
    out = {}
    n, h = 16, 1.0 / 16
    for e in EPS:
        eps = np.full((n, n), e)
        G = dense.dense_G(n, n, h, 2 * math.pi)
        A = dense.dense_A_from_G(G, dense.contrast(eps))
        AR = dense.dense_A_from_G(G, dense.reg_contrast(eps))
        out[e] = (A, AR, np.linalg.eigvals(A), np.linalg.eigvals(AR @ A))
    return out


@pytest.mark.parametrize("e", EPS)
def test_homogeneous_map(homogeneous, e):
    """P5: for A = I - chi G, spec(A_R A) is the image of spec(A) under Eq. (5.3); A, A_R commute."""
    A, AR, la, lra = homogeneous[e]
    assert np.max(np.abs(A @ AR - AR @ A)) < 1e-11 * np.max(np.abs(A))
    mapped = deflation.regularized_eig_map(la, e)
    # each mapped eigenvalue has a partner in the computed spectrum and vice versa
    d1 = np.min(np.abs(mapped[:, None] - lra[None, :]), axis=1)
    d2 = np.min(np.abs(lra[:, None] - mapped[None, :]), axis=1)
    scale = np.max(np.abs(lra))
    assert np.max(d1) < 1e-9 * scale and np.max(d2) < 1e-9 * scale


@pytest.mark.parametrize("e", EPS)
def test_essential_spectrum_segment(homogeneous, e):
    """P7: most eigenvalues of A cluster on the segment [1, eps_r] (Eq. (3.20))."""
    _, _, la, _ = homogeneous[e]
    t = np.clip(np.real((la - 1) * np.conj(e - 1)) / abs(e - 1) ** 2, 0, 1)
    dist = np.abs(la - (1 + t * (e - 1)))
    frac = np.mean(dist < 0.05 * abs(e))
    assert frac >= 0.8, frac


def test_wedge_bound_soft(homogeneous):
    """P9 (soft): lossless eps = 16 > 1 puts the eigenvalues in Im(lambda) <= 0 (Eq. (3.21))."""
    _, _, la, _ = homogeneous[EPS[0]]
    assert np.max(la.imag) <= 0.01 * np.max(np.abs(la))


def test_lossless_segment_image():
    """P8: the segment [1, 16] maps to [1, 4.515625] (Section 5)."""
    g = GOLDEN["lossless_image_upper_end"]
    R = deflation.deflation_radius([g["eps_r"]], samples=100001)
    assert R == pytest.approx(g["value"], rel=1e-9)
    R1000 = deflation.deflation_radius([g["eps_r"], 1.0])
    assert abs(R1000 - g["value"]) < 1e-5
    lam = 1 + np.linspace(0, 1, 1001) * 15
    img = deflation.regularized_eig_map(lam, 16.0)
    assert np.min(img) == pytest.approx(1.0) and np.max(np.abs(img.imag)) == 0


@pytest.mark.parametrize("regularized", [False, True])
def test_deflation_moves_eigenvalues_to_one(regularized):
    """P6: spec(Atilde P^-1) = {1 (x r)} U (spec(Atilde) minus the r deflated values)."""
    n, h = 10, 0.1
    eps = W.core_shell(n, side=1.0, r_core=0.2, r_shell=0.45, eps_core=-16 + 1.5j, eps_shell=16).eps_r
    A = dense.dense_A(eps, h)
    At = dense.dense_AR(eps, h) @ A if regularized else A
    r = 8
    D = deflation.Deflation(At, r)
    assert np.allclose(D.V.conj().T @ D.V, np.eye(r), atol=1e-12)
    assert np.allclose(np.sort_complex(np.linalg.eigvals(D.T)), np.sort_complex(D.eigs), atol=1e-8 * abs(D.eigs[0]))
    lam = np.linalg.eigvals(At @ D.matrix())
    ones = np.abs(lam - 1.0) < 1e-8
    assert np.count_nonzero(ones) >= r
    full = np.linalg.eigvals(At)
    rest = [z for z in full if np.min(np.abs(z - D.eigs)) > 1e-9 * abs(z)]
    for z in rest:
        assert np.min(np.abs(lam - z)) < 1e-8 * max(1.0, abs(z))
    assert np.min(np.abs(D.eigs)) >= np.max(np.abs(rest)) - 1e-9


def test_deflation_from_products_equals_dense():
    """The product-only deflation (ARPACK eigs + modified Gram-Schmidt, Section 5) gives the
    same preconditioner as the dense eigendecomposition: P^-1 depends only on the span of
    the r eigenvectors, and the eigenvalues agree."""
    n, h = 10, 0.1
    eps = W.core_shell(n, side=1.0, r_core=0.2, r_shell=0.45, eps_core=-16 + 1.5j, eps_shell=16).eps_r
    At = dense.dense_AR(eps, h) @ dense.dense_A(eps, h)
    r = 8
    D = deflation.Deflation(At, r)
    Dp = deflation.Deflation.from_operator(lambda v: dense.matvec(At, v), (2, n, n), r, tol=1e-13)
    assert np.allclose(Dp.V.conj().T @ Dp.V, np.eye(r), atol=1e-12)
    assert np.max(np.abs(Dp.eigs - D.eigs)) < 1e-9 * abs(D.eigs[0])
    assert np.max(np.abs(Dp.matrix() - D.matrix())) < 1e-8


def test_negative_core_segment_image_reaches_the_origin():
    """Why restarted GMRES stalls on the core-shell object: the essential spectrum of A
    contains the segment [1, eps] of every permittivity value (Eq. (3.20)); for the
    plasma-like core eps = -2 + 0.1i that segment passes within |Im eps| / 3 = 0.0333 of
    the origin, and its image under the regularised map of Eq. (5.3) passes closer still
    (0.0167), because the map fixes 0.  The shell eps = 20 + 0.5i maps into the disc of
    the deflation radius 5.514, so only eigenvalues beyond it are discrete outliers.
    The discrete spectrum of a small grid already shows the small eigenvalues."""
    e = -2 + 0.1j
    t = np.linspace(0.0, 1.0, 200001)
    seg = 1.0 + t * (e - 1.0)
    assert np.min(np.abs(seg)) == pytest.approx(0.1 / abs(e - 1.0) * 1.0, rel=1e-3)
    img = deflation.regularized_eig_map(seg, e)
    assert np.min(np.abs(img)) < 0.0168 and np.min(np.abs(img)) > 0.0166
    p = W.config2(512)
    R = deflation.deflation_radius(np.unique(p.eps_r))
    # close to the lossless closed form 1 + (eps - 1)^2 / (4 eps) at eps = 20 (Section 5)
    assert R == pytest.approx(1.0 + 19.0 ** 2 / 80.0, abs=2e-3)
    q = W.config2(24)
    lam = np.linalg.eigvals(dense.dense_AR(q.eps_r, q.h) @ dense.dense_A(q.eps_r, q.h))
    assert np.min(np.abs(lam)) < 0.05
