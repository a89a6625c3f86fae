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
