"""Pins for the oracle's FFT product and sampled-row sums against the dense matrix (P1)."""
import math

import numpy as np
import pytest

from oracle import dense, fftmv, rows
from paper_1104_4263_gb300 import workloads as W

K = 2 * math.pi


@pytest.mark.parametrize("n1,n2,M", [(16, 16, None), (12, 7, None), (9, 10, (24, 27))])
def test_fft_operator_equals_dense(n1, n2, M):
    rng = W.rng_for(90, n1 * 100 + n2)
    eps = W.random_field(rng, n1, n2, -4.0, 16.0)
    h = 0.07
    kw = {} if M is None else {"M1": M[0], "M2": M[1]}
    op = fftmv.FFTOperator(eps, h, **kw)
    A = dense.dense_A(eps, h)
    AR = dense.dense_AR(eps, h)
    x = W.random_vector(rng, n1, n2)
    y = dense.matvec(A, x)
    assert np.linalg.norm(op.apply(x) - y) / np.linalg.norm(y) < 1e-13
    yr = dense.matvec(AR @ A, x)
    assert np.linalg.norm(op.apply_regularized(x) - yr) / np.linalg.norm(yr) < 1e-13


def test_rows_equal_dense():
    rng = W.rng_for(91)
    n1, n2, h = 11, 8, 0.09
    eps = W.random_field(rng, n1, n2)
    x = W.random_vector(rng, n1, n2)
    y = dense.matvec(dense.dense_A(eps, h), x).reshape(-1)
    idx = rng.choice(2 * n1 * n2, size=25, replace=False)
    got = rows.rows_apply(dense.contrast(eps), x, h, idx)
    assert np.max(np.abs(got - y[idx])) / np.max(np.abs(y)) < 1e-13


def test_plane_wave_is_series_with_unit_eps():
    """The incident field equals the cylinder series with eps_r = 1 (no scatterer)."""
    from oracle import cylinder
    n, h = 12, 0.1
    for psi in (0.0, 0.7, 2.5):
        b = dense.plane_wave(n, n, h, psi)
        X1, X2 = W.mesh(n, n, h)
        E1, E2, _ = cylinder.field(1.0, 0.3, X1, X2, psi)
        assert np.max(np.abs(b - np.stack([E1, E2]))) < 1e-10
