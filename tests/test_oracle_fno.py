"""Pins for the oracle's Fourier neural operator (the learned preconditioner's reference)."""
import math

import numpy as np
import pytest

from oracle import fno


def _net(seed=0, H=6, W=8, c_in=6, c_out=4, width=4, modes=2, layers=2, hidden=5):
    rng = np.random.default_rng(seed)
    p = fno.init_params(rng, c_in, c_out, width, modes, layers, hidden)
    x = rng.standard_normal((c_in, H, W))
    return rng, p, x


def _brute_spectral_conv(h, R1, R2, m):
    """The definition with explicit DFT sums: X_k = sum_n h_n e^{-i theta_k n} on the kept
    modes, Y = sum_i X R, and y_n = (1/HW) sum_k c(k2) Re(Y_k e^{i theta_k n})."""
    C_in, H, W = h.shape
    C_out = R1.shape[1]
    n1, n2 = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    y = np.zeros((C_out, H, W))
    kept = [(k1, k2, R1[:, :, k1, k2]) for k1 in range(m) for k2 in range(m)]
    kept += [(H - m + j, k2, R2[:, :, j, k2]) for j in range(m) for k2 in range(m)]
    for k1, k2, R in kept:
        e = np.exp(2j * math.pi * (k1 * n1 / H + k2 * n2 / W))
        X = np.array([np.sum(h[i] * np.conj(e)) for i in range(C_in)])
        Y = X @ R
        c = 1.0 if k2 == 0 or 2 * k2 == W else 2.0
        for o in range(C_out):
            y[o] += c * np.real(Y[o] * e) / (H * W)
    return y


def test_spectral_conv_is_the_truncated_dft_definition():
    rng = np.random.default_rng(1)
    h = rng.standard_normal((3, 6, 8))
    R1 = rng.standard_normal((3, 2, 2, 2)) + 1j * rng.standard_normal((3, 2, 2, 2))
    R2 = rng.standard_normal((3, 2, 2, 2)) + 1j * rng.standard_normal((3, 2, 2, 2))
    got = fno.spectral_conv(h, R1, R2, 2)
    assert np.allclose(got, _brute_spectral_conv(h, R1, R2, 2), rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("k1", [1, 7])          # a mode of the R1 block and one of the R2 block
def test_single_mode_closed_form(k1):
    """h = cos(theta_k . n) for one kept mode k = (k1, k2) with k2 > 0 and weight r on that
    mode only: K h = |r| cos(theta_k . n + arg r) (the rfft2 half keeps k, not -k)."""
    H, W, m, k2 = 8, 8, 2, 1
    n1, n2 = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    theta = 2 * math.pi * (k1 * n1 / H + k2 * n2 / W)
    h = np.cos(theta)[None]
    r = 0.7 - 1.3j
    R1 = np.zeros((1, 1, m, m), np.complex128)
    R2 = np.zeros((1, 1, m, m), np.complex128)
    if k1 < m:
        R1[0, 0, k1, k2] = r
    else:
        R2[0, 0, k1 - (H - m), k2] = r
    y = fno.spectral_conv(h, R1, R2, m)[0]
    assert np.allclose(y, abs(r) * np.cos(theta + np.angle(r)), atol=1e-13)


def test_periodic_shift_equivariance():
    """Every stage is pointwise or a periodic convolution, so shifts commute with the net."""
    _, p, x = _net(2, H=8, W=8)
    y, _ = fno.forward(p, x)
    ys, _ = fno.forward(p, np.roll(x, (3, 5), axis=(1, 2)))
    assert np.allclose(ys, np.roll(y, (3, 5), axis=(1, 2)), rtol=1e-12, atol=1e-12)


def test_zero_spectral_weights_give_a_pointwise_network():
    """With R = 0 the operator is the same small MLP applied at every grid point."""
    _, p, x = _net(3)
    for l in range(p["layers"]):
        p[f"R1_{l}"][:] = 0
        p[f"R2_{l}"][:] = 0
    y, _ = fno.forward(p, x)
    from scipy.special import erf
    g = lambda t: 0.5 * t * (1 + erf(t / math.sqrt(2)))      # GELU from erf
    for i, j in [(0, 0), (2, 5), (5, 7)]:
        v = p["P"] @ x[:, i, j] + p["p"]
        for l in range(p["layers"]):
            v = p[f"W{l}"] @ v + p[f"w{l}"]
            if l < p["layers"] - 1:
                v = g(v)
        out = p["Q2"] @ g(p["Q1"] @ v + p["q1"]) + p["q2"]
        assert np.allclose(y[:, i, j], out, rtol=1e-12, atol=1e-13)


def test_gradients_match_central_differences():
    """Every parameter (real and imaginary parts of the spectral weights) and the input:
    the hand-derived backward pass against central differences of L = <g, y>."""
    rng, p, x = _net(4)
    gy = rng.standard_normal(fno.forward(p, x)[0].shape)
    loss = lambda pp, xx: float(np.sum(gy * fno.forward(pp, xx)[0]))
    _, tape = fno.forward(p, x)
    grads = fno.backward(p, tape, gy)
    eps = 1e-6
    names = [k for k in p if k not in ("layers", "modes")] + ["x"]
    for name in names:
        arr = x if name == "x" else p[name]
        g = grads[name]
        idx = [tuple(rng.integers(0, s) for s in arr.shape) for _ in range(4)]
        for ix in idx:
            for part in ((1.0,) if not np.iscomplexobj(arr) else (1.0, 1j)):
                old = arr[ix]
                arr[ix] = old + eps * part
                lp = loss(p, x)
                arr[ix] = old - eps * part
                lm = loss(p, x)
                arr[ix] = old
                fd = (lp - lm) / (2 * eps)
                an = g[ix].real if part == 1.0 else g[ix].imag
                assert abs(fd - an) <= 1e-6 * max(1.0, abs(fd)), (name, ix, part, fd, an)


def test_modes_must_fit_the_grid():
    h = np.zeros((1, 6, 8))
    R = np.zeros((1, 1, 4, 4), np.complex128)
    with pytest.raises(ValueError):
        fno.spectral_conv(h, R, R, 4)           # 2 m > H
