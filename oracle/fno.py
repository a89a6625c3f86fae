"""Fourier neural operator: reference forward and backward passes in float64.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  The learned right preconditioner of
the flexible GMRES solves is a Fourier neural operator as defined by Li, Kovachki,
Azizzadenesheli, Liu, Bhattacharya, Stuart and Anandkumar, "Fourier neural operator for
parametric partial differential equations" (ICLR 2021).  Restated on an H x W periodic
grid with real channels:

  lifting     h_0     = P x + p                         pointwise affine, C_in -> C
  layer l     a_l     = W_l h_l + w_l + K_l h_l
              h_{l+1} = GELU(a_l), except after the last layer (h_L = a_{L-1})
  projection  y       = Q2 GELU(Q1 h_L + q1) + q2       pointwise, C -> hidden -> C_out

The spectral convolution K of a layer, per input channel i and output channel o:
  X = rfft2(h)                        (half spectrum, k2 = 0 .. W/2)
  Y[o, k] = sum_i X[i, k] R[i, o, k]  for the kept modes k = (k1, k2), k2 in [0, m) and
            k1 in [0, m) (weights R1) or k1 in [H - m, H) (weights R2); Y = 0 elsewhere
  K h = irfft2(Y)
GELU(x) = x Phi(x), Phi the standard normal distribution function.

The backward pass is derived by hand.  irfft2 of a half spectrum is the real-linear map
  y[n] = (1 / HW) sum_k c(k2) Re(Y_k exp(i theta_k . n)),  c = 1 for k2 in {0, W/2}, else 2,
so the gradient of <g, y> with respect to Y_k (d/dRe + i d/dIm) is c(k2) rfft2(g)_k / HW.
For a complex product Y = a b the gradients are G conj(b) (for a) and G conj(a) (for b).
rfft2 of real h restricted to the kept modes has the adjoint  h -> HW Re(ifft2(D)),  with
D the mode gradients placed in a full H x W spectrum and zeros elsewhere.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import ndtr

_SQRT_2PI = math.sqrt(2.0 * math.pi)


def gelu(x):
    return x * ndtr(x)


def gelu_grad(x):
    return ndtr(x) + x * np.exp(-0.5 * x * x) / _SQRT_2PI


def init_params(rng: np.random.Generator, c_in: int, c_out: int, width: int, modes: int, layers: int,
                hidden: int) -> dict:
    """Random parameters of the shapes above (scaled so that activations stay O(1))."""
    def lin(o, i):
        return rng.standard_normal((o, i)) / math.sqrt(i), 0.1 * rng.standard_normal(o)

    p = {}
    p["P"], p["p"] = lin(width, c_in)
    for l in range(layers):
        p[f"W{l}"], p[f"w{l}"] = lin(width, width)
        s = 1.0 / width
        for name in (f"R1_{l}", f"R2_{l}"):
            p[name] = s * (rng.standard_normal((width, width, modes, modes))
                           + 1j * rng.standard_normal((width, width, modes, modes)))
    p["Q1"], p["q1"] = lin(hidden, width)
    p["Q2"], p["q2"] = lin(c_out, hidden)
    p["layers"] = layers
    p["modes"] = modes
    return p


def _check_modes(H: int, W: int, m: int):
    if not (1 <= m and 2 * m <= H and m <= W // 2):
        raise ValueError("modes must satisfy 2 m <= H and m <= W / 2")


def spectral_conv(h: np.ndarray, R1: np.ndarray, R2: np.ndarray, m: int) -> np.ndarray:
    """K h for h of shape (C_in, H, W); R1, R2 of shape (C_in, C_out, m, m)."""
    _, H, W = h.shape
    _check_modes(H, W, m)
    X = np.fft.rfft2(h, axes=(1, 2))
    Y = np.zeros((R1.shape[1], H, W // 2 + 1), dtype=np.complex128)
    Y[:, :m, :m] = np.einsum("ixy,ioxy->oxy", X[:, :m, :m], R1)
    Y[:, H - m:, :m] = np.einsum("ixy,ioxy->oxy", X[:, H - m:, :m], R2)
    return np.fft.irfft2(Y, s=(H, W), axes=(1, 2))


def spectral_conv_backward(g: np.ndarray, h: np.ndarray, R1: np.ndarray, R2: np.ndarray, m: int):
    """Gradients of <g, K h> with respect to h (real) and R1, R2 (d/dRe + i d/dIm)."""
    _, H, W = h.shape
    X = np.fft.rfft2(h, axes=(1, 2))
    c = np.full(W // 2 + 1, 2.0)
    c[0] = 1.0
    if W % 2 == 0:
        c[W // 2] = 1.0
    G = np.fft.rfft2(g, axes=(1, 2)) * (c / (H * W))
    G1, G2 = G[:, :m, :m], G[:, H - m:, :m]
    X1, X2 = X[:, :m, :m], X[:, H - m:, :m]
    dR1 = np.einsum("oxy,ixy->ioxy", G1, np.conj(X1))
    dR2 = np.einsum("oxy,ixy->ioxy", G2, np.conj(X2))
    D = np.zeros((h.shape[0], H, W), dtype=np.complex128)
    D[:, :m, :m] = np.einsum("oxy,ioxy->ixy", G1, np.conj(R1))
    D[:, H - m:, :m] = np.einsum("oxy,ioxy->ixy", G2, np.conj(R2))
    dh = H * W * np.real(np.fft.ifft2(D, axes=(1, 2)))
    return dh, dR1, dR2


def _affine(A, a, h):
    return np.einsum("oi,ihw->ohw", A, h) + a[:, None, None]


def forward(p: dict, x: np.ndarray):
    """Output y (C_out, H, W) for input x (C_in, H, W), and the tape for `backward`."""
    L, m = p["layers"], p["modes"]
    tape = {"x": x}
    h = _affine(p["P"], p["p"], x)
    for l in range(L):
        tape[f"h{l}"] = h
        a = _affine(p[f"W{l}"], p[f"w{l}"], h) + spectral_conv(h, p[f"R1_{l}"], p[f"R2_{l}"], m)
        tape[f"a{l}"] = a
        h = gelu(a) if l < L - 1 else a
    tape["hL"] = h
    u = _affine(p["Q1"], p["q1"], h)
    tape["u"] = u
    y = _affine(p["Q2"], p["q2"], gelu(u))
    return y, tape


def _affine_backward(A, h, d):
    return np.einsum("ohw,ihw->oi", d, h), d.sum(axis=(1, 2)), np.einsum("oi,ohw->ihw", A, d)


def backward(p: dict, tape: dict, gy: np.ndarray) -> dict:
    """Gradients of <gy, forward(p, x)> with respect to every parameter and to x ("x")."""
    L, m = p["layers"], p["modes"]
    grads = {}
    s = gelu(tape["u"])
    grads["Q2"], grads["q2"], ds = _affine_backward(p["Q2"], s, gy)
    du = ds * gelu_grad(tape["u"])
    grads["Q1"], grads["q1"], dh = _affine_backward(p["Q1"], tape["hL"], du)
    for l in reversed(range(L)):
        da = dh * gelu_grad(tape[f"a{l}"]) if l < L - 1 else dh
        h = tape[f"h{l}"]
        grads[f"W{l}"], grads[f"w{l}"], dh_lin = _affine_backward(p[f"W{l}"], h, da)
        dh_sp, grads[f"R1_{l}"], grads[f"R2_{l}"] = spectral_conv_backward(da, h, p[f"R1_{l}"], p[f"R2_{l}"], m)
        dh = dh_lin + dh_sp
    grads["P"], grads["p"], grads["x"] = _affine_backward(p["P"], tape["x"], dh)
    return grads
