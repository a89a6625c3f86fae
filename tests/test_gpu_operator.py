"""GPU parity of the FFT-speed products with the CPU oracle (through the C ABI).

Every comparison checks the whole vector twice: in the 2-norm, ||y - y_ref|| / ||y_ref||,
and element by element, max |y - y_ref| / max |y_ref| (a padding, crop or edge-row
mistake confined to a few cells fails the second even where the norm hides it).

Tolerances: FP64 products within 1e-10 in both measures (the FP64 gate).  Complex64
products within 2e-5 in the norm and 5e-5 per element (relative to the largest
entry): single-precision rounding (6e-8) grows like the number of radix stages and the
Green-spectrum dynamic range over two FFT passes per direction, and one element's
error can exceed the root-mean-square error by a small factor.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import dense, fftmv, rows  # noqa: E402
from paper_1104_4263_gb300 import die, workloads as W  # noqa: E402

FP64_TOL = 1e-10
C64_TOL = 2e-5
C64_ELEM_TOL = 5e-5


def rel(a, b):
    """Relative 2-norm error; also asserts the element-wise bound of the same precision
    (FP64 when a is complex128, complex64 otherwise), so that every norm check below is
    accompanied by an element-by-element one."""
    a = np.asarray(a)
    e = float(np.max(np.abs(a - b)) / np.max(np.abs(b)))
    assert e < (FP64_TOL if a.dtype == np.complex128 else C64_ELEM_TOL), ("element-wise", e)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def dev(x, dtype=torch.complex128):
    return torch.from_numpy(np.ascontiguousarray(x)).to(dtype).cuda()


# grids: tiny, ragged (odd, non-square), a 3*2^a FFT size (n=33 -> M=96 is 3*32), n=61
CASES = [(2, 2), (5, 3), (16, 16), (12, 7), (33, 20), (24, 33), (61, 9)]


@pytest.mark.parametrize("n1,n2", CASES)
def test_apply_matches_dense(n1, n2):
    rng = W.rng_for(100, n1 * 1000 + n2)
    eps = W.random_field(rng, n1, n2, -4.0, 16.0)
    h = 0.8 / max(n1, n2)
    x = W.random_vector(rng, n1, n2)
    A = dense.dense_A(eps, h)
    AR = dense.dense_AR(eps, h)
    op = die.Operator(eps, h)
    xt = dev(x)
    assert rel(op.apply(xt).cpu().numpy(), dense.matvec(A, x)) < FP64_TOL
    assert rel(op.apply_regularized(xt).cpu().numpy(), dense.matvec(AR @ A, x)) < FP64_TOL
    assert rel(op.apply_regularizer(xt).cpu().numpy(), dense.matvec(AR, x)) < FP64_TOL
    op32 = die.Operator(eps, h, prec=die.DIE_FP32_INNER)
    x32 = dev(x, torch.complex64)
    assert rel(op32.apply(x32).cpu().numpy(), dense.matvec(A, x)) < C64_TOL
    assert rel(op32.apply_regularized(x32).cpu().numpy(), dense.matvec(AR @ A, x)) < C64_TOL


@pytest.mark.parametrize("n1,n2,M", [(40, 40, (96, 96)), (40, 40, (96, 128)), (50, 30, (192, 64))])
def test_apply_explicit_fft_sizes(n1, n2, M):
    rng = W.rng_for(101, n1 + n2)
    eps = W.random_field(rng, n1, n2)
    h = 0.02
    x = W.random_vector(rng, n1, n2)
    ref = fftmv.FFTOperator(eps, h)
    op = die.Operator(eps, h, M1=M[0], M2=M[1])
    assert (op.M1, op.M2) == M
    xt = dev(x)
    assert rel(op.apply(xt).cpu().numpy(), ref.apply(x)) < FP64_TOL
    assert rel(op.apply_regularized(xt).cpu().numpy(), ref.apply_regularized(x)) < FP64_TOL


@pytest.mark.parametrize("n", [64, 96, 128, 200, 256])
def test_apply_matches_fft_oracle(n):
    p = W.core_shell(n, side=n / 64.0, r_core=1.5 * n / 512, r_shell=2.5 * n / 512)
    rng = W.rng_for(102, n)
    x = W.random_vector(rng, n, n)
    ref = fftmv.FFTOperator(p.eps_r, p.h)
    op = die.Operator(p.eps_r, p.h)
    xt = dev(x)
    assert rel(op.apply(xt).cpu().numpy(), ref.apply(x)) < FP64_TOL
    assert rel(op.apply_regularized(xt).cpu().numpy(), ref.apply_regularized(x)) < FP64_TOL
    op32 = die.Operator(p.eps_r, p.h, prec=die.DIE_FP32_INNER)
    assert rel(op32.apply_regularized(dev(x, torch.complex64)).cpu().numpy(), ref.apply_regularized(x)) < C64_TOL


# Grids with n = M/2 and M = 2^a >= 256 along a direction take the compile-time FFT
# kernels there; these mix them with the general kernels in the other direction.
@pytest.mark.parametrize("n1,n2", [(128, 200), (200, 128), (256, 64), (128, 1024)])
def test_apply_mixed_fast_and_general_passes(n1, n2):
    rng = W.rng_for(105, n1 * 10000 + n2)
    eps = W.random_field(rng, n1, n2, lo=1.0, hi=9.0, loss=0.5)
    h = 2.0 / max(n1, n2)
    x = W.random_vector(rng, n1, n2)
    ref = fftmv.FFTOperator(eps, h)
    op = die.Operator(eps, h)
    xt = dev(x)
    assert rel(op.apply(xt).cpu().numpy(), ref.apply(x)) < FP64_TOL
    assert rel(op.apply_regularized(xt).cpu().numpy(), ref.apply_regularized(x)) < FP64_TOL
    op32 = die.Operator(eps, h, prec=die.DIE_FP32_INNER)
    x32 = dev(x, torch.complex64)
    assert rel(op32.apply(x32).cpu().numpy(), ref.apply(x)) < C64_TOL
    assert rel(op32.apply_regularized(x32).cpu().numpy(), ref.apply_regularized(x)) < C64_TOL


@pytest.mark.parametrize("n", [1024, 2048])
def test_large_grids_match_fft_oracle(n):
    """The compile-time kernels at L = 2048 and 4096 (the largest transform)."""
    p = W.core_shell(n, side=n / 64.0, r_core=1.5 * n / 512, r_shell=2.5 * n / 512)
    rng = W.rng_for(106, n)
    x = W.random_vector(rng, n, n)
    ref = fftmv.FFTOperator(p.eps_r, p.h, workers=8)
    yr = ref.apply_regularized(x)
    op = die.Operator(p.eps_r, p.h)
    assert rel(op.apply_regularized(dev(x)).cpu().numpy(), yr) < FP64_TOL
    del op
    op32 = die.Operator(p.eps_r, p.h, prec=die.DIE_FP32_INNER)
    assert rel(op32.apply_regularized(dev(x, torch.complex64)).cpu().numpy(), yr) < C64_TOL


@pytest.mark.parametrize("n1,n2,prec", [(512, 512, "c64"), (256, 256, "c128"), (128, 200, "c128"), (33, 20, "c64")])
def test_apply_batch_equals_single_products(n1, n2, prec):
    """Batched products (one launch per pass over all right-hand sides) are bit-identical
    to one product per vector, for both the compile-time and the general FFT passes."""
    rng = W.rng_for(107, n1 * 10000 + n2)
    eps = W.random_field(rng, n1, n2, lo=1.0, hi=9.0, loss=0.5)
    h = 2.0 / max(n1, n2)
    op = die.Operator(eps, h, prec=die.DIE_FP64 if prec == "c128" else die.DIE_FP32_INNER)
    dt = torch.complex128 if prec == "c128" else torch.complex64
    X = torch.stack([dev(W.random_vector(rng, n1, n2), dt) for _ in range(5)])
    for reg in (False, True):
        Y = op.apply_batch(X, regularized=reg)
        for k in range(5):
            yk = op.apply_regularized(X[k].clone()) if reg else op.apply(X[k].clone())
            assert torch.equal(Y[k], yk)
    Yi = X.clone()
    op.apply_batch(Yi, Yi, regularized=True)
    assert torch.equal(Yi, op.apply_batch(X, regularized=True))


def test_in_place_apply():
    p = W.config1(16)
    rng = W.rng_for(103)
    x = W.random_vector(rng, 16, 16)
    op = die.Operator(p.eps_r, p.h)
    xt = dev(x)
    ref = op.apply_regularized(xt).clone()
    op.apply_regularized(xt, xt)
    assert torch.equal(xt, ref)


def test_plane_wave_matches_oracle():
    op = die.Operator(np.ones((9, 13), dtype=complex), 0.07)
    for psi in (0.0, 0.3, 2.0, -1.0):
        b = op.plane_wave(psi).cpu().numpy()
        assert np.max(np.abs(b - dense.plane_wave(13, 9, 0.07, psi))) < 1e-12


def test_full_size_core_shell_512():
    """512^2 core-shell workload: the whole product against the (pinned) CPU FFT oracle,
    and 64 seeded rows against exact dense sums."""
    p = W.config2(512)
    rng = W.rng_for(104)
    x = W.random_vector(rng, 512, 512)
    op = die.Operator(p.eps_r, p.h)
    y = op.apply(dev(x)).cpu().numpy()
    ref = fftmv.FFTOperator(p.eps_r, p.h, workers=8)
    assert rel(y, ref.apply(x)) < FP64_TOL
    idx = rng.choice(2 * 512 * 512, size=64, replace=False)
    got = y.reshape(-1)[idx]
    exact = rows.rows_apply(dense.contrast(p.eps_r), x, p.h, idx)
    assert np.max(np.abs(got - exact)) / np.max(np.abs(y)) < FP64_TOL
    yr = op.apply_regularized(dev(x)).cpu().numpy()
    yref = ref.apply_regularized(x)
    assert rel(yr, yref) < FP64_TOL
    op32 = die.Operator(p.eps_r, p.h, prec=die.DIE_FP32_INNER)
    assert rel(op32.apply_regularized(dev(x, torch.complex64)).cpu().numpy(), yref) < C64_TOL


def test_singular_permittivity_rejected():
    eps = np.full((8, 8), 4.0 + 0j)
    eps[3, 5] = 0.0
    with pytest.raises(die.DieError) as e:
        die.Operator(eps, 0.1)
    assert e.value.code == 4
    eps[3, 5] = np.nan
    with pytest.raises(die.DieError):
        die.Operator(eps, 0.1)


def test_eps_on_device_matches_host():
    p = W.config1(20)
    rng = W.rng_for(105)
    x = dev(W.random_vector(rng, 20, 20))
    a = die.Operator(p.eps_r, p.h).apply(x)
    b = die.Operator(torch.from_numpy(p.eps_r).cuda(), p.h).apply(x)
    assert torch.equal(a, b)


def _edge_inputs(n1, n2, rng):
    """Inputs that reach the grid's edges and the padding boundary: non-zero only on the
    last row (x2 = n2 - 1) and the last column (x1 = n1 - 1) of both components, a single
    hot cell in the far corner of component 2, and a single hot cell in the middle of
    component 1."""
    out = []
    x = np.zeros((2, n2, n1), dtype=np.complex128)
    x[:, n2 - 1, :] = rng.standard_normal((2, n1)) + 1j * rng.standard_normal((2, n1))
    x[:, :, n1 - 1] = rng.standard_normal((2, n2)) + 1j * rng.standard_normal((2, n2))
    out.append(("last row and column", x))
    x = np.zeros((2, n2, n1), dtype=np.complex128)
    x[1, n2 - 1, n1 - 1] = 1.0 - 0.5j
    out.append(("corner cell", x))
    x = np.zeros((2, n2, n1), dtype=np.complex128)
    x[0, n2 // 2, n1 // 2] = 0.25 + 1.0j
    out.append(("middle cell", x))
    return out


@pytest.mark.parametrize("n1,n2", [(12, 7), (33, 20), (61, 9)])
def test_edge_and_hot_cell_inputs_dense(n1, n2):
    """Edge rows/columns and single hot cells against the dense oracle, element by element."""
    rng = W.rng_for(108, n1 * 1000 + n2)
    eps = W.random_field(rng, n1, n2, -4.0, 16.0)
    h = 0.8 / max(n1, n2)
    A = dense.dense_A(eps, h)
    AR = dense.dense_AR(eps, h)
    op = die.Operator(eps, h)
    op32 = die.Operator(eps, h, prec=die.DIE_FP32_INNER)
    for name, x in _edge_inputs(n1, n2, rng):
        ya, yr = dense.matvec(A, x), dense.matvec(AR @ A, x)
        assert rel(op.apply(dev(x)).cpu().numpy(), ya) < FP64_TOL, name
        assert rel(op.apply_regularized(dev(x)).cpu().numpy(), yr) < FP64_TOL, name
        assert rel(op32.apply(dev(x, torch.complex64)).cpu().numpy(), ya) < C64_TOL, name
        assert rel(op32.apply_regularized(dev(x, torch.complex64)).cpu().numpy(), yr) < C64_TOL, name


@pytest.mark.parametrize("n", [128, 512])
def test_edge_and_hot_cell_inputs_fast_path(n):
    """The same inputs on grids of the compile-time FFT kernels (n = M / 2), against the
    pinned FFT oracle, element by element."""
    p = W.core_shell(n, side=n / 64.0, r_core=1.5 * n / 512, r_shell=2.5 * n / 512)
    rng = W.rng_for(109, n)
    ref = fftmv.FFTOperator(p.eps_r, p.h, workers=8)
    op = die.Operator(p.eps_r, p.h)
    op32 = die.Operator(p.eps_r, p.h, prec=die.DIE_FP32_INNER)
    for name, x in _edge_inputs(n, n, rng):
        ya, yr = ref.apply(x), ref.apply_regularized(x)
        assert rel(op.apply(dev(x)).cpu().numpy(), ya) < FP64_TOL, name
        assert rel(op.apply_regularized(dev(x)).cpu().numpy(), yr) < FP64_TOL, name
        assert rel(op32.apply(dev(x, torch.complex64)).cpu().numpy(), ya) < C64_TOL, name
        assert rel(op32.apply_regularized(dev(x, torch.complex64)).cpu().numpy(), yr) < C64_TOL, name


def test_set_permittivity_equals_fresh_operator():
    """dieop_set_permittivity: the products of an operator given a new map equal those of an
    operator created with it (bit for bit: same Green spectra, same contrasts); a deflation
    handle of the old map is rejected; a map violating the existence condition is refused
    and leaves the previous one in place."""
    rng = W.rng_for(140)
    e1 = W.random_field(rng, 40, 33, 1.0, 9.0)
    e2 = W.random_field(rng, 40, 33, -4.0, 16.0)
    h = 0.03
    op = die.Operator(e1, h)
    D = die.Deflation(op, 4, tol=1e-4, regularized=True)
    x = dev(W.random_vector(rng, 40, 33))
    op.set_permittivity(e2)
    fresh = die.Operator(e2, h)
    assert torch.equal(op.apply(x), fresh.apply(x))
    assert torch.equal(op.apply_regularized(x), fresh.apply_regularized(x))
    with pytest.raises(die.DieError):
        op.solve(op.plane_wave(0.0), regularized=True, deflation=D, max_iters=5)
    bad = e2.copy()
    bad[3, 4] = 0.0
    with pytest.raises(die.DieError) as e:
        op.set_permittivity(bad)
    assert e.value.code == 4
    assert torch.equal(op.apply(x), fresh.apply(x))
    op.set_permittivity(torch.from_numpy(e1).cuda())
    assert torch.equal(op.apply(x), die.Operator(e1, h).apply(x))
