"""Pins for the oracle's restarted GMRES (P10)."""
import math

import numpy as np
import pytest

from oracle import deflation, dense, fftmv, gmres
from paper_1104_4263_gb300 import workloads as W


def test_full_gmres_is_exact():
    rng = np.random.default_rng(5)
    n = 40
    A = np.eye(n) * 3 + 0.3 * (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / math.sqrt(n)
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    res = gmres.gmres(lambda x: A @ x, b, restart=n, tol=1e-13, max_iters=n)
    assert res.converged and res.iters <= n
    assert np.linalg.norm(res.x - np.linalg.solve(A, b)) / np.linalg.norm(res.x) < 1e-12


def test_distinct_eigenvalue_count():
    """Full GMRES on a diagonalisable matrix with k distinct eigenvalues stops in <= k steps."""
    rng = np.random.default_rng(6)
    vals = np.array([1.0, 2 + 1j, -3.0, 0.5j + 4, 7.0])
    d = np.repeat(vals, 8)
    S = np.eye(40) + 0.1 * rng.standard_normal((40, 40))
    A = S @ np.diag(d) @ np.linalg.inv(S)
    b = rng.standard_normal(40) + 0j
    res = gmres.gmres(lambda x: A @ x, b, restart=40, tol=1e-10, max_iters=40)
    assert res.converged and res.iters <= 5


def test_residual_history_monotone_within_cycle():
    rng = np.random.default_rng(7)
    A = np.eye(60) + 0.9 * rng.standard_normal((60, 60)) / math.sqrt(60)
    b = rng.standard_normal(60) + 0j
    res = gmres.gmres(lambda x: A @ x, b, restart=60, tol=1e-12, max_iters=60)
    h = np.array(res.history)
    assert np.all(np.diff(h) <= 1e-14)


@pytest.fixture(scope="module")
def small_problem():
    n = 10
    eps = W.core_shell(n, side=1.0, r_core=0.2, r_shell=0.42, eps_core=-2 + 0.1j, eps_shell=20 + 0.5j).eps_r
    h = 0.1
    A = dense.dense_A(eps, h)
    AR = dense.dense_AR(eps, h)
    b = dense.plane_wave(n, n, h, 0.0)
    x = np.linalg.solve(A, b.reshape(-1)).reshape(b.shape)
    return eps, h, A, AR, b, x


def test_all_forms_reach_the_same_solution(small_problem):
    """Plain, regularised, deflated and regularised+deflated GMRES agree with the direct solve."""
    eps, h, A, AR, b, x = small_problem
    kappa = np.linalg.cond(A)
    tol = 1e-11
    Ap = lambda v: dense.matvec(A, v)
    Arp = lambda v: dense.matvec(AR @ A, v)
    bR = dense.matvec(AR, b)
    D = deflation.Deflation(AR @ A, 10)
    D0 = deflation.Deflation(A, 10)
    full = b.size                               # restart = 2N: full GMRES, exact in <= 2N steps
    runs = [gmres.gmres(Ap, b, full, tol, full),
            gmres.gmres(Arp, bR, full, tol, full),
            gmres.gmres(Ap, b, full, tol, full, precond=D0.apply),
            gmres.gmres(Arp, bR, 60, tol, 3000, precond=D.apply)]
    for r in runs:
        assert r.converged
        assert np.linalg.norm(r.x - x) / np.linalg.norm(x) < 10 * kappa * tol


def test_exact_preconditioner_converges_in_one_step(small_problem):
    eps, h, A, AR, b, x = small_problem
    Ainv = np.linalg.inv(A)
    res = gmres.gmres(lambda v: dense.matvec(A, v), b, 10, 1e-12, 10,
                      precond=lambda v: dense.matvec(Ainv, v))
    assert res.iters == 1 and res.converged


def test_fft_gmres_matches_dense_gmres():
    p = W.config1(16)
    b = dense.plane_wave(16, 16, p.h, 0.3)
    op = fftmv.FFTOperator(p.eps_r, p.h)
    A = dense.dense_A(p.eps_r, p.h)
    r1 = gmres.gmres(op.apply, b, 20, 1e-10, 3000)
    r2 = gmres.gmres(lambda v: dense.matvec(A, v), b, 20, 1e-10, 3000)
    assert r1.iters == pytest.approx(r2.iters, abs=2)
    assert np.linalg.norm(r1.x - r2.x) / np.linalg.norm(r2.x) < 1e-8


def test_regularised_deflated_beats_plain_under_restart():
    """Sections 4-5: with restart 60 the plain system stalls on a core-shell object while
    A_R A P^-1 converges (the behaviour the paper's Table 2 reports)."""
    n = 12
    eps = W.core_shell(n, side=1.2, r_core=0.25, r_shell=0.5, eps_core=-2 + 0.1j, eps_shell=20 + 0.5j).eps_r
    h = 0.1
    A = dense.dense_A(eps, h)
    AR = dense.dense_AR(eps, h)
    b = dense.plane_wave(n, n, h, 0.0)
    plain = gmres.gmres(lambda v: dense.matvec(A, v), b, 60, 1e-10, 1500)
    D = deflation.Deflation(AR @ A, 10)
    reg = gmres.gmres(lambda v: dense.matvec(AR @ A, v), dense.matvec(AR, b), 60, 1e-10, 1500,
                      precond=D.apply)
    assert not plain.converged and reg.converged and reg.iters < 600


def _random_system(seed, n=48):
    rng = np.random.default_rng(seed)
    A = np.eye(n) * 2 + 0.8 * (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / math.sqrt(n)
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    return rng, A, b


def test_fgmres_with_fixed_preconditioner_is_right_preconditioned_gmres():
    """Flexible GMRES with one linear preconditioner for every step takes the iterates of
    right-preconditioned GMRES (the same Krylov space of A M, the same minimisation)."""
    rng, A, b = _random_system(11)
    Mx = np.eye(48) + 0.3 * rng.standard_normal((48, 48)) / math.sqrt(48)
    kw = dict(restart=7, tol=1e-10, max_iters=400)
    ref = gmres.gmres(lambda x: A @ x, b, precond=lambda v: Mx @ v, **kw)
    got = gmres.fgmres(lambda x: A @ x, b, precond=lambda v, j: Mx @ v, **kw)
    assert (got.iters, got.cycles) == (ref.iters, ref.cycles)
    assert np.allclose(got.history, ref.history, rtol=1e-9, atol=1e-15)
    assert np.linalg.norm(got.x - ref.x) <= 1e-9 * np.linalg.norm(ref.x)
    plain = gmres.gmres(lambda x: A @ x, b, **kw)
    ident = gmres.fgmres(lambda x: A @ x, b, **kw)
    assert ident.iters == plain.iters and np.allclose(ident.x, plain.x, rtol=1e-10, atol=1e-14)


def test_full_fgmres_with_a_nonlinear_preconditioner_is_exact():
    """With a preconditioner that changes every step (here a nonlinear map of v and j) the
    full flexible method still minimises the residual over the span of its z_j: with as
    many steps as unknowns it returns the solution of A x = b."""
    rng, A, b = _random_system(12, n=30)
    B = rng.standard_normal((30, 30)) / math.sqrt(30)

    def nonlinear(v, j):
        return v + 0.2 * np.tanh(np.abs(B @ v)) * v * (1 + 0.1 * j)

    res = gmres.fgmres(lambda x: A @ x, b, restart=30, tol=1e-13, max_iters=30, precond=nonlinear)
    assert res.converged
    assert np.linalg.norm(res.x - np.linalg.solve(A, b)) <= 1e-11 * np.linalg.norm(res.x)
    # the residual estimates are those of the minimisation: non-increasing within the cycle
    assert np.all(np.diff(res.history) <= 1e-14)
    # and the last estimate is the true residual
    assert abs(res.history[-1] - res.rel_res) <= 1e-10
