"""The TM (E-wave) variant on the GPU against the TM oracle (oracle/tm.py), through the C
ABI: products (element by element), the plane wave, a solve to the FP64 gate, the
deflation of Eq. (4.12) and the closed-form cylinder.  A TM field is the first plane of
the two-plane layout; the second plane is zero and must stay exactly zero."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import tm  # noqa: E402
from paper_1104_4263_gb300 import die, workloads as W  # noqa: E402


def _field(e3):
    return torch.from_numpy(np.stack([e3, np.zeros_like(e3)])).cuda()


def _elem(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.mark.parametrize("n1,n2", [(12, 7), (33, 20), (64, 64), (128, 128)])
def test_tm_product_matches_dense(n1, n2):
    rng = W.rng_for(130, n1 * 1000 + n2)
    eps = W.random_field(rng, n1, n2, -4.0, 16.0)
    h = 0.8 / max(n1, n2)
    x = rng.standard_normal((n2, n1)) + 1j * rng.standard_normal((n2, n1))
    ref = (tm.dense_A(eps, h) @ x.reshape(-1)).reshape(n2, n1)
    op = die.Operator(eps, h, pol=die.DIE_TM)
    y = op.apply(_field(x)).cpu().numpy()
    assert _elem(y[0], ref) < 1e-10
    assert np.all(y[1] == 0)
    op32 = die.Operator(eps, h, pol=die.DIE_TM, prec=die.DIE_FP32_INNER)
    y32 = op32.apply(_field(x).to(torch.complex64)).cpu().numpy()
    assert _elem(y32[0], ref) < 5e-5 and np.all(y32[1] == 0)


def test_tm_plane_wave():
    op = die.Operator(np.ones((9, 13), dtype=complex), 0.07, pol=die.DIE_TM)
    for psi in (0.0, 0.9, -2.3):
        b = op.plane_wave(psi).cpu().numpy()
        assert np.max(np.abs(b[0] - tm.plane_wave(13, 9, 0.07, psi))) < 1e-12 and np.all(b[1] == 0)


def test_tm_solve_fp64_gate_and_series():
    """The config-1 cylinder in TM: GMRES(20) to 1e-13 equals the dense direct solve to
    1e-10 relative (element by element too); against the closed form the error is that of
    the discretisation (oracle pin: below 0.2 at 32^2)."""
    p = W.config1(32)
    A = tm.dense_A(p.eps_r, p.h)
    b = tm.plane_wave(32, 32, p.h, 0.0)
    xd = np.linalg.solve(A, b.reshape(-1)).reshape(32, 32)
    op = die.Operator(p.eps_r, p.h, pol=die.DIE_TM)
    u, rep = op.solve(op.plane_wave(0.0), restart=20, tol=1e-13, max_iters=40000)
    assert rep["converged"]
    ug = u.cpu().numpy()
    assert np.all(ug[1] == 0)
    assert np.linalg.norm(ug[0] - xd) / np.linalg.norm(xd) < 1e-10 and _elem(ug[0], xd) < 1e-10
    X1, X2 = W.mesh(32, 32, p.h)
    ser = tm.cylinder_field(4.0, 1.0, X1, X2, 0.0)
    assert np.linalg.norm(ug[0] - ser) / np.linalg.norm(ser) < 0.2


def test_tm_deflation():
    """Deflating the r largest-magnitude TM eigenvalues (Eq. (4.12), Table 1's method): the
    eigenvalues equal the dense ones, the basis lies in the first plane, and the deflated
    solve reaches the direct solution."""
    n = 16
    eps = W.core_shell(n, side=1.0, r_core=0.2, r_shell=0.45, eps_core=2.5 + 20j, eps_shell=16.0).eps_r
    h = 1.0 / n
    A = tm.dense_A(eps, h)
    lam = np.linalg.eigvals(A)
    lam = lam[np.argsort(-np.abs(lam))]
    op = die.Operator(eps, h, pol=die.DIE_TM)
    r = 6
    D = die.Deflation(op, r, tol=1e-10, regularized=False)
    assert D.converged and D.r == r
    for z in lam[:r]:
        assert np.min(np.abs(D.eigenvalues - z)) < 1e-7 * abs(z)
    x = torch.zeros((2, n, n), dtype=torch.complex128, device="cuda")
    x[0] = torch.randn((n, n), dtype=torch.complex128)
    assert bool((D.apply(x)[1] == 0).all())
    b = op.plane_wave(0.4)
    xd = np.linalg.solve(A, b.cpu().numpy()[0].reshape(-1))
    u, rep = op.solve(b, restart=40, tol=1e-10, max_iters=20000, deflation=D)
    assert rep["converged"], rep
    assert np.linalg.norm(u.cpu().numpy()[0].reshape(-1) - xd) / np.linalg.norm(xd) < 1e-7
