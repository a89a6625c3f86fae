"""GPU parity of the TE system with magnetic contrast (DIE_TE_MAG) with oracle/te_mag.py.

Products element by element against the dense 3N oracle (FP64 1e-10, complex64 5e-5 of
the largest entry) on ragged and power-of-two grids, and against exact rows of the
oracle's couplings on a 128^2 grid; the regularised product A(chi'_e, chi_m) A(chi_e, chi_m);
solves against the dense direct solution (FP64 gate 1e-10) and against the closed-form
magneto-dielectric cylinder series; a regularised, deflated FP32-inner solve; without
magnetic contrast the electric planes agree with the two-plane TE operator.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import green, te_mag  # noqa: E402
from paper_1104_4263_gb300 import die, workloads as W  # noqa: E402

K = 2 * math.pi


def elem_rel(a, b):
    return float(np.max(np.abs(np.asarray(a) - b)) / np.max(np.abs(b)))


def maps(n1, n2, seed):
    rng = W.rng_for(31, seed)
    eps = W.random_field(rng, n1, n2, lo=1.0, hi=9.0)
    mu = W.random_field(rng, n1, n2, lo=1.0, hi=4.0, loss=0.3)
    return eps, mu


def field(n1, n2, seed):
    rng = W.rng_for(32, seed)
    return np.stack([W.random_vector(rng, n1, n2)[0] for _ in range(3)])


@pytest.mark.parametrize("n1,n2,h", [(11, 9, 0.07), (16, 16, 0.05), (24, 20, 0.04)])
def test_products_match_dense_oracle(n1, n2, h):
    eps, mu = maps(n1, n2, n1)
    x = field(n1, n2, n2)
    A = te_mag.dense_A(eps, mu, h)
    AR = te_mag.dense_AR(eps, mu, h)
    ref = (A @ x.reshape(-1)).reshape(x.shape)
    refr = (AR @ (A @ x.reshape(-1))).reshape(x.shape)
    op = die.Operator(eps, h, pol=die.DIE_TE_MAG, mu_r=mu)
    xt = torch.from_numpy(x).cuda()
    assert elem_rel(op.apply(xt).cpu().numpy(), ref) < 1e-10
    assert elem_rel(op.apply_regularized(xt).cpu().numpy(), refr) < 1e-10
    op32 = die.Operator(eps, h, pol=die.DIE_TE_MAG, mu_r=mu, prec=die.DIE_FP32_INNER)
    x32 = xt.to(torch.complex64)
    assert elem_rel(op32.apply(x32).cpu().numpy(), ref) < 5e-5
    assert elem_rel(op32.apply_regularized(x32).cpu().numpy(), refr) < 5e-5


def exact_rows(eps, mu, h, x, rows):
    """y at the selected (plane, node) outputs from the oracle's couplings, O(N) each."""
    n2, n1 = eps.shape
    i1 = np.tile(np.arange(n1), n2)
    i2 = np.repeat(np.arange(n2), n1)
    xc = ((np.arange(n1) + 0.5) * h - 0.5 * n1 * h)[i1]
    yc = ((np.arange(n2) + 0.5) * h - 0.5 * n2 * h)[i2]
    chi = [(eps - 1.0).reshape(-1), (eps - 1.0).reshape(-1), (mu - 1.0).reshape(-1)]
    xs = x.reshape(3, -1)
    out = []
    for l, n in rows:
        d1, d2 = xc[n] - xc, yc[n] - yc
        G11, G22, G12 = green.green_tensor(d1, d2, K, h)
        G13, G23, G33 = te_mag.coupling(d1, d2, K, h)
        Gl = ((G11, G12, G13), (G12, G22, G23), (G13, G23, G33))[l]
        out.append(xs[l, n] - sum(np.sum(Gl[q] * chi[q] * xs[q]) for q in range(3)))
    return np.array(out)


def test_sampled_rows_at_128():
    n, h = 128, 1.0 / 40
    eps, mu = maps(n, n, 128)
    x = field(n, n, 128)
    op = die.Operator(eps, h, pol=die.DIE_TE_MAG, mu_r=mu)
    y = op.apply(torch.from_numpy(x).cuda()).cpu().numpy().reshape(3, -1)
    rng = np.random.default_rng(5)
    rows = [(l, int(m)) for l in range(3) for m in rng.integers(0, n * n, 8)] + [(0, 0), (1, n * n - 1), (2, n - 1)]
    ref = exact_rows(eps, mu, h, x, rows)
    got = np.array([y[l, m] for l, m in rows])
    assert np.max(np.abs(got - ref)) < 1e-10 * np.max(np.abs(ref))


def test_electric_planes_agree_with_te_without_magnetic_contrast():
    n1, n2, h = 40, 36, 0.03
    eps, _ = maps(n1, n2, 7)
    x = field(n1, n2, 7)
    mag = die.Operator(eps, h, pol=die.DIE_TE_MAG)            # mu_r = 1
    te = die.Operator(eps, h)
    y3 = mag.apply(torch.from_numpy(x).cuda()).cpu().numpy()
    y2 = te.apply(torch.from_numpy(np.ascontiguousarray(x[:2])).cuda()).cpu().numpy()
    assert elem_rel(y3[:2], y2) < 1e-12


def test_fp64_solve_matches_direct_solution():
    n1, n2, h = 14, 12, 0.06
    eps, mu = maps(n1, n2, 3)
    op = die.Operator(eps, h, pol=die.DIE_TE_MAG, mu_r=mu)
    b = op.plane_wave(0.6)
    ref_b = te_mag.plane_wave(n1, n2, h, 0.6)
    assert elem_rel(b.cpu().numpy(), ref_b) < 1e-14
    x, rep = op.solve(b, restart=60, tol=1e-13, max_iters=5000)
    assert rep["converged"]
    u = np.linalg.solve(te_mag.dense_A(eps, mu, h), ref_b.reshape(-1)).reshape(3, n2, n1)
    assert np.linalg.norm(x.cpu().numpy() - u) / np.linalg.norm(u) < 1e-10


@pytest.mark.parametrize("eps,mu", [(1.0, 4.0), (2.0, 2.0)])
def test_cylinder_solve_matches_series(eps, mu):
    """The GPU solution on the 40^2 grid against the series at the equal-area radius, as
    the oracle's pin (measured there: 2.0% and 6.2%)."""
    n, side, R = 40, 1.25, 0.5
    p = W.cylinder(n, side, R, 2.0)
    mask = p.eps_r != 1.0
    r_eff = math.sqrt(mask.sum() * p.h ** 2 / math.pi)
    op = die.Operator(np.where(mask, eps, 1.0).astype(np.complex128), p.h, pol=die.DIE_TE_MAG,
                      mu_r=np.where(mask, mu, 1.0).astype(np.complex128))
    x, rep = op.solve(op.plane_wave(0.0), restart=80, tol=1e-10, max_iters=20000)
    assert rep["converged"]
    X1, X2 = W.mesh(n, n, p.h)
    ref = np.stack(te_mag.cylinder_field(eps, mu, r_eff, X1, X2, 0.0))
    assert np.linalg.norm(x.cpu().numpy() - ref) / np.linalg.norm(ref) < 0.07


def test_regularised_deflated_mixed_solve():
    """A_R A P^-1 (r = 6, deflation built with complex64 products), FP32-inner GMRES(20) on a
    magneto-dielectric core-shell: converges, and the field matches the FP64 direct solution."""
    n, h = 24, 1.0 / 16
    p = W.core_shell(n, side=n * h, r_core=0.35, r_shell=0.6, eps_core=4.0 + 0.2j, eps_shell=9.0 + 0.3j)
    mu = np.where(np.abs(p.eps_r - 1.0) > 0, 2.0 + 0.1j, 1.0).astype(np.complex128)
    op = die.Operator(p.eps_r, h, pol=die.DIE_TE_MAG, mu_r=mu)
    D = die.Deflation(op, 6, tol=1e-4, regularized=True, inner=die.DIE_FP32_INNER)
    b = op.plane_wave(0.0)
    x, rep = op.solve(b, restart=20, tol=1e-9, max_iters=4000, regularized=True, inner=die.DIE_FP32_INNER,
                      deflation=D)
    assert rep["converged"]
    u = np.linalg.solve(te_mag.dense_A(p.eps_r, mu, h), te_mag.plane_wave(n, n, h, 0.0).reshape(-1))
    assert np.linalg.norm(x.cpu().numpy().reshape(-1) - u) / np.linalg.norm(u) < 1e-6


def test_permeability_errors():
    eps, mu = maps(10, 10, 1)
    te = die.Operator(eps, 0.05)
    with pytest.raises(die.DieError):
        te.set_permeability(mu)
    op = die.Operator(eps, 0.05, pol=die.DIE_TE_MAG, mu_r=mu)
    x = torch.from_numpy(field(10, 10, 1)).cuda()
    y0 = op.apply(x).cpu()
    bad = mu.copy()
    bad[3, 4] = np.nan
    with pytest.raises(die.DieError):
        op.set_permeability(bad)
    assert torch.equal(op.apply(x).cpu(), y0)                  # the previous map is kept
