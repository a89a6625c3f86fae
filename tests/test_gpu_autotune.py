"""The tile-height schedule of the complex64 row passes (dieop_autotune).

The rows of a row-pass block are independent transforms, each run by the same threads
and stages whatever the block's height, so every schedule must give bit-identical
products: plain and regularised products, batched products, and a deflated FP32-inner
solve (whose first row pass also applies the deflation).  The autotuner must time every
valid height, keep the default unless another height is at least 3% faster, and reuse the
choice for operators of the same sizes.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1104_4263_gb300 import die, workloads as W  # noqa: E402


def heights(n):
    """Valid tile heights for an n x n grid with M1 = 2n (at most 512 threads per block)."""
    L = 2 * n
    return [t for t in (1, 2, 4, 8) if t * (L // 16) <= 512]


def c64_vec(op, seed, nrhs=None):
    rng = W.rng_for(0, seed)
    shape = (2 * op.N,) if nrhs is None else (nrhs, 2 * op.N)
    x = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    return torch.from_numpy(x.astype(np.complex64)).cuda()


@pytest.mark.parametrize("n", [128, 512, 2048])
def test_every_tile_height_gives_identical_products(n):
    p = W.config2(n)
    op = die.Operator(p.eps_r, p.h, prec=die.DIE_FP32_INNER)
    x = c64_vec(op, 1)
    xb = c64_vec(op, 2, nrhs=3).reshape(3, 2, n, n)
    ref = None
    for t in heights(n):
        op.set_tile_rows(t)
        assert op.tile_rows == t
        out = (op.apply(x).cpu(), op.apply_regularized(x).cpu(),
               op.apply_batch(xb, regularized=True).cpu())
        if ref is None:
            ref = out
        else:
            for a, b in zip(out, ref):
                assert torch.equal(a, b), (n, t)


def test_every_tile_height_gives_identical_deflated_solves():
    p = W.config2(128)
    op = die.Operator(p.eps_r, p.h)
    D = die.Deflation(op, 8, tol=1e-4, regularized=True, inner=die.DIE_FP32_INNER)
    b = op.plane_wave(0.3)
    ref = None
    for t in heights(128):
        op.set_tile_rows(t)
        x, rep = op.solve(b, restart=20, tol=1e-12, max_iters=60, regularized=True, inner=die.DIE_FP32_INNER,
                          deflation=D)
        x = x.cpu()
        if ref is None:
            ref = (x, rep["rel_res_solved"])
        else:
            assert torch.equal(x, ref[0]) and rep["rel_res_solved"] == ref[1], t


def test_autotune_times_every_height_and_reuses_its_choice():
    p = W.config2(256)
    op = die.Operator(p.eps_r, p.h)
    r = op.autotune(force=True)
    valid = heights(256)
    assert r["tile_rows"] in valid and op.tile_rows == r["tile_rows"]
    for t, us in r["us_per_product"].items():
        assert (us > 0) == (t in valid), (t, us)
    us = r["us_per_product"]
    default = 4
    alt = min((t for t in valid if t != default), key=lambda t: us[t])
    assert r["tile_rows"] == (alt if us[alt] < 0.97 * us[default] else default), us
    op2 = die.Operator(W.config2(256).eps_r, p.h)           # same sizes: the choice is reused
    r2 = op2.autotune()
    assert r2["tile_rows"] == r["tile_rows"] and op2.tile_rows == r["tile_rows"]
    assert all(us == 0 for us in r2["us_per_product"].values())


def test_tile_height_limits():
    q = W.config2(2048)
    op = die.Operator(q.eps_r, q.h)
    for bad in (3, 4, 8, 16, -1):              # 4 rows of 4096-point rows already need 1024 threads
        with pytest.raises(die.DieError):
            op.set_tile_rows(bad)
    op.set_tile_rows(1)
    assert op.tile_rows == 1
    op.set_tile_rows(0)
    assert op.tile_rows == 2
    small = die.Operator(W.config1(20).eps_r, W.config1(20).h)   # not a compile-time length: one schedule
    assert small.tile_rows == 0
    with pytest.raises(die.DieError):
        small.set_tile_rows(2)
    assert small.autotune()["tile_rows"] == 0
