"""The byte and flop model behind the bench's achieved GB/s and roofline fractions."""
import importlib.util
import os
import types

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_module", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _grid(n):
    p = types.SimpleNamespace(n1=n, n2=n, N=n * n)
    op = types.SimpleNamespace(M1=2 * n, M2=2 * n)
    return p, op


@pytest.mark.parametrize("n,s", [(512, 8), (512, 16), (256, 8), (1024, 8)])
def test_product_bytes_closed_forms(bench, n, s):
    """Per regularised product at M = 2n: K1 reads u (2N) and chi (N), writes W (4N);
    each K2 reads and writes W and reads the three quarter spectra; K3K1 reads W, u, chi'
    and writes v and W; K3 reads W and v and writes y (element size s throughout)."""
    p, op = _grid(n)
    N = n * n
    b = bench.product_bytes(p, op, s)
    assert b["rows_fwd"] == 7 * N * s
    assert b["cols_green"] == 2 * (8 * N * s + 3 * (n + 1) ** 2 * s)
    assert b["rows_inv_fwd"] == 13 * N * s
    assert b["rows_inv"] == 8 * N * s
    total = sum(b.values())
    assert total == 44 * N * s + 6 * (n + 1) ** 2 * s        # about 50 N s


def test_product_bytes_at_the_bench_size(bench):
    p, op = _grid(512)
    assert sum(bench.product_bytes(p, op, 8).values()) == pytest.approx(104.9e6, rel=1e-3)


def test_deflated_first_pass_and_fp64_output(bench):
    """The deflated first row pass reads r complex64 basis vectors, the FP64 Arnoldi vector
    (read and written back normalised) and writes z; the complex128 output of the
    FP32-inner products counts 16 bytes in the last pass."""
    p, op = _grid(512)
    N, r = 512 * 512, 20
    b = bench.product_bytes(p, op, 8, out_s=16, defl_r=r)
    assert b["rows_fwd"] == r * 2 * N * 8 + 2 * 2 * N * 16 + 2 * N * 8 + N * 8 + 4 * N * 8
    assert b["rows_inv"] == 4 * N * 8 + 2 * N * 8 + 2 * N * 16


def test_projection_flops_per_cycle(bench):
    """Step j of a cycle projects on j + 1 vectors (8 flops per element each) and forms the
    norm of w (4); per cycle one residual norm (4) and the FP64 deflation projections (8 r)."""
    p, op = _grid(64)
    n = 2 * 64 * 64
    m, r, cycles = 30, 20, 3
    kind, flops = bench.work_model("dots", p, op, r, m, cycles, 0, 0)
    assert kind == "alu"
    assert flops == cycles * (8 * m * (m + 1) // 2 + 4 * m + 4 + 8 * r) * n + 4 * n
