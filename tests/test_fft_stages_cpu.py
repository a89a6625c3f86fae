"""The Stockham stages of the product kernels, run on the host.

The stage code of `csrc/fft_fast.cuh` and `csrc/fft.cuh` (stage loads, twiddles, radix-R
DFTs and stores through the padded shared-memory layout) is host-callable.
`fft_stages_host.cu` runs every thread of a transform group through
* each compile-time plan of the fast kernels (L = 256 ... 4096), and
* the runtime-plan stages of the general kernels through the planner's plans for 2^a and
  3 * 2^a lengths (16 or 12 values per thread),
forward and inverse, FP64 and FP32, and compares the result with the plain DFT sum
evaluated in long double.  This pins the FFT building blocks of the GPU path on a machine
without a GPU; the GPU parity tests check the complete products against the oracle.
"""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
LENGTHS = (256, 512, 1024, 2048, 4096)               # compile-time plans (fast kernels)
GENERAL_LENGTHS = (16, 32, 64, 128, 512, 1024, 24, 48, 96, 192, 384, 768, 1536)   # runtime plans


def _nvcc():
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    return None


@pytest.fixture(scope="module")
def stage_errors(tmp_path_factory):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not available")
    exe = str(tmp_path_factory.mktemp("fft_stages") / "fft_stages_host")
    src = os.path.join(HERE, "fft_stages_host.cu")
    r = subprocess.run([nvcc, "-std=c++17", "-O1", "--expt-relaxed-constexpr", "-x", "cu", src, "-o", exe],
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-4000:]
    out = subprocess.run([exe], capture_output=True, text=True, timeout=600, check=True).stdout
    errs = {}
    for line in out.splitlines():
        L, direction, prec, err = line.split()
        errs[(L, direction, prec)] = float(err)
    return errs


def test_every_plan_is_run(stage_errors):
    lengths = [str(L) for L in LENGTHS] + ["gen%d" % L for L in GENERAL_LENGTHS]
    want = {(L, d, p) for L in lengths for d in ("fwd", "inv") for p in ("f64", "f32")}
    assert set(stage_errors) == want


@pytest.mark.parametrize("prec,tol", [("f64", 1e-14), ("f32", 1e-6)])
def test_stages_equal_plain_dft(stage_errors, prec, tol):
    # FP64: a few ulps of the largest output; FP32: single-precision rounding over
    # log16(L) radix-16/8 stages (measured 1e-7 .. 2e-7)
    bad = {k: v for k, v in stage_errors.items() if k[2] == prec and not v <= tol}
    assert not bad, bad
