"""The small dense FP64 routines of the deflation eigensolver, run on the host.

`csrc/small_dense.cuh` holds the Schur decomposition that the deflation build (Krylov-Schur)
runs in one GPU thread: Householder reduction to Hessenberg form, shifted complex QR,
reordering of the Schur form by decreasing |T_ii|, and a Gauss-Jordan inverse for
T^-1 - I.  The code is host-callable; `small_dense_host.cu` runs it on seeded matrices
(orders 1 to 64, general, triangular and with a shifted spectrum as the Rayleigh quotients
have), and this test checks the decomposition's defining properties and its eigenvalues
against numpy's.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def _nvcc():
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    return None


@pytest.fixture(scope="module")
def cases(tmp_path_factory):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not available")
    exe = str(tmp_path_factory.mktemp("small_dense") / "small_dense_host")
    r = subprocess.run([nvcc, "-std=c++17", "-O1", "-x", "cu", os.path.join(HERE, "small_dense_host.cu"), "-o", exe],
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-4000:]
    out = subprocess.run([exe], capture_output=True, text=True, timeout=300, check=True).stdout
    res, cur = {}, None
    for line in out.splitlines():
        f = line.split()
        if f[0] == "case":
            n = int(f[2])
            cur = {"n": n, "rc": int(f[3]), "unit": float(f[4]), "below": float(f[5]), "rec": float(f[6]),
                   "sorted": int(f[7]), "inv": float(f[8]), "B": np.zeros((n, n), np.complex128),
                   "eig": np.zeros(n, np.complex128)}
            res[f[1]] = cur
        elif f[0] == "b":
            cur["B"][int(f[1]), int(f[2])] = float(f[3]) + 1j * float(f[4])
        elif f[0] == "t":
            cur["eig"][int(f[1])] = float(f[2]) + 1j * float(f[3])
    return res


def test_every_case_ran(cases):
    assert set(cases) == {"one", "two", "random5", "random17", "random40", "shifted64", "upper12"}


def test_schur_decomposition_properties(cases):
    """Z unitary, T upper triangular, Z T Z^* = B, |T_ii| non-increasing (relative to max|B|)."""
    for name, c in cases.items():
        assert c["rc"] == 0, name
        assert c["unit"] <= 1e-13, (name, c["unit"])
        assert c["below"] == 0.0, (name, c["below"])
        assert c["rec"] <= 1e-13 * max(1, c["n"]), (name, c["rec"])
        assert c["sorted"] == 1, name


def test_eigenvalues_match_numpy(cases):
    from scipy.optimize import linear_sum_assignment
    for name, c in cases.items():
        ref = np.linalg.eigvals(c["B"])
        cost = np.abs(c["eig"][:, None] - ref[None, :])
        i, j = linear_sum_assignment(cost)
        scale = np.abs(c["B"]).max()
        assert cost[i, j].max() <= 1e-10 * scale, (name, cost[i, j].max())


def test_inverse(cases):
    for name, c in cases.items():
        assert 0 <= c["inv"] <= 1e-11 * max(1, c["n"]), (name, c["inv"])
