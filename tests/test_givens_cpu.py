"""The GMRES Givens step of the device solver, run on the host.

`givens_column` (csrc/krylov.cuh) is the arithmetic of the kernel that, one step behind the
Arnoldi steps, rotates each new Hessenberg column into R and rotates beta e1 (the
least-squares problem min || beta e1 - H y || of restarted GMRES, Saad & Schultz).
`givens_host.cu` runs it on seeded Hessenberg matrices with real non-negative subdiagonals
(as Arnoldi produces).  Pins: after j + 1 steps |g[j+1]| equals the least-squares residual
computed by numpy; R is the triangular factor of a unitary reduction of H (same singular
values); and R y = g gives numpy's least-squares solution.
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
    exe = str(tmp_path_factory.mktemp("givens") / "givens_host")
    r = subprocess.run([nvcc, "-std=c++17", "-O1", "-x", "cu", os.path.join(HERE, "givens_host.cu"), "-o", exe],
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-4000:]
    out = subprocess.run([exe], capture_output=True, text=True, timeout=300, check=True).stdout
    res, cur = {}, None
    for line in out.splitlines():
        f = line.split()
        if f[0] == "case":
            m = int(f[2])
            cur = {"m": m, "beta": float(f[3]), "H": np.zeros((m + 1, m), np.complex128), "est": np.zeros(m),
                   "R": np.zeros((m, m), np.complex128), "g": np.zeros(m + 1, np.complex128)}
            res[f[1]] = cur
        elif f[0] == "h":
            cur["H"][int(f[1]), int(f[2])] = float(f[3]) + 1j * float(f[4])
        elif f[0] == "est":
            cur["est"][int(f[1])] = float(f[2])
        elif f[0] == "r":
            cur["R"][int(f[1]), int(f[2])] = float(f[3]) + 1j * float(f[4])
        elif f[0] == "g":
            cur["g"][int(f[1])] = float(f[2]) + 1j * float(f[3])
    return res


def test_every_case_ran(cases):
    assert set(cases) == {"m1", "m5", "m30", "m64", "zero_column"}


def test_residual_estimates_are_least_squares_residuals(cases):
    for name, c in cases.items():
        H, m = c["H"], c["m"]
        e1 = np.zeros(m + 1, np.complex128)
        e1[0] = c["beta"]
        for j in range(m):
            y, *_ = np.linalg.lstsq(H[:j + 2, :j + 1], e1[:j + 2], rcond=None)
            ref = np.linalg.norm(e1[:j + 2] - H[:j + 2, :j + 1] @ y)
            assert abs(c["est"][j] - ref) <= 1e-12 * c["beta"] + 1e-10 * ref, (name, j, c["est"][j], ref)


def test_r_is_the_rotated_hessenberg_and_solves_the_least_squares_problem(cases):
    for name, c in cases.items():
        H, R, g, m = c["H"], c["R"], c["g"], c["m"]
        assert np.allclose(np.linalg.svd(R, compute_uv=False), np.linalg.svd(H, compute_uv=False),
                           rtol=1e-12, atol=1e-13), name
        e1 = np.zeros(m + 1, np.complex128)
        e1[0] = c["beta"]
        y_ref, *_ = np.linalg.lstsq(H, e1, rcond=None)
        y = np.linalg.solve(R, g[:m])
        kappa = np.linalg.cond(H)         # both solutions carry rounding of order eps * kappa
        assert np.linalg.norm(y - y_ref) <= 100 * 2.2e-16 * kappa * np.linalg.norm(y_ref), (name, kappa)
        assert abs(abs(g[m]) - c["est"][-1]) <= 1e-15 * c["beta"], name
