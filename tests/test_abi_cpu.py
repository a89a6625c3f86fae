"""CPU-side checks of the C ABI: the library loads without a GPU, exports every symbol
the header declares, and its host-only helpers behave (no device work here)."""
import ctypes as ct
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", h) for h in sorted(os.listdir(os.path.join(ROOT, "include")))
           if h.endswith(".h")]


def declared_functions():
    src = "\n".join(open(h).read() for h in HEADERS)
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = set(re.findall(r"^\s*(?:[A-Za-z_][\w\s\*]*?)\b([a-z_][a-z0-9_]*)\s*\(", src, flags=re.M))
    return sorted(n for n in names if n not in {"if", "while", "for", "sizeof", "defined"})


@pytest.fixture(scope="module")
def lib():
    from paper_1104_4263_gb300 import build, die
    if not os.path.exists(build.LIB):
        build.build()
    return die.lib()


def test_header_declares_the_core_calls():
    names = declared_functions()
    for n in ["dieop_create", "dieop_apply", "dieop_apply_regularized", "gmres_solve", "deflation_build",
              "dieop_destroy", "deflation_destroy", "die_status_str"]:
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    handle = ct.CDLL(os.path.join(ROOT, "paper_1104_4263_gb300", "_lib", "libdie.so"))
    missing = [n for n in declared_functions() if not hasattr(handle, n)]
    assert not missing, missing


def test_binding_covers_every_symbol():
    from paper_1104_4263_gb300 import die
    assert set(declared_functions()) == set(die.EXPORTS)


def test_status_strings(lib):
    assert lib.die_status_str(0) == b"ok"
    assert b"singular" in lib.die_status_str(4)
    assert lib.die_abi_version() == 3


def test_struct_layouts_match_the_binding(lib):
    """The ctypes mirrors of the public structures have the library's sizes."""
    import ctypes as ct
    from paper_1104_4263_gb300 import die
    sizes = (ct.c_longlong * 4)()
    assert lib.die_abi_sizes(sizes, 4) == 0
    assert list(sizes) == [ct.sizeof(t) for t in die.STRUCTS]
    assert lib.die_abi_sizes(None, 4) == 1 and lib.die_abi_sizes(sizes, 5) == 1


def test_deflation_radius_host(lib):
    """Section 5 radius: lossless eps = 16 -> 1 + 15^2/64 (sampled at 1000 points)."""
    from paper_1104_4263_gb300 import die
    R = die.deflation_radius(np.array([16.0 + 0j, 1.0 + 0j]))
    assert abs(R - 4.515625) < 1e-5
    # agrees with the oracle's independent routine on a lossy, inhomogeneous map
    from oracle import deflation
    eps = np.array([-16 + 1.5j, 2.5 + 20j, 16.0, 1.0])
    assert die.deflation_radius(eps) == pytest.approx(deflation.deflation_radius(eps), rel=1e-12)
    assert lib.die_deflation_radius(None, 1, 10) < 0


def test_invalid_arguments_rejected_without_gpu(lib):
    from paper_1104_4263_gb300 import die
    out = ct.c_void_p()
    d = die.Desc(1, 8, 0.1, 0.0, 0, 0, 0)          # n1 < 2
    eps = np.ones(8, dtype=np.complex128)
    assert lib.dieop_create(ct.byref(d), eps.ctypes.data_as(ct.c_void_p), 0, None, ct.byref(out)) == 1
    d = die.Desc(8, 8, -1.0, 0.0, 0, 0, 0)         # h <= 0
    assert lib.dieop_create(ct.byref(d), eps.ctypes.data_as(ct.c_void_p), 0, None, ct.byref(out)) == 1
    assert out.value is None
    assert lib.gmres_solve(None, None, None, None, None, None, None) == 1
    assert lib.dieop_apply(None, None, None, None) == 1
    assert lib.dieop_apply_batch(None, 1, None, None, 0, None) == 1
    assert lib.gmres_solve_batch(None, None, None, 1, None, None, None, None) == 1
    opts = die.GmresOpts(30, 100, 1e-6, 0, 0, 0, 0, 0.0)
    dummy = ct.c_void_p(1)                       # never dereferenced: the checks below return first
    for nrhs in (0, 17):                          # outside [1, 16]
        assert lib.gmres_solve_batch(dummy, None, ct.byref(opts), nrhs, dummy, dummy, None, None) == 1
    for nrhs in (0, 1025):                        # outside [1, 1024]
        assert lib.dieop_apply_batch(dummy, nrhs, dummy, dummy, 1, None) == 1
    assert lib.gmres_solve_many(0, dummy, None, ct.byref(opts), dummy, dummy, None, None) == 1
    assert lib.gmres_solve_many(1, None, None, ct.byref(opts), dummy, dummy, None, None) == 1
    nulls = ct.cast((ct.c_void_p * 1)(None), ct.c_void_p)     # ops[0] == NULL
    assert lib.gmres_solve_many(1, nulls, None, ct.byref(opts), nulls, nulls, None, None) == 1
    # the magnetic-contrast operator and the tile schedule
    d = die.Desc(8, 8, 0.1, 0.0, 0, 0, 0, 3)          # no such polarisation
    assert lib.dieop_create(ct.byref(d), eps.ctypes.data_as(ct.c_void_p), 0, None, ct.byref(out)) == 1
    assert lib.dieop_set_permeability(None, None, 0, None) == 1
    assert lib.dieop_set_tile_rows(None, 4) == 1
    assert lib.dieop_tile_rows(None) == 0
    assert lib.dieop_autotune(None, 0, None, None, None) == 1


def test_solve_many_argument_checks_without_gpu():
    """The binding rejects mismatched lists and tensors that are not contiguous complex128
    CUDA vectors of the operator's size before calling the library."""
    import types

    import torch

    from paper_1104_4263_gb300 import die
    op = types.SimpleNamespace(N=16, handle=None)
    with pytest.raises(ValueError):
        die.solve_many([op, op], [torch.zeros(2, 4, 4, dtype=torch.complex128)])
    with pytest.raises(TypeError):            # a CPU tensor
        die.solve_many([op], [torch.zeros(2, 4, 4, dtype=torch.complex128)])
    with pytest.raises(TypeError):            # wrong dtype
        die.solve_many([op], [torch.zeros(2, 4, 4, dtype=torch.complex64)])


def test_memory_plan_reproduces_the_sinusoidal_example(lib):
    """Section 5's worked example (tests/golden): 4 GB, beta 0.0011, restart 8 r, 15 points per
    wavelength and eps up to 15 allow [a/lambda]_max = 4; at a/lambda = 4 the grid has
    233 x 233 = 54289 points (3N = 162867), r = 3 N beta = 180 (rounded up) and the restarts
    are 8 r and 9 r."""
    import json
    import math
    from paper_1104_4263_gb300 import die
    g = json.load(open(os.path.join(ROOT, "tests", "golden", "paper_values.json")))["memory_plan_sinusoidal"]
    plan = die.memory_plan(g["memory_bytes"], g["beta"], g["restart_over_r"], g["points_per_wavelength"],
                           g["eps_max"])
    assert round(plan["a_over_lambda_max"]) == g["a_over_lambda_max"]
    assert plan["alpha"] == pytest.approx(15 * math.sqrt(15))
    side = round(plan["alpha"] * g["a_over_lambda_max"] + 1)      # grid points per side, 233
    N = side * side
    assert 3 * N == g["three_n"]
    r = math.ceil(3 * N * g["beta"])                                # beta is "approximately 0.0011"
    assert r == g["r"]
    assert g["restart_over_r"] * r == g["restart_preconditioned"] and (g["restart_over_r"] + 1) * r == g["restart_original"]
    out = (ct.c_double * 3)()
    assert lib.die_memory_plan(-1.0, 0.1, 1.0, 15.0, 4.0, out) == 1
