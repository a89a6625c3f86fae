"""deflation_apply_noalloc against deflation_apply, through the C ABI.

The no-allocation entry point serves callers that cannot allocate device memory (a
host program whose device memory is all owned by its own pool, or a loop that must
not trigger the synchronisation cudaMalloc/cudaFree can cause).  It must give the
same z = P^-1 x as the ordinary entry point, call after call, although every call
reuses one static scratch array inside the library.
"""
import ctypes as ct

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1104_4263_gb300 import die, workloads as W  # noqa: E402

# Both paths launch the same two kernels with the same grid on the same data, and the
# reduction sums in a fixed order, so the results are bitwise equal (no tolerance).


@pytest.mark.parametrize("r", [11, 128])
def test_noalloc_matches_deflation_apply_twice(r):
    """r = 11 and r = 128 (the largest rank the static array holds): two calls in a row,
    then one in place, each bitwise equal to deflation_apply."""
    n = 12
    eps = W.core_shell(n, side=1.2, r_core=0.25, r_shell=0.5, eps_core=-2 + 0.1j, eps_shell=20 + 0.5j).eps_r
    op = die.Operator(eps, 0.1)
    # r = 128 on 288 unknowns: a short Krylov-Schur basis and few restarts suffice, since
    # this test needs a valid rank-128 handle, not converged eigenpairs
    D = (die.Deflation(op, r, tol=1e-8, regularized=True) if r < 64 else
         die.Deflation(op, r, tol=1e-6, regularized=True, krylov_dim=r + 8, max_restarts=2))
    assert D.r == r
    lib = die.lib()
    stream = ct.c_void_p(torch.cuda.current_stream().cuda_stream)
    rng = W.rng_for(120, r)
    for call in range(2):
        x = torch.from_numpy(W.random_vector(rng, n, n)).cuda()
        ref = D.apply(x)
        z = torch.full_like(x, complex("nan"))
        code = lib.deflation_apply_noalloc(D.handle, ct.c_void_p(x.data_ptr()), ct.c_void_p(z.data_ptr()), stream)
        assert code == 0, die.STATUS.get(code, code)
        torch.cuda.synchronize()
        assert torch.equal(z, ref), (call, float((z - ref).abs().max()))
    # in place, as deflation_apply allows
    x = torch.from_numpy(W.random_vector(rng, n, n)).cuda()
    ref = D.apply(x)
    assert lib.deflation_apply_noalloc(D.handle, ct.c_void_p(x.data_ptr()), ct.c_void_p(x.data_ptr()), stream) == 0
    torch.cuda.synchronize()
    assert torch.equal(x, ref)


def test_noalloc_rejects_null_arguments():
    lib = die.lib()
    assert lib.deflation_apply_noalloc(None, None, None, None) == 1


def test_noalloc_rejects_rank_above_its_array():
    """A rank-129 handle (deflation_build allows up to 256) is refused with DIE_EINVAL by
    the no-allocation entry point, whose static array holds rank 128, and nothing is
    written; the ordinary entry point serves it."""
    n = 12
    eps = W.core_shell(n, side=1.2, r_core=0.25, r_shell=0.5, eps_core=-2 + 0.1j, eps_shell=20 + 0.5j).eps_r
    op = die.Operator(eps, 0.1)
    D = die.Deflation(op, 129, tol=1e-6, regularized=True, krylov_dim=137, max_restarts=2)
    assert D.r == 129
    lib = die.lib()
    x = torch.from_numpy(W.random_vector(W.rng_for(120, 129), n, n)).cuda()
    z = torch.full_like(x, complex("nan"))
    stream = ct.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.deflation_apply_noalloc(D.handle, ct.c_void_p(x.data_ptr()), ct.c_void_p(z.data_ptr()), stream) == 1
    torch.cuda.synchronize()
    assert torch.isnan(z.real).all()
    assert torch.isfinite(D.apply(x).real).all()
