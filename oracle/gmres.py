"""Restarted GMRES(m) with an optional right preconditioner (paper Sections 4-5).

The paper solves A u = b, A_R A u = A_R b and their right-preconditioned forms
A P^-1 v = b, u = P^-1 v (Eq. (4.12), and A_R A P^-1 v = A_R b in Section 5) with
restarted GMRES.  This is the plain textbook method: within a cycle the Krylov
basis is built by modified Gram-Schmidt, and the iterate is the minimiser of
|| beta e1 - H y || solved directly with a dense least-squares routine; between
cycles the residual is recomputed from scratch.  x0 = 0 unless given.

Stopping: relative residual of the solved system, ||b - Atilde x|| / ||b|| <= tol
(with right preconditioning this is the unpreconditioned residual of Atilde).
`iters` counts applications of Atilde (inner Arnoldi steps).
"""
from __future__ import annotations

import dataclasses

import numpy as np


@dataclasses.dataclass
class GmresResult:
    x: np.ndarray
    converged: bool
    iters: int
    cycles: int
    rel_res: float                   # true residual of the solved system at exit
    history: list                    # per-step residual estimates (relative)


def gmres(apply, b, restart: int, tol: float, max_iters: int, precond=None, x0=None) -> GmresResult:
    """Solve apply(x) = b with GMRES(restart), right preconditioner `precond` (x = P^-1 v)."""
    b = np.asarray(b, dtype=np.complex128)
    shape = b.shape
    bv = b.reshape(-1)
    bnorm = np.linalg.norm(bv)
    x = np.zeros_like(bv) if x0 is None else np.array(x0, dtype=np.complex128).reshape(-1)
    P = (lambda v: v) if precond is None else (lambda v: precond(v.reshape(shape)).reshape(-1))
    Aop = lambda v: apply(v.reshape(shape)).reshape(-1)
    history: list = []
    iters = 0
    cycles = 0
    if bnorm == 0.0:
        return GmresResult(np.zeros(shape, np.complex128), True, 0, 0, 0.0, history)
    while True:
        r = bv - Aop(x)
        beta = np.linalg.norm(r)
        if beta / bnorm <= tol or iters >= max_iters:
            break
        cycles += 1
        V = [r / beta]
        H = np.zeros((restart + 1, restart), dtype=np.complex128)
        e1 = np.zeros(restart + 1, dtype=np.complex128)
        e1[0] = beta
        k = 0
        y = np.zeros(0, dtype=np.complex128)
        for j in range(restart):
            w = Aop(P(V[j]))
            iters += 1
            for i in range(j + 1):                       # modified Gram-Schmidt
                H[i, j] = np.vdot(V[i], w)
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            k = j + 1
            y, *_ = np.linalg.lstsq(H[:k + 1, :k], e1[:k + 1], rcond=None)
            est = np.linalg.norm(e1[:k + 1] - H[:k + 1, :k] @ y) / bnorm
            history.append(est)
            if est <= tol or iters >= max_iters or H[j + 1, j] == 0.0:
                break
            V.append(w / H[j + 1, j])
        d = sum(y[i] * V[i] for i in range(k))
        x = x + P(d)
    rel = np.linalg.norm(bv - Aop(x)) / bnorm
    return GmresResult(x.reshape(shape), rel <= tol, iters, cycles, rel, history)


def fgmres(apply, b, restart: int, tol: float, max_iters: int, precond=None, x0=None) -> GmresResult:
    """Flexible GMRES(restart) (Saad, "A flexible inner-outer preconditioned GMRES
    algorithm", SIAM J. Sci. Comput. 14, 1993): the right preconditioner may change from
    step to step, or be nonlinear (a learned map).  Step j applies z_j = precond(v_j, j),
    keeps z_j, and extends the Arnoldi relation A Z_j = V_{j+1} H_j; the cycle's update
    is x += Z_k y with y the minimiser of || beta e1 - H y ||.  With a fixed linear
    preconditioner the iterates are those of right-preconditioned GMRES.  Same stopping
    rule and counters as `gmres`; precond=None is the identity."""
    b = np.asarray(b, dtype=np.complex128)
    shape = b.shape
    bv = b.reshape(-1)
    bnorm = np.linalg.norm(bv)
    x = np.zeros_like(bv) if x0 is None else np.array(x0, dtype=np.complex128).reshape(-1)
    M = (lambda v, j: v) if precond is None else (lambda v, j: np.asarray(precond(v.reshape(shape), j)).reshape(-1))
    Aop = lambda v: apply(v.reshape(shape)).reshape(-1)
    history: list = []
    iters = 0
    cycles = 0
    if bnorm == 0.0:
        return GmresResult(np.zeros(shape, np.complex128), True, 0, 0, 0.0, history)
    while True:
        r = bv - Aop(x)
        beta = np.linalg.norm(r)
        if beta / bnorm <= tol or iters >= max_iters:
            break
        cycles += 1
        V = [r / beta]
        Z = []
        H = np.zeros((restart + 1, restart), dtype=np.complex128)
        e1 = np.zeros(restart + 1, dtype=np.complex128)
        e1[0] = beta
        k = 0
        y = np.zeros(0, dtype=np.complex128)
        for j in range(restart):
            Z.append(M(V[j], iters))
            w = Aop(Z[j])
            iters += 1
            for i in range(j + 1):                       # modified Gram-Schmidt
                H[i, j] = np.vdot(V[i], w)
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            k = j + 1
            y, *_ = np.linalg.lstsq(H[:k + 1, :k], e1[:k + 1], rcond=None)
            est = np.linalg.norm(e1[:k + 1] - H[:k + 1, :k] @ y) / bnorm
            history.append(est)
            if est <= tol or iters >= max_iters or H[j + 1, j] == 0.0:
                break
            V.append(w / H[j + 1, j])
        x = x + sum(y[i] * Z[i] for i in range(k))
    rel = np.linalg.norm(bv - Aop(x)) / bnorm
    return GmresResult(x.reshape(shape), rel <= tol, iters, cycles, rel, history)
