"""Deflating right preconditioner and deflation radius (paper Sections 4-5).

Eq. (4.12):  P^-1 = I + V (T^-1 - I_r) V^*,   Eq. (4.13): T = V^* Atilde V,
where V (2N x r) is an orthonormal basis, obtained by modified Gram-Schmidt, of the
eigenvectors of the r largest-magnitude eigenvalues of the system matrix Atilde.
Here the eigenpairs come from a dense eigendecomposition (small grids only).

Deflation radius (Section 5): each segment [1, eps_r(x)] radially emerging from
1 + 0i is mapped through the homogeneous eigenvalue map of Eq. (5.3),
lambda' = [1 + (eps_b / eps)(1 - lambda)] lambda, and the largest |lambda'| over
all segments is the radius beyond which eigenvalues are deflated.
"""
from __future__ import annotations

import numpy as np


def largest_eigs(Atilde: np.ndarray, r: int):
    """The r eigenpairs of largest |lambda| (ties: larger |lambda| first, then lower index)."""
    w, X = np.linalg.eig(Atilde)
    order = sorted(range(len(w)), key=lambda i: (-abs(w[i]), i))[:r]
    return w[order], X[:, order]


def mgs(X: np.ndarray) -> np.ndarray:
    """Modified Gram-Schmidt orthonormalisation of the columns of X."""
    Q = np.array(X, dtype=np.complex128, copy=True)
    for j in range(Q.shape[1]):
        for i in range(j):
            Q[:, j] -= np.vdot(Q[:, i], Q[:, j]) * Q[:, i]
        Q[:, j] /= np.linalg.norm(Q[:, j])
    return Q


def largest_eigs_op(apply, n: int, r: int, tol: float = 1e-10, seed: int = 0):
    """The r eigenpairs of largest |lambda| of the linear map `apply` on C^n, by the
    implicitly restarted Arnoldi method of ARPACK (scipy.sparse.linalg.eigs), which is
    what the Matlab eigs of Section 5 runs; for grids whose dense matrix is too large.
    Ordered as largest_eigs."""
    from scipy.sparse.linalg import LinearOperator, eigs
    rng = np.random.default_rng(seed)
    v0 = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    op = LinearOperator((n, n), matvec=lambda v: np.asarray(apply(v)).reshape(-1), dtype=np.complex128)
    w, X = eigs(op, k=r, which="LM", tol=tol, v0=v0)
    order = sorted(range(len(w)), key=lambda i: (-abs(w[i]), i))[:r]
    return w[order], X[:, order]


class Deflation:
    """P^-1 = I + V (T^-1 - I) V^* for the r largest-magnitude eigenvalues of Atilde."""

    def __init__(self, Atilde: np.ndarray, r: int):
        self.eigs, X = largest_eigs(Atilde, r)
        self.V = mgs(X)
        self.T = self.V.conj().T @ Atilde @ self.V
        self.M = np.linalg.inv(self.T) - np.eye(r)

    @classmethod
    def from_operator(cls, apply, shape, r: int, tol: float = 1e-10, seed: int = 0) -> "Deflation":
        """The same preconditioner from products only (Section 5: eigs, then the eigenvectors
        orthonormalised by modified Gram-Schmidt, then T = V^* Atilde V from r products).
        apply maps an array of `shape` to one of `shape`."""
        n = int(np.prod(shape))
        flat = lambda v: np.asarray(apply(np.asarray(v).reshape(shape))).reshape(-1)
        self = cls.__new__(cls)
        self.eigs, X = largest_eigs_op(flat, n, r, tol, seed)
        self.V = mgs(X)
        AV = np.stack([flat(self.V[:, i]) for i in range(r)], axis=1)
        self.T = self.V.conj().T @ AV
        self.M = np.linalg.inv(self.T) - np.eye(r)
        return self

    def apply(self, x: np.ndarray) -> np.ndarray:
        shape = x.shape
        v = x.reshape(-1)
        return (v + self.V @ (self.M @ (self.V.conj().T @ v))).reshape(shape)

    def matrix(self) -> np.ndarray:
        n = self.V.shape[0]
        return np.eye(n) + self.V @ self.M @ self.V.conj().T


def regularized_eig_map(lam, eps):
    """Eq. (5.3): lambda' = [1 + (1 - lambda)/eps] lambda  (eps relative to eps_b = 1)."""
    return (1.0 + (1.0 - lam) / eps) * lam


def deflation_radius(eps_values, samples: int = 1000) -> float:
    """max |lambda'| over the images of the segments [1, eps] (Section 5)."""
    t = np.linspace(0.0, 1.0, samples)
    R = 0.0
    for e in np.unique(np.asarray(eps_values, dtype=np.complex128).reshape(-1)):
        lam = 1.0 + t * (e - 1.0)
        R = max(R, float(np.max(np.abs(regularized_eig_map(lam, e)))))
    return R
