"""Eigenvalue adjoint on the sparsity patterns of A and B.  Test infrastructure only.

For a simple eigenvalue lambda_i of (A, B) with right vector x_i (A x = lambda B x) and
left vector y_i (y^* A = lambda y^* B),

    d lambda_i = y_i^* (dA - lambda_i dB) x_i / (y_i^* B x_i)

(first-order perturbation of a simple eigenvalue).  For a real loss L of the
eigenvalues with G_i = dL/dRe(lambda_i) + i dL/dIm(lambda_i), the gradient with respect
to an entry a_pq (in the same convention, d/dRe + i d/dIm) is

    dL/da_pq = sum_i G_i conj(c_i),   c_i = conj(y_ip) x_iq / (y_i^* B x_i),
    dL/db_pq = sum_i G_i conj(-lambda_i c_i),

and for real matrices the real part is the gradient.  Left vectors come from the pencil
(A^*, B^*) at the shift conj(sigma), whose eigenvalues are conj(lambda); pairs are
matched by nearest eigenvalue.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def pair(lam_right: np.ndarray, mu_left: np.ndarray, rtol: float = 1e-6) -> np.ndarray:
    """perm with lam_right[i] ~ conj(mu_left[perm[i]]); raises if a match is missing or
    not unique within rtol * |lambda|."""
    target = np.conj(mu_left)
    perm = np.empty(lam_right.size, dtype=int)
    for i, lam in enumerate(lam_right):
        d = np.abs(target - lam)
        j = int(np.argmin(d))
        tol = rtol * max(abs(lam), 1e-300)
        if d[j] > tol or np.sum(d <= tol) != 1:
            raise ValueError(f"no unique left eigenvalue for lambda_{i} = {lam}")
        perm[i] = j
    if len(set(perm.tolist())) != perm.size:
        raise ValueError("left/right pairing is not one-to-one")
    return perm


def eig_grad(A, B, lam: np.ndarray, X: np.ndarray, Y: np.ndarray, G: np.ndarray):
    """(dL/dA.data, dL/dB.data or None) on the CSR patterns of A and B (in CSR order).
    X, Y: n x k right and left vectors, paired column by column with lam."""
    A = sp.csr_matrix(A)
    BX = X if B is None else sp.csr_matrix(B) @ X
    d = np.einsum("pi,pi->i", Y.conj(), BX)                       # y_i^* B x_i
    alpha = G / np.conj(d)

    def scatter(M, coef):
        M = sp.csr_matrix(M)
        rows = np.repeat(np.arange(M.shape[0]), np.diff(M.indptr))
        cols = M.indices
        out = np.einsum("ei,ei,i->e", Y[rows], X[cols].conj(), coef)
        return out if np.iscomplexobj(M.data) else out.real

    dA = scatter(A, alpha)
    dB = None if B is None else scatter(B, -np.conj(lam) * alpha)
    return dA, dB
