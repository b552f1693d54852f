"""GPLHR-EIG, Algorithm 3 of the paper (Appendix A), in plain FP64/complex128 NumPy.
Test infrastructure only (see the package docstring).

The eigenvector-based variant of GPLHR: the iterate is a block X of approximate
eigenvectors with unit columns, the eigenvalue approximations are the bilinear forms
alpha_j = x_j^* A x_j, beta_j = x_j^* B x_j (diagonal Lambda_A, Lambda_B), the trial and
test subspaces are built as in Algorithm 2 with the diagonal factors in place of
M_A, M_B, and the projected pair (U^* A Z, U^* B Z) is solved by a full
eigendecomposition whose eigenvectors, ordered by the distance of their eigenvalues to
sigma, give the new X and P.

Readings (shared with the CUDA path):
* Step 21 subtracts Q(Q^* Qhat) after orth; Qhat is orthonormalised again after that
  subtraction (as for Algorithm 2).
* Step 27 (P = Z Ybar(:, k+1:2k), the thick restart) is the default; p_mode="lobpcg"
  disables it and keeps the LOBPCG-style P of step 25, as the algorithm's footnote allows.
* Eigenvectors of the projected pair: the right eigenvectors of its complex QZ form
  (the triangular pencil's by back substitution, rotated back by the right Schur
  vectors), each scaled to unit norm; order as in Algorithm 2 (|alpha - sigma beta| /
  |beta| ascending, ties by Re, then Im).
* Convergence: pair j passes when
      ||beta_j A x_j - alpha_j B x_j|| / ((|beta_j| ||A||_1 + |alpha_j| ||B||_1) ||x_j||) <= tol
  for all k pairs at once (the algorithm has no soft locking).
"""
from __future__ import annotations

import dataclasses

import numpy as np

from .gplhr import Pencil, onenorm, orth, tri_eigvecs
from .ordqz import ordqz
from .precond import build as build_precond


def projected_eigvecs(Phi: np.ndarray, Psi: np.ndarray, sigma: complex, nvec: int):
    """The nvec eigenpairs of (Phi, Psi) nearest sigma: (alpha, beta, Y), Y with unit
    columns, via the ordered complex QZ (Phi Y_R = Y_L R_A, ...) and back substitution."""
    RA, RB, YL, YR = ordqz(Phi, Psi, sigma)
    Zt = tri_eigvecs(RA[:nvec, :nvec], RB[:nvec, :nvec])
    Y = YR[:, :nvec] @ Zt
    Y = Y / np.linalg.norm(Y, axis=0)[None, :]
    return np.diag(RA)[:nvec].copy(), np.diag(RB)[:nvec].copy(), Y


@dataclasses.dataclass
class EigResult:
    X: np.ndarray
    alpha: np.ndarray
    beta: np.ndarray
    lam: np.ndarray
    resid: np.ndarray
    iters: int
    converged: bool
    history: list


def _rayleigh(pen: Pencil, X: np.ndarray):
    AX = pen.Amul(X)
    BX = pen.Bmul(X)
    a = np.einsum("ij,ij->j", X.conj(), AX)
    b = np.einsum("ij,ij->j", X.conj(), BX)
    return AX, BX, a, b


def _resid(pen: Pencil, X, AX, BX, a, b) -> np.ndarray:
    E = AX * b[None, :] - BX * a[None, :]
    den = (np.abs(b) * pen.normA + np.abs(a) * pen.normB) * np.linalg.norm(X, axis=0)
    return np.linalg.norm(E, axis=0) / den


def solve_eig(A, B, sigma, X0, m: int = 1, tol: float = 1e-8, maxit: int = 500, precond: str = "none",
              block_size: int = 1, T=None, p_mode: str = "thick", callback=None) -> EigResult:
    """Algorithm 3 until all k pairs meet ``tol`` or ``maxit`` iterations."""
    if p_mode not in ("thick", "lobpcg"):
        raise ValueError(f"unknown p_mode {p_mode!r}")
    if T is None:
        T = build_precond(A, B, sigma, precond, block_size)
    pen = Pencil(A, B, sigma, T)
    sig = pen.sigma
    generalized = pen.B is not None
    X = np.asarray(X0, dtype=np.complex128).copy()
    k = X.shape[1]
    X = X / np.linalg.norm(X, axis=0)[None, :]                      # steps 1-2
    AX, BX, a, b = _rayleigh(pen, X)
    Qb = AX - sig * BX
    P = None
    hist = []
    res = _resid(pen, X, AX, BX, a, b)
    it = 0
    while not np.all(res <= tol) and it < maxit:
        V = orth(X)                                                  # step 4
        Q = orth(Qb)
        proj_V = lambda Y: Y - V @ (V.conj().T @ Y)                  # noqa: E731
        proj_Q = lambda Y: Y - Q @ (Q.conj().T @ Y)                  # noqa: E731
        proj_right = proj_Q if generalized else proj_V
        T_L = lambda Y: proj_V(pen.Tmul(proj_right(Y)))              # noqa: E731
        W = orth(T_L(AX * b[None, :] - BX * a[None, :]))             # steps 5-10
        S = []
        S_prev = W
        for _ in range(m):                                           # steps 11-18
            Sl = T_L(pen.Amul(S_prev) * b[None, :] - pen.Bmul(S_prev) * a[None, :])
            Sl = Sl - W @ (W.conj().T @ Sl)
            if S:
                Sc = np.hstack(S)
                Sl = Sl - Sc @ (Sc.conj().T @ Sl)
            Sl = orth(Sl)
            S.append(Sl)
            S_prev = Sl
        blocks = [W] + S
        if P is not None:                                            # step 19
            Sc = np.hstack(S) if S else np.zeros((pen.n, 0), dtype=np.complex128)
            P = P - V @ (V.conj().T @ P)
            P = P - W @ (W.conj().T @ P)
            P = P - Sc @ (Sc.conj().T @ P)
            P = orth(P)
            blocks.append(P)
        K = np.hstack(blocks)
        Z = np.hstack([V, K])                                        # step 20
        AZ = np.hstack([pen.Amul(V), pen.Amul(K)])
        BZ = np.hstack([pen.Bmul(V), pen.Bmul(K)])
        Qh = orth(AZ[:, k:] - sig * BZ[:, k:])                      # step 21
        Qh = orth(Qh - Q @ (Q.conj().T @ Qh))
        U = np.hstack([Q, Qh])                                       # step 22
        _, _, Yb = projected_eigvecs(U.conj().T @ AZ, U.conj().T @ BZ, sig, 2 * k)   # step 23
        Y = Yb[:, :k]                                                # step 24
        P = K @ Y[k:, :]                                             # step 25
        X = V @ Y[:k, :] + P                                         # step 26
        if p_mode == "thick":
            P = Z @ Yb[:, k:2 * k]                                   # step 27
        X = X / np.linalg.norm(X, axis=0)[None, :]                  # step 28
        AX, BX, a, b = _rayleigh(pen, X)
        Qb = AX - sig * BX                                           # step 26: Q <- (A - sigma B) X
        it += 1
        res = _resid(pen, X, AX, BX, a, b)
        hist.append(res.copy())
        if callback is not None:
            callback(X, a, b, res)
    with np.errstate(divide="ignore", invalid="ignore"):
        lam = a / b
    return EigResult(X, a, b, lam, res, it, bool(np.all(res <= tol)), hist)
