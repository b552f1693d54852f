"""Preconditioner T ~ (A - sigma B)^{-1} (Sec. 4 of the paper).  Test infrastructure only.

* "none":          T = I.
* "jacobi":        T = diag(A - sigma B)^{-1}.  When every diagonal entry is the
                   same number (relative spread <= 1e-12) T is a multiple of I,
                   and since every output of T passes through a projector and an
                   orthonormalisation, the iteration is the one with T = I; the
                   oracle then uses T = I (this also covers a shift that makes the
                   constant diagonal vanish).  A zero entry otherwise is singular.
* "block_jacobi":  T = blockdiag(D_1^{-1}, ..., D_nb^{-1}), D_b the bs x bs diagonal
                   block of A - sigma B on rows/cols [b bs, (b+1) bs) (the last block
                   is n mod bs wide when bs does not divide n).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


class SingularPreconditioner(ValueError):
    pass


class Preconditioner:
    def __init__(self, kind: str, diag=None, blocks=None, bs: int = 1):
        self.kind = kind          # "identity" | "jacobi" | "block_jacobi"
        self.diag_inv = diag
        self.blocks_inv = blocks  # list of dense inverse blocks
        self.bs = bs

    def apply(self, X: np.ndarray) -> np.ndarray:
        if self.kind == "identity":
            return X.copy()
        if self.kind == "jacobi":
            return self.diag_inv[:, None] * X
        out = np.empty_like(X)
        for b, Dinv in enumerate(self.blocks_inv):
            r0 = b * self.bs
            r1 = r0 + Dinv.shape[0]
            out[r0:r1] = Dinv @ X[r0:r1]
        return out


def shifted(A: sp.spmatrix, B, sigma: complex) -> sp.csr_matrix:
    n = A.shape[0]
    Bm = sp.identity(n, format="csr") if B is None else B
    return sp.csr_matrix(A.astype(np.complex128) - sigma * Bm.astype(np.complex128))


def build(A, B, sigma: complex, kind: str, bs: int = 1, inner_steps: int = 0):
    """The preconditioner of kind (with block size bs); inner_steps > 0 wraps it as the
    basic preconditioner T0 of that many block GMRES steps on (A - sigma B) w = r
    (oracle.gmres)."""
    T0 = _build(A, B, sigma, kind, bs)
    if inner_steps > 0:
        from .gmres import BlockGmres
        return BlockGmres(shifted(A, B, sigma), T0, inner_steps)
    return T0


def _build(A, B, sigma: complex, kind: str, bs: int = 1) -> Preconditioner:
    if kind == "none":
        return Preconditioner("identity")
    K = shifted(A, B, sigma)
    if kind == "jacobi":
        d = K.diagonal()
        amax = np.abs(d).max()
        if amax == 0 or np.abs(d - d[0]).max() <= 1e-12 * amax:
            return Preconditioner("identity")
        if np.any(d == 0):
            raise SingularPreconditioner("zero diagonal entry in A - sigma B")
        return Preconditioner("jacobi", diag=1.0 / d)
    if kind == "block_jacobi":
        n = K.shape[0]
        blocks = []
        for r0 in range(0, n, bs):
            r1 = min(n, r0 + bs)
            D = K[r0:r1, r0:r1].toarray()
            if np.linalg.matrix_rank(D) < D.shape[0]:
                raise SingularPreconditioner(f"singular diagonal block at row {r0}")
            blocks.append(np.linalg.inv(D))
        return Preconditioner("block_jacobi", blocks=blocks, bs=bs)
    raise ValueError(f"unknown preconditioner {kind!r}")
