"""T as an inner linear solve (Sec. 4): s steps of block GMRES on (A - sigma B) W = R.
Test infrastructure only (see the package docstring).

Definition (zero initial guess, right preconditioning by a basic preconditioner T0,
Sec. 4): with K = A - sigma B and the block Krylov space

    K_s = span{R, (K T0) R, ..., (K T0)^{s-1} R}      (n x s k, block columns),

T R = T0 Y*, where Y* in K_s minimises the Frobenius norm ||R - K T0 Y||_F; since the
columns decouple, every column of R is minimised over the whole block space.  The
oracle builds an orthonormal basis of K_s by block Arnoldi (block classical
Gram-Schmidt applied twice, Householder QR of each new block), so that
K T0 V_s = V_{s+1} H with H block upper Hessenberg and R = V_1 B0, and solves the
small least-squares problem min ||E1 B0 - H Y||_F with numpy's lstsq.

Readings: the paper's experiments run single-vector GMRES per column (Sec. 5.3) and
recommend block solvers for speed (Sec. 4); this is the block form.  The number of
steps s is fixed (no inner tolerance).  If the space stops growing (an exact
solution inside K_j), the Householder QR of a zero block still returns orthonormal
columns with a zero H entry and lstsq returns the minimum-norm minimiser, which is
then the exact solution.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


class BlockGmres:
    """T = s steps of right-preconditioned block GMRES on (A - sigma B) W = R."""

    def __init__(self, K: sp.spmatrix, T0, steps: int):
        if steps < 1:
            raise ValueError("block GMRES needs at least one step")
        self.K = sp.csr_matrix(K)
        self.T0 = T0
        self.steps = steps
        self.kind = "gmres"

    def apply(self, R: np.ndarray) -> np.ndarray:
        R = np.asarray(R, dtype=np.complex128)
        n, w = R.shape
        s = self.steps
        V1, B0 = np.linalg.qr(R)
        basis = [V1]
        H = np.zeros(((s + 1) * w, s * w), dtype=np.complex128)
        for j in range(s):
            Wj = self.K @ self.T0.apply(basis[j])          # K T0 v_j
            for _ in range(2):                             # block CGS, twice
                for i in range(j + 1):
                    h = basis[i].conj().T @ Wj
                    H[i * w:(i + 1) * w, j * w:(j + 1) * w] += h
                    Wj = Wj - basis[i] @ h
            Vn, Rn = np.linalg.qr(Wj)
            H[(j + 1) * w:(j + 2) * w, j * w:(j + 1) * w] = Rn
            basis.append(Vn)
        E = np.zeros(((s + 1) * w, w), dtype=np.complex128)
        E[:w] = B0
        Y = np.linalg.lstsq(H, E, rcond=None)[0]
        return self.T0.apply(np.hstack(basis[:s]) @ Y)
