"""torch.autograd wrapper around gplhr_grad: eigenvalues of a sparse pencil as a
differentiable function of the stored values of A (and B).

    lam = eigenvalues(A_vals, pattern_A, sigma, k, m, ..., B_vals=None, pattern_B=None)
    loss(lam).backward()            # fills A_vals.grad (and B_vals.grad)

Forward solves GPLHR on (A, B) at sigma and on (A^*, B^*) at conj(sigma) through the C
ABI; backward calls gplhr_grad, whose kernel scatters
y_i^*(dA - lambda_i dB) x_i / (y_i^* B x_i) onto the CSR patterns.  With
recompute=True the contexts (and their n x s blocks) are released after forward and
both solves are repeated, from the same seeded start block, in backward.  This module
only marshals arguments; all arithmetic runs in libgplhr.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import torch

from . import gplhr as G


def _csr(pattern, vals: np.ndarray) -> sp.csr_matrix:
    indptr, indices, n = pattern
    return sp.csr_matrix((vals, indices, indptr), shape=(n, n))


def _solve_pair(A, B, sigma, k, m, opts, V0):
    right = G.GPLHR(A, B, sigma, k, m, **opts)
    right.solve(V0)
    AH = sp.csr_matrix(A.conj().T)
    BH = None if B is None else sp.csr_matrix(B.conj().T)
    lopts = dict(opts)
    if lopts.get("T") is not None:          # an explicit T ~ (A - sigma B)^{-1}: use T^*
        lopts["T"] = sp.csr_matrix(lopts["T"].conj().T)
    left = G.GPLHR(AH, BH, np.conj(sigma), k, m, **lopts)
    left.solve(V0)
    return right, left


class _Eigenvalues(torch.autograd.Function):
    @staticmethod
    def forward(fctx, a_vals, b_vals, pattern_A, pattern_B, sigma, k, m, opts, V0, recompute):
        A = _csr(pattern_A, a_vals.detach().cpu().numpy())
        B = None if b_vals is None else _csr(pattern_B, b_vals.detach().cpu().numpy())
        right, left = _solve_pair(A, B, sigma, k, m, opts, V0)
        lam = right.vectors()["lam"]
        fctx.meta = (pattern_A, pattern_B, sigma, k, m, opts, V0, recompute)
        fctx.save_for_backward(a_vals, b_vals if b_vals is not None else torch.empty(0))
        fctx.has_b = b_vals is not None
        if recompute:
            right.close()
            left.close()
            fctx.solvers = None
        else:
            fctx.solvers = (right, left)
        return torch.from_numpy(lam.astype(np.complex128))

    @staticmethod
    def backward(fctx, grad_lam):
        a_vals, b_vals = fctx.saved_tensors
        pattern_A, pattern_B, sigma, k, m, opts, V0, recompute = fctx.meta
        if fctx.solvers is None:
            A = _csr(pattern_A, a_vals.detach().cpu().numpy())
            B = _csr(pattern_B, b_vals.detach().cpu().numpy()) if fctx.has_b else None
            right, left = _solve_pair(A, B, sigma, k, m, opts, V0)
        else:
            right, left = fctx.solvers
        g = grad_lam.detach().cpu().numpy().astype(np.complex128)
        dA = torch.zeros_like(a_vals, device="cuda")
        dB = torch.zeros_like(b_vals, device="cuda") if fctx.has_b else None
        G.gplhr_grad(right.ctx, left.ctx, g, dA, dB)
        right.close()
        left.close()
        fctx.solvers = None
        gA = dA.to(a_vals.device)
        gB = dB.to(b_vals.device) if dB is not None else None
        return gA, gB, None, None, None, None, None, None, None, None


def eigenvalues(A_vals: torch.Tensor, pattern_A, sigma: complex, k: int, m: int = 1,
                B_vals: torch.Tensor | None = None, pattern_B=None, precond: str = "none",
                block_size: int = 1, T=None, tol: float = 1e-10, maxit: int = 500,
                V0: np.ndarray | None = None, seed: int = 0, recompute: bool = False):
    """The k eigenvalues of (A, B) nearest sigma (complex128 tensor), differentiable with
    respect to A_vals (and B_vals).  pattern = (indptr, indices, n) of the CSR matrix."""
    n = pattern_A[2]
    if V0 is None:
        V0 = np.random.default_rng(seed).standard_normal((n, k))
    opts = dict(precond=precond, block_size=block_size, T=T, tol=tol, maxit=maxit)
    return _Eigenvalues.apply(A_vals, B_vals, pattern_A, pattern_B, complex(sigma), k, m, opts,
                              V0, recompute)
