"""Pins for deflation in the oracle (Sec. 3.6, last paragraph): k Schur vectors from one
GPLHR run, k more from GPLHR on the deflated pair; together they are the 2k eigenvalues
nearest sigma (dense LAPACK), and the two blocks form one partial (generalized) Schur
form A [V1 V2] = [Q1 Q2] [[R_A1, Q1^* A V2], [0, R_A2]] (likewise B), with V2 orthogonal
to V1 and Q2 to Q1: what the paper states the deflated solve provides."""
import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from oracle import gplhr as G
from oracle.precond import Preconditioner
from paper_1506_06829_gb300 import problems as P


def _nearest(ev, sigma, k):
    return ev[np.argsort(np.abs(ev - sigma))[:k]]


def _match(got, want, rtol):
    for mu in want:
        assert np.min(np.abs(got - mu)) <= rtol * abs(mu), (mu, got)


def test_deflation_standard_two_stages():
    A = P.schroedinger2d(12, 0.3)
    n, k = A.shape[0], 3
    sigma = -2.0 - 0.5j
    ev = sla.eigvals(A.toarray())
    T = Preconditioner("block_jacobi", blocks=[np.linalg.inv(A.toarray() - sigma * np.eye(n))], bs=n)
    r1 = G.solve(A, None, sigma, P.start_block(n, k, 1), m=1, tol=1e-11, maxit=200, T=T)
    assert r1.converged
    r2 = G.solve(A, None, sigma, P.start_block(n, k, 2), m=1, tol=1e-11, maxit=200, T=T,
                 deflate=(r1.V, None))
    assert r2.converged
    lam = np.concatenate([r1.lam, r2.lam])
    _match(lam, _nearest(ev, sigma, 2 * k), 1e-9)
    V = np.hstack([r1.V, r2.V])
    assert np.linalg.norm(V.conj().T @ V - np.eye(2 * k)) < 1e-10
    R = np.zeros((2 * k, 2 * k), dtype=complex)
    R[:k, :k], R[k:, k:] = r1.R, r2.R
    R[:k, k:] = r1.V.conj().T @ (A @ r2.V)
    assert np.linalg.norm(A @ V - V @ R) < 1e-8 * G.onenorm(A)


def test_deflation_generalized_two_stages():
    N = 6
    A, B = P.convdiff3d(N, (0.4, 0.2, 0.1)), P.mass3d(N)
    sigma = 300.0 + 40.0j
    n, k = A.shape[0], 4
    Tm = np.linalg.inv(A.toarray() - sigma * B.toarray())
    T = Preconditioner("block_jacobi", blocks=[Tm], bs=n)
    ev = sla.eigvals(A.toarray(), B.toarray())
    r1 = G.solve(A, B, sigma, P.start_block(n, k, 3), m=1, tol=1e-11, maxit=200, T=T)
    assert r1.converged
    r2 = G.solve(A, B, sigma, P.start_block(n, k, 4), m=1, tol=1e-11, maxit=200, T=T,
                 deflate=(r1.V, r1.Q))
    assert r2.converged
    _match(np.concatenate([r1.lam, r2.lam]), _nearest(ev, sigma, 2 * k), 1e-9)
    V, Q = np.hstack([r1.V, r2.V]), np.hstack([r1.Q, r2.Q])
    assert np.linalg.norm(V.conj().T @ V - np.eye(2 * k)) < 1e-10
    assert np.linalg.norm(Q.conj().T @ Q - np.eye(2 * k)) < 1e-10
    for M, R1, R2 in ((A, r1.RA, r2.RA), (B, r1.RB, r2.RB)):
        R = np.zeros((2 * k, 2 * k), dtype=complex)
        R[:k, :k], R[k:, k:] = R1, R2
        R[:k, k:] = r1.Q.conj().T @ (M @ r2.V)
        assert np.linalg.norm(M @ V - Q @ R) < 1e-8 * G.onenorm(A)
