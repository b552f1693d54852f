"""Pins for the oracle's GPLHR-EIG (Algorithm 3, Appendix A).

* It reaches the k eigenvalues nearest sigma of dense LAPACK, with eigenvector backward
  errors below tol, on a non-normal standard problem and a generalized pencil.
* Its eigenvalues are the Rayleigh quotients of its vectors (the appendix's
  motivation): alpha_j / beta_j = x_j^* A x_j / x_j^* B x_j for the returned X, and for a
  Hermitian A they obey the quadratic bound |rho - lambda| <= r^2 / delta,
  r = min over values of ||A x - value x|| for the unit vector x, delta the distance from
  rho to the rest of the spectrum (on this test's iterates the harmonic Ritz values meet
  the bound too, so the bound checks accuracy, the first check the definition).
* When the first trial subspace is the whole space ((m + 2) k = n), one iteration returns
  exact eigenvectors.
"""
import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from oracle import gplhr_eig as E
from oracle.precond import Preconditioner
from paper_1506_06829_gb300 import problems as P


def _nearest(ev, sigma, k):
    return ev[np.argsort(np.abs(ev - sigma))[:k]]


def test_eig_standard_nonnormal_vs_lapack():
    A = P.schroedinger2d(12, 0.3)
    n, k, sigma = A.shape[0], 3, -2.0 - 0.5j
    T = Preconditioner("block_jacobi", blocks=[np.linalg.inv(A.toarray() - sigma * np.eye(n))], bs=n)
    r = E.solve_eig(A, None, sigma, P.start_block(n, k, 11), m=1, tol=1e-11, maxit=200, T=T)
    assert r.converged
    ev = sla.eigvals(A.toarray())
    for mu in _nearest(ev, sigma, k):
        assert np.min(np.abs(r.lam - mu)) <= 1e-9 * abs(mu)
    R = A @ r.X - r.X * r.lam[None, :]
    assert np.all(np.linalg.norm(R, axis=0) <= 1e-9 * abs(A).sum(axis=0).max())


def test_eig_values_are_rayleigh_quotients_of_returned_vectors():
    N = 6
    A, B = P.convdiff3d(N, (0.4, 0.2, 0.1)), P.mass3d(N)
    n, k, sigma = A.shape[0], 4, 300.0 + 40.0j
    T = Preconditioner("block_jacobi", blocks=[np.linalg.inv(A.toarray() - sigma * B.toarray())], bs=n)
    r = E.solve_eig(A, B, sigma, P.start_block(n, k, 14), m=1, tol=1e-6, maxit=200, T=T)
    for j in range(k):
        x = r.X[:, j]
        rq = (x.conj() @ (A @ x)) / (x.conj() @ (B @ x))
        assert abs(r.lam[j] - rq) <= 1e-12 * abs(rq)


def test_eig_generalized_vs_lapack():
    N = 6
    A, B = P.convdiff3d(N, (0.4, 0.2, 0.1)), P.mass3d(N)
    n, k, sigma = A.shape[0], 4, 300.0 + 40.0j
    T = Preconditioner("block_jacobi", blocks=[np.linalg.inv(A.toarray() - sigma * B.toarray())], bs=n)
    r = E.solve_eig(A, B, sigma, P.start_block(n, k, 12), m=1, tol=1e-11, maxit=200, T=T)
    assert r.converged
    ev = sla.eigvals(A.toarray(), B.toarray())
    for mu in _nearest(ev, sigma, k):
        assert np.min(np.abs(r.lam - mu)) <= 1e-9 * abs(mu)


def test_eig_rayleigh_quotients_are_quadratically_accurate():
    n, k = 400, 3
    d = np.linspace(1.0, 50.0, n) ** 1.3
    rng = np.random.default_rng(8)
    U = np.linalg.qr(rng.standard_normal((n, n)))[0]
    A = sp.csr_matrix(U @ np.diag(d) @ U.T)                  # Hermitian, known spectrum
    sigma = 0.0                                               # the lower end of the spectrum
    T = Preconditioner("identity")
    hist = []
    E.solve_eig(A, None, sigma, P.start_block(n, k, 13), m=2, tol=1e-300, maxit=30, T=T,
                callback=lambda X, a, b, res: hist.append((X.copy(), a / b)))
    checked = 0
    for X, rho in hist:
        for j in range(k):
            x = X[:, j] / np.linalg.norm(X[:, j])
            # the smallest residual any value gives for this x (independent of rho)
            r = np.linalg.norm(A @ x - (x.conj() @ (A @ x)) * x)
            i = np.argmin(np.abs(d - rho[j].real))
            delta = np.min(np.abs(np.delete(d, i) - rho[j].real))
            if r < 0.3 * delta:                               # the bound's range of validity
                assert abs(rho[j] - d[i]) <= r * r / delta * (1 + 1e-6) + 1e-12 * d.max(), (j, r)
                checked += 1
    assert checked >= k


def test_eig_whole_space_one_iteration_exact():
    rng = np.random.default_rng(9)
    n, k, m = 12, 2, 4                                         # (m + 2) k = n
    A = sp.csr_matrix(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    sigma = 0.2 - 0.3j
    r = E.solve_eig(A, None, sigma, rng.standard_normal((n, k)), m=m, tol=1e-300, maxit=1,
                    T=Preconditioner("identity"))
    ev = sla.eigvals(A.toarray())
    want = _nearest(ev, sigma, k)
    for mu in want:
        assert np.min(np.abs(r.lam - mu)) <= 1e-10 * np.abs(ev).max()
    assert np.all(r.resid <= 1e-13)
