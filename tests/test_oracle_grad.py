"""Pins for the oracle's eigenvalue adjoint (oracle/grad.py): central finite differences
of the eigenvalues themselves (dense LAPACK eigensolves of perturbed matrices), the
per-edge chain rule of the differentiation workload, and agreement between vectors
from GPLHR (right solve on (A, B), left solve on (A^*, B^*)) and from dense LAPACK."""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

from oracle import gplhr as OG
from oracle.grad import eig_grad, pair
from oracle.precond import Preconditioner
from paper_1506_06829_gb300 import problems as P


def _nearest(ev, sigma, k):
    return ev[np.argsort(np.abs(ev - sigma))[:k]]


def _loss(A, B, sigma, k, G):
    ev = sla.eigvals(A, B) if B is not None else sla.eigvals(A)
    lam = _nearest(ev, sigma, k)
    return lam, float(np.sum((np.conj(G) * lam).real))


def _dense_vectors(A, B, lam):
    w, vl, vr = sla.eig(A, B, left=True, right=True) if B is not None else \
        sla.eig(A, left=True, right=True)
    idx = [int(np.argmin(np.abs(w - l))) for l in lam]
    return vr[:, idx], vl[:, idx]


@pytest.mark.parametrize("complex_A,with_B", [(False, False), (False, True), (True, True)])
def test_adjoint_matches_central_differences(complex_A, with_B):
    rng = np.random.default_rng(31)
    n, k = 9, 3
    A = rng.standard_normal((n, n)) + (1j * rng.standard_normal((n, n)) if complex_A else 0)
    B = (np.eye(n) + 0.2 * rng.standard_normal((n, n))) if with_B else None
    sigma = 0.3 + 0.2j
    G = rng.standard_normal(k) + 1j * rng.standard_normal(k)
    lam, _ = _loss(A, B, sigma, k, G)
    X, Y = _dense_vectors(A, B, lam)
    dA, dB = eig_grad(sp.csr_matrix(A), None if B is None else sp.csr_matrix(B), lam, X, Y, G)
    delta = 1e-6
    # every entry of A (and B): real part, and imaginary part for complex A
    for (p, q) in [(0, 0), (1, 4), (7, 2), (8, 8), (3, 6)]:
        e = np.zeros((n, n))
        e[p, q] = 1.0
        fd = (_loss(A + delta * e, B, sigma, k, G)[1] - _loss(A - delta * e, B, sigma, k, G)[1]) / (2 * delta)
        got = dA[p * n + q]
        assert abs(np.real(got) - fd) <= 1e-6 * max(1.0, abs(fd)), (p, q, got, fd)
        if complex_A:
            fdi = (_loss(A + 1j * delta * e, B, sigma, k, G)[1]
                   - _loss(A - 1j * delta * e, B, sigma, k, G)[1]) / (2 * delta)
            assert abs(np.imag(got) - fdi) <= 1e-6 * max(1.0, abs(fdi))
        if with_B:
            fdb = (_loss(A, B + delta * e, sigma, k, G)[1] - _loss(A, B - delta * e, sigma, k, G)[1]) / (2 * delta)
            assert abs(np.real(dB[p * n + q]) - fdb) <= 1e-6 * max(1.0, abs(fdb))


def test_edge_chain_rule_matches_finite_differences():
    """Gradient of sum Re(lambda_i) w.r.t. the per-edge convection field b (6 x 6 grid)."""
    N, k = 6, 3
    pr = P.config5(N)
    b = pr.meta["b"]
    A = pr.A
    sigma = pr.sigma + 7.0
    ev = sla.eigvals(A.toarray())
    lam = _nearest(ev, sigma, k)
    X, Y = _dense_vectors(A.toarray(), None, lam)
    G = np.ones(k, dtype=np.complex128)             # L = sum Re(lambda_i)
    dA, _ = eig_grad(A, None, lam, X, Y, G)
    J = P.edge_jacobian(N, A)
    db = J.T @ dA
    delta = 1e-6
    for e in [0, 5, 17, 29, 44, 59]:
        bp, bm = b.copy(), b.copy()
        bp[e] += delta
        bm[e] -= delta
        Lp = np.sum(_nearest(sla.eigvals(P.convdiff2d_edges(N, bp).toarray()), sigma, k).real)
        Lm = np.sum(_nearest(sla.eigvals(P.convdiff2d_edges(N, bm).toarray()), sigma, k).real)
        fd = (Lp - Lm) / (2 * delta)
        assert abs(db[e] - fd) <= 1e-5 * max(1.0, abs(fd)), (e, db[e], fd)


def test_gplhr_left_right_vectors_give_the_dense_gradient():
    """Right solve on (A, B) at sigma, left solve on (A^*, B^*) at conj(sigma), paired by
    eigenvalue: the adjoint equals the one from dense LAPACK eigenvectors."""
    N = 6
    A, B = P.convdiff3d(N, (0.4, 0.2, 0.1)), P.mass3d(N)
    sigma = 300.0 + 40.0j
    n, k = A.shape[0], 4
    AH, BH = sp.csr_matrix(A.conj().T), sp.csr_matrix(B.conj().T)
    Tr = Preconditioner("block_jacobi", blocks=[np.linalg.inv(A.toarray() - sigma * B.toarray())], bs=n)
    Tl = Preconditioner("block_jacobi",
                        blocks=[np.linalg.inv(AH.toarray() - np.conj(sigma) * BH.toarray())], bs=n)
    V0 = P.start_block(n, k, 5)
    r = OG.solve(A, B, sigma, V0, m=1, tol=1e-12, maxit=200, T=Tr)
    l = OG.solve(AH, BH, np.conj(sigma), V0, m=1, tol=1e-12, maxit=200, T=Tl)
    assert r.converged and l.converged

    def vecs(res):
        Zv = OG.tri_eigvecs(res.RA, res.RB)
        Xv = res.V @ Zv
        return Xv / np.linalg.norm(Xv, axis=0)

    X, Yl = vecs(r), vecs(l)
    perm = pair(r.lam, l.lam)
    Y = Yl[:, perm]
    G = np.array([1.0, 0.5 - 0.25j, -1.0j, 2.0])
    dA, dB = eig_grad(A, B, r.lam, X, Y, G)
    Xd, Yd = _dense_vectors(A.toarray(), B.toarray(), r.lam)
    dA2, dB2 = eig_grad(A, B, r.lam, Xd, Yd, G)
    assert np.linalg.norm(dA - dA2) <= 1e-7 * np.linalg.norm(dA2)
    assert np.linalg.norm(dB - dB2) <= 1e-7 * np.linalg.norm(dB2)


def test_pair_rejects_missing_match():
    with pytest.raises(ValueError):
        pair(np.array([1.0 + 1j, 2.0]), np.array([1.0 - 1j, 3.0]))
