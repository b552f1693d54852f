"""Pins for the oracle's Algorithm 2 (GPLHR) and its building blocks.

Each GPLHR run is checked against answers fixed independently of the oracle:
exact spectra of diagonal pencils, closed-form spectra of the stencil operators
(sine eigenvectors), dense LAPACK eigenvalues of small copies, and the
invariants the paper states (orthonormal V and Q, Prop. 3.2, Eq. gschur2,
the residual identity after Alg. 2).
"""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

from oracle import gplhr as G
from oracle.precond import Preconditioner, build as build_precond
from paper_1506_06829_gb300 import problems as P


def _subspace_angle(X, Y):
    return float(np.max(sla.subspace_angles(X, Y)))


# ----------------------------------------------------------------- orth ------

def _gram_schmidt_twice(X):
    """Independent brute-force orthonormalisation: modified Gram-Schmidt, twice,
    column by column in plain Python loops."""
    n, k = X.shape
    Qm = np.zeros_like(X, dtype=np.complex128)
    for j in range(k):
        v = X[:, j].astype(np.complex128)
        for _ in range(2):
            for i in range(j):
                v = v - Qm[:, i] * np.vdot(Qm[:, i], v)
        Qm[:, j] = v / np.linalg.norm(v)
    return Qm


def test_orth_is_unique_positive_qr():
    rng = np.random.default_rng(11)
    X = rng.standard_normal((40, 6)) + 1j * rng.standard_normal((40, 6))
    Qm = G.orth(X)
    assert np.allclose(Qm.conj().T @ Qm, np.eye(6), atol=1e-13)
    R = Qm.conj().T @ X
    assert np.allclose(np.tril(R, -1), 0, atol=1e-12)
    assert np.all(np.abs(np.diag(R).imag) < 1e-12) and np.all(np.diag(R).real > 0)
    assert np.allclose(Qm, _gram_schmidt_twice(X), atol=1e-12)


# -------------------------------------------------------------- precond ------

def test_block_jacobi_inverts_diagonal_blocks():
    pr = P.config3(12)
    sigma = pr.sigma
    T = build_precond(pr.A, None, sigma, "block_jacobi", 16)
    K = (pr.A - sigma * sp.identity(pr.n)).toarray()
    TK = T.apply(K)
    n, bs = pr.n, 16
    for r0 in range(0, n, bs):          # n = 144: 9 blocks, the last one is full
        r1 = min(n, r0 + bs)
        assert np.allclose(TK[r0:r1, r0:r1], np.eye(r1 - r0), atol=1e-10)


def test_block_jacobi_ragged_tail_and_jacobi():
    rng = np.random.default_rng(12)
    n = 21
    A = sp.csr_matrix(rng.standard_normal((n, n)) + 5 * np.eye(n))
    T = build_precond(A, None, 0.5 + 0.25j, "block_jacobi", 8)
    K = A.toarray() - (0.5 + 0.25j) * np.eye(n)
    TK = T.apply(K)
    for r0, r1 in ((0, 8), (8, 16), (16, 21)):
        assert np.allclose(TK[r0:r1, r0:r1], np.eye(r1 - r0), atol=1e-12)
    Tj = build_precond(A, None, 0.5 + 0.25j, "jacobi")
    assert np.allclose(Tj.apply(np.diag(K)[:, None])[:, 0], 1.0)
    # constant diagonal -> identity (any constant scaling of T is the same iteration)
    Ac = P.config1(8)
    Tc = build_precond(Ac.A, None, Ac.sigma, "jacobi")
    assert Tc.kind == "identity"


# ------------------------------------------------------------- GPLHR ---------

def _exact_T(A, B, sigma):
    n = A.shape[0]
    Bm = np.eye(n) if B is None else B.toarray()
    return Preconditioner("block_jacobi", blocks=[np.linalg.inv(A.toarray() - sigma * Bm)], bs=n)


def test_gplhr_diagonal_standard_exact_answer():
    n, k = 200, 4
    d = np.arange(1, n + 1, dtype=float)
    A = sp.diags(d).tocsr()
    V0 = np.random.default_rng(0).standard_normal((n, k))
    T = Preconditioner("jacobi", diag=1.0 / (d - 50.3))
    r = G.solve(A, None, 50.3, V0, m=1, tol=1e-10, maxit=50, T=T)
    assert r.converged
    assert np.allclose(np.sort(r.lam.real), [49, 50, 51, 52], atol=1e-9)
    E = np.zeros((n, k))
    E[[48, 49, 50, 51], range(k)] = 1
    assert _subspace_angle(r.V, E) < 1e-8


def test_gplhr_diagonal_generalized_exact_answer():
    n, k = 200, 4
    d = np.arange(1, n + 1, dtype=float)
    b = np.linspace(1, 2, n)
    A, B = sp.diags(d).tocsr(), sp.diags(b).tocsr()
    lam = d / b
    V0 = np.random.default_rng(1).standard_normal((n, k))
    T = Preconditioner("jacobi", diag=1.0 / (d - 30.0 * b))
    r = G.solve(A, B, 30.0, V0, m=1, tol=1e-10, maxit=50, T=T)
    assert r.converged
    want = lam[np.argsort(np.abs(lam - 30.0))[:k]]
    assert np.allclose(np.sort(r.lam.real), np.sort(want), rtol=1e-11)
    # partial generalized Schur form A V = Q R_A, B V = Q R_B (Eq. gschur)
    # Schur residuals within a small multiple of tol * (||A||_1 + |lam| ||B||_1)
    scale = 10 * np.sqrt(k) * 1e-10 * (d.max() + 30.0 * b.max())
    assert np.linalg.norm(A @ r.V - r.Q @ r.RA) < scale
    assert np.linalg.norm(B @ r.V - r.Q @ r.RB) < scale


def test_gplhr_generalized_stencil_closed_form():
    """gamma = 0 3-D pencil (A, M x M x M): closed-form spectrum (sine vectors).
    k = 3 targets a triple eigenvalue (the cube's symmetry), a degenerate case."""
    N, k = 6, 3
    A = P.convdiff3d(N, (0.0, 0.0, 0.0))
    B = P.mass3d(N)
    ev = P.sym_pencil3d_eigs(N)
    es = np.unique(np.round(np.sort(ev), 9))
    sigma = es[2] * 0.97 + 1.0j          # just below the third distinct eigenvalue
    dist = np.sort(np.abs(ev - sigma))
    assert dist[k] > 1.05 * dist[k - 1]   # the k-th and (k+1)-th are well separated
    want = ev[np.argsort(np.abs(ev - sigma))[:k]]
    V0 = P.start_block(A.shape[0], k, 7)
    r = G.solve(A, B, sigma, V0, m=1, tol=1e-10, maxit=100, T=_exact_T(A, B, sigma))
    assert r.converged
    # ev has multiplicities; compare as multisets
    assert np.allclose(np.sort(r.lam.real), np.sort(want), rtol=1e-10)
    assert np.abs(r.lam.imag).max() < 1e-8 * np.abs(r.lam).max()
    assert np.allclose(r.V.conj().T @ r.V, np.eye(k), atol=1e-12)
    assert np.allclose(r.Q.conj().T @ r.Q, np.eye(k), atol=1e-12)


def test_gplhr_convection_diffusion_closed_form():
    """Non-normal 2-D convection-diffusion: closed-form real spectrum.  Eigenvalue
    error bound: kappa(lambda) * backward error (H1 non-normality)."""
    N, k = 16, 4
    pr = P.config1(N)
    ev = pr.meta["closed_form"]
    sigma = np.sort(ev)[2] + 0.3        # near the low end of the spectrum
    want = ev[np.argsort(np.abs(ev - sigma))[:k]]
    r = G.solve(pr.A, None, sigma, pr.start_block(), m=1, tol=1e-10, maxit=200,
                T=_exact_T(pr.A, None, sigma))
    assert r.converged
    # dense eigenvectors give kappa(lambda) = ||x|| ||y|| / |y^* x|
    w, vl, vr = sla.eig(pr.A.toarray(), left=True, right=True)
    for lam in r.lam:
        i = np.argmin(np.abs(w - lam))
        kappa = 1.0 / abs(np.vdot(vl[:, i], vr[:, i]))
        j = np.argmin(np.abs(want - lam.real))
        bound = max(1e-12, 10 * kappa * 1e-10 * (G.onenorm(pr.A) + abs(lam)))
        assert abs(lam - want[j]) <= bound, (lam, want[j], kappa)
    assert np.max(r.resid) <= 1e-10


def test_gplhr_complex_scaled_free_closed_form():
    """V = 0 complex-scaled Laplacian: lambda = e^{-2 i theta} (4/h^2)(sin^2 + sin^2)."""
    N, k = 12, 6
    A = P.schroedinger2d(N, 0.3, with_potential=False)
    ev = P.schroedinger2d_free_eigs(N, 0.3)
    sigma = ev[np.argsort(np.abs(ev))[4]] * 1.02 + 0.5j
    want = ev[np.argsort(np.abs(ev - sigma))[:k]]
    V0 = P.start_block(A.shape[0], k, 3)
    r = G.solve(A, None, sigma, V0, m=2, tol=1e-11, maxit=200, precond="block_jacobi",
                block_size=12)
    assert r.converged
    for lam in r.lam:
        assert np.min(np.abs(want - lam)) <= 1e-9 * abs(lam)
    for mu in want:
        assert np.min(np.abs(r.lam - mu)) <= 1e-9 * abs(mu)


def test_gplhr_schroedinger_small_vs_dense_lapack():
    """Config-3 operator (potential well) on a 24 x 24 grid vs dense zgeev."""
    pr = P.config3(24)
    k = pr.k
    ev = sla.eigvals(pr.A.toarray())
    want = ev[np.argsort(np.abs(ev - pr.sigma))[:k]]
    r = G.solve(pr.A, None, pr.sigma, pr.start_block(), m=pr.m, tol=1e-10, maxit=300,
                precond="block_jacobi", block_size=pr.block_size)
    assert r.converged
    for mu in want:
        assert np.min(np.abs(r.lam - mu)) <= 1e-8 * abs(mu)
    n = pr.n
    assert np.allclose(r.V.conj().T @ r.V, np.eye(k), atol=1e-12)
    # B = I output: A V = V R (Eq. schur), R upper triangular; M_B -> I (Sec. 3.4)
    assert np.linalg.norm(pr.A @ r.V - r.V @ r.R) <= 1e-8 * G.onenorm(pr.A)
    assert np.allclose(np.tril(r.R, -1), 0, atol=1e-8 * G.onenorm(pr.A))
    assert np.linalg.norm(r.MB - np.eye(k)) <= 1e-6


def test_prop32_and_residual_identity_one_step():
    """After one iteration: (A - sigma B) V = Q (R_A - sigma R_B) (Prop. 3.2), and the
    identity (I - QQ^*)(W_A M_B - W_B M_A) = (I - QQ^*)(A V M_B - B V M_A)."""
    N = 6
    A = P.convdiff3d(N, (0.4, 0.2, 0.1))
    B = P.mass3d(N)
    sigma = 800.0 + 50.0j
    T = build_precond(A, B, sigma, "block_jacobi", 6)
    pen = G.Pencil(A, B, sigma, T)
    st = G.init_state(pen, P.start_block(A.shape[0], 3, 5), 1)
    for _ in range(3):
        st = G.iterate(pen, st)
    Ac, Bc = pen.A, pen.B
    lhs = Ac @ st.V - sigma * (Bc @ st.V)
    rhs = st.Q @ (st.RA - sigma * st.RB)
    assert np.linalg.norm(lhs - rhs) <= 1e-11 * np.linalg.norm(lhs)
    AV, BV = Ac @ st.V, Bc @ st.V
    WA, WB = AV - st.Q @ st.RA, BV - st.Q @ st.RB
    X1 = WA @ st.MB - WB @ st.MA
    X2 = AV @ st.MB - BV @ st.MA
    proj = lambda X: X - st.Q @ (st.Q.conj().T @ X)
    assert np.linalg.norm(proj(X1) - proj(X2)) <= 1e-12 * np.linalg.norm(X2)
    assert np.allclose(st.V.conj().T @ st.V, np.eye(3), atol=1e-13)


def test_residual_measure_on_exact_and_perturbed_pairs():
    """residuals() is the backward error ||Ax - lam Bx|| / ((||A||_1 + |lam| ||B||_1)||x||)."""
    rng = np.random.default_rng(21)
    n, k = 30, 3
    A = sp.csr_matrix(rng.standard_normal((n, n)))
    B = sp.csr_matrix(np.eye(n) + 0.1 * rng.standard_normal((n, n)))
    AA, BB, Ql, Zr = sla.qz(A.toarray(), B.toarray(), output="complex")
    T = Preconditioner("identity")
    pen = G.Pencil(A, B, 0.0, T)
    st = G.State(Zr[:, :k], Ql[:, :k], None, AA[:k, :k], BB[:k, :k], None, None, 0, 1, 1)
    assert np.max(G.residuals(pen, st)) < 1e-14
    # one exact eigenpair perturbed by a known vector: brute-force backward error
    w, X = sla.eig(A.toarray(), B.toarray())
    x = X[:, 0] + 1e-6 * rng.standard_normal(n)
    lam = w[0]
    want = np.linalg.norm(A @ x - lam * (B @ x)) / (
        (np.abs(A.toarray()).sum(0).max() + abs(lam) * np.abs(B.toarray()).sum(0).max())
        * np.linalg.norm(x))
    st1 = G.State(x[:, None] / np.linalg.norm(x), None, None, np.array([[lam]]),
                  np.array([[1.0 + 0j]]), None, None, 0, 1, 1)
    assert np.isclose(G.residuals(pen, st1)[0], want, rtol=1e-10)
