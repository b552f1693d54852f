"""Pins for the oracle's inner block GMRES preconditioner (oracle/gmres.py), T R = T0 Y*
with Y* = argmin over the block Krylov space K_s(K T0, R) of ||R - K T0 Y||_F (Sec. 4):

* a Krylov space that fills C^n gives the exact solve K W = R;
* first-order optimality, checked against an independent monomial basis of K_s: the
  residual R - K W is orthogonal to K T0 K_s, and T0^{-1} W lies in K_s (right
  preconditioning: a left-preconditioned or wrong-operator solve fails both);
* s = 1, one column: the closed form w = a T0 r, a = (K T0 r)^* r / ||K T0 r||^2;
* the residual norm never grows with s (nested spaces)."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import gplhr as OG
from oracle.gmres import BlockGmres
from oracle.precond import build, shifted
from paper_1506_06829_gb300 import problems as P


def _problem(n_side=6, sigma=30.0 + 4.0j):
    A = P.convdiff2d(n_side, 0.4, 0.2)
    return A, shifted(A, None, sigma), sigma


def _diag_blocks(K, bs):
    """blockdiag of K's bs x bs diagonal blocks (T0^{-1} of block Jacobi), built from K."""
    n = K.shape[0]
    D = np.zeros((n, n), dtype=np.complex128)
    Kd = K.toarray()
    for r0 in range(0, n, bs):
        r1 = min(n, r0 + bs)
        D[r0:r1, r0:r1] = Kd[r0:r1, r0:r1]
    return D


@pytest.mark.parametrize("kind,bs", [("none", 1), ("block_jacobi", 4)])
def test_full_krylov_space_gives_the_exact_solve(kind, bs):
    A, K, sigma = _problem(6)                       # n = 36
    n, k = K.shape[0], 3
    T = build(A, None, sigma, kind, bs, inner_steps=n // k)
    rng = np.random.default_rng(1)
    R = rng.standard_normal((n, k)) + 1j * rng.standard_normal((n, k))
    W = T.apply(R)
    assert np.linalg.norm(K @ W - R) <= 1e-9 * np.linalg.norm(R)


@pytest.mark.parametrize("s,k", [(1, 2), (3, 2), (4, 3)])
def test_minimal_residual_over_the_block_krylov_space(s, k):
    A, K, sigma = _problem(7)                       # n = 49
    n, bs = K.shape[0], 7
    T0 = build(A, None, sigma, "block_jacobi", bs)
    T = BlockGmres(K, T0, s)
    rng = np.random.default_rng(2)
    R = rng.standard_normal((n, k)) + 1j * rng.standard_normal((n, k))
    W = T.apply(R)
    # monomial basis of K_s(K T0, R), columns scaled to unit norm (no Arnoldi involved)
    blocks, X = [], R
    for _ in range(s):
        blocks.append(X / np.linalg.norm(X, axis=0))
        X = K @ T0.apply(blocks[-1])
    Mb = np.hstack(blocks)
    KTM = K @ T0.apply(Mb)
    res = R - K @ W
    assert np.linalg.norm(KTM.conj().T @ res) <= 1e-9 * np.linalg.norm(KTM) * np.linalg.norm(R)
    Y = _diag_blocks(K, bs) @ W                      # T0^{-1} W
    coef = np.linalg.lstsq(Mb, Y, rcond=None)[0]
    assert np.linalg.norm(Y - Mb @ coef) <= 1e-9 * np.linalg.norm(Y)


def test_one_step_one_column_closed_form():
    A, K, sigma = _problem(5)
    T0 = build(A, None, sigma, "block_jacobi", 5)
    r = np.random.default_rng(3).standard_normal((K.shape[0], 1)) + 0j
    z = T0.apply(r)
    Kz = K @ z
    a = (Kz.conj().T @ r)[0, 0] / np.vdot(Kz, Kz)
    w = BlockGmres(K, T0, 1).apply(r)
    assert np.linalg.norm(w - a * z) <= 1e-12 * np.linalg.norm(a * z)


def test_residual_never_grows_with_the_step_count():
    A, K, sigma = _problem(8)
    T0 = build(A, None, sigma, "jacobi")
    R = np.random.default_rng(4).standard_normal((K.shape[0], 4)) + 0j
    norms = [np.linalg.norm(R - K @ BlockGmres(K, T0, s).apply(R)) for s in range(1, 7)]
    assert all(b <= a * (1 + 1e-12) for a, b in zip(norms, norms[1:])), norms
    assert norms[-1] < norms[0]


def test_inner_gmres_cuts_outer_iterations():
    """Behaviour, not a pin: on a small copy of the complex Schroedinger workload
    (block-Jacobi 16), 3 inner steps need fewer GPLHR iterations than T0 alone."""
    pr = P.config3(24)
    V0 = P.start_block(pr.n, 4, 1003)
    its = []
    for s in (0, 3):
        r = OG.solve(pr.A, None, pr.sigma, V0, m=1, tol=1e-8, maxit=300, precond="block_jacobi",
                     block_size=16, inner_steps=s)
        assert r.converged
        its.append(r.iters)
    assert its[1] < its[0], its
