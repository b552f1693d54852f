"""Pins for the oracle's Q-free Schur algebra and ordered QZ (Sec. 2.2, Alg. 2 step 2).

Every check compares against something other than the oracle itself: the
diagonal values the paper states after Eqs. G1_fix/G2_fix, Theorem 1's identity
on an exact generalized Schur form from LAPACK, and LAPACK's unordered
generalized eigenvalues (zggev) for the ordered QZ.
"""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle.ordqz import distance, ordqz
from oracle.schur import g_factors, m_factors


def _rand_tri(rng, k, scale=1.0):
    R = np.triu(rng.standard_normal((k, k)) + 1j * rng.standard_normal((k, k)))
    return R * scale


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_lemma1_unit_diagonal_and_stated_diagonals(seed):
    rng = np.random.default_rng(seed)
    k = 9
    RA = _rand_tri(rng, k)
    RB = _rand_tri(rng, k)
    # force both branches of Eqs. G1_fix/G2_fix, plus a zero and an infinite eigenvalue
    RA[0, 0] = 1e-3 * RB[0, 0]
    RB[1, 1] = 1e-3 * RA[1, 1]
    RA[2, 2] = 0.0
    RB[3, 3] = 0.0
    MA, MB, G = m_factors(RA, RB)
    assert np.allclose(np.diag(G), 1.0, atol=1e-14)                # Lemma 1
    assert np.allclose(np.tril(G, -1), 0.0)
    for j in range(k):                                            # text after Eq. G2_fix
        a, b = RA[j, j], RB[j, j]
        if abs(a) < abs(b):
            assert np.isclose(MA[j, j], a / b, rtol=1e-13, atol=1e-15)
            assert np.isclose(MB[j, j], 1.0, rtol=1e-13)
        else:
            assert np.isclose(MA[j, j], a, rtol=1e-13)
            assert np.isclose(MB[j, j], b, rtol=1e-13, atol=1e-15)
    assert np.allclose(np.tril(MA, -1), 0.0) and np.allclose(np.tril(MB, -1), 0.0)
    g1, g2 = g_factors(RA, RB)
    assert np.allclose(np.diag(RA) * g1 + np.diag(RB) * g2, 1.0)


@pytest.mark.parametrize("seed", [3, 4])
def test_theorem1_qfree_form_on_exact_schur(seed):
    """A V M_B = B V M_A for an exact partial generalized Schur form (Thm 1)."""
    rng = np.random.default_rng(seed)
    n, k = 14, 5
    A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    B = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    AA, BB, Ql, Zr = sla.qz(A, B, output="complex")
    V = Zr[:, :k]
    RA, RB = AA[:k, :k], BB[:k, :k]
    assert np.allclose(A @ V, Ql[:, :k] @ RA, atol=1e-12)
    MA, MB, _ = m_factors(RA, RB)
    E = A @ V @ MB - B @ V @ MA
    assert np.linalg.norm(E) <= 1e-12 * (np.linalg.norm(A) + np.linalg.norm(B))
    lam = np.diag(MA) / np.diag(MB)
    assert np.allclose(lam, np.diag(RA) / np.diag(RB), rtol=1e-12)


def test_standard_case_limits():
    """For B = I and an exact Schur form, M_A -> R and M_B -> I (Sec. 3.4)."""
    rng = np.random.default_rng(5)
    R = _rand_tri(rng, 6)
    MA, MB, _ = m_factors(R, np.eye(6))
    big = np.abs(np.diag(R)) >= 1.0
    # |R(j,j)| >= 1 takes the second branch (M_A(j,j) = R(j,j), M_B(j,j) = 1)
    assert np.allclose(np.diag(MA)[big], np.diag(R)[big])
    R2 = R.copy()
    np.fill_diagonal(R2, 2.0 + np.arange(6))     # all |R(j,j)| >= |1|
    MA2, MB2, _ = m_factors(R2, np.eye(6))
    assert np.allclose(MA2, R2, atol=1e-13) and np.allclose(MB2, np.eye(6), atol=1e-13)


@pytest.mark.parametrize("seed,sigma", [(6, 0.3 + 0.1j), (7, -1.0 + 0.0j), (8, 2.0 - 1.0j)])
def test_ordqz_against_lapack_eigvals(seed, sigma):
    rng = np.random.default_rng(seed)
    s = 17
    Phi = rng.standard_normal((s, s)) + 1j * rng.standard_normal((s, s))
    Psi = rng.standard_normal((s, s)) + 1j * rng.standard_normal((s, s))
    RA, RB, YL, YR = ordqz(Phi, Psi, sigma)
    I = np.eye(s)
    assert np.allclose(YL.conj().T @ YL, I, atol=1e-13)
    assert np.allclose(YR.conj().T @ YR, I, atol=1e-13)
    assert np.allclose(np.tril(RA, -1), 0) and np.allclose(np.tril(RB, -1), 0)
    assert np.allclose(Phi @ YR, YL @ RA, atol=1e-12)
    assert np.allclose(Psi @ YR, YL @ RB, atol=1e-12)
    lam = np.diag(RA) / np.diag(RB)
    ref = sla.eigvals(Phi, Psi)                         # LAPACK zggev, independent path
    d_ref = np.sort(np.abs(ref - sigma))
    d = np.abs(lam - sigma)
    assert np.all(np.diff(d) >= -1e-12 * d.max())       # non-decreasing distance
    assert np.allclose(np.diag(RB).imag, 0) and np.all(np.diag(RB).real >= 0)
    assert np.allclose(d, d_ref, rtol=1e-10)
    # multiset match of the eigenvalues themselves
    for mu in ref:
        assert np.min(np.abs(lam - mu)) <= 1e-10 * max(1, abs(mu))


def test_ordqz_infinite_eigenvalue_last():
    rng = np.random.default_rng(9)
    s = 6
    Phi = rng.standard_normal((s, s)) + 0j
    Psi = rng.standard_normal((s, s)) + 0j
    Psi[:, 0] = 0.0                                    # singular B part: one infinite eigenvalue
    RA, RB, YL, YR = ordqz(Phi, Psi, 0.1)
    assert abs(RB[-1, -1]) <= 1e-12 * np.abs(Psi).max()
    assert all(np.isfinite(distance(RA[j, j], RB[j, j], 0.1)) for j in range(s - 1))
