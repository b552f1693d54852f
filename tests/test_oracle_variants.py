"""Pins for the oracle's variants of the search directions P (Sec. 3.5, compared in the
paper's Table 2) and of the projector before T (Table 3).

* LOBPCG-style P (Eq. P_lobpcg): the paper states that P = V^(i-1) and
  P = V^(i) - V^(i-1) C give the same trial subspace; the harmonic extraction depends on
  the subspaces only, so runs with C = I, with a random invertible C and with
  P = V^(i-1) produce the same iterates to rounding, and differ from runs without P.
* No P (Eq. trial_partial): the trial subspace has (m + 2) k columns; when that is n,
  every iteration extracts from the whole space and returns the exact eigenvalues
  nearest sigma (dense LAPACK), also after the first iteration, where a P would
  otherwise have been appended.
* Without the right projector: when B = I and T = I the left projector (I - VV^*)
  absorbs the right one, so both forms give the same iterates; with T != I or B != I
  they differ.
"""
import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from oracle import gplhr as G
from oracle.precond import Preconditioner
from paper_1506_06829_gb300 import problems as P


def _run(A, B, sigma, V0, m, T, iters, **kw):
    pen = G.Pencil(A, B, sigma, T)
    st = G.init_state(pen, V0, m, **kw)
    out = []
    for _ in range(iters):
        st = G.iterate(pen, st)
        out.append((st.V.copy(), np.diag(st.RA) / np.diag(st.RB)))
    return out


def _angle(X, Y):
    return float(np.max(sla.subspace_angles(X, Y)))


def _pencil():
    # convection-diffusion plus a varying diagonal (with its constant diagonal alone the
    # Jacobi preconditioner would be a multiple of I)
    A0 = P.convdiff2d(12, 0.3, 0.2)
    n = A0.shape[0]
    A = (A0 + sp.diags(np.linspace(0.0, 0.5, n) * A0.diagonal().max())).tocsr()
    d = A.diagonal()
    sigma = (0.45 + 0.03j) * d.max()   # complex: no conjugate pairs tied in distance
    T = Preconditioner("jacobi", diag=1.0 / (d - sigma))
    V0 = np.random.default_rng(3).standard_normal((n, 3))
    return A, sigma, T, V0


def test_lobpcg_p_equals_previous_v_and_any_invertible_c():
    A, sigma, T, V0 = _pencil()
    k = V0.shape[1]
    rng = np.random.default_rng(4)
    C = np.eye(k) + 0.3 * (rng.standard_normal((k, k)) + 1j * rng.standard_normal((k, k)))
    runs = {
        "lobpcg": _run(A, None, sigma, V0, 1, T, 4, p_mode="lobpcg"),
        "lobpcg_C": _run(A, None, sigma, V0, 1, T, 4, p_mode="lobpcg", lobpcg_C=C),
        "previous": _run(A, None, sigma, V0, 1, T, 4, p_mode="previous"),
        "none": _run(A, None, sigma, V0, 1, T, 4, p_mode="none"),
    }
    for i in range(4):
        V, lam = runs["lobpcg"][i]
        for other in ("lobpcg_C", "previous"):
            V2, lam2 = runs[other][i]
            assert np.allclose(lam, lam2, rtol=1e-9, atol=0), (other, i)
            assert _angle(V, V2) < 1e-8, (other, i)
    # from the second iteration on P is in the trial subspace: the iterates move
    V, lam = runs["lobpcg"][3]
    Vn, lamn = runs["none"][3]
    assert np.max(np.abs(lam - lamn)) > 1e-6 * np.max(np.abs(lam))


def test_no_p_whole_space_gives_exact_eigenvalues():
    rng = np.random.default_rng(5)
    n, k, m = 12, 2, 4                       # (m + 2) k = n
    A = sp.csr_matrix(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    sigma = 0.3 + 0.1j
    ev = sla.eigvals(A.toarray())
    want = ev[np.argsort(np.abs(ev - sigma))[:k]]
    T = Preconditioner("identity")
    V0 = rng.standard_normal((n, k))
    for V, lam in _run(A, None, sigma, V0, m, T, 3, p_mode="none"):
        for mu in want:
            assert np.min(np.abs(lam - mu)) < 1e-9 * np.max(np.abs(ev))


def test_right_projector_absorbed_when_t_and_b_are_identity():
    A, sigma, _, V0 = _pencil()
    T = Preconditioner("identity")
    with_p = _run(A, None, sigma, V0, 1, T, 3, right_proj=True)
    without = _run(A, None, sigma, V0, 1, T, 3, right_proj=False)
    for (V, lam), (V2, lam2) in zip(with_p, without):
        assert np.allclose(lam, lam2, rtol=1e-10, atol=0)
        assert _angle(V, V2) < 1e-9
    # with T != I the two forms differ, also when B = I (so the omitted projector is not
    # replaced by another one)
    _, _, Tj, _ = _pencil()
    s1 = _run(A, None, sigma, V0, 1, Tj, 2, right_proj=True)
    s2 = _run(A, None, sigma, V0, 1, Tj, 2, right_proj=False)
    assert np.max(np.abs(s1[1][1] - s2[1][1])) > 1e-8 * np.max(np.abs(s1[1][1]))
    # generalized: (I - VV^*) T (I - QQ^*) differs from (I - VV^*) T
    n = A.shape[0]
    B = P.convdiff2d_mass(12, 0.3, 0.2)[1]
    Vg0 = np.random.default_rng(6).standard_normal((n, 3))
    g1 = _run(A, B, sigma, Vg0, 1, T, 2, right_proj=True)
    g2 = _run(A, B, sigma, Vg0, 1, T, 2, right_proj=False)
    assert np.max(np.abs(g1[1][1] - g2[1][1])) > 1e-8 * np.max(np.abs(g1[1][1]))
