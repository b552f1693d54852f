"""GPU parity of the eigenvalue adjoint (gplhr_grad) against the CPU oracle's adjoint,
and of the torch.autograd path against finite differences.

Tolerance: the adjoint is linear in x_i and y_i, which both solves deliver to their
residual tolerance (1e-11 here) times the eigenvector condition; 1e-7 relative on the
whole gradient vector is well above that and far below any formula error (a wrong sign,
conjugation or index changes the result by O(1))."""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

torch = pytest.importorskip("torch")

from oracle.grad import eig_grad
from paper_1506_06829_gb300 import gplhr as G
from paper_1506_06829_gb300 import problems as P

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _dense_pairs(A, B, sigma, k):
    Ad = A.toarray()
    Bd = None if B is None else B.toarray()
    w, vl, vr = sla.eig(Ad, Bd, left=True, right=True) if Bd is not None else sla.eig(Ad, left=True, right=True)
    idx = np.argsort(np.abs(w - sigma))[:k]
    return w[idx], vr[:, idx], vl[:, idx]


def _exact_T(A, B, sigma):
    n = A.shape[0]
    Bd = np.eye(n) if B is None else B.toarray()
    return sp.csr_matrix(np.linalg.inv(A.toarray() - sigma * Bd))


@pytest.mark.parametrize("case", ["edges_real_B_I", "generalized_real", "complex_A"])
def test_gplhr_grad_matches_oracle_adjoint(case):
    if case == "edges_real_B_I":
        pr = P.config5(8)
        A, B, sigma, k = pr.A, None, pr.sigma + 3.0, 4
    elif case == "generalized_real":
        A, B = P.convdiff3d(6, (0.4, 0.2, 0.1)), P.mass3d(6)
        sigma, k = 300.0 + 40.0j, 4
    else:
        # complex-scaled Schroedinger plus a seeded complex diagonal: the square's symmetry
        # would otherwise give exact double eigenvalues, whose individual derivatives do
        # not exist (gplhr_grad refuses them)
        rng = np.random.default_rng(4)
        A0 = P.schroedinger2d(10, 0.3)
        A = sp.csr_matrix(A0 + sp.diags(rng.uniform(-2, 2, A0.shape[0]) + 1j * rng.uniform(-1, 1, A0.shape[0])))
        B, sigma, k = None, -2.0 - 0.5j, 5
    n = A.shape[0]
    V0 = P.start_block(n, k, 9)
    AH = sp.csr_matrix(A.conj().T)
    BH = None if B is None else sp.csr_matrix(B.conj().T)
    with G.GPLHR(A, B, sigma, k, 1, "csr", T=_exact_T(A, B, sigma), tol=1e-11, maxit=100) as r, \
         G.GPLHR(AH, BH, np.conj(sigma), k, 1, "csr", T=_exact_T(AH, BH, np.conj(sigma)), tol=1e-11,
                 maxit=100) as l:
        r.solve(V0)
        l.solve(V0)
        lam = r.vectors()["lam"]
        Gv = np.linspace(1.0, 2.0, k) + 1j * np.linspace(-0.5, 0.5, k)
        cplx = np.iscomplexobj(A.data)
        dA = np.zeros(A.nnz, dtype=np.complex128 if cplx else np.float64)
        dB = None if B is None else np.zeros(B.nnz)
        G.gplhr_grad(r.ctx, l.ctx, Gv, dA, dB)
        # device outputs as well
        dA_dev = torch.zeros(A.nnz, dtype=torch.complex128 if cplx else torch.float64, device="cuda:0")
        G.gplhr_grad(r.ctx, l.ctx, Gv, dA_dev, None)
    lam_d, X, Y = _dense_pairs(A, B, sigma, k)
    order = [int(np.argmin(np.abs(lam_d - l_))) for l_ in lam]
    refA, refB = eig_grad(A, B, lam, X[:, order], Y[:, order], Gv)
    assert np.linalg.norm(dA - refA) <= 1e-7 * np.linalg.norm(refA)
    assert np.linalg.norm(dA_dev.cpu().numpy() - refA) <= 1e-7 * np.linalg.norm(refA)
    if B is not None:
        assert np.linalg.norm(dB - refB) <= 1e-7 * np.linalg.norm(refB)


def test_autograd_edge_field_against_finite_differences():
    """torch.autograd path on the per-edge field of an 8 x 8 copy of the differentiation
    workload: d(sum Re lambda)/db against central differences (step 1e-6) on 12 edges."""
    from paper_1506_06829_gb300.autograd import eigenvalues
    N, k = 8, 4
    pr = P.config5(N)
    b = pr.meta["b"]
    sigma = pr.sigma + 3.0
    J = P.edge_jacobian(N, pr.A)
    pattern = (pr.A.indptr, pr.A.indices, pr.n)
    T = _exact_T(pr.A, None, sigma)
    bt = torch.tensor(b, dtype=torch.float64, requires_grad=True)
    Jt = torch.tensor(J.toarray())
    L0 = torch.tensor(P.convdiff2d_edges(N, np.zeros_like(b)).data)   # b-independent part
    for recompute in (False, True):
        vals = L0 + Jt @ bt
        lam = eigenvalues(vals, pattern, sigma, k, 1, precond="csr", T=T, tol=1e-11, maxit=100,
                          recompute=recompute)
        loss = lam.real.sum()
        g, = torch.autograd.grad(loss, bt)
        delta = 1e-6
        for e in [0, 3, 11, 20, 33, 47, 55, 60, 71, 90, 101, 111]:
            def L(bb):
                ev = sla.eigvals(P.convdiff2d_edges(N, bb).toarray())
                return np.sort(ev[np.argsort(np.abs(ev - sigma))[:k]].real).sum()
            bp, bm = b.copy(), b.copy()
            bp[e] += delta
            bm[e] -= delta
            fd = (L(bp) - L(bm)) / (2 * delta)
            assert abs(g[e].item() - fd) <= 1e-5 * max(1.0, abs(fd)), (e, g[e].item(), fd)


def test_gplhr_grad_refuses_a_degenerate_eigenvalue():
    """Exact double eigenvalues (square-domain symmetry): no unique left/right pairing."""
    A = P.schroedinger2d(10, 0.3)
    n, k = A.shape[0], 4
    AH = sp.csr_matrix(A.conj().T)
    V0 = P.start_block(n, k, 9)
    with G.GPLHR(A, None, -2.0 - 0.5j, k, 1, "csr", T=_exact_T(A, None, -2.0 - 0.5j), tol=1e-11) as r, \
         G.GPLHR(AH, None, -2.0 + 0.5j, k, 1, "csr", T=_exact_T(AH, None, -2.0 + 0.5j), tol=1e-11) as l:
        r.solve(V0)
        l.solve(V0)
        with pytest.raises(G.GplhrError) as e:
            G.gplhr_grad(r.ctx, l.ctx, np.ones(k, dtype=complex), np.zeros(A.nnz, dtype=complex))
        assert e.value.status == G.GPLHR_EINVAL


def test_differentiation_workload_gates_on_the_32x32_copy():
    """The differentiation workload's checks on its 32 x 32 copy (n = 1024, sigma = 4/h^2 at
    the centre of the spectrum, k = 8, B = I), both solves with the exact shift-invert T:

    * the workload's loss L1 = sum Re lambda_i: its gradient w.r.t. the per-edge field
      against the dense-eigendecomposition gradient.  sigma sits in the 32-fold Laplacian
      eigenvalue split by the skew convection: the two real eigenvalues of the 8 have
      opposite gradients and the six complex ones have real parts constant to first order,
      so the sum nearly cancels (|grad L1| ~ 1e-10 against 0.1 per eigenvalue).  The
      error is therefore measured against the scale of its terms, sum_i |grad Re lambda_i|;
    * a loss without that cancellation, L2 = sum |lambda_i - sigma|^2, at 1e-6 relative
      to the dense gradient;
    * L2 against central differences (step 1e-6) of dense LAPACK eigenvalues on 32 seeded
      edges: the differences carry about 1e-12 absolute rounding in each eigenvalue, i.e.
      ~3e-5 relative noise at this gradient size; 1e-3 relative is the gate."""
    from oracle.grad import eig_grad
    from paper_1506_06829_gb300.autograd import eigenvalues
    N, k = 32, 8
    pr = P.config5(N)
    b, sigma = pr.meta["b"], pr.sigma
    J = P.edge_jacobian(N, pr.A)
    pattern = (pr.A.indptr, pr.A.indices, pr.n)
    T = _exact_T(pr.A, None, sigma)
    L0 = torch.tensor(P.convdiff2d_edges(N, np.zeros_like(b)).data)
    Jt = torch.tensor(J.toarray())
    lam_d, X, Y = _dense_pairs(pr.A, None, sigma, k)
    grads = {}
    for name in ("L1", "L2"):
        bt = torch.tensor(b, dtype=torch.float64, requires_grad=True)
        lam = eigenvalues(L0 + Jt @ bt, pattern, sigma, k, 1, precond="csr", T=T, tol=1e-12, maxit=50)
        loss = lam.real.sum() if name == "L1" else ((lam - sigma).abs() ** 2).sum()
        g, = torch.autograd.grad(loss, bt)
        grads[name] = g.numpy()
        for mu in lam.detach().numpy():
            assert np.min(np.abs(lam_d - mu)) <= 1e-9 * abs(mu)
    # dense references: per-eigenvalue gradients of Re lambda_i, and the two losses
    per = [J.T @ eig_grad(pr.A, None, lam_d[i:i + 1], X[:, i:i + 1], Y[:, i:i + 1], np.ones(1))[0]
           for i in range(k)]
    ref1 = np.sum(per, axis=0)
    scale1 = np.sum([np.linalg.norm(p) for p in per])
    ref2 = J.T @ eig_grad(pr.A, None, lam_d, X, Y, 2.0 * (lam_d - sigma))[0]
    assert np.linalg.norm(grads["L1"] - ref1) <= 1e-6 * scale1
    assert np.linalg.norm(grads["L2"] - ref2) <= 1e-6 * np.linalg.norm(ref2)
    # central differences of L2 on 32 seeded edges
    rng = np.random.default_rng(1005)
    edges = rng.choice(b.size, size=32, replace=False)
    delta = 1e-6

    def L2(bb):
        ev = sla.eigvals(P.convdiff2d_edges(N, bb).toarray())
        near = ev[np.argsort(np.abs(ev - sigma))[:k]]
        return float(np.sum(np.abs(near - sigma) ** 2))

    fd = np.empty(edges.size)
    for i, e in enumerate(edges):
        bp, bm = b.copy(), b.copy()
        bp[e] += delta
        bm[e] -= delta
        fd[i] = (L2(bp) - L2(bm)) / (2 * delta)
    assert np.linalg.norm(grads["L2"][edges] - fd) <= 1e-3 * np.linalg.norm(fd)
