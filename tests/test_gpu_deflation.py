"""GPU tests of deflation (gplhr_set_deflation, Sec. 3.6): a second solve on the deflated
pair returns the next k eigenvalues nearest sigma (dense LAPACK, the oracle's deflated
solve), and the two blocks form one partial (generalized) Schur form."""
import numpy as np
import pytest
import scipy.linalg as sla

torch = pytest.importorskip("torch")

from oracle import gplhr as OG
from oracle.precond import Preconditioner
from paper_1506_06829_gb300 import gplhr as G
from paper_1506_06829_gb300 import problems as P
import scipy.sparse as sp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _match(got, want, rtol):
    for mu in want:
        assert np.min(np.abs(got - mu)) <= rtol * abs(mu), (mu, got)


@pytest.mark.parametrize("generalized", [False, True])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_two_stage_deflated_solve(generalized, precision):
    if generalized:
        N = 6
        A, B = P.convdiff3d(N, (0.4, 0.2, 0.1)), P.mass3d(N)
        sigma, k = 300.0 + 40.0j, 4
        Tm = np.linalg.inv(A.toarray() - sigma * B.toarray())
        ev = sla.eigvals(A.toarray(), B.toarray())
    else:
        A, B = P.schroedinger2d(12, 0.3), None
        sigma, k = -2.0 - 0.5j, 3
        Tm = np.linalg.inv(A.toarray() - sigma * np.eye(A.shape[0]))
        ev = sla.eigvals(A.toarray())
    n = A.shape[0]
    Tcsr = sp.csr_matrix(Tm)
    s1 = G.GPLHR(A, B, sigma, k, 1, "csr", T=Tcsr, tol=1e-11, maxit=200, precision=precision)
    s1.solve(P.start_block(n, k, 3))
    v1 = s1.vectors()
    s2 = G.GPLHR(A, B, sigma, k, 1, "csr", T=Tcsr, tol=1e-11, maxit=200, precision=precision)
    G.gplhr_set_deflation(s2.ctx, v1["V"], v1["Q"] if generalized else None)
    info = s2.solve(P.start_block(n, k, 4))
    v2 = s2.vectors()
    s1.close()
    s2.close()
    assert info.nconv == k
    want = ev[np.argsort(np.abs(ev - sigma))[:2 * k]]
    _match(np.concatenate([v1["lam"], v2["lam"]]), want, 1e-9)
    # the oracle's deflated solve finds the same second block
    To = Preconditioner("block_jacobi", blocks=[Tm], bs=n)
    o = OG.solve(A, B, sigma, P.start_block(n, k, 4), m=1, tol=1e-11, maxit=200, T=To,
                 deflate=(v1["V"], v1["Q"] if generalized else None))
    _match(v2["lam"], o.lam, 1e-9)
    # one partial Schur form
    V = np.hstack([v1["V"], v2["V"]])
    Q = np.hstack([v1["Q"], v2["Q"]])
    assert np.linalg.norm(V.conj().T @ V - np.eye(2 * k)) < 1e-10
    pairs = ((A, v1["RA"], v2["RA"]), (B, v1["RB"], v2["RB"])) if generalized else ((A, v1["RA"], v2["RA"]),)
    for M, R1, R2 in pairs:
        R = np.zeros((2 * k, 2 * k), dtype=complex)
        R[:k, :k], R[k:, k:] = R1, R2
        R[:k, k:] = v1["Q"].conj().T @ (M @ v2["V"]) if generalized else v1["V"].conj().T @ (A @ v2["V"])
        L = Q if generalized else V
        assert np.linalg.norm(M @ V - L @ R) < 1e-8 * OG.onenorm(A)
