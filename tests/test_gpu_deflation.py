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


@pytest.mark.parametrize("generalized", [False, True])
def test_spectrum_slices_deflate_their_neighbours(generalized):
    """Spectrum slicing composed with deflation (Sec. 3.6, last paragraph): three slices
    of one pencil whose shifts are close enough that their k nearest eigenvalues overlap.
    Slice i deflates the Schur vectors that slices 0..i-1 found, so the slices return
    disjoint sets: together the k nearest eigenvalues of sigma_0, then of sigma_1 among
    those not found yet, and so on (dense LAPACK), and all their Schur vectors form one
    orthonormal basis of a partial (generalized) Schur form."""
    if generalized:
        # mild convection (cell Peclet 0.2, 0.1): a strongly non-normal pencil would tie the
        # comparison with LAPACK to its eigenvalue condition numbers instead
        A, B = P.convdiff2d_mass(14, 0.2, 0.1)
        ev = sla.eigvals(A.toarray(), B.toarray())
        Bd = B.toarray()
    else:
        A, B = P.schroedinger2d(14, 0.3), None
        ev = sla.eigvals(A.toarray())
        Bd = np.eye(A.shape[0])
    n, k = A.shape[0], 3
    near = ev[np.argsort(np.abs(ev - ev[np.argmin(np.abs(ev))]))]
    # shifts between consecutive low eigenvalues, so neighbouring k-sets overlap
    shifts = [complex(near[2]), complex(0.5 * (near[2] + near[4])), complex(near[4])]
    Vs, Qs, lams = [], [], []
    found = np.zeros(0, dtype=complex)
    for i, sg in enumerate(shifts):
        Tcsr = sp.csr_matrix(np.linalg.inv(A.toarray() - (sg + 1e-3) * Bd))
        s = G.GPLHR(A, B, sg + 1e-3, k, 1, "csr", T=Tcsr, tol=1e-11, maxit=200)
        if Vs:
            G.gplhr_set_deflation(s.ctx, np.hstack(Vs), np.hstack(Qs) if generalized else None)
        info = s.solve(P.start_block(n, k, 60 + i))
        v = s.vectors()
        s.close()
        assert info.nconv == k
        rest = np.array([mu for mu in ev if np.min(np.abs(found - mu), initial=np.inf) > 1e-8 * abs(mu)])
        want = rest[np.argsort(np.abs(rest - (sg + 1e-3)))[:k]]
        _match(v["lam"], want, 1e-9)
        _match(want, v["lam"], 1e-9)
        found = np.concatenate([found, v["lam"]])
        Vs.append(v["V"])
        Qs.append(v["Q"])
    V = np.hstack(Vs)
    assert np.linalg.norm(V.conj().T @ V - np.eye(V.shape[1])) < 1e-10
    L = np.hstack(Qs) if generalized else V
    R = L.conj().T @ (A @ V)
    assert np.linalg.norm(np.tril(R, -1)) < 1e-8 * OG.onenorm(A)      # one triangular factor
    assert np.linalg.norm(A @ V - L @ R) < 1e-8 * OG.onenorm(A)
