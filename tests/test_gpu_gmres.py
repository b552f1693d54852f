"""GPU parity of the inner block GMRES preconditioner (T = s block GMRES steps on
(A - sigma B) W = R, right-preconditioned by T0; Sec. 4) against the oracle's
BlockGmres, through gplhr_precond_apply, and of whole solves that use it.

Tolerance: T R is the unique minimiser over the block Krylov space mapped by T0, so the
two sides agree up to rounding amplified by the conditioning of the small
least-squares problem (the basis is orthonormal, so that is the conditioning of
(A - sigma B) T0 on the space, here below 1e4): 1e-9 relative to ||T R|| leaves a wide
margin and is far below what a wrong operator, shift, preconditioner side or
coefficient changes (O(1))."""
import numpy as np
import pytest
import scipy.sparse as sp

torch = pytest.importorskip("torch")

from oracle import gplhr as OG
from oracle.precond import build as oracle_precond
from paper_1506_06829_gb300 import gplhr as G
from paper_1506_06829_gb300 import problems as P

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    G.lib()


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex128)).to(DEV)


def _case(name):
    if name == "schroedinger":
        pr = P.config3(32)
        return pr.A, None, pr.sigma, 8, 8, "block_jacobi", 16, 4
    if name == "generalized_ragged":
        A, B = P.convdiff3d(10, (0.4, 0.2, 0.1)), P.mass3d(10)
        return A, B, 900.0 + 60.0j, 8, 5, "block_jacobi", 8, 3
    if name == "constant_jacobi":
        pr = P.config1(40)
        return pr.A, None, pr.sigma, 4, 4, "jacobi", 1, 6
    if name == "schroedinger_16k":
        pr = P.config3(128)
        return pr.A, None, pr.sigma, 16, 16, "block_jacobi", 16, 2
    raise ValueError(name)


@pytest.mark.parametrize("name", ["schroedinger", "generalized_ragged", "constant_jacobi", "schroedinger_16k"])
def test_gmres_preconditioner_matches_oracle(name):
    A, B, sigma, k, w, kind, bs, s = _case(name)
    n = A.shape[0]
    rng = np.random.default_rng(21)
    Xh = rng.standard_normal((n, w)) + 1j * rng.standard_normal((n, w))
    Xh[:, 0] *= 1e3                                   # columns of different scales
    ctx = G.gplhr_create(A, B, sigma, k, 1, precond=kind, block_size=bs, inner_steps=s)
    try:
        X = _dev(Xh)
        Y = torch.zeros_like(X)
        G.gplhr_precond_apply(ctx, X, Y)
        ref = oracle_precond(A, B, sigma, kind, bs, inner_steps=s).apply(Xh)
        err = np.linalg.norm(Y.cpu().numpy() - ref) / np.linalg.norm(ref)
        assert err <= 1e-9, err
        G.gplhr_precond_apply(ctx, X, X)              # in place
        assert np.linalg.norm(X.cpu().numpy() - ref) <= 1e-9 * np.linalg.norm(ref)
    finally:
        G.gplhr_destroy(ctx)


def test_gmres_limits_are_checked():
    A = P.config3(16).A
    for s, k in ((33, 1), (13, 32)):
        with pytest.raises(G.GplhrError) as e:
            G.gplhr_create(A, None, -2.0 - 0.5j, k, 1, precond="block_jacobi", block_size=16,
                           inner_steps=s)
        assert e.value.status == G.GPLHR_EINVAL


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_solve_with_inner_gmres_matches_oracle(precision):
    """Small copy of the complex Schroedinger workload (48 x 48, k = 4, m = 1,
    block-Jacobi 16) with 3 inner steps: converged eigenvalues equal the oracle's (same
    T) to 1e-8 relative, every residual <= tol, and the FP64 run takes the oracle's
    iteration count (to within one)."""
    pr = P.config3(48)
    k, s, tol = 4, 3, 1e-9
    V0 = P.start_block(pr.n, k, 1003)
    ref = OG.solve(pr.A, None, pr.sigma, V0, m=1, tol=tol, maxit=200, precond="block_jacobi",
                   block_size=16, inner_steps=s)
    assert ref.converged
    with G.GPLHR(pr.A, None, pr.sigma, k, 1, precond="block_jacobi", block_size=16, tol=tol,
                 maxit=200, precision=precision, inner_steps=s) as g:
        info = g.solve(V0)
        lam = g.vectors()["lam"]
    assert info.nconv == k and max(info.resid[:k]) <= tol
    assert info.n_inner == s * info.n_prec
    order = [int(np.argmin(np.abs(ref.lam - l))) for l in lam]
    assert np.max(np.abs(lam - ref.lam[order]) / np.abs(ref.lam[order])) <= 1e-8
    if precision == "fp64":
        assert abs(info.iters - ref.iters) <= 1, (info.iters, ref.iters)
