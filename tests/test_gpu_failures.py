"""Failure detection on the GPU without a GPU fault (bounded waits and host-visible
statuses).

* A tensor-core kernel whose pipeline wait runs out: the context option wait_probe makes
  the combination's epilogue wait on an mbarrier whose phase nothing completes, and
  wait_limit bounds that wait to a few tests.  The kernel then ends its roles, waits for
  its own products in flight, frees its tensor memory and raises the error flag: the call
  returns GPLHR_ETIMEOUT, and the context and the GPU stay usable.
* A singular block-Jacobi block (or a zero Jacobi entry) of A - sigma B: GPLHR_ESINGULAR
  from gplhr_create.
* A NaN in the start block: GPLHR_ENUMERIC from gplhr_solve.
"""
import numpy as np
import pytest
import scipy.sparse as sp

torch = pytest.importorskip("torch")

from paper_1506_06829_gb300 import gplhr as G
from paper_1506_06829_gb300 import problems as P

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _rand(rng, n, w):
    return rng.standard_normal((n, w)) + 1j * rng.standard_normal((n, w))


def test_tensor_core_wait_runs_out_and_everything_stays_usable():
    rng = np.random.default_rng(31)
    n, w = 4096, 8
    Xh, Ch = _rand(rng, n, w), _rand(rng, w, w)
    X, C = torch.from_numpy(Xh).to(DEV), torch.from_numpy(Ch).to(DEV)
    ctx = G.gplhr_create(sp.identity(n, format="csr"), None, 0.5, w, 1, wait_probe=True, wait_limit=64)
    try:
        Y = torch.zeros((n, w), dtype=torch.complex128, device=DEV)
        with pytest.raises(G.GplhrError) as e:
            G.gplhr_combine(ctx, X, C, Y)
        assert e.value.status == G.GPLHR_ETIMEOUT
        # the same context still computes (its Gram products do not take the probe), and
        # a DFMA combination on it is exact to rounding
        Gm = torch.zeros((w, w), dtype=torch.complex128, device=DEV)
        G.gplhr_gram(ctx, X, X, Gm, "tensor")
        ref = Xh.conj().T @ Xh
        assert np.max(np.abs(Gm.cpu().numpy() - ref)) <= 1e-13 * np.max(np.abs(ref))
        G.gplhr_combine(ctx, X, C, Y, False, "dfma")
        assert np.max(np.abs(Y.cpu().numpy() - Xh @ Ch)) <= 1e-13 * np.max(np.abs(Xh @ Ch))
        # a whole solve on the probed context ends with the time-out status too
        with pytest.raises(G.GplhrError) as e:
            G.gplhr_solve(ctx, rng.standard_normal((n, w)))
        assert e.value.status == G.GPLHR_ETIMEOUT
    finally:
        G.gplhr_destroy(ctx)
    torch.cuda.synchronize()
    # a fresh context on the same GPU: the tensor-core combination is correct again
    ctx = G.gplhr_create(sp.identity(n, format="csr"), None, 0.5, w, 1)
    try:
        Y = torch.zeros((n, w), dtype=torch.complex128, device=DEV)
        G.gplhr_combine(ctx, X, C, Y)
        assert np.max(np.abs(Y.cpu().numpy() - Xh @ Ch)) <= 1e-13 * np.max(np.abs(Xh @ Ch))
    finally:
        G.gplhr_destroy(ctx)


def test_singular_block_jacobi_block_is_esingular():
    A = P.config3(12).A.tolil()
    sigma = 1.0 + 0.5j
    A[0:8, 0:8] = 0.0
    for i in range(8):
        A[i, i] = sigma                             # the first 8 x 8 block of A - sigma I is 0
    A = sp.csr_matrix(A)
    with pytest.raises(G.GplhrError) as e:
        G.gplhr_create(A, None, sigma, 4, 1, "block_jacobi", 8)
    assert e.value.status == G.GPLHR_ESINGULAR
    assert "block 0" in str(e.value)


def test_zero_jacobi_entry_is_esingular():
    A = P.config3(12).A.tolil()
    sigma = complex(A[5, 5])                         # diag(A - sigma I) vanishes at row 5 only
    with pytest.raises(G.GplhrError) as e:
        G.gplhr_create(sp.csr_matrix(A), None, sigma, 4, 1, "jacobi")
    assert e.value.status == G.GPLHR_ESINGULAR


def test_nan_in_start_block_is_enumeric():
    pr = P.config3(12)
    V0 = pr.start_block()
    V0[7, 2] = np.nan
    with G.GPLHR(pr.A, None, pr.sigma, pr.k, pr.m, pr.precond, pr.block_size) as s:
        with pytest.raises(G.GplhrError) as e:
            s.solve(V0)
        assert e.value.status == G.GPLHR_ENUMERIC
