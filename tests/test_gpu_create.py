"""gplhr_create rejects malformed CSR input (EINVAL, no device fault), on matrices large
enough (>= 2^20 nonzeros) for the host checks to split their rows over threads."""
import numpy as np
import pytest
import scipy.sparse as sp

from paper_1506_06829_gb300 import gplhr as G

pytestmark = pytest.mark.gpu


def _tridiag(n):
    return sp.diags([np.full(n - 1, -1.0), np.full(n, 4.0), np.full(n - 1, -1.0)], [-1, 0, 1], format="csr")


def _raw(A):
    """A CSR copy whose arrays scipy will not check or fix."""
    M = sp.csr_matrix(A.shape)
    M.data, M.indices, M.indptr = A.data.copy(), A.indices.copy(), A.indptr.copy()
    return M


@pytest.mark.parametrize("where", ["early", "late"])
def test_create_rejects_malformed_csr(where):
    n = 400000
    A = _tridiag(n)
    assert A.nnz >= 1 << 20
    r = 17 if where == "early" else n - 23
    # a row pointer far beyond nnz, then a decrease: no column index past nnz may be read
    M = _raw(A)
    M.indptr[r] = A.nnz + 10 ** 7
    # columns out of order in a row
    M2 = _raw(A)
    e = M2.indptr[r]
    M2.indices[e], M2.indices[e + 1] = M2.indices[e + 1], M2.indices[e]
    # a column out of range
    M3 = _raw(A)
    M3.indices[M3.indptr[r]] = n + 5
    for bad in (M, M2, M3):
        with pytest.raises(G.GplhrError) as err:
            G.gplhr_create(bad, None, 0.5, 4, 1)
        assert err.value.status == G.GPLHR_EINVAL
    # the well-formed matrix is accepted
    ctx = G.gplhr_create(A, None, 0.5, 4, 1)
    G.gplhr_destroy(ctx)
