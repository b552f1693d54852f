"""GPU tests of CUDA-graph replay of the iteration (opts.graphs): the captured segments
launch the same kernels in the same order as the plain path, so solves and iterates
agree bit for bit, through state changes that select other graphs (locking, the
mixed mode's switch to FP64, P appearing after the first iteration)."""
import numpy as np
import pytest
import scipy.sparse as sp

torch = pytest.importorskip("torch")

from paper_1506_06829_gb300 import gplhr as G
from paper_1506_06829_gb300 import problems as P

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _cases():
    pr = P.config3(16)
    A, B = P.convdiff3d(8, (0.4, 0.2, 0.1)), P.mass3d(8)
    T = sp.csr_matrix(np.linalg.inv(A.toarray() - (300 + 40j) * B.toarray()))
    return [
        ("standard, block-Jacobi, locking", dict(A=pr.A, B=None, sigma=pr.sigma, k=pr.k, m=pr.m, precond=pr.precond,
                                                block_size=pr.block_size), pr.start_block()),
        ("generalized, exact T, m = 2", dict(A=A, B=B, sigma=300 + 40j, k=4, m=2, precond="csr", T=T),
         P.start_block(A.shape[0], 4, 3)),
        ("generalized, mixed precision", dict(A=A, B=B, sigma=300 + 40j, k=4, m=1, precond="csr", T=T,
                                             precision="mixed"), P.start_block(A.shape[0], 4, 5)),
        ("standard, DFMA combinations, Gram pencil", dict(A=pr.A, B=None, sigma=pr.sigma, k=4, m=1,
                                                          precond=pr.precond, block_size=pr.block_size,
                                                          fp64_gemm="dfma", pencil="gram"),
         P.start_block(pr.A.shape[0], 4, 7)),
    ]


@pytest.mark.parametrize("case", range(4))
def test_graph_replay_solve_equals_plain_solve(case):
    name, kw, V0 = _cases()[case]
    out = {}
    for graphs in (False, True):
        s = G.GPLHR(tol=1e-10, maxit=300, graphs=graphs, **kw)
        info = s.solve(V0, allow_notconv=True)
        vec = s.vectors()
        out[graphs] = (info.iters, info.nconv, info.n_spmm, info.h2d_bytes, info.d2h_bytes, vec["lam"], vec["V"])
        s.close()
    a, b = out[False], out[True]
    assert a[:5] == b[:5], (name, a[:5], b[:5])
    assert np.array_equal(a[5], b[5]) and np.array_equal(a[6], b[6]), name


def test_graph_replay_in_batched_iterations():
    ps = P.config4(n_pencils=4, slice_grid=24, n_slices=3)
    res = {}
    for graphs in (False, True):
        solvers = [G.GPLHR(p.A, p.B, p.sigma, p.k, p.m, p.precond, p.block_size, tol=p.tol, maxit=10 ** 6,
                           graphs=graphs) for p in ps]
        for s, p in zip(solvers, ps):
            s.start(p.start_block())
        st, infos, sts = G.gplhr_iterate_batched([s.ctx for s in solvers], 6)
        assert st == G.GPLHR_OK, sts
        res[graphs] = [(info.iters, s.vectors()["lam"]) for s, info in zip(solvers, infos)]
        for s in solvers:
            s.close()
    for (ia, la), (ib, lb) in zip(res[False], res[True]):
        assert ia == ib == 6 and np.array_equal(la, lb)
