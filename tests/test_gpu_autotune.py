"""GPU tests of the SpMM autotuner (opts.autotune): every launch shape computes each row
in the same lane group, so autotuned solves equal default ones bit for bit; the
reported shape is one of the candidates, measured no slower than the default."""
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
        (dict(A=pr.A, B=None, sigma=pr.sigma, k=pr.k, m=pr.m, precond=pr.precond, block_size=pr.block_size),
         pr.start_block()),
        (dict(A=A, B=B, sigma=300 + 40j, k=4, m=1, precond="csr", T=T, precision="mixed"),
         P.start_block(A.shape[0], 4, 5)),
    ]


@pytest.mark.parametrize("case", range(2))
def test_autotuned_solve_equals_default_solve(case):
    kw, V0 = _cases()[case]
    out = {}
    for tune in (False, True):
        s = G.GPLHR(tol=1e-10, maxit=300, autotune=tune, **kw)
        info = s.solve(V0, allow_notconv=True)
        vec = s.vectors()
        out[tune] = (info.iters, info.nconv, vec["lam"], vec["V"])
        if tune:
            fp32 = kw.get("precision") == "mixed"
            for w in range(1, kw["k"] + 1):
                for ph in ((False, True) if fp32 else (False,)):
                    t, g, us, ud = G.gplhr_spmm_shape(s.ctx, w, ph)
                    assert t in (64, 128, 256) and g in (2, 4, 8, 16, 64)
                    assert 0 < us <= ud
        else:
            assert G.gplhr_spmm_shape(s.ctx, 1)[:2] == (256, 8)
        s.close()
    a, b = out[False], out[True]
    assert a[:2] == b[:2]
    assert np.array_equal(a[2], b[2]) and np.array_equal(a[3], b[3])
