"""GPU tests of the batched entry points: many pencils of uneven size, and many shifts
over one pencil (spectrum slicing), solved concurrently; each context's result is the
one a solve on its own gives (the kernels are deterministic and contexts share
nothing), and slices find the eigenvalues nearest their own shifts."""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

torch = pytest.importorskip("torch")

from paper_1506_06829_gb300 import gplhr as G
from paper_1506_06829_gb300 import problems as P

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _pencils():
    out = []
    for N in (12, 16, 20, 24):                       # uneven sizes
        pr = P.config3(N)
        out.append((pr.A, None, pr.sigma, pr.k, pr.m, pr.precond, pr.block_size, pr.start_block()))
    A, B = P.convdiff3d(6, (0.4, 0.2, 0.1)), P.mass3d(6)
    T = sp.csr_matrix(np.linalg.inv(A.toarray() - (300 + 40j) * B.toarray()))
    out.append((A, B, 300 + 40j, 4, 1, "csr", 1, P.start_block(A.shape[0], 4, 3), T))
    return out


def _make(p, tol=1e-10):
    A, B, sigma, k, m, prec, bs, V0 = p[:8]
    T = p[8] if len(p) > 8 else None
    return G.GPLHR(A, B, sigma, k, m, prec, bs, T=T, tol=tol, maxit=400), V0


def test_batched_solve_equals_individual_solves():
    ps = _pencils()
    solo = []
    for p in ps:
        s, V0 = _make(p)
        info = s.solve(V0)
        solo.append((info.iters, s.vectors()["lam"]))
        s.close()
    solvers = [_make(p) for p in ps]
    st, infos, sts = G.gplhr_solve_batched([s.ctx for s, _ in solvers], [v for _, v in solvers], nthreads=3)
    assert st == G.GPLHR_OK and all(x == G.GPLHR_OK for x in sts)
    for (s, _), info, (it, lam) in zip(solvers, infos, solo):
        assert info.iters == it
        assert np.array_equal(s.vectors()["lam"], lam)
        s.close()


def test_spectrum_slicing_one_pencil_many_shifts():
    A = P.schroedinger2d(16, 0.3)
    ev = sla.eigvals(A.toarray())
    shifts = [-2.0 - 0.5j, 40.0 - 20.0j, 120.0 - 60.0j]
    k = 3
    n = A.shape[0]
    # each slice with its own exact shift-invert preconditioner: the test is about the slicing
    Ts = [sp.csr_matrix(np.linalg.inv(A.toarray() - sg * np.eye(n))) for sg in shifts]
    solvers = [G.GPLHR(A, None, sg, k, 2, "csr", T=T, tol=1e-10, maxit=200) for sg, T in zip(shifts, Ts)]
    V0s = [P.start_block(A.shape[0], k, 50 + i) for i in range(len(shifts))]
    st, infos, sts = G.gplhr_solve_batched([s.ctx for s in solvers], V0s)
    assert st == G.GPLHR_OK, sts
    for s, sg in zip(solvers, shifts):
        lam = s.vectors()["lam"]
        want = ev[np.argsort(np.abs(ev - sg))[:k]]
        for mu in want:
            assert np.min(np.abs(lam - mu)) <= 1e-8 * abs(mu)
        s.close()


def test_iterate_batched_on_the_batched_workload_copy():
    """A small copy of the batched workload (4 pencils of uneven size + 3 slices of a 24^2
    pencil): every context advances exactly niter iterations and stays finite."""
    ps = P.config4(n_pencils=4, slice_grid=24, n_slices=3)
    solvers = [G.GPLHR(p.A, p.B, p.sigma, p.k, p.m, p.precond, p.block_size, tol=p.tol, maxit=10 ** 6)
               for p in ps]
    for s, p in zip(solvers, ps):
        s.start(p.start_block())
    st, infos, sts = G.gplhr_iterate_batched([s.ctx for s in solvers], 5)
    assert st == G.GPLHR_OK, sts
    for s, info in zip(solvers, infos):
        assert info.iters == 5
        assert np.all(np.isfinite(s.vectors()["lam"]))
        s.close()


def _spec(p, tol=1e-10):
    A, B, sigma, k, m, prec, bs, V0 = p[:8]
    d = dict(A=A, B=B, sigma=sigma, k=k, m=m, precond=prec, block_size=bs, tol=tol, maxit=400)
    if len(p) > 8:
        d["T"] = p[8]
    return d


def test_create_batched_equals_individual_creates():
    """gplhr_create_batched (contexts created concurrently by host threads) gives contexts
    whose batched solves equal solves of contexts created one by one."""
    ps = _pencils()
    solo = []
    for p in ps:
        s, V0 = _make(p)
        info = s.solve(V0)
        solo.append((info.iters, s.vectors()["lam"]))
        s.close()
    ctxs = G.gplhr_create_batched([_spec(p) for p in ps], nthreads=4)
    try:
        st, infos, sts = G.gplhr_solve_batched(ctxs, [p[7] for p in ps], nthreads=3)
        assert st == G.GPLHR_OK and all(x == G.GPLHR_OK for x in sts)
        for c, p, info, (it, lam) in zip(ctxs, ps, infos, solo):
            assert info.iters == it
            assert np.array_equal(G.gplhr_vectors(c, p[0].shape[0], p[3])["lam"], lam)
    finally:
        for c in ctxs:
            G.gplhr_destroy(c)


def test_create_batched_is_all_or_nothing():
    """One invalid entry (k = 33) fails the whole call: EINVAL, the message names the
    entry, and no context is left behind."""
    ps = _pencils()
    specs = [_spec(p) for p in ps]
    specs[2]["k"] = 33
    with pytest.raises(G.GplhrError) as e:
        G.gplhr_create_batched(specs, nthreads=4)
    assert e.value.status == G.GPLHR_EINVAL
    assert "context 2" in str(e.value)
