"""GPU tests of the persistent batched iteration (gplhr_solve_persistent /
gplhr_iterate_persistent): every device segment of an iteration runs for all contexts of
a batch in one launch of the persistent kernel, which runs each context's recorded
launches in order (each waits, bounded, for its context's previous launch) and the
contexts independently.

Checks: whole solves of pencils of uneven size (standard and generalized, block-Jacobi
and an explicit sparse T, FP64 and mixed precision, soft locking) give the eigenvalues
that per-context solves and dense LAPACK give; lockstep iterations of a copy of the
batched workload (pencils and slices of one pencil) track per-context iterations; one
pencil of the batch against the CPU oracle; three launches per iteration of the whole
batch; a wait that runs out returns ETIMEOUT and leaves the GPU usable; contexts
the kernel cannot run are refused before any launch."""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

torch = pytest.importorskip("torch")

from oracle import gplhr as OG
from paper_1506_06829_gb300 import gplhr as G
from paper_1506_06829_gb300 import problems as P

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _pencils():
    out = []
    for N in (12, 16, 20, 24):                       # uneven sizes, k = 16, m = 2, block-Jacobi 16
        pr = P.config3(N)
        out.append(dict(A=pr.A, B=None, sigma=pr.sigma, k=pr.k, m=pr.m, precond=pr.precond,
                        block_size=pr.block_size, V0=pr.start_block()))
    A, B = P.convdiff3d(6, (0.4, 0.2, 0.1)), P.mass3d(6)
    T = sp.csr_matrix(np.linalg.inv(A.toarray() - (300 + 40j) * B.toarray()))
    out.append(dict(A=A, B=B, sigma=300 + 40j, k=4, m=1, precond="csr", block_size=1, T=T,
                    V0=P.start_block(A.shape[0], 4, 3)))
    return out


def _solver(p, precision="fp64", tol=1e-10, **kw):
    return G.GPLHR(p["A"], p["B"], p["sigma"], p["k"], p["m"], p["precond"], p["block_size"], T=p.get("T"),
                   tol=tol, maxit=400, precision=precision, **kw)


def _dense_nearest(p):
    A = p["A"].toarray()
    ev = sla.eigvals(A) if p["B"] is None else sla.eigvals(A, p["B"].toarray())
    return ev[np.argsort(np.abs(ev - p["sigma"]))[:p["k"]]]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_persistent_solve_matches_per_context_solves(precision):
    ps = _pencils()
    solo = []
    for p in ps:
        s = _solver(p, precision)
        info = s.solve(p["V0"])
        solo.append((info.iters, s.vectors()["lam"]))
        s.close()
    solvers = [_solver(p, precision) for p in ps]
    st, infos, sts, stats = G.gplhr_solve_persistent([s.ctx for s in solvers], [p["V0"] for p in ps],
                                                     nthreads=4)
    assert st == G.GPLHR_OK and all(x == G.GPLHR_OK for x in sts), (st, sts, G.gplhr_last_error())
    # three launches per iteration of the batch, each replacing many recorded launches
    maxit = max(i.iters for i in infos)
    assert stats.launches <= 3 * maxit and stats.ops > 20 * stats.launches, (stats.launches, stats.ops, maxit)
    for s, p, info, (it, lam) in zip(solvers, ps, infos, solo):
        v = s.vectors()
        assert info.nconv == p["k"] and float(np.max(v["resid"])) <= 1e-10
        assert abs(info.iters - it) <= 2, (info.iters, it)
        for mu in lam:                                # the per-context solve's eigenvalues
            assert np.min(np.abs(v["lam"] - mu)) <= 1e-9 * abs(mu)
        for mu in _dense_nearest(p):                  # and dense LAPACK's
            assert np.min(np.abs(v["lam"] - mu)) <= 1e-8 * abs(mu)
        s.close()


def test_persistent_pencil_against_oracle():
    """One Schroedinger pencil (20^2, k = 16, m = 2, block-Jacobi 16) solved inside a batch
    with two others: the oracle from the same start block converges in the same number of
    iterations (within 2) to the same eigenvalues."""
    ps = _pencils()[1:4]
    solvers = [_solver(p, tol=1e-8) for p in ps]
    st, infos, sts, _ = G.gplhr_solve_persistent([s.ctx for s in solvers], [p["V0"] for p in ps])
    assert st == G.GPLHR_OK, sts
    p = ps[1]
    ref = OG.solve(p["A"], None, p["sigma"], p["V0"], m=p["m"], tol=1e-8, maxit=400, precond=p["precond"],
                   block_size=p["block_size"])
    assert ref.converged
    v = solvers[1].vectors()
    assert abs(infos[1].iters - ref.iters) <= 2, (infos[1].iters, ref.iters)
    for mu in ref.lam:
        assert np.min(np.abs(v["lam"] - mu)) <= 1e-8 * abs(mu)
    for s in solvers:
        s.close()


def _max_rel_gap(la, lb):
    """Largest relative distance from a value of lb to the nearest value of la."""
    return max(np.min(np.abs(la - mu)) / abs(mu) for mu in lb)


def test_persistent_iterations_track_per_context_iterations():
    """Lockstep iterations of a batch follow per-context iterations from the same start
    blocks: 4 iterations of the uneven Schroedinger pencils and the generalized pencil
    (well-conditioned eigenvalues) give the same Ritz values to 1e-9; 6 iterations of a
    copy of the batched workload (4 convection-diffusion pencils with B = M x M and 3 slices
    of a 24^2 pencil, T = I) agree to 1e-9 on the contexts whose iterations are stable under
    rounding-sized changes (the others are chaotic there; see below)."""
    ps = _pencils()
    a = [_solver(p) for p in ps]
    b = [_solver(p) for p in ps]
    for s, t, p in zip(a, b, ps):
        s.start(p["V0"])
        t.start(p["V0"])
    st, infos, sts, stats = G.gplhr_iterate_persistent([s.ctx for s in a], 4)
    assert st == G.GPLHR_OK, (sts, G.gplhr_last_error())
    for s, t, info in zip(a, b, infos):
        ti = t.iterate(4)                             # both stop early at convergence
        assert info.iters == ti.iters
        assert _max_rel_gap(s.vectors()["lam"], t.vectors()["lam"]) <= 1e-9
    for s in a + b:
        s.close()

    # A copy of the batched workload: T = I on interior eigenvalues of non-normal pencils.
    # Some of these iterations are chaotic: the oracle's own Ritz values after 6 iterations
    # move by 1e-5 .. 0.2 when the start block changes by 1e-13 (computed below), so only
    # the contexts whose oracle trajectory is stable under that perturbation are compared
    # value by value; the others must take their 6 iterations and stay finite.  The pencils
    # and shifts are real, so the conjugate of an iteration is an iteration too: k columns
    # take one member of a conjugate pair of Ritz values, and which one (their distances to
    # sigma tie) can follow rounding; the comparison allows the mirror image.
    qs = P.config4(n_pencils=4, slice_grid=24, n_slices=3)

    def oracle6(p, V0):
        return OG.solve(p.A, p.B, p.sigma, V0, m=p.m, tol=1e-30, maxit=6, precond=p.precond,
                        block_size=p.block_size).lam

    rng = np.random.default_rng(7)
    stable = []
    for p in qs:
        V0 = p.start_block()
        la, lb = oracle6(p, V0), oracle6(p, V0 + 1e-13 * rng.standard_normal(V0.shape))
        stable.append(_max_rel_gap(la, lb) <= 1e-10)
    assert sum(stable) >= 2, stable

    def make():
        ss = [G.GPLHR(p.A, p.B, p.sigma, p.k, p.m, p.precond, p.block_size, tol=p.tol, maxit=10 ** 6)
              for p in qs]
        for s, p in zip(ss, qs):
            s.start(p.start_block())
        return ss

    a, b = make(), make()
    st, infos, sts, stats = G.gplhr_iterate_persistent([s.ctx for s in a], 6)
    assert st == G.GPLHR_OK, (sts, G.gplhr_last_error())
    assert stats.launches == 3 * 6
    for s in b:
        s.iterate(6)
    for sa, sb, info, ok in zip(a, b, infos, stable):
        assert info.iters == 6
        la, lb = sa.vectors()["lam"], sb.vectors()["lam"]
        assert np.all(np.isfinite(la))
        if ok:  # real pencils, real shifts: a trajectory and its complex conjugate are equivalent
            assert min(_max_rel_gap(la, lb), _max_rel_gap(la, np.conj(lb))) <= 1e-9
    for s in a + b:
        s.close()


def test_persistent_wait_timeout_then_gpu_usable():
    """opts.wait_probe makes every wait for a previous launch ask for one CTA more than it
    has, so the first such wait (wait_limit = 64 tests, ~1.3 ms) runs out, the call
    returns ETIMEOUT and nothing hangs; a fresh batch then iterates normally on the same
    GPU."""
    ps = _pencils()[:2]
    probe = [_solver(p, wait_limit=64, wait_probe=True) for p in ps]
    for s, p in zip(probe, ps):
        s.start(p["V0"])
    st, infos, sts, _ = G.gplhr_iterate_persistent([s.ctx for s in probe], 2)
    assert st == G.GPLHR_ETIMEOUT and all(x == G.GPLHR_ETIMEOUT for x in sts), (st, sts)
    for s in probe:
        s.close()
    fresh = [_solver(p) for p in ps]
    for s, p in zip(fresh, ps):
        s.start(p["V0"])
    st, infos, sts, stats = G.gplhr_iterate_persistent([s.ctx for s in fresh], 2)
    assert st == G.GPLHR_OK and stats.launches == 6, (sts, G.gplhr_last_error())
    for s in fresh:
        assert np.all(np.isfinite(s.vectors()["lam"]))
        s.close()


def test_persistent_refuses_what_it_cannot_run():
    ps = _pencils()
    a, b = _solver(ps[0]), _solver(ps[1])
    gm = _solver(ps[2], inner_steps=2)
    try:
        # not started
        st, _, _, stats = G.gplhr_iterate_persistent([a.ctx, b.ctx], 1)
        assert st == G.GPLHR_EINVAL and stats.launches == 0
        a.start(ps[0]["V0"])
        b.start(ps[1]["V0"])
        gm.start(ps[2]["V0"])
        # a context twice
        st, _, _, stats = G.gplhr_iterate_persistent([a.ctx, b.ctx, a.ctx], 1)
        assert st == G.GPLHR_EINVAL and "twice" in G.gplhr_last_error()
        # inner GMRES (least squares on the host inside T)
        st, _, _, stats = G.gplhr_iterate_persistent([a.ctx, gm.ctx], 1)
        assert st == G.GPLHR_EINVAL and "GMRES" in G.gplhr_last_error()
        assert stats.launches == 0
    finally:
        for s in (a, b, gm):
            s.close()
