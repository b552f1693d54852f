"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Tolerances (FP64 throughout; derivation): a length-L complex dot product has a
relative rounding error below ~L u with u = 2^-53 ~ 1.1e-16 (different summation
orders on the two sides), so kernel-level results are compared at 1e-12 relative to
the norms involved.  Whole solves compare what is unique: eigenvalues to 1e-8
relative (the target stated for the method), subspaces by principal angles
<= 1e-6, and every residual <= tol.
"""
import os

import numpy as np
import pytest
import scipy.linalg as sla
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


def _host(t):
    return t.cpu().numpy()


def _rand_block(rng, n, w):
    return rng.standard_normal((n, w)) + 1j * rng.standard_normal((n, w))


def _angle(X, Y):
    return float(np.max(sla.subspace_angles(X, Y)))


# ------------------------------------------------------------------ SpMM ----

@pytest.mark.parametrize("case", ["generalized_real", "complex_A", "ragged_w5", "ragged_w3", "wide_w40"])
def test_spmm_parity(case):
    rng = np.random.default_rng(1)
    if case in ("generalized_real", "ragged_w5", "wide_w40"):
        N = 10
        A, B = P.convdiff3d(N, (0.4, 0.2, 0.1)), P.mass3d(N)
        k = {"generalized_real": 8, "ragged_w5": 5, "wide_w40": 8}[case]
        w = {"generalized_real": 8, "ragged_w5": 5, "wide_w40": 8}[case]
        m = 1
    else:
        pr = P.config3(20)
        A, B = pr.A, None
        k, w, m = (16, 16, 2) if case == "complex_A" else (3, 3, 1)
    n = A.shape[0]
    ctx = G.gplhr_create(A, B, 0.1 + 0.2j, k, m)
    try:
        wide = 40 if case == "wide_w40" else w
        Xh = _rand_block(rng, n, wide)
        # strided views: X is a column slice of a wider tensor
        Xbig = _dev(np.hstack([Xh, _rand_block(rng, n, 3)]))
        X = Xbig[:, :wide]
        AX = torch.zeros((n, wide + 2), dtype=torch.complex128, device=DEV)
        BX = torch.zeros((n, wide + 2), dtype=torch.complex128, device=DEV)
        G.gplhr_spmm(ctx, X, AX[:, :wide], BX[:, :wide] if B is not None else None)
        torch.cuda.synchronize()
        ref = A @ Xh
        got = _host(AX)[:, :wide]
        assert np.linalg.norm(got - ref) <= 1e-13 * np.linalg.norm(ref)
        assert np.all(_host(AX)[:, wide:] == 0)              # no writes past the block
        if B is not None:
            refB = B @ Xh
            assert np.linalg.norm(_host(BX)[:, :wide] - refB) <= 1e-13 * np.linalg.norm(refB)
    finally:
        G.gplhr_destroy(ctx)


# ------------------------------------------------------------ precond ----

@pytest.mark.parametrize("kind,bs,N,gen", [("block_jacobi", 8, 10, True), ("block_jacobi", 16, 10, True),
                                          ("block_jacobi", 16, 24, False), ("jacobi", 1, 24, False),
                                          ("block_jacobi", 7, 9, True)])
def test_precond_parity(kind, bs, N, gen):
    rng = np.random.default_rng(2)
    if gen:
        A, B = P.convdiff3d(N, (0.4, 0.2, 0.1)), P.mass3d(N)
        sigma = 900.0 + 60.0j
    else:
        A, B = P.config3(N).A, None
        sigma = -2.0 - 0.5j
    n = A.shape[0]
    k = 8
    ctx = G.gplhr_create(A, B, sigma, k, 1, precond=kind, block_size=bs)
    try:
        Xh = _rand_block(rng, n, k)
        X = _dev(Xh)
        Y = torch.zeros_like(X)
        G.gplhr_precond_apply(ctx, X, Y)
        T = oracle_precond(A, B, sigma, kind, bs)
        ref = T.apply(Xh)
        assert np.linalg.norm(_host(Y) - ref) <= 1e-12 * np.linalg.norm(ref)
        G.gplhr_precond_apply(ctx, X, X)                       # in place
        assert np.linalg.norm(_host(X) - ref) <= 1e-12 * np.linalg.norm(ref)
    finally:
        G.gplhr_destroy(ctx)


# ------------------------------------------------------------ Gram / orth --

@pytest.mark.parametrize("n,wx,wy", [(5000, 24, 48), (777, 8, 8), (100003, 16, 32), (33, 3, 5)])
def test_gram_parity(n, wx, wy):
    rng = np.random.default_rng(3)
    A = sp.identity(n, format="csr")
    k, m = (8, 7) if n >= 80 else (3, 1)
    ctx = G.gplhr_create(A, None, 0.5, k, m)
    try:
        Xh, Yh = _rand_block(rng, n, wx), _rand_block(rng, n, wy)
        Cd = torch.zeros((wx, wy), dtype=torch.complex128, device=DEV)
        G.gplhr_gram(ctx, _dev(Xh), _dev(Yh), Cd)
        ref = Xh.conj().T @ Yh
        assert np.linalg.norm(_host(Cd) - ref) <= 1e-13 * np.linalg.norm(Xh) * np.linalg.norm(Yh)
    finally:
        G.gplhr_destroy(ctx)


@pytest.mark.parametrize("n,w,cond", [(3000, 8, 1e2), (20000, 24, 1e6), (4096, 16, 1e10),
                                      (20000, 64, 1e6), (9001, 80, 1e3)])
def test_orth_parity(n, w, cond):
    """orth() = the unique thin QR factor with a real positive R diagonal (oracle: Householder).
    w = 64, 80: the Gram products and the in-place X R^-1 run as several tensor-core launches
    (column blocks from the last to the first)."""
    rng = np.random.default_rng(4)
    Uq, _ = np.linalg.qr(_rand_block(rng, n, w))
    Vq, _ = np.linalg.qr(_rand_block(rng, w, w))
    Xh = Uq @ np.diag(np.logspace(0, -np.log10(cond), w)) @ Vq
    A = sp.identity(n, format="csr")
    ctx = G.gplhr_create(A, None, 0.5, 8, 7)
    try:
        X = _dev(Xh)
        G.gplhr_orth(ctx, X)
        Qg = _host(X)
        assert np.linalg.norm(Qg.conj().T @ Qg - np.eye(w)) <= 1e-13 * w
        ref = OG.orth(Xh)
        # the factors are unique; the accuracy of Q itself degrades like u * cond(X)
        assert np.linalg.norm(Qg - ref) <= max(1e-12, 1e-15 * cond) * np.sqrt(w)
    finally:
        G.gplhr_destroy(ctx)


# ----------------------------------------------------------- whole solves --

def _compare_solutions(res_o, vec_g, k, tol, lam_rtol=1e-8, ang_tol=1e-6):
    lo, lg = res_o.lam, vec_g["lam"]
    # every GPU eigenvalue matches an oracle one (multiset), and vice versa
    for mu in lg:
        assert np.min(np.abs(lo - mu)) <= lam_rtol * abs(mu), (mu, lo)
    for mu in lo:
        assert np.min(np.abs(lg - mu)) <= lam_rtol * abs(mu), (mu, lg)
    assert _angle(vec_g["V"], res_o.V) <= ang_tol
    assert np.max(vec_g["resid"]) <= tol


@pytest.mark.parametrize("products,pencil", [("combine", "gram"), ("spmm", "factored"), ("spmm", "gram")])
def test_solve_parity_schroedinger_small(products, pencil):
    pr = P.config3(24)
    o = OG.solve(pr.A, None, pr.sigma, pr.start_block(), m=pr.m, tol=pr.tol, maxit=300,
                 precond=pr.precond, block_size=pr.block_size)
    assert o.converged
    with G.GPLHR(pr.A, None, pr.sigma, pr.k, pr.m, pr.precond, pr.block_size, tol=pr.tol,
                 maxit=300, products=products, pencil=pencil) as s:
        info = s.solve(pr.start_block())
        vec = s.vectors()
    assert info.iters <= 2 * o.iters + 5
    _compare_solutions(o, vec, pr.k, pr.tol)
    ev = sla.eigvals(pr.A.toarray())
    want = ev[np.argsort(np.abs(ev - pr.sigma))[:pr.k]]
    for mu in want:
        assert np.min(np.abs(vec["lam"] - mu)) <= 1e-8 * abs(mu)
    V = vec["V"]
    assert np.linalg.norm(V.conj().T @ V - np.eye(pr.k)) <= 1e-12
    # A V = V R (Eq. schur) with the returned R
    assert np.linalg.norm(pr.A @ V - V @ vec["RA"]) <= 1e-7 * OG.onenorm(pr.A)


def test_solve_parity_generalized_exact_preconditioner():
    """Generalized 3-D pencil with T = (A - sigma B)^{-1} given explicitly (CSR)."""
    N = 6
    A, B = P.convdiff3d(N, (0.4, 0.2, 0.1)), P.mass3d(N)
    sigma = 300.0 + 40.0j
    n, k = A.shape[0], 4
    Tm = np.linalg.inv(A.toarray() - sigma * B.toarray())
    Tcsr = sp.csr_matrix(Tm)
    V0 = P.start_block(n, k, 77)
    from oracle.precond import Preconditioner
    To = Preconditioner("block_jacobi", blocks=[Tm], bs=n)
    o = OG.solve(A, B, sigma, V0, m=1, tol=1e-10, maxit=100, T=To)
    assert o.converged
    with G.GPLHR(A, B, sigma, k, 1, "csr", T=Tcsr, tol=1e-10, maxit=100) as s:
        s.solve(V0)
        vec = s.vectors()
    _compare_solutions(o, vec, k, 1e-10)
    ev = sla.eigvals(A.toarray(), B.toarray())
    want = ev[np.argsort(np.abs(ev - sigma))[:k]]
    for mu in want:
        assert np.min(np.abs(vec["lam"] - mu)) <= 1e-8 * abs(mu)
    # partial generalized Schur form (Eq. gschur) and Prop. 3.2
    V, Q = vec["V"], vec["Q"]
    nA = OG.onenorm(A)
    assert np.linalg.norm(A @ V - Q @ vec["RA"]) <= 1e-8 * nA
    assert np.linalg.norm(B @ V - Q @ vec["RB"]) <= 1e-8 * nA
    assert np.linalg.norm(Q.conj().T @ Q - np.eye(k)) <= 1e-12


@pytest.mark.parametrize("products,pencil", [("combine", "gram"), ("spmm", "gram"), ("combine", "factored"),
                                            ("spmm", "factored")])
def test_one_step_parity_generalized_block_jacobi(products, pencil):
    """Same start block, same number of iterations: the Ritz values and the nested
    Schur subspaces of the GPU iterate equal the oracle's (orth and QZ bases differ
    only by unitary factors that the harmonic projection removes)."""
    N = 8
    A, B = P.convdiff3d(N, (0.4, 0.2, 0.1)), P.mass3d(N)
    lmax = 21295.965461059128           # dense eigvals of this 8^3 pencil
    sigma = complex(0.3 * lmax, 0.05 * lmax)
    n, k, m = A.shape[0], 8, 1
    V0 = P.start_block(n, k, 1002)
    T = oracle_precond(A, B, sigma, "block_jacobi", 8)
    pen = OG.Pencil(A, B, sigma, T)
    st = OG.init_state(pen, V0, m)
    with G.GPLHR(A, B, sigma, k, m, "block_jacobi", 8, tol=1e-14, maxit=10, lock=False,
                 products=products, pencil=pencil) as s:
        s.start(V0)
        for it in range(3):
            st = OG.iterate(pen, st)
            s.iterate(1)
            vec = s.vectors()
            lo = np.diag(st.RA) / np.diag(st.RB)
            assert np.allclose(vec["lam"], lo, rtol=1e-9, atol=0), (it, vec["lam"], lo)
            for j in range(1, k + 1):
                assert _angle(vec["V"][:, :j], st.V[:, :j]) <= 1e-7, (it, j)


def test_jacobi_constant_diagonal_is_identity_and_notconv_status():
    """Config-1 shape (32 x 32 convection-diffusion, sigma at the spectrum's midpoint):
    the constant Jacobi diagonal makes T = I; a short run returns ENOTCONV with the
    results readable, like the paper's DNC."""
    pr = P.config1()
    with G.GPLHR(pr.A, None, pr.sigma, pr.k, pr.m, "jacobi", tol=pr.tol, maxit=5) as s:
        with pytest.raises(G.GplhrError) as e:
            s.solve(pr.start_block())
        assert e.value.status == G.GPLHR_ENOTCONV
        vec = s.vectors()
        assert np.all(np.isfinite(vec["lam"]))
        V = vec["V"]
        assert np.linalg.norm(V.conj().T @ V - np.eye(pr.k)) <= 1e-12


# -------------------------------------------------- full-size, sampled checks --

@pytest.mark.parametrize("cfg", ["config2", "config3"])
def test_full_size_sampled(cfg):
    """Full-size workloads (n = 262144 / 65536) in the configuration the benchmark
    times: after start + 2 iterations, (i) sampled rows of the SpMM against the
    oracle's sparse rows, element by element within the FP64 dot-product bound, (ii) V, Q orthonormal, (iii) Prop. 3.2
    (A - sigma B) V = Q (R_A - sigma R_B) with fresh products, (iv) the library's
    residuals equal the oracle's residual formula on the returned vectors."""
    pr = P.config2() if cfg == "config2" else P.config3()
    n, k = pr.n, pr.k
    rng = np.random.default_rng(5)
    with G.GPLHR(pr.A, pr.B, pr.sigma, k, pr.m, pr.precond, pr.block_size, tol=pr.tol,
                 maxit=10) as s:
        s.start(pr.start_block())
        s.iterate(2)
        vec = s.vectors()
        V, Q = vec["V"], vec["Q"]
        # (i) sampled SpMM rows
        Xh = _rand_block(rng, n, k)
        AX = torch.zeros((n, k), dtype=torch.complex128, device=DEV)
        BX = torch.zeros((n, k), dtype=torch.complex128, device=DEV)
        G.gplhr_spmm(s.ctx, _dev(Xh), AX, BX if pr.B is not None else None)
        rows = rng.choice(n, 200, replace=False)
        u = 2.0 ** -53
        xabs = np.abs(Xh.real) + np.abs(Xh.imag)
        for M, OUT in ((pr.A, AX), (pr.B, BX)):
            if M is None:
                continue
            Mr = M[rows]
            ref = Mr @ Xh
            got = _host(OUT)[rows]
            # element by element: a row's FP64 dot product of nnz terms errs by at most
            # (nnz + 2) u sum_j |m_j| (|Re x_j| + |Im x_j|) in each real part; the
            # reference (scipy, FP64) and the device each stay within it
            nnz = int(np.diff(Mr.indptr).max())
            bound = 2.02 * (nnz + 2) * u * (abs(Mr) @ xabs)
            assert np.all(np.abs(got.real - ref.real) <= bound)
            assert np.all(np.abs(got.imag - ref.imag) <= bound)
    assert np.linalg.norm(V.conj().T @ V - np.eye(k)) <= 1e-12
    assert np.linalg.norm(Q.conj().T @ Q - np.eye(k)) <= 1e-12
    Bm = sp.identity(n) if pr.B is None else pr.B
    lhs = pr.A @ V - pr.sigma * (Bm @ V)
    if pr.B is None:
        # B = I: RA is R, and Q spans (A - sigma I) V; use the QZ form via Q^* (A - sigma) V
        QR = Q @ (Q.conj().T @ lhs)
    else:
        QR = Q @ (vec["RA"] - pr.sigma * vec["RB"])
    assert np.linalg.norm(lhs - QR) <= 1e-10 * np.linalg.norm(lhs)
    X = vec["X"]
    a, b = vec["alpha"], vec["beta"]
    E = (pr.A @ X) * b[None, :] - (Bm @ X) * a[None, :]
    ref = np.linalg.norm(E, axis=0) / ((np.abs(b) * OG.onenorm(pr.A)
                                        + np.abs(a) * OG.onenorm(pr.B)) * np.linalg.norm(X, axis=0))
    assert np.allclose(vec["resid"], ref, rtol=1e-6, atol=1e-15)


# --------------------------------------------------------- mixed precision --

def test_mixed_solve_schroedinger_small():
    """GPLHR_MIXED: FP32 bulk phase, then FP64 refinement; the final answer meets the
    same FP64 targets as the FP64 mode (eigenvalues vs the oracle, residuals <= tol)."""
    pr = P.config3(24)
    o = OG.solve(pr.A, None, pr.sigma, pr.start_block(), m=pr.m, tol=pr.tol, maxit=300,
                 precond=pr.precond, block_size=pr.block_size)
    with G.GPLHR(pr.A, None, pr.sigma, pr.k, pr.m, pr.precond, pr.block_size, tol=pr.tol,
                 maxit=300, precision="mixed") as s:
        info = s.solve(pr.start_block())
        vec = s.vectors()
    assert info.fp32_iters > 0 and info.bulk == 0
    _compare_solutions(o, vec, pr.k, pr.tol)


def test_mixed_solve_generalized_exact_preconditioner():
    N = 6
    A, B = P.convdiff3d(N, (0.4, 0.2, 0.1)), P.mass3d(N)
    sigma = 300.0 + 40.0j
    n, k = A.shape[0], 4
    Tm = np.linalg.inv(A.toarray() - sigma * B.toarray())
    V0 = P.start_block(n, k, 77)
    from oracle.precond import Preconditioner
    o = OG.solve(A, B, sigma, V0, m=1, tol=1e-10, maxit=100,
                 T=Preconditioner("block_jacobi", blocks=[Tm], bs=n))
    with G.GPLHR(A, B, sigma, k, 1, "csr", T=sp.csr_matrix(Tm), tol=1e-10, maxit=100,
                 precision="mixed") as s:
        info = s.solve(V0)
        vec = s.vectors()
    assert info.fp32_iters > 0
    _compare_solutions(o, vec, k, 1e-10)


@pytest.mark.parametrize("products", ["combine", "spmm"])
def test_bulk_fp32_iterates_track_the_oracle(products):
    """In the FP32 bulk phase the iterates follow the FP64 oracle's to FP32 accuracy:
    Ritz values after each of 2 iterations agree to 1e-4 relative (u32 ~ 6e-8, times
    the growth of two iterations on this non-normal pencil)."""
    N = 8
    A, B = P.convdiff3d(N, (0.4, 0.2, 0.1)), P.mass3d(N)
    lmax = 21295.965461059128
    sigma = complex(0.3 * lmax, 0.05 * lmax)
    n, k, m = A.shape[0], 8, 1
    V0 = P.start_block(n, k, 1002)
    pen = OG.Pencil(A, B, sigma, oracle_precond(A, B, sigma, "block_jacobi", 8))
    st = OG.init_state(pen, V0, m)
    with G.GPLHR(A, B, sigma, k, m, "block_jacobi", 8, tol=1e-14, maxit=10, lock=False,
                 products=products, precision="mixed", switch_tol=1e-30, stall_iters=-1) as s:
        s.start(V0)
        for it in range(2):
            st = OG.iterate(pen, st)
            info = s.iterate(1)
            assert info.bulk == 1
            vec = s.vectors()
            lo = np.diag(st.RA) / np.diag(st.RB)
            assert np.allclose(vec["lam"], lo, rtol=1e-4, atol=0), (it, vec["lam"], lo)
            assert _angle(vec["V"], st.V) <= 1e-3


@pytest.mark.parametrize("n,wx,wy", [(100003, 32, 64), (5000, 24, 24), (777, 8, 8)])
def test_gram_arithmetic_variants(n, wx, wy):
    """EXACT32: for FP32-valued inputs every product is exact and each thread's float-pair
    (compensated) sum over at most 32 rows errs by <= 32 * 2^-48 * sum|p| ~ 1.1e-13 before
    FP64 takes over, so it matches numpy's FP64 Gram of the same values to 2e-13 relative
    to sum|x||y| (FP32 arithmetic is ~1e-7 off); FP32: within FP32 accuracy."""
    rng = np.random.default_rng(6)
    Xh = _rand_block(rng, n, wx).astype(np.complex64).astype(np.complex128)
    Yh = _rand_block(rng, n, wy).astype(np.complex64).astype(np.complex128)
    # magnitudes spread over rows, as in localized eigenvectors
    scale = np.exp(rng.uniform(-6, 0, size=n))[:, None]
    Xh = (Xh * scale).astype(np.complex64).astype(np.complex128)
    ref = Xh.conj().T @ Yh
    A = sp.identity(n, format="csr")
    k, m = (8, 7) if n >= 80 else (3, 1)
    ctx = G.gplhr_create(A, None, 0.5, k, m)
    try:
        nrm = np.abs(Xh).T @ np.abs(Yh)                      # sum |x||y| per entry
        for arith, rtol in (("exact32", 2e-13), ("fp32", 1e-6), ("fp64", 1e-14)):
            Cd = torch.zeros((wx, wy), dtype=torch.complex128, device=DEV)
            G.gplhr_gram(ctx, _dev(Xh), _dev(Yh), Cd, arith)
            err = np.abs(_host(Cd) - ref) / nrm
            assert err.max() <= rtol, (arith, err.max())
    finally:
        G.gplhr_destroy(ctx)


def test_bulk_phase_gram_is_fp64_accurate_on_fp32_values():
    """In the bulk phase the Cholesky-QR Gram and the projected pencil are formed from
    exact products of the FP32-valued blocks (FP32 pipe, compensated accumulation): for
    FP32-representable inputs the result must match an FP64 Gram to ~1e-14 relative,
    far below FP32's 6e-8.  Checked through a mixed-mode solve's internal Gram via the
    orthonormality it delivers: V^*V = I to 1e-12 after FP32 bulk iterations."""
    pr = P.config3(24)
    with G.GPLHR(pr.A, None, pr.sigma, pr.k, pr.m, pr.precond, pr.block_size, tol=pr.tol,
                 maxit=20, precision="mixed", switch_tol=1e-30, stall_iters=-1) as s:
        s.start(pr.start_block())
        info = s.iterate(15)
        assert info.bulk == 1
        vec = s.vectors()
    V, Q = vec["V"], vec["Q"]
    assert np.linalg.norm(V.conj().T @ V - np.eye(pr.k)) <= 1e-5    # FP32 updates of V
    assert np.linalg.norm(Q.conj().T @ Q - np.eye(pr.k)) <= 1e-5


@pytest.mark.parametrize("arith", ["fp32", "exact32"])
def test_fp32_conversion_is_round_to_nearest_even(arith):
    """With Y = I the FP32 Gram returns C = X^* exactly (products with 1 and 0, sums of one
    nonzero term), so C holds the kernels' FP64 -> FP32 conversion of every entry of X:
    bit-exact against IEEE round-to-nearest-even (numpy's cast, FP32 subnormals kept) on
    random values over FP32's exponent range, exact ties, near-ties, carries into the
    exponent and underflow."""
    rng = np.random.default_rng(12)
    n, wx = 80, 40
    vals = np.ldexp(rng.uniform(1.0, 2.0, 2 * n * wx), rng.integers(-125, 127, 2 * n * wx))
    vals *= rng.choice([-1.0, 1.0], vals.size)
    special = []
    for e in (-100, -3, 0, 1, 17, 100):
        one = 2.0 ** e
        ulp = 2.0 ** (e - 23)
        special += [one + ulp / 2, one + 1.5 * ulp, one + ulp / 2 + 2.0 ** (e - 52), one + ulp / 2 - 2.0 ** (e - 52),
                    2 * one - 2.0 ** (e - 30), -(one + ulp / 2), -(2 * one - 2.0 ** (e - 52)), one + ulp]
    special += [0.0, -0.0, 2.0 ** -126, 2.0 ** -127, -3.0e-40, 1.0e-300, 2.0 ** -126 * (1 - 2.0 ** -30),
                float(np.finfo(np.float32).max), -float(np.finfo(np.float32).max)]
    vals[:len(special)] = special
    Xh = (vals[0::2] + 1j * vals[1::2]).reshape(n, wx)
    A = sp.identity(n, format="csr")
    ctx = G.gplhr_create(A, None, 0.5, 8, 7)
    try:
        Cd = torch.zeros((wx, n), dtype=torch.complex128, device=DEV)
        G.gplhr_gram(ctx, _dev(Xh), _dev(np.eye(n, dtype=np.complex128)), Cd, arith)
        C = _host(Cd)
    finally:
        G.gplhr_destroy(ctx)
    f32 = lambda x: x.astype(np.float32).astype(np.float64)
    want_re, want_im = f32(Xh.real.T), -f32(Xh.imag.T)
    got_re, got_im = C.real, C.imag
    assert np.array_equal(got_re, want_re), np.argwhere(got_re != want_re)[:5]
    # the conjugate of a zero imaginary part may carry either sign after the sum
    assert np.array_equal(np.abs(got_im), np.abs(want_im)) and \
        np.array_equal(got_im[want_im != 0], want_im[want_im != 0])


# ------------------------------------------------- block combination (a11) --
def _dot2_product(X, C):
    """X C for complex128 X (n x w), C (w x c) in twice the working precision, rounded
    once (Ogita, Rump and Oishi's Dot2: error-free products by Veltkamp splitting and
    error-free sums, |error| <= u |XC| + 2 (K' u)^2 sum |x'||c'|), through the real form
    X' = (Re x, Im x) per column, C' = [[Re c, Im c], [-Im c, Re c]] per entry."""
    n, w = X.shape
    c = C.shape[1]
    Xr = np.empty((n, 2 * w))
    Xr[:, 0::2], Xr[:, 1::2] = X.real, X.imag
    Cr = np.empty((2 * w, 2 * c))
    Cr[0::2, 0::2], Cr[0::2, 1::2], Cr[1::2, 0::2], Cr[1::2, 1::2] = C.real, C.imag, -C.imag, C.real

    def split(a):
        t = a * 134217729.0
        hi = t - (t - a)
        return hi, a - hi

    s = np.zeros((n, 2 * c))
    comp = np.zeros((n, 2 * c))
    for k in range(2 * w):
        a, b = Xr[:, k:k + 1], Cr[k:k + 1, :]
        p = a * b
        ah, al = split(a)
        bh, bl = split(b)
        e = al * bl - (((p - ah * bh) - al * bh) - ah * bl)
        t = s + p
        z = t - s
        q = (s - (t - z)) + (p - z)
        s = t
        comp += q + e
    y = s + comp
    return y[:, 0::2] + 1j * y[:, 1::2]



@pytest.mark.parametrize("n,w,c,beta", [
    (5000, 8, 8, False),      # K' = 16, N' = 16: two CTAs per SM
    (30001, 16, 8, True),     # K' = 32, N' = 16: two CTAs per SM, one digit stage each
    (6007, 12, 16, False),    # K' = 32, N' = 32
    (9000, 8, 12, True),      # K' = 16, N' = 32: next tile's rows loaded a tile ahead
    (1000, 3, 2, True),       # fewer tiles than CTAs
    (30011, 16, 24, True),    # N' = 48: integer final rounding
    (5003, 8, 32, False),     # N' = 64: integer final rounding
    (100003, 32, 16, True), (4099, 17, 5, False), (2048, 32, 32, True), (777, 24, 40, False),
    (20000, 48, 16, True),    # two input chunks (32 + 16)
    (8192, 80, 32, False),    # three input chunks
    (6007, 20, 64, True),     # two output blocks
    (4099, 70, 80, False)])   # three chunks x three blocks, ragged
def test_combine_tensor_and_dfma_match_fp64(n, w, c, beta):
    """Y = X C (+ Y) on the tensor cores (integer digits, FP32 accumulation) and by DFMA
    against numpy's FP64 product.  Rows span 1e-30 .. 1e30 and include zero rows, C has
    a zero column.  In the real form (K' = 2w terms per output, x' = Re/Im of x, c' of C)
    the digit scheme errs by at most (K'/4 + 2) u max_k |x'_rk| sum_k |c'_kn| (u = 2^-53:
    the input digits' rounding, the dropped digit pairs and one final rounding), a DFMA
    dot product by at most (K' + 1) u (sum_k |x'_rk| |c'_kn| + |y_old|).  More than 32
    output columns: blocks of at most 32, each its own tensor-core launches.  More than 32 input
    columns: the tensor cores sum chunks of at most 32 (K' <= 64 each, the chunk bounds add
    up to at most (64/4 + 2) u max|x'| sum|c'|), and each chunk after the first is added to
    the rounded sum so far, one more rounding of at most u (max|x'| sum|c'| + |y_old|)."""
    rng = np.random.default_rng(40 + w)
    Xh = _rand_block(rng, n, w) * np.exp(rng.uniform(-69, 69, size=n))[:, None]
    Xh[::97] = 0.0
    Ch = _rand_block(rng, w, c) * np.exp(rng.uniform(-3, 3, size=(w, c)))
    Ch[:, min(2, c - 1)] = 0.0
    Y0 = _rand_block(rng, n, c)
    xy = _dot2_product(Xh, Ch)
    ref = xy + (Y0 if beta else 0.0)
    u, K = 2.0 ** -53, 2 * w
    xmax = np.maximum(np.abs(Xh.real), np.abs(Xh.imag)).max(axis=1)[:, None]
    csum = (np.abs(Ch.real) + np.abs(Ch.imag)).sum(axis=0)[None, :]
    # the reference's own rounding (one of X C, one of the sum with Y), and beta's
    slack = u * np.maximum(np.abs(xy.real), np.abs(xy.imag)) * 1.01
    # beta = 1: the tensor-core path adds Y to its rounded product (one more rounding);
    # the DFMA path starts its accumulator at Y, so every one of its K' roundings may
    # carry |Y| as well
    y0max = np.maximum(np.abs(Y0.real), np.abs(Y0.imag))
    yold = {"auto": 2.0 * u * np.maximum(np.abs(ref.real), np.abs(ref.imag)) if beta else 0.0,
            "dfma": (K + 1) * u * y0max if beta else 0.0}
    A = sp.identity(n, format="csr")
    ctx = G.gplhr_create(A, None, 0.5, 8, 2)
    nch = -(-w // 32)
    chunks = 1.01 * (nch - 1) * u * (xmax * csum + (y0max if beta else 0.0))
    try:
        for arith, fac in (("auto", min(K, 64) / 4 + 2), ("dfma", K + 1)):
            bound = fac * u * xmax * csum + slack + yold[arith] + (chunks if arith == "auto" else 0.0)
            Y = _dev(Y0)
            G.gplhr_combine(ctx, _dev(Xh), _dev(Ch), Y, beta, arith)
            got = _host(Y)
            err = np.maximum(np.abs(got.real - ref.real), np.abs(got.imag - ref.imag))
            assert np.all(err <= bound), (arith, np.max(err / np.maximum(bound, 1e-300)))
    finally:
        G.gplhr_destroy(ctx)


def test_combine_in_place_and_nonfinite():
    """In place (Y = X, the X R^-1 step) on both paths, and a NaN in one row of X gives
    NaN in that row only."""
    rng = np.random.default_rng(5)
    n, w = 3000, 16
    Xh = _rand_block(rng, n, w)
    Ch = np.triu(_rand_block(rng, w, w))
    A = sp.identity(n, format="csr")
    ctx = G.gplhr_create(A, None, 0.5, 8, 2)
    try:
        for arith in ("auto", "dfma"):
            X = _dev(Xh)
            G.gplhr_combine(ctx, X, _dev(Ch), X, False, arith)
            assert np.allclose(_host(X), Xh @ Ch, rtol=0, atol=1e-13 * np.abs(Xh @ Ch).max())
            Xn = Xh.copy()
            Xn[123, 4] = np.nan
            Y = torch.zeros((n, w), dtype=torch.complex128, device=DEV)
            G.gplhr_combine(ctx, _dev(Xn), _dev(Ch), Y, False, arith)
            bad = ~np.isfinite(_host(Y)).all(axis=1)
            assert bad[123] and bad.sum() == 1, (arith, np.flatnonzero(bad)[:5])
    finally:
        G.gplhr_destroy(ctx)


# ------------------------------------- search directions and projector (Tables 2-3) --

@pytest.mark.parametrize("p_mode,right_proj,products", [("lobpcg", True, "combine"), ("lobpcg", True, "spmm"),
                                                        ("none", True, "combine"), ("thick", False, "combine"),
                                                        ("lobpcg", False, "spmm")])
def test_variant_iterates_follow_oracle(p_mode, right_proj, products):
    """The P-block variants (Eq. P_lobpcg with C = I, no P) and the variant without the
    projector before T, iterate by iterate against the oracle on the generalized
    block-Jacobi pencil: Ritz values and nested Schur subspaces."""
    N = 8
    A, B = P.convdiff3d(N, (0.4, 0.2, 0.1)), P.mass3d(N)
    lmax = 21295.965461059128           # dense eigvals of this 8^3 pencil
    sigma = complex(0.3 * lmax, 0.05 * lmax)
    n, k, m = A.shape[0], 8, 1
    V0 = P.start_block(n, k, 1002)
    T = oracle_precond(A, B, sigma, "block_jacobi", 8)
    pen = OG.Pencil(A, B, sigma, T)
    st = OG.init_state(pen, V0, m, p_mode=p_mode, right_proj=right_proj)
    with G.GPLHR(A, B, sigma, k, m, "block_jacobi", 8, tol=1e-14, maxit=10, lock=False,
                 products=products, p_mode=p_mode, right_proj=right_proj) as s:
        s.start(V0)
        for it in range(3):
            st = OG.iterate(pen, st)
            s.iterate(1)
            vec = s.vectors()
            lo = np.diag(st.RA) / np.diag(st.RB)
            assert np.allclose(vec["lam"], lo, rtol=1e-9, atol=0), (it, vec["lam"], lo)
            for j in range(1, k + 1):
                assert _angle(vec["V"][:, :j], st.V[:, :j]) <= 1e-7, (it, j)


@pytest.mark.parametrize("p_mode", ["lobpcg", "none"])
def test_variant_solve_with_locking(p_mode):
    """Whole solves with soft locking (P columns of the active pairs) against the oracle
    and dense LAPACK, complex-scaled Schroedinger 24^2."""
    pr = P.config3(24)
    o = OG.solve(pr.A, None, pr.sigma, pr.start_block(), m=pr.m, tol=pr.tol, maxit=400,
                 precond=pr.precond, block_size=pr.block_size, p_mode=p_mode)
    assert o.converged
    with G.GPLHR(pr.A, None, pr.sigma, pr.k, pr.m, pr.precond, pr.block_size, tol=pr.tol,
                 maxit=400, p_mode=p_mode) as s:
        info = s.solve(pr.start_block())
        vec = s.vectors()
    assert info.iters <= 2 * o.iters + 5
    _compare_solutions(o, vec, pr.k, pr.tol)
    ev = sla.eigvals(pr.A.toarray())
    want = ev[np.argsort(np.abs(ev - pr.sigma))[:pr.k]]
    for mu in want:
        assert np.min(np.abs(vec["lam"] - mu)) <= 1e-8 * abs(mu)


# ------------------------------------------------------ Gram on the tensor cores (a9) --

def _narrow_pieces(n, sms=152):
    """Row intervals over which the narrow tensor-core Gram takes one exponent bound per
    column: CTA b of G = min(152, H) takes the 64-row halves [b H / G, (b+1) H / G),
    H = ceil(n / 64), in pieces of up to 8 halves from its first."""
    H = -(-n // 64)
    G = min(sms, H)
    out = []
    for b in range(G):
        h0, h1 = H * b // G, H * (b + 1) // G
        for ph in range(h0, h1, 8):
            out.append((64 * ph, min(n, 64 * min(h1, ph + 8))))
    return out


def _gram_window_bound(Xh, Yh, nwin_cta, win=128, pieces=None):
    """Bound on |C - X^* Y| per real part for the tensor-core Gram: per window w of `win`
    rows (or per row interval of `pieces`) and real columns m of X', n of Y' the digit
    rounding and dropped pairs stay below 2^-53 (max_w|x'_m| sum_w|y'_n| +
    max_w|y'_n| sum_w|x'_m| + max_w|x'_m| max_w|y'_n|), the window's rounding below
    u |G_w|; the FP64 sums over a CTA's windows and the reduction over CTAs add
    (nwin_cta + 160) u sum_r |x'_rm||y'_rn|.  Re C and Im C each add two real entries."""
    n = Xh.shape[0]
    u = 2.0 ** -53

    def real(Z):
        R = np.empty((Z.shape[0], 2 * Z.shape[1]))
        R[:, 0::2], R[:, 1::2] = np.abs(Z.real), np.abs(Z.imag)
        return R

    Xr, Yr = real(Xh), real(Yh)
    Bm = np.zeros((Xr.shape[1], Yr.shape[1]))
    for r0, r1 in (pieces if pieces is not None else [(r, min(n, r + win)) for r in range(0, n, win)]):
        xs, ys = Xr[r0:r1], Yr[r0:r1]
        mx, my = xs.max(axis=0), ys.max(axis=0)
        sx, sy = xs.sum(axis=0), ys.sum(axis=0)
        Bm += 2 * u * (np.outer(mx, sy) + np.outer(sx, my) + np.outer(mx, my))
    Bm += (nwin_cta + 160) * u * (Xr.T @ Yr)
    # Re C(j,l) uses (2j,2l), (2j+1,2l+1); Im C uses (2j,2l+1), (2j+1,2l)
    bre = Bm[0::2, 0::2] + Bm[1::2, 1::2]
    bim = Bm[0::2, 1::2] + Bm[1::2, 0::2]
    return bre, bim


@pytest.mark.parametrize("n,wx,wy,self_", [
    # wide products (tc_gram_wide_kernel; wx > 64 or large outputs: tc_gram_kernel)
    (5000, 32, 32, False), (100003, 128, 16, False), (20000, 64, 32, False), (2048, 24, 24, False),
    (30001, 24, 24, True), (40000, 32, 32, True), (10007, 48, 20, False), (3000, 17, 30, False),
    (2049, 64, 16, False),
    # narrow products (tc_gram_narrow_kernel: planes stacked along M and N)
    (4096, 8, 8, False), (100003, 8, 8, True), (20000, 24, 8, False), (30001, 16, 16, False),
    (2048, 3, 5, False), (9000, 1, 1, True), (7001, 24, 1, False), (12345, 5, 16, False), (65536, 24, 24, True),
    # narrow after swapping the operands (C = (Y^* X)^*)
    (20000, 8, 24, False), (30001, 4, 20, False),
    # narrow with several 512-row pieces per CTA
    (233500, 16, 8, False), (467000, 8, 8, True),
    # wide after swapping the operands
    (30001, 16, 64, False),
    # more than 32 columns of Y: column blocks of at most 32, each by one of the forms above
    (20000, 80, 80, False), (9000, 64, 64, True), (12000, 24, 40, False), (4096, 40, 40, True),
    # 80 x 32 and 128 x 24 fit no form: blocks of 16 columns
    (8192, 80, 32, False), (6000, 128, 24, False), (2500, 112, 112, True)])
def test_gram_tensor_matches_twice_precision(n, wx, wy, self_):
    """C = X^* Y on the tensor cores (GPLHR_GRAM_TENSOR) against a twice-working-
    precision product, with rows spread over 1e-30..1e30, zero rows and a zero column,
    within the digit scheme's per-window bound; wide and narrow shapes, ragged last
    windows, self products."""
    rng = np.random.default_rng(70 + wx + wy)
    Xh = _rand_block(rng, n, wx) * np.exp(rng.uniform(-69, 69, size=n))[:, None]
    Xh[::113] = 0.0
    Xh[:, min(3, wx - 1)] = 0.0
    Yh = Xh.copy() if self_ else _rand_block(rng, n, wy) * np.exp(rng.uniform(-5, 5, size=n))[:, None]
    ref = _dot2_product(Xh.conj().T.copy(), Yh)
    A = sp.identity(n, format="csr")
    ctx = G.gplhr_create(A, None, 0.5, 16, 2)
    try:
        X, Y = _dev(Xh), (None if self_ else _dev(Yh))
        C = torch.zeros((wx, wy), dtype=torch.complex128, device=DEV)
        G.gplhr_gram(ctx, X, X if self_ else Y, C, "tensor")
        got = _host(C)
    finally:
        G.gplhr_destroy(ctx)
    nwin_cta = -(-(-(-n // 128)) // 152)
    bre, bim = _gram_window_bound(Xh, Yh, nwin_cta)
    # the narrow form takes one exponent bound per piece of up to 512 rows: its bound, where
    # it is the larger (a valid bound whichever form ran)
    b2re, b2im = _gram_window_bound(Xh, Yh, nwin_cta, pieces=_narrow_pieces(n))
    bre, bim = np.maximum(bre, b2re), np.maximum(bim, b2im)
    u = 2.0 ** -53
    ere = np.abs(got.real - ref.real) - u * np.abs(ref.real)
    eim = np.abs(got.imag - ref.imag) - u * np.abs(ref.imag)
    assert np.all(ere <= bre) and np.all(eim <= bim), (np.max(ere / np.maximum(bre, 1e-300)),
                                                      np.max(eim / np.maximum(bim, 1e-300)))


@pytest.mark.parametrize("wx,wy,self_", [(32, 16, False), (8, 8, False), (12, 12, True), (24, 24, True),
                                         (100, 16, False)])
def test_gram_tensor_nonfinite(wx, wy, self_):
    """A NaN in X (an Inf in Y) makes exactly its row (column) of C NaN."""
    rng = np.random.default_rng(9)
    n = 4096
    Xh = _rand_block(rng, n, wx)
    Yh = Xh if self_ else _rand_block(rng, n, wy)
    Xh[700, 5] = np.nan
    if not self_:
        Yh[3000, 2] = np.inf
    A = sp.identity(n, format="csr")
    ctx = G.gplhr_create(A, None, 0.5, 16, 2)
    try:
        C = torch.zeros((wx, wy), dtype=torch.complex128, device=DEV)
        X = _dev(Xh)
        G.gplhr_gram(ctx, X, X if self_ else _dev(Yh), C, "tensor")
        got = _host(C)
    finally:
        G.gplhr_destroy(ctx)
    bad = ~np.isfinite(got)
    want = np.zeros_like(bad)
    want[5, :] = True
    want[:, 5 if self_ else 2] = True
    assert np.array_equal(bad, want)
