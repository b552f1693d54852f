"""Seeded synthetic pencils (A, B) and start blocks for the GPLHR workloads.

This module builds INPUTS only: sparse operators in CSR form, shifts, and seeded
Gaussian start blocks.  It holds none of the eigensolver's arithmetic, imports
neither the CUDA binding nor the CPU oracle, and is shared by both, by the tests
and by the benchmark.

The paper's own test matrices (Matrix Market / IFISS, Table 1 of Sec. 5) are not
available here; these PDE operators stand in for its problem classes: a
non-normal standard problem (convection-diffusion), a generalized problem with a
mass matrix B and a complex shift, and a complex non-Hermitian (complex-scaled)
operator.

Conventions
-----------
* Grid unknowns are numbered with x fastest: ``idx = i + N*j (+ N*N*l)``.
* CSR arrays: ``indptr`` int32 (n+1), ``indices`` int32 (nnz, sorted per row),
  ``data`` float64 or complex128.
* ``B is None`` means B = I.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import scipy.sparse as sp


@dataclasses.dataclass
class Problem:
    """One pencil with its solver settings."""
    name: str
    A: sp.csr_matrix
    B: sp.csr_matrix | None          # None  =>  B = I
    sigma: complex
    k: int
    m: int
    precond: str                      # "none" | "jacobi" | "block_jacobi"
    block_size: int
    tol: float
    seed: int
    meta: dict = dataclasses.field(default_factory=dict)

    @property
    def n(self) -> int:
        return self.A.shape[0]

    def start_block(self) -> np.ndarray:
        return start_block(self.n, self.k, self.seed)


def start_block(n: int, k: int, seed: int) -> np.ndarray:
    """Seeded real Gaussian n-by-k start block V0 (column-major semantics;
    returned as a C-contiguous numpy array of shape (n, k))."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((n, k))


def _csr(M) -> sp.csr_matrix:
    M = sp.csr_matrix(M)
    M.sum_duplicates()
    M.sort_indices()
    M.indptr = M.indptr.astype(np.int32)
    M.indices = M.indices.astype(np.int32)
    return M


def tridiag(n: int, lo, di, up) -> sp.csr_matrix:
    """n-by-n tridiagonal matrix with constant sub-, main and super-diagonal."""
    return sp.diags([np.full(n - 1, lo), np.full(n, di), np.full(n - 1, up)],
                    [-1, 0, 1], format="csr")


def convdiff_1d(N: int, gamma: float, h: float) -> sp.csr_matrix:
    """1-D central-difference -u'' + b u' on N interior points, cell Peclet
    gamma = b*h/2:  row (-(1+gamma), 2, -(1-gamma)) / h^2."""
    return tridiag(N, -(1.0 + gamma), 2.0, -(1.0 - gamma)) / (h * h)


def kron_sum(mats) -> sp.csr_matrix:
    """Kronecker sum with the first factor fastest-varying:
    sum_d I x ... x M_d x ... x I, ordered so that mats[0] acts on x."""
    sizes = [M.shape[0] for M in mats]
    total = None
    for d, M in enumerate(mats):
        term = None
        for e in reversed(range(len(mats))):
            F = M if e == d else sp.identity(sizes[e], format="csr")
            term = F if term is None else sp.kron(term, F, format="csr")
        total = term if total is None else total + term
    return total


def kron_prod(mats) -> sp.csr_matrix:
    """Kronecker product with mats[0] acting on the fastest index."""
    out = None
    for M in reversed(mats):
        out = M if out is None else sp.kron(out, M, format="csr")
    return out


# ---------------------------------------------------------------------------
# Standard problem: 2-D convection-diffusion (B = I)
# ---------------------------------------------------------------------------

def convdiff2d_eigs(N: int, gx: float, gy: float) -> np.ndarray:
    """Closed-form spectrum of the 2-D operator built by ``convdiff2d``:
    (4 - 2 sqrt(1-gx^2) cos(j pi h) - 2 sqrt(1-gy^2) cos(l pi h)) / h^2,
    h = 1/(N+1), j, l = 1..N.  (Each 1-D factor is diagonally similar to a
    symmetric tridiagonal matrix.)"""
    h = 1.0 / (N + 1)
    c = np.cos(np.arange(1, N + 1) * math.pi * h)
    ex = (2.0 - 2.0 * math.sqrt(1 - gx * gx) * c) / (h * h)
    ey = (2.0 - 2.0 * math.sqrt(1 - gy * gy) * c) / (h * h)
    return (ex[:, None] + ey[None, :]).ravel()


def convdiff2d(N: int, gx: float, gy: float) -> sp.csr_matrix:
    h = 1.0 / (N + 1)
    return _csr(kron_sum([convdiff_1d(N, gx, h), convdiff_1d(N, gy, h)]))


def config1(N: int = 32) -> Problem:
    """2-D convection-diffusion, 5-point, N x N interior grid (n = 1024 at N = 32),
    gamma = (0.5, 0.3), B = I, k = 4 nearest the midpoint of the spectrum, m = 1,
    Jacobi on A - sigma I, tol 1e-8, seed 1001.

    The midpoint of the closed-form spectrum is exactly 4/h^2, which is also the
    constant diagonal of A, so diag(A - sigma I) vanishes: the Jacobi
    preconditioner is undefined there and reduces to T = I (any constant scaling
    of T leaves the iteration unchanged)."""
    A = convdiff2d(N, 0.5, 0.3)
    ev = convdiff2d_eigs(N, 0.5, 0.3)
    sigma = 0.5 * (ev.min() + ev.max())
    return Problem(f"convdiff2d_{N}x{N}", A, None, complex(sigma, 0.0), k=4, m=1,
                   precond="jacobi", block_size=1, tol=1e-8, seed=1001,
                   meta={"N": N, "gamma": (0.5, 0.3), "closed_form": ev})


# ---------------------------------------------------------------------------
# Generalized problem: 3-D convection-diffusion with a Q1-type mass matrix
# ---------------------------------------------------------------------------

def mass_1d(N: int) -> sp.csr_matrix:
    """1-D mass matrix M = tridiag(1/6, 2/3, 1/6) (unscaled)."""
    return tridiag(N, 1.0 / 6.0, 2.0 / 3.0, 1.0 / 6.0)


def convdiff3d(N: int, gammas) -> sp.csr_matrix:
    h = 1.0 / (N + 1)
    return _csr(kron_sum([convdiff_1d(N, g, h) for g in gammas]))


def mass3d(N: int) -> sp.csr_matrix:
    M = mass_1d(N)
    return _csr(kron_prod([M, M, M]))


def sym_pencil3d_eigs(N: int) -> np.ndarray:
    """Closed-form spectrum of (A, B) for gamma = 0:
    lambda = (mu_1 + mu_2 + mu_3) / (nu_1 nu_2 nu_3), mu = (2 - 2 cos t)/h^2,
    nu = (2 + cos t)/3, t = j pi/(N+1).  The sine vectors diagonalise both the
    1-D difference operator and the 1-D mass matrix."""
    h = 1.0 / (N + 1)
    t = np.arange(1, N + 1) * math.pi * h
    mu = (2.0 - 2.0 * np.cos(t)) / (h * h)
    nu = (2.0 + np.cos(t)) / 3.0
    lam = ((mu[:, None, None] + mu[None, :, None] + mu[None, None, :])
           / (nu[:, None, None] * nu[None, :, None] * nu[None, None, :]))
    return lam.ravel()


# Largest-modulus eigenvalue of the 64^3 pencil with gamma = (0.4, 0.2, 0.1)
# (ARPACK on B^{-1} A; its imaginary part came out exactly 0), frozen as a literal.
# Written by ``python -m paper_1506_06829_gb300.lambda_max 64``.
CONFIG2_LAMBDA_MAX = 1359896.7265743553


def config2(N: int = 64, lambda_max: float | None = None) -> Problem:
    """3-D convection-diffusion, 7-point, N^3 (n = 262144 at N = 64),
    gamma = (0.4, 0.2, 0.1); B = M x M x M with M = tridiag(1/6, 2/3, 1/6)
    (27-point, SPD); sigma = (0.3 + 0.05i) lambda_max; k = 8, m = 1;
    block-Jacobi 8 x 8 on A - sigma B; tol 1e-10; seed 1002."""
    gam = (0.4, 0.2, 0.1)
    A = convdiff3d(N, gam)
    B = mass3d(N)
    if lambda_max is None:
        lambda_max = CONFIG2_LAMBDA_MAX if N == 64 else None
    if lambda_max is None:
        raise ValueError("config2 needs lambda_max for this N")
    sigma = complex(0.3 * lambda_max, 0.05 * lambda_max)
    return Problem(f"convdiff3d_{N}^3_mass", A, B, sigma, k=8, m=1,
                   precond="block_jacobi", block_size=8, tol=1e-10, seed=1002,
                   meta={"N": N, "gamma": gam, "lambda_max": lambda_max})


# ---------------------------------------------------------------------------
# Complex non-Hermitian problem: complex-scaled 2-D Schroedinger operator
# ---------------------------------------------------------------------------

def neg_laplacian2d(N: int, h: float) -> sp.csr_matrix:
    T = tridiag(N, -1.0, 2.0, -1.0) / (h * h)
    return _csr(kron_sum([T, T]))


def schroedinger2d(N: int, theta: float, depth: float = 5.0, width: float = 0.02,
                   with_potential: bool = True) -> sp.csr_matrix:
    """A = exp(-2 i theta) L_h + diag(V) on the N x N interior grid of [-1, 1]^2,
    h = 2/(N+1); L_h the 5-point negative Laplacian; V = -depth exp(-|x|^2/width)
    (the potential is not complex-scaled)."""
    h = 2.0 / (N + 1)
    L = neg_laplacian2d(N, h).astype(np.complex128)
    A = np.exp(-2j * theta) * L
    if with_potential:
        x = -1.0 + h * np.arange(1, N + 1)
        X, Y = np.meshgrid(x, x, indexing="xy")      # X varies fastest in ravel
        V = -depth * np.exp(-(X ** 2 + Y ** 2) / width)
        A = A + sp.diags(V.ravel().astype(np.complex128))
    return _csr(A)


def schroedinger2d_free_eigs(N: int, theta: float) -> np.ndarray:
    """Closed form for V = 0: exp(-2 i theta) (4/h^2)(sin^2(j pi/(2(N+1)))
    + sin^2(l pi/(2(N+1)))), h = 2/(N+1)."""
    h = 2.0 / (N + 1)
    s = np.sin(np.arange(1, N + 1) * math.pi / (2 * (N + 1))) ** 2
    return (np.exp(-2j * theta) * (4.0 / (h * h)) * (s[:, None] + s[None, :])).ravel()


def config3(N: int = 256) -> Problem:
    """Complex-scaled Schroedinger, 256 x 256 (n = 65536), theta = 0.3,
    V = -5 exp(-|x|^2/0.02) on [-1, 1]^2, B = I, k = 16 nearest
    sigma = -2 - 0.5i, m = 2, block-Jacobi 16 x 16, tol 1e-8, seed 1003."""
    A = schroedinger2d(N, 0.3)
    return Problem(f"schroedinger2d_{N}x{N}", A, None, complex(-2.0, -0.5), k=16, m=2,
                   precond="block_jacobi", block_size=16, tol=1e-8, seed=1003,
                   meta={"N": N, "theta": 0.3})


def csr_arrays(M: sp.csr_matrix):
    """(indptr int32, indices int32, data) views of a CSR matrix."""
    return (np.ascontiguousarray(M.indptr, dtype=np.int32),
            np.ascontiguousarray(M.indices, dtype=np.int32),
            np.ascontiguousarray(M.data))


# ---------------------------------------------------------------------------
# Differentiation workload: 2-D convection-diffusion with a per-edge field b_e
# ---------------------------------------------------------------------------

def edges2d(N: int):
    """Interior edges (p, q = p + e_d) of the N x N grid, x edges first, then y edges."""
    idx = np.arange(N * N).reshape(N, N)          # idx[j, i] = i + N j
    ex = np.stack([idx[:, :-1].ravel(), idx[:, 1:].ravel()], axis=1)
    ey = np.stack([idx[:-1, :].ravel(), idx[1:, :].ravel()], axis=1)
    return np.concatenate([ex, ey], axis=0)


def convdiff2d_edges(N: int, b: np.ndarray) -> sp.csr_matrix:
    """5-point -Laplacian (4/h^2 diagonal, -1/h^2 neighbours, h = 1/(N+1)) plus a
    central-difference convection term per interior edge e = (p, q): +b_e/(2h) at (p, q)
    and -b_e/(2h) at (q, p).  Linear in b: A(b) = L + sum_e b_e E_e."""
    h = 1.0 / (N + 1)
    L = neg_laplacian2d(N, h)
    E = edges2d(N)
    c = b / (2.0 * h)
    C = sp.coo_matrix((np.concatenate([c, -c]), (np.concatenate([E[:, 0], E[:, 1]]),
                                                 np.concatenate([E[:, 1], E[:, 0]]))),
                      shape=L.shape)
    return _csr(L + C)


def edge_jacobian(N: int, A: sp.csr_matrix) -> sp.csr_matrix:
    """J (nnz(A) x n_edges) with dA.data / db = J: entry (p, q) of edge e gets +1/(2h),
    entry (q, p) gets -1/(2h).  Maps a gradient on A's CSR values to one on b."""
    h = 1.0 / (N + 1)
    E = edges2d(N)
    A = sp.csr_matrix(A)
    pos = {}
    for p in range(A.shape[0]):
        for j in range(A.indptr[p], A.indptr[p + 1]):
            pos[(p, int(A.indices[j]))] = j
    rows, cols, vals = [], [], []
    for e, (p, q) in enumerate(E):
        rows += [pos[(int(p), int(q))], pos[(int(q), int(p))]]
        cols += [e, e]
        vals += [1.0 / (2.0 * h), -1.0 / (2.0 * h)]
    return sp.csr_matrix((vals, (rows, cols)), shape=(A.nnz, E.shape[0]))


def config5(N: int = 256) -> Problem:
    """Per-edge convection field b_e ~ U[0.2, 0.6] (seed 1005) on the N x N 5-point
    operator (n = 65536 at N = 256), B = I, k = 8 nearest sigma = 4/h^2 (the centre of
    the spectrum), m = 1, FP64; gradient of sum Re(lambda_i) w.r.t. b."""
    E = edges2d(N)
    rng = np.random.default_rng(1005)
    b = rng.uniform(0.2, 0.6, size=E.shape[0])
    A = convdiff2d_edges(N, b)
    h = 1.0 / (N + 1)
    return Problem(f"convdiff2d_edges_{N}x{N}", A, None, complex(4.0 / (h * h), 0.0), k=8, m=1,
                   precond="jacobi", block_size=1, tol=1e-8, seed=1005,
                   meta={"N": N, "b": b})


# ---------------------------------------------------------------------------
# Batched workload: many convection-diffusion pencils, and shifts over one pencil
# ---------------------------------------------------------------------------

def convdiff2d_mass(N: int, gx: float, gy: float):
    """(A, B): 5-point convection-diffusion and the 2-D mass matrix M x M (9-point)."""
    M = mass_1d(N)
    return convdiff2d(N, gx, gy), _csr(kron_prod([M, M]))


def separable_interval(N: int, gx: float, gy: float):
    """Real spectral interval of the separable approximation (mu_x + mu_y)/(nu_x nu_y),
    mu = (2 - 2 sqrt(1-g^2) cos t)/h^2, nu = (2 + cos t)/3, t = j pi h: exact when the
    pencil's 1-D factors share eigenvectors (gamma = 0), an approximation otherwise."""
    h = 1.0 / (N + 1)
    t = np.arange(1, N + 1) * math.pi * h
    mux = (2 - 2 * math.sqrt(1 - gx * gx) * np.cos(t)) / (h * h)
    muy = (2 - 2 * math.sqrt(1 - gy * gy) * np.cos(t)) / (h * h)
    nu = (2 + np.cos(t)) / 3
    lam = (mux[:, None] + muy[None, :]) / (nu[:, None] * nu[None, :])
    return float(lam.min()), float(lam.max())


def config4(n_pencils: int = 64, slice_grid: int = 128, n_slices: int = 16):
    """64 independent pencils (convection-diffusion, B = M x M) with grid sides drawn
    uniformly from 16..96 and gamma_x, gamma_y ~ U[0.1, 0.9] (seed 1004), k = 4 each,
    sigma at the midpoint of the separable approximation's real interval; plus one
    128 x 128 pencil sliced by 16 shifts at the centres of 16 equal sub-intervals of that
    interval, k = 8 per shift.  m = 1, Jacobi on A - sigma B, tol 1e-8."""
    rng = np.random.default_rng(1004)
    sides = rng.integers(16, 97, size=n_pencils)
    gam = rng.uniform(0.1, 0.9, size=(n_pencils, 2))
    out = []
    for i in range(n_pencils):
        N = int(sides[i])
        A, B = convdiff2d_mass(N, gam[i, 0], gam[i, 1])
        lo, hi = separable_interval(N, gam[i, 0], gam[i, 1])
        out.append(Problem(f"pencil{i}_{N}x{N}", A, B, complex(0.5 * (lo + hi), 0.0), k=4, m=1,
                           precond="jacobi", block_size=1, tol=1e-8, seed=1004 + 1 + i,
                           meta={"N": N, "gamma": tuple(gam[i])}))
    gx, gy = rng.uniform(0.1, 0.9, size=2)
    A, B = convdiff2d_mass(slice_grid, gx, gy)
    lo, hi = separable_interval(slice_grid, gx, gy)
    for s in range(n_slices):
        sig = lo + (s + 0.5) * (hi - lo) / n_slices
        out.append(Problem(f"slice{s}_{slice_grid}x{slice_grid}", A, B, complex(sig, 0.0), k=8, m=1,
                           precond="jacobi", block_size=1, tol=1e-8, seed=2004 + s,
                           meta={"N": slice_grid, "gamma": (gx, gy), "slice": s}))
    return out
