"""GPLHR, Algorithm 2 of the paper, in plain FP64/complex128 NumPy.
Test infrastructure only (see the package docstring).

Notation follows Sec. 3: V (right Schur basis, n x k), Q (left Schur basis),
R_A, R_B (k x k upper triangular), M_A, M_B (Q-free factors, Eq. M), W, S_l, P
(correction blocks), Z (trial basis), U = [Q, Qhat] (test basis).

Readings where the paper is silent or ambiguous (each is also applied by the
CUDA path):
* orth(X) (Alg. 1 footnote): the unique thin QR factor whose R has a real
  positive diagonal (Householder QR, then a column phase fix).
* Alg. 2 step 22 subtracts Q(Q^* Qhat) after orth, which leaves U without
  orthonormal columns although Prop. 3.1 assumes them; Qhat is orthonormalised
  again after that subtraction.
* Soft locking (Sec. 3.6): q leading converged pairs are kept in V and Q; W, S_l
  and P carry only the k - q active columns; the active recurrence for S_l uses
  the trailing blocks M_A(q:, q:), M_B(q:, q:) (the correction of a locked
  column is zero, and M_A, M_B are upper triangular); the thick-restart block is
  P = Z Ybar_R(:, k+1 : 2k-q), and when q grows P keeps its leading k - q columns
  (the Schur vectors nearest sigma after V).  m <- min(floor(m0 k/(k - q)), 20).
* Convergence (Sec. 5.1 measures eigen-residuals of vectors made from V): the
  eigenvector of the j-th pair is x_j = V z_j, z_j the eigenvector of the upper
  triangular pencil (R_A, R_B) for its j-th diagonal pair (alpha_j, beta_j),
  and pair j passes when
      ||beta_j A x - alpha_j B x|| / ((|beta_j| ||A||_1 + |alpha_j| ||B||_1) ||x||) <= tol,
  i.e. ||A x - lambda B x|| / ((||A||_1 + |lambda| ||B||_1) ||x||) <= tol.
  Locking is in order (lock_update): the q locked pairs count as converged, and q
  grows by the run of pairs q, q+1, ... that pass.  The iteration stops when all k
  pairs are locked (without locking: when all k pass).
* Search directions P (Sec. 3.5; the paper compares the options in Table 2):
  "thick" is P = Z Ybar_R(:, k+1:2k) (Eq. P1, the default); "lobpcg" is
  P = V^(i) - V^(i-1) C (Eq. P_lobpcg) with C = I, since the paper leaves C open and
  every invertible C gives the same trial subspace once P is orthogonalised against
  V^(i) (span{V, V - V_old C} = span{V, V_old}); "previous" is P = V^(i-1), the other
  option the paper names with the same subspace; "none" drops P (Eq. trial_partial).
  Under soft locking a lobpcg / previous P keeps the columns of the active pairs
  q..k-1, a thick P its leading k - q columns.
* The right projector before T (Table 3) can be omitted: T_L = (I - VV^*) T instead of
  (I - VV^*) T (I - QQ^*) (or (I - VV^*) T (I - VV^*) when B = I).
* Deflation (Sec. 3.6, last paragraph): given k1 computed right and left Schur vectors
  V1, Q1, further ones come from GPLHR on the deflated pair ((I - Q1 Q1^*) A (I - V1 V1^*),
  (I - Q1 Q1^*) B (I - V1 V1^*)), or (I - V1 V1^*) A (I - V1 V1^*) with B = I.  That pair
  is singular on span(V1) (both maps vanish there), so the trial subspace must stay
  orthogonal to V1: the paper is silent on how, and the reading here deflates T too,
  T_d = (I - V1 V1^*) T (I - Q1 Q1^*) ((I - V1 V1^*) T (I - V1 V1^*) with B = I), and
  projects the start block.  Residual norms keep ||A||_1, ||B||_1 of the original pair.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.sparse as sp

from .ordqz import ordqz
from .precond import Preconditioner, build as build_precond
from .schur import m_factors

MMAX = 20  # cap on the adapted m (Sec. 3.6)


def orth(X: np.ndarray) -> np.ndarray:
    """Orthonormal basis of col(X): thin QR with R(j,j) real positive."""
    if X.shape[1] == 0:
        return X.copy()
    Qm, R = np.linalg.qr(X)
    d = np.diag(R)
    mag = np.abs(d)
    ph = np.where(mag > 0, d / np.where(mag > 0, mag, 1.0), 1.0)
    return Qm * ph[None, :]


def onenorm(M) -> float:
    """||M||_1 (max column sum of |entries|); 1 for M = None (B = I)."""
    if M is None:
        return 1.0
    return float(np.abs(M).sum(axis=0).max())


class Pencil:
    """(A, B, sigma, T) with B = None meaning B = I."""

    def __init__(self, A, B, sigma: complex, T: Preconditioner, deflate=None):
        self.A = sp.csr_matrix(A).astype(np.complex128)
        self.B = None if B is None else sp.csr_matrix(B).astype(np.complex128)
        self.sigma = complex(sigma)
        self.T = T
        # deflation basis (V1, Q1); Q1 is ignored (taken as V1) when B = I
        self.V1 = self.Q1 = None
        if deflate is not None:
            self.V1 = np.asarray(deflate[0], dtype=np.complex128)
            self.Q1 = self.V1 if self.B is None else np.asarray(deflate[1], dtype=np.complex128)
        self.n = self.A.shape[0]
        self.normA = onenorm(self.A)
        self.normB = onenorm(self.B)
        self.n_mv = 0       # products with A (and with B when B != I), column blocks
        self.n_prec = 0     # applications of T, column blocks

    def _pv(self, X):
        return X if self.V1 is None else X - self.V1 @ (self.V1.conj().T @ X)

    def _pq(self, X):
        return X if self.Q1 is None else X - self.Q1 @ (self.Q1.conj().T @ X)

    def Amul(self, X):
        self.n_mv += 1
        return self._pq(self.A @ self._pv(X))

    def Bmul(self, X):
        if self.B is None:
            return X.copy()
        return self._pq(self.B @ self._pv(X))

    def Tmul(self, X):
        self.n_prec += 1
        return self._pv(self.T.apply(self._pq(X)))


@dataclasses.dataclass
class State:
    V: np.ndarray
    Q: np.ndarray
    P: np.ndarray | None
    RA: np.ndarray
    RB: np.ndarray
    MA: np.ndarray
    MB: np.ndarray
    q: int
    m: int
    m0: int
    it: int = 0
    p_mode: str = "thick"         # "thick" | "lobpcg" | "previous" | "none"
    right_proj: bool = True       # projector before T (Table 3)
    lobpcg_C: np.ndarray | None = None   # C of Eq. P_lobpcg (None: identity)

    @property
    def k(self) -> int:
        return self.V.shape[1]

    def copy(self) -> "State":
        return dataclasses.replace(
            self, V=self.V.copy(), Q=self.Q.copy(),
            P=None if self.P is None else self.P.copy(),
            RA=self.RA.copy(), RB=self.RB.copy(), MA=self.MA.copy(), MB=self.MB.copy())


def init_state(pen: Pencil, V0: np.ndarray, m: int, p_mode: str = "thick", right_proj: bool = True,
               lobpcg_C: np.ndarray | None = None) -> State:
    """Steps 1-4 of Algorithm 2."""
    if p_mode not in ("thick", "lobpcg", "previous", "none"):
        raise ValueError(f"unknown p_mode {p_mode!r}")
    V = orth(np.asarray(V0, dtype=np.complex128))
    AV = pen.Amul(V)
    BV = pen.Bmul(V)
    Q = orth(AV - pen.sigma * BV)
    RA, RB, YL, YR = ordqz(Q.conj().T @ AV, Q.conj().T @ BV, pen.sigma)
    V = V @ YR
    Q = Q @ YL
    MA, MB, _ = m_factors(RA, RB)
    return State(V, Q, None, RA, RB, MA, MB, q=0, m=m, m0=m, p_mode=p_mode, right_proj=right_proj,
                 lobpcg_C=lobpcg_C)


def iterate(pen: Pencil, st: State) -> State:
    """Steps 6-29 of Algorithm 2 (one pass of the while loop)."""
    V, Q, P, RA, RB, MA, MB = st.V, st.Q, st.P, st.RA, st.RB, st.MA, st.MB
    k, q, m = st.k, st.q, st.m
    sig = pen.sigma
    generalized = pen.B is not None

    def proj_V(X):
        return X - V @ (V.conj().T @ X)

    def proj_Q(X):
        return X - Q @ (Q.conj().T @ X)

    proj_right = proj_Q if generalized else proj_V

    def T_L(X):  # projected preconditioner, Eqs. prec_gen / prec (right projector optional)
        return proj_V(pen.Tmul(proj_right(X) if st.right_proj else X))

    AV = pen.Amul(V)
    BV = pen.Bmul(V)
    # Steps 6-11: projected preconditioned residual (active columns q: only).
    if generalized:
        WA = AV - Q @ RA
        WB = BV - Q @ RB
        Rres = (WA @ MB - WB @ MA)[:, q:]
    else:
        Rres = (AV @ MB - V @ MA)[:, q:]
    W = orth(T_L(Rres))                                    # step 12
    MAa = MA[q:, q:]
    MBa = MB[q:, q:]
    S = []
    S_prev = W
    for _ in range(m):                                     # steps 13-20
        Sl = T_L(pen.Amul(S_prev) @ MBa - pen.Bmul(S_prev) @ MAa)
        Sl = Sl - W @ (W.conj().T @ Sl)
        if S:
            Sc = np.hstack(S)
            Sl = Sl - Sc @ (Sc.conj().T @ Sl)
        Sl = orth(Sl)
        S.append(Sl)
        S_prev = Sl
    Sc = np.hstack(S) if S else np.zeros((pen.n, 0), dtype=np.complex128)
    blocks = [W] + S
    if P is not None:                                      # soft locking: k - q columns
        P = P[:, q:] if st.p_mode in ("lobpcg", "previous") else P[:, :k - q]
    if P is not None and P.shape[1] > 0:                   # step 21
        P = P - V @ (V.conj().T @ P)
        P = P - W @ (W.conj().T @ P)
        P = P - Sc @ (Sc.conj().T @ P)
        P = orth(P)
        blocks.append(P)
    K = np.hstack(blocks)
    Z = np.hstack([V, K])                                  # step 22
    AK = pen.Amul(K)
    BK = pen.Bmul(K)
    Qh = orth(AK - sig * BK)                               # step 23
    Qh = Qh - Q @ (Q.conj().T @ Qh)
    Qh = orth(Qh)
    U = np.hstack([Q, Qh])                                 # step 24
    AZ = np.hstack([AV, AK])
    BZ = np.hstack([BV, BK])
    RAb, RBb, YLb, YRb = ordqz(U.conj().T @ AZ, U.conj().T @ BZ, sig)
    kk = k - q
    YR = YRb[:, :k]                                        # step 25
    YL = YLb[:, :k]
    RA = RAb[:k, :k]
    RB = RBb[:k, :k]
    V_old = V
    V = Z @ YR                                             # steps 26-27
    Q = U @ YL
    if st.p_mode == "thick":
        P = Z @ YRb[:, k:k + kk]                           # step 28 (thick restart, Eq. P1)
    elif st.p_mode == "lobpcg":                            # Eq. P_lobpcg, all k columns
        P = V - (V_old if st.lobpcg_C is None else V_old @ st.lobpcg_C)
    elif st.p_mode == "previous":
        P = V_old.copy()
    else:
        P = None
    MA, MB, _ = m_factors(RA, RB)                          # steps 29-30
    return dataclasses.replace(st, V=V, Q=Q, P=P, RA=RA, RB=RB, MA=MA, MB=MB,
                               it=st.it + 1)


def tri_eigvecs(RA: np.ndarray, RB: np.ndarray) -> np.ndarray:
    """Columns z_j with (beta_j RA - alpha_j RB) z_j = 0, z_j(j) = 1 and
    z_j(i) = 0 for i > j (back substitution on the upper triangular pencil).
    A pivot below eps * scale is replaced by eps * scale."""
    k = RA.shape[0]
    Zv = np.zeros((k, k), dtype=np.complex128)
    nA = np.linalg.norm(RA)
    nB = np.linalg.norm(RB)
    eps = np.finfo(np.float64).eps
    for j in range(k):
        a, b = RA[j, j], RB[j, j]
        C = b * RA - a * RB
        small = eps * max(abs(b) * nA + abs(a) * nB, np.finfo(np.float64).tiny)
        z = np.zeros(k, dtype=np.complex128)
        z[j] = 1.0
        for i in range(j - 1, -1, -1):
            rhs = -(C[i, i + 1:j + 1] @ z[i + 1:j + 1])
            piv = C[i, i]
            if abs(piv) < small:
                piv = small
            z[i] = rhs / piv
        Zv[:, j] = z
    return Zv


def residuals(pen: Pencil, st: State, AV=None, BV=None) -> np.ndarray:
    """Backward-error residual of each of the k pairs (see module docstring)."""
    if AV is None:
        AV = pen._pq(pen.A @ pen._pv(st.V))
    if BV is None:
        BV = st.V if pen.B is None else pen._pq(pen.B @ pen._pv(st.V))
    Zv = tri_eigvecs(st.RA, st.RB)
    a = np.diag(st.RA)
    b = np.diag(st.RB)
    X = st.V @ Zv
    E = (AV @ Zv) * b[None, :] - (BV @ Zv) * a[None, :]
    num = np.linalg.norm(E, axis=0)
    den = (np.abs(b) * pen.normA + np.abs(a) * pen.normB) * np.linalg.norm(X, axis=0)
    return num / den


def lock_update(res: np.ndarray, tol: float, q: int, m: int, m0: int) -> tuple[int, int]:
    """Soft locking and the adaptation of m (Sec. 3.6), after the residuals ``res`` of
    the k pairs of an iteration.

    Locked pairs count as converged and stay locked, and locking is in order: pair j
    can be locked only once pairs 0..j-1 are locked.  So q grows by the run of pairs
    q, q+1, ... that meet ``tol`` (whatever the current residuals of the locked pairs
    0..q-1).  When q grows and pairs remain, m becomes the largest integer with
    m (k - q) <= m0 k, i.e. floor(m0 k / (k - q)), capped at MMAX = 20; otherwise m is
    kept.  q = k means every pair is locked: the iteration has converged.
    Returns the new (q, m)."""
    k = len(res)
    lead = q
    while lead < k and res[lead] <= tol:
        lead += 1
    if lead > q and lead < k:
        return lead, min(m0 * k // (k - lead), MMAX)
    return lead, m


@dataclasses.dataclass
class Result:
    V: np.ndarray
    Q: np.ndarray
    RA: np.ndarray
    RB: np.ndarray
    MA: np.ndarray
    MB: np.ndarray
    alpha: np.ndarray
    beta: np.ndarray
    lam: np.ndarray
    resid: np.ndarray
    iters: int
    converged: bool
    n_mv: int
    n_prec: int
    history: list
    R: np.ndarray | None = None   # B = I:  R = M_A M_B^{-1}  (step 31, see solve())


def solve(A, B, sigma, V0, m: int = 1, tol: float = 1e-8, maxit: int = 500,
          precond: str = "none", block_size: int = 1, T: Preconditioner | None = None,
          lock: bool = True, callback=None, inner_steps: int = 0, p_mode: str = "thick",
          right_proj: bool = True, lobpcg_C: np.ndarray | None = None, deflate=None) -> Result:
    """Run Algorithm 2 until all k pairs meet ``tol`` or ``maxit`` iterations.
    inner_steps > 0: T is that many block GMRES steps preconditioned by ``precond``.
    p_mode, right_proj, lobpcg_C: the variants of Sec. 3.5 and Tables 2-3 (module
    docstring).  deflate = (V1, Q1): solve the deflated pair (module docstring)."""
    if deflate is not None and inner_steps > 0:
        raise ValueError("deflation with an inner GMRES preconditioner is not supported")
    if T is None:
        T = build_precond(A, B, sigma, precond, block_size, inner_steps)
    pen = Pencil(A, B, sigma, T, deflate)
    st = init_state(pen, pen._pv(np.asarray(V0, dtype=np.complex128)), m, p_mode, right_proj, lobpcg_C)
    k = st.k
    hist = []
    res = residuals(pen, st)
    converged = bool(np.all(res <= tol))
    while not converged and st.it < maxit:
        st = iterate(pen, st)
        res = residuals(pen, st)
        hist.append(res.copy())
        if callback is not None:
            callback(st, res)
        if lock:
            st.q, st.m = lock_update(res, tol, st.q, st.m, st.m0)
            converged = st.q == k       # every pair locked (a locked pair has converged)
        else:
            converged = bool(np.all(res <= tol))
    a = np.diag(st.RA).copy()
    b = np.diag(st.RB).copy()
    with np.errstate(divide="ignore", invalid="ignore"):
        lam = a / b
    R = None
    if pen.B is None:
        # Step 31 prints R = M_B^{-1} M_A; Eq. gschur2 with B = I gives A V = V M_A M_B^{-1}
        # at every iterate.  The two coincide when M_B = I, the converged limit.
        R = st.MA @ np.linalg.inv(st.MB)
    return Result(st.V, st.Q, st.RA, st.RB, st.MA, st.MB, a, b, lam, res, st.it,
                  converged, pen.n_mv, pen.n_prec, hist, R)
