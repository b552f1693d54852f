"""Pins for soft locking and the adaptation of m in the oracle (Sec. 3.6).

The paper's rules: converged Schur vectors are kept in V and Q and their columns are
removed from W, S_1..S_m and P; locking is in order (v_{j+1} only after v_1..v_j are
locked); and when q pairs are locked, m is raised to the largest integer with
m (k - q) <= m0 k, at most 20.

Two kinds of pins, neither of which retypes the oracle's formula:
* brute force on tiny inputs: every convergence pattern of up to 6 pairs, every q and
  m0 in a small range, against the rules as the paper states them (a search over the
  admissible q and over the integers m);
* a whole oracle solve on a diagonal pencil whose start block makes pair 1 (and 2)
  converge long before pair 0, observed through what the iteration actually does: the
  width of the blocks multiplied by A in the Krylov-Arnoldi steps is k - q, and their
  number is m.  Out-of-order locking, a missing m update, a missing or wrong cap, and
  a q that can shrink are planted in the oracle below and must fail these pins.
"""
import itertools

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import gplhr as G
from oracle.precond import Preconditioner

TOL = 1e-10


# ------------------------------------------------------------ brute force ----

def _admissible_q(conv, q0):
    """Largest q' with q' >= q0 (locked pairs stay locked) such that every pair in
    q0..q'-1 has converged (locking in order, each pair only once its predecessors are
    locked), found by trying every q'."""
    best = q0
    for t in range(q0, len(conv) + 1):
        if all(conv[q0:t]):
            best = t
    return best


def _largest_m(k, q, m0):
    """The largest integer m with m (k - q) <= m0 k, then at most 20 (by search)."""
    m = max(mm for mm in range(0, 1000) if mm * (k - q) <= m0 * k)
    return min(m, 20)


def _check_rule(fn):
    for k in range(1, 7):
        for pattern in itertools.product((False, True), repeat=k):
            res = np.where(pattern, TOL / 2, 2 * TOL)
            for q0 in range(0, k):
                for m0 in range(0, 5):
                    m_now = m0 + 3           # any current m: kept when q does not grow
                    q, m = fn(res, TOL, q0, m_now, m0)
                    qe = _admissible_q(pattern, q0)
                    if qe == k:              # every pair locked: the iteration stops
                        assert q == k, (pattern, q0, q)
                        continue
                    me = _largest_m(k, qe, m0) if qe > q0 else m_now
                    assert (q, m) == (qe, me), (pattern, q0, m0, (q, m), (qe, me))


def test_lock_rule_brute_force():
    _check_rule(G.lock_update)


# --------------------------------------------------------- observed solve ----

def _scenario(lock_fn):
    """Diagonal pencil, B = I, sigma = 0, T = I, k = 4, m0 = 6.  Start block: e_2 and e_3
    (eigenvalues 2 and 3) almost exactly, e_1 polluted by a far eigenvector, and a random
    column.  Pairs 1 and 2 meet the tolerance from the first iteration on, pair 0 only
    later; pair 3 (eigenvalue 3.9, next to 3.93) last.  Returns per iteration the
    residuals and the widths of the blocks multiplied by A."""
    n = 300
    rng = np.random.default_rng(0)
    d = np.concatenate([[1.0, 2.0, 3.0, 3.9, 3.93], np.linspace(6, 400, n - 5)])
    V0 = rng.standard_normal((n, 4)) * 1e-3
    V0[:, 0] = 1e-11 * rng.standard_normal(n)
    V0[1, 0] = 1.0
    V0[0, 1], V0[60, 1] = 1.0, 0.3
    V0[:, 2] = 1e-11 * rng.standard_normal(n)
    V0[2, 2] = 1.0
    V0[:, 3] = rng.standard_normal(n)
    widths = []
    log = []
    orig_amul, orig_lock = G.Pencil.Amul, G.lock_update

    def amul(self, X):
        widths.append(X.shape[1])
        return orig_amul(self, X)

    def cb(st, res):
        log.append((res.copy(), len(widths)))

    G.Pencil.Amul, G.lock_update = amul, lock_fn
    try:
        r = G.solve(sp.diags(d).tocsr(), None, 0.0, V0, m=6, tol=TOL, maxit=60,
                    T=Preconditioner("identity"), callback=cb)
    finally:
        G.Pencil.Amul, G.lock_update = orig_amul, orig_lock
    iters = []
    for i, (res, nw) in enumerate(log):   # widths[0] is A V0 of the start (steps 1-4)
        lo = 1 if i == 0 else log[i - 1][1]
        iters.append((res, widths[lo:nw]))
    return r, iters


def _observed(ws, k):
    """(q, m) the iteration ran with: its products are A V (k columns), the m
    Krylov-Arnoldi blocks (k - q columns each) and A [W S P]."""
    krylov = ws[1:-1]
    assert len(set(krylov)) <= 1
    return (k - krylov[0] if krylov else None), len(krylov)


def _pin_scenario(lock_fn):
    r, iters = _scenario(lock_fn)
    k = 4
    out_of_order = 0
    for i in range(1, len(iters)):
        res_prev = iters[i - 1][0]
        q, m = _observed(iters[i][1], k)
        conv = res_prev <= TOL
        if conv[1] and conv[2] and not conv[0]:
            out_of_order += 1
            assert (q, m) == (0, 6), (i, q, m)        # pairs 1, 2 converged: not locked
        if conv[0] and conv[1] and conv[2] and not conv[3]:
            assert (q, m) == (3, 20), (i, q, m)       # floor(6*4/1) = 24 capped at 20
    assert out_of_order >= 3
    assert any(_observed(ws, k) == (3, 20) for _, ws in iters)
    assert r.converged
    lam = np.sort(r.lam.real)
    assert np.allclose(lam, [1.0, 2.0, 3.0, 3.9], rtol=1e-9)


def test_lock_rule_in_a_solve():
    _pin_scenario(G.lock_update)


# ------------------------------------------------------ planted mistakes ----

_ORACLE_LOCK = G.lock_update        # the mutants below start from it

def _any_order(res, tol, q, m, m0):
    k = len(res)
    c = int(np.sum(res <= tol))
    return (c, min(m0 * k // max(k - c, 1), 20)) if c > q else (q, m)


def _no_m_update(res, tol, q, m, m0):
    return _ORACLE_LOCK(res, tol, q, m, m0)[0], m


def _no_cap(res, tol, q, m, m0):
    k = len(res)
    q2, m2 = _ORACLE_LOCK(res, tol, q, m, m0)
    return (q2, m0 * k // (k - q2)) if q < q2 < k else (q2, m2)


def _cap_10(res, tol, q, m, m0):
    q2, m2 = _ORACLE_LOCK(res, tol, q, m, m0)
    return q2, min(m2, 10)


def _ceil(res, tol, q, m, m0):
    k = len(res)
    q2, m2 = _ORACLE_LOCK(res, tol, q, m, m0)
    return (q2, min(-(-m0 * k // (k - q2)), 20)) if q < q2 < k else (q2, m2)


def _can_shrink(res, tol, q, m, m0):
    k = len(res)
    lead = 0
    while lead < k and res[lead] <= tol:
        lead += 1
    return (lead, min(m0 * k // max(k - lead, 1), 20)) if lead != q else (q, m)


def _relock_from_zero(res, tol, q, m, m0):
    """Counts the leading run from pair 0, so a locked pair whose residual rose above
    tol blocks the locking of converged pairs after it."""
    k = len(res)
    lead = 0
    while lead < k and res[lead] <= tol:
        lead += 1
    if lead > q and lead < k:
        return lead, min(m0 * k // (k - lead), 20)
    return max(q, lead), m


@pytest.mark.parametrize("mutant", [_any_order, _no_m_update, _no_cap, _cap_10, _ceil, _can_shrink,
                                    _relock_from_zero],
                         ids=lambda f: f.__name__)
def test_planted_lock_mistakes_fail_a_pin(mutant):
    failed = []
    for pin in (_check_rule, _pin_scenario):
        try:
            pin(mutant)
        except AssertionError:
            failed.append(pin.__name__)
    assert failed, f"{mutant.__name__} passed every pin"
