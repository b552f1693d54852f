"""Sorted complex QZ of a small pencil (footnote to step 2 of Algorithm 2).
Test infrastructure only.

ordqz(Phi, Psi, sigma) returns the FULL generalized Schur decomposition

    Phi = YL RA YR^*,   Psi = YL RB YR^*,   YL, YR unitary, RA, RB upper triangular,

with the diagonal ordered so that |RA(i,i)/RB(i,i) - sigma| is non-decreasing.
Library primitives: LAPACK's complex QZ (scipy.linalg.qz) and its adjacent-swap
reordering ZTGEXC; the ordering itself is a plain selection sort that moves the
nearest remaining eigenvalue to the next leading position.

Normalisation: the diagonal of RB is made real non-negative (the convention of
LAPACK's complex QZ before reordering, lost by adjacent swaps), by scaling row j
of RA and RB by a unit phase t_j and column j of YL by conj(t_j).  The paper's
remark that M_A -> R and M_B -> I for B = I (Sec. 3.4) relies on it.

Distance (reading of the paper's sort rule, which names only |lambda - sigma|):
|alpha - sigma beta| / |beta|, +inf when beta = 0 (an infinite eigenvalue goes
last); ties are broken by Re(lambda), then Im(lambda).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
from scipy.linalg.lapack import ztgexc


def distance(alpha: complex, beta: complex, sigma: complex) -> float:
    if beta == 0:
        return np.inf
    return abs(alpha - sigma * beta) / abs(beta)


def sort_key(alpha: complex, beta: complex, sigma: complex):
    d = distance(alpha, beta, sigma)
    if not np.isfinite(d):
        return (np.inf, np.inf, np.inf)
    lam = alpha / beta
    return (d, lam.real, lam.imag)


def ordqz(Phi: np.ndarray, Psi: np.ndarray, sigma: complex):
    """Returns (RA, RB, YL, YR) with Phi YR = YL RA, Psi YR = YL RB."""
    Phi = np.asarray(Phi, dtype=np.complex128)
    Psi = np.asarray(Psi, dtype=np.complex128)
    s = Phi.shape[0]
    RA, RB, YL, YR = sla.qz(Phi, Psi, output="complex")
    for pos in range(s - 1):
        keys = [sort_key(RA[j, j], RB[j, j], sigma) for j in range(pos, s)]
        best = pos + min(range(len(keys)), key=lambda t: keys[t])
        if best != pos:
            RA, RB, YL, YR, info = ztgexc(RA, RB, YL, YR, best + 1, pos + 1)
            if info != 0:
                raise np.linalg.LinAlgError(f"ztgexc failed (info={info})")
    # ZTGEXC keeps exact zeros below the diagonal only up to rounding.
    RA = np.triu(RA)
    RB = np.triu(RB)
    for j in range(s):
        mag = abs(RB[j, j])
        if mag > 0:
            t = np.conj(RB[j, j]) / mag
            RA[j, :] *= t
            RB[j, :] *= t
            RB[j, j] = mag
            YL[:, j] *= np.conj(t)
    return RA, RB, YL, YR
