"""Q-free Schur factors (Sec. 2.2 of the paper).  Test infrastructure only.

Given upper triangular R_A, R_B of a partial generalized Schur form
A V = Q R_A, B V = Q R_B (Eq. gschur), Lemma 1 and Theorem 1 build

    G1, G2 diagonal (Eqs. G1_fix, G2_fix, i.e. tau_j = 0 if |R_A(j,j)| < |R_B(j,j)|
                     and tau_j = 1 otherwise),
    G   = R_A G1 + R_B G2           (unit upper triangular, Lemma 1),
    M_A = G2 G^{-1} R_A,  M_B = I - G1 G^{-1} R_A      (Eq. M),

so that A V M_B = B V M_A (Eq. gschur2) with M_A(j,j)/M_B(j,j) = lambda_j.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


def g_factors(RA: np.ndarray, RB: np.ndarray):
    """Diagonals of G1 and G2 per Eqs. G1_fix and G2_fix."""
    a = np.diag(RA).astype(np.complex128)
    b = np.diag(RB).astype(np.complex128)
    g1 = np.zeros_like(a)
    g2 = np.zeros_like(a)
    for j in range(a.size):
        if abs(a[j]) < abs(b[j]):
            g1[j] = 0.0
            g2[j] = 1.0 / b[j]
        else:
            g1[j] = (1.0 - b[j]) / a[j]
            g2[j] = 1.0
    return g1, g2


def m_factors(RA: np.ndarray, RB: np.ndarray):
    """(M_A, M_B, G) of Theorem 1 with the fixed tau choice."""
    RA = np.asarray(RA, dtype=np.complex128)
    RB = np.asarray(RB, dtype=np.complex128)
    g1, g2 = g_factors(RA, RB)
    G1 = np.diag(g1)
    G2 = np.diag(g2)
    G = RA @ G1 + RB @ G2
    # G is unit upper triangular: G^{-1} R_A by a triangular solve.
    GinvRA = sla.solve_triangular(G, RA, lower=False)
    MA = G2 @ GinvRA
    MB = np.eye(RA.shape[0]) - G1 @ GinvRA
    return MA, MB, G
