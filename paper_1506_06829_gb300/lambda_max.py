"""Largest-modulus eigenvalue of the 64^3 convection-diffusion / mass pencil.

Input preparation for the generalized workload (its shift is
sigma = (0.3 + 0.05i) lambda_max): ARPACK on B^{-1} A, with B (SPD, condition
number <= 27) applied by conjugate gradients.  Prints the value that
``problems.CONFIG2_LAMBDA_MAX`` holds.

    python -m paper_1506_06829_gb300.lambda_max [N]
"""
import sys

import numpy as np
import scipy.sparse.linalg as spla

from . import problems as P


def lambda_max(N: int = 64, tol: float = 1e-10) -> complex:
    A = P.convdiff3d(N, (0.4, 0.2, 0.1))
    B = P.mass3d(N)
    n = A.shape[0]

    def binv_a(x):
        y, info = spla.cg(B, A @ x, rtol=1e-14, maxiter=500)
        if info != 0:
            raise RuntimeError("CG on B did not converge")
        return y

    op = spla.LinearOperator((n, n), matvec=binv_a, dtype=np.float64)
    v0 = np.random.default_rng(2024).standard_normal(n)
    w = spla.eigs(op, k=1, which="LM", tol=tol, v0=v0, ncv=64, maxiter=20000,
                  return_eigenvectors=False)
    return complex(w[0])


if __name__ == "__main__":
    N = int(sys.argv[1]) if len(sys.argv) > 1 else 64
    print(repr(lambda_max(N)))
