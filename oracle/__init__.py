"""CPU oracle for the GPLHR eigensolver (Vecharynski, Yang & Xue, arXiv 1506.06829).

TEST INFRASTRUCTURE ONLY.  Plain, slow, FP64/complex128 NumPy/SciPy code that
follows the paper step by step, used to check the CUDA path.  Only ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference`` legs
of ``bench.py`` may import it.  It shares no code with the CUDA path
(``paper_1506_06829_gb300``); the only common module is the seeded input
generator ``paper_1506_06829_gb300.problems``, which holds none of the method's
arithmetic.

Modules
-------
schur     -- Lemma 1 / Theorem 1: G1, G2 (Eqs. G1_fix, G2_fix), G, M_A, M_B (Eq. M).
ordqz     -- full generalized Schur form of a small pencil, ordered by distance
             of the eigenvalues to sigma (Alg. 2 footnote to step 2).
precond   -- T ~ (A - sigma B)^{-1}: identity, Jacobi, block-Jacobi (Sec. 4).
gplhr     -- Algorithm 2 (GPLHR) with soft locking and m-adaptation (Sec. 3.6).
vectors   -- eigenvectors from Schur vectors and residual measures (Sec. 2.1).
grad      -- eigenvalue adjoint d lambda = y^*(dA - lambda dB)x / (y^* B x).

Parity pins: every function is checked in ``tests/test_oracle_*.py`` against
closed forms, library eigensolvers on small dense copies and invariants stated
by the paper.  No function here is "parity unpinned".
"""
