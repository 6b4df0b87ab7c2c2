"""Plain FP64 CPU oracle for the accuracy-controlled H^2 direct solver.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The CUDA library never imports, links or executes it, and it shares
no code with the CUDA library: the only common module is the seeded input
generator ``paper_1703_06155_gb300.inputs``, which holds none of the method.

Everything here is slow, sequential, complex128 numpy, written from the paper
(Ma & Jiao, "Accuracy directly controlled fast direct solutions of general
H^2-matrices", 2017).  Each function cites the section / equation / algorithm
it follows.  Library primitives (matmul, SVD, Hermitian eigensolver,
Householder QR, triangular solve) are used as single steps.

Modules
  kernel  - matrix entries of the scalar volume-integral-equation stand-in
  tree    - cluster tree (Sec. II) and block partition (eq. 1)
  h2      - exact nested-basis H^2 construction, matvec, dense assembly
  dense   - own dense LU with partial pivoting, solve, inverse (brute force)
  factor  - Algorithms 1-4 (factorization), eq. 35 (inverse), Alg. 5-6 (solve),
            adjoint solve, iterative refinement
  adjoint - dense derivative of the solve in the per-cell contrast (general
            and reduced forms, probe objective, finite differences)
"""
