"""FP64 CPU oracle for the Nystrom-preconditioned matrix-free NGD hot path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports, links or runs
this package: only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s
CPU-baseline / reference legs use it.  It shares no code with the CUDA library
(``paper_2505_11638_gb300/csrc``); the two meet only through the seeded input
arrays of ``paper_2505_11638_gb300.inputs``.

It is deliberately plain and slow: NumPy float64, one function per step of the
paper, library primitives (matmul, QR, Cholesky, SVD) used as single steps and
nothing blocked, fused or reordered.

Modules
  mlp      tanh MLP (Sec. 2.3), forward-Laplacian residual and loss (Sec. 2.2.1,
           Eq. energy_poisson), explicit Jacobian rows, JVP, VJP (Thm. 1).
  gramian  G = J^T diag(w) J (Thm. 1, Eq. G_matrixfree), matvec, diagonal
           (Eq. gram_diagonal), direct damped solve (Alg. 2).
  philox   Philox4x32-10 counter RNG (Salmon et al., SC'11) and Box-Muller, the
           Gaussian test matrix of App. A.
  nystrom  randomized Nystrom approximation (App. A, Alg. randomized_nystrom) and
           the preconditioner of Alg. 4 (Eq. nystrom_inverse).
  solve    preconditioned CG (Sec. 3/4, Alg. 3), Armijo line search and one NGD
           step (Alg. 1 with Alg. 3 and Alg. 4).

Every function of ``mlp``, ``gramian``, ``philox``, ``nystrom`` and ``solve`` is
pinned by a ``-m "not gpu"`` test against something other than itself (closed
forms, finite differences, published known-answer vectors, invariants, brute
force).  No function here is "parity unpinned".
"""
