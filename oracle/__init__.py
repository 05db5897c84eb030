"""CPU FP64 oracle of spaND with first- and second-order sparsification.

TEST INFRASTRUCTURE ONLY.  This package is the slow, plain reference that the
CUDA path is checked against.  Only the tests, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import it; the product library never
calls it and shares no code with it (the two only share the seeded input
generators of ``spand_inputs``, which contain none of the method).

Contents, each written from the paper (arXiv 2007.00789):

* ``partition`` -- geometric nested dissection and the per-level clusters
  (interiors / interface pieces) that the spaND partitioning of §3 needs;
* ``rrqr``      -- Algorithm 1: early-stopping column-pivoted Householder QR
  and the extraction of E / E_2 and Q_c^T A_pw;
* ``spand``     -- Algorithm 2 (eliminate interiors, scale interfaces,
  sparsify interfaces, recurse), the preconditioner apply
  M = L^{-T} L^{-1}, and PCG with a zero initial guess (§4).

Floating point is float64 throughout; dense steps use library primitives
(Cholesky, triangular solve, matmul) exactly where the paper's formulas
name those operations.

Parity pins: every function is checked by ``tests/test_oracle_*.py`` against
closed forms or brute force (exact block Cholesky at eps = 0, the two-level
error identities of §2.1-2.2, Propositions 1-3, Theorem 1, the Poisson
eigenpairs of §4.1.1).  The per-cluster ranks and CG iteration counts of the
large grid workloads are "parity unpinned": the paper prints no value for
those shapes, so they are checked only for self-consistency.
"""
