"""Plain FP64 CPU oracle for the inverse-free spectral divide-and-conquer.

TEST INFRASTRUCTURE ONLY.  This package is the slow, obviously-correct
restatement of Ballard, Demmel and Dumitriu, "Minimizing Communication for
Eigenproblems and the Singular Value Decomposition" (arXiv 1011.3077), written
from the paper's algorithms in their order and notation.  Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py`` (its ``cpu_baseline`` leg and
``--impl reference`` arm) may import it.  The CUDA product path never imports,
links or executes anything here, and this package shares no code with it.

Library primitives used as single steps: numpy's matrix product ``@``, ``sqrt``,
``log``, ``cos``/``sin``, ``sort`` and ``median``.  No LAPACK routine is called:
every factorization (Householder QR, RQ, Jacobi, Hessenberg, Francis QR) is
written out here.

Modules
  philox     Philox4x32-10 counter generator and Box-Muller normals (Sec. 2,
             the Gaussian matrix of Algorithm 1).
  householder  Householder QR with explicit Q, RQ by index reversal (Sec. 3
             intro: QR/RQ/QL/LQ routines).
  irs        Implicit repeated squaring (Algorithm 3) and the region maps of
             Sec. 3.3 (Moebius line -> unit circle) and Sec. 3.5 (circles).
  rurv       Haar matrix, RURV (Algorithm 1), GRURV (Algorithm 2).
  split      Similarity, symmetrisation and the block-size choice (Algorithms
             4-6, Sec. 4.2.1 prefix-sum / max formulation).
  leaves     Small-problem solvers ("the standard algorithm", Sec. 3.6):
             cyclic Jacobi, Hessenberg + Francis double-shift QR.
  solve      One divide step (RSEP / RNEP / RGNEP) and the recursive drivers
             (Sec. 3.3-3.5 strategies).
  svd        RSVD through the symmetric embedding (Sec. 3.2).
  trevc      Eigenvectors from the Schur form (the eigenvector section).
  complex_qr   Complex Householder QR / RQ and the Haar unitary.
  complex_leaf Complex Hessenberg + single-shift QR (complex Schur leaves).
  cplane     The complex-plane strategy of Sec. 3.3: lines at random angles,
             the 2-step radius shrink and convex enclosures of clusters.

Parity status of each function is stated in its docstring; functions with no
independent pin say "parity unpinned".
"""
