"""FP64 CPU oracle for the SPAI-preconditioned CG hot path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may use it.  It shares no code with the CUDA library (no kernels,
headers, helpers or constant tables); the two meet only in the seeded inputs of
``workloads``.

Contents (each function cites the passage of the paper it follows):

* ``pattern``  - sparsity pattern of G (full / lower / upper) and the explicit
  transpose with its value permutation (Sec. 3.2.2: G keeps A's pattern).
* ``fsai``     - classical factorised sparse approximate inverse, the
  Kolotilina-Yeremin construction the paper cites beside Eq. 1 (M^-1 = G G^T).
* ``gnn``      - the encoder-processor-decoder GNN forward pass (Sec. 3.2.2,
  Eqs. 3-5) with the dimension-agnostic norm of Sec. 3.3.
* ``pcg``      - CSR mat-vec, the preconditioner apply of Eq. 2 and
  Algorithm 1 (App. A) with residual replacement.
* ``spectrum`` - kappa and Kaporin's condition number of M^-1 A (Sec. 4.5),
  dense, and the Ritz values of the CG / Lanczos tridiagonal matrix.
* ``sai``      - the scale-invariant aligned-identity loss with probe vectors
  (Sec. 3.3, Eqs. 7-8), forward value.
* ``train``    - its gradient with respect to G and, by reverse-mode
  differentiation of Eqs. 3-5, with respect to the GNN's weights (Sec. 3.3).

All arithmetic is float64 (the paper fixes no precision).  The code is written
for readability, not speed: plain numpy with no blocking or fusion.
"""
from . import pattern, fsai, gnn, pcg, sai, spectrum, train  # noqa: F401
