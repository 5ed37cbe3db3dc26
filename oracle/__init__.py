"""Plain, slow FP64 CPU oracle of the Newton-step linear solve (test infrastructure).

This package is test infrastructure.  Only the test-suite, the smoke check
and the benchmark's CPU-baseline leg may import it; the CUDA library never
calls it, and it shares no code with the CUDA path.

It restates, in numpy, what the paper's hot path computes:

* ``assembly``  -- FastHashReduction's result (Sec. 5.2, Alg. FastHashReduction /
  FastSegmentReduction) by its definition: the sum of all blocks that share
  a key (r, c), r <= c, sorted by key; and the two-level affine-body
  reduction (Sec. 5.1).
* ``partition`` -- the level-0 domain partition with padding (Sec. 3.2,
  Eq. num_subdomains, supplement Algorithm 1).  METIS is replaced by a
  deterministic recursive coordinate bisection of the rest positions, fully
  specified in that module.
* ``mas``       -- connectivity-enhanced MAS levels (supplement Algorithms 2-5),
  level matrices (Algorithm 1 of the paper), per-domain inverses, and the
  preconditioner apply of supplement Eq. 4-6.
* ``pcg``       -- preconditioned conjugate gradients (Sec. 3.2), and the
  symmetric block SpMV (Sec. 5.3) by its definition: ``pcg.spmv`` on the
  stored blocks, ``pcg.SymmetricMatrix`` as a scipy BSR operator.
* ``adjoint``   -- gradients of a loss through x = H^-1 b.
* ``strain_limit`` -- the cubic strain-limiting energy of Sec. 4 and its
  analytic eigensystem.
* ``elastic``   -- stable Neo-Hookean element Hessians (PSD-projected, pulled
  back to the node blocks) and lumped masses of a tet mesh (Sec. 3.1).
* ``newton``    -- Newton's method on the implicit-Euler incremental potential
  (Fig. framework; supplement Eq. 1).
* ``cloth``     -- the stiff-cloth element Hessians: membrane with the cubic
  strain limit of Sec. 4, hinge bending, lumped masses.

Every floating-point quantity is float64.
"""
