"""Plain FP64 CPU oracle of the hierarchically preconditioned eigensolver.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline / reference leg may import, call or execute
anything in this package.  The CUDA library never imports it, and it imports
nothing from the library: the two share only the seeded input generators in
``workloads``.

Modules:
  rng     -- SplitMix64 counter generator (random vectors the method draws)
  mmd     -- decomposition build (Sections 2.2-2.3)
  solvers -- CG, flexible PCG, Operator OP, B-solve (Sections 4-5)
  eig     -- Algorithms 2-6 with the level-0 completion
  grad    -- eigenvalue / eigenvector gradients w.r.t. the CSR values
"""
