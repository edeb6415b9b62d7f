"""FP64 CPU oracle for the defect-correction monolithic AMG solve phase.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import or run anything in this package;
the CUDA library and its Python binding never do, and there is no CPU fallback
through it.

It restates the paper's solve phase step by step in plain numpy / scipy FP64,
sharing no code with the CUDA path:

* ``vanka``  - additive Vanka relaxation (Sec. 3.3.1, Eq. vanka) with every
  patch system solved by dense LU with partial pivoting;
* ``dlsc``   - the DLSC relaxation (Sec. 3.3.2, Alg. 2) with Chebyshev
  semi-iterations;
* ``cycle``  - the defect-correction cycle (Eq. TG-operator-full) around the
  Galerkin V-cycle on the P1isoP2/P1 hierarchy (Eq. TG-operator), with an
  exact bordered solve on the coarsest level;
* ``krylov`` - restarted flexible GMRES with right preconditioning (Sec. 4);
  ``cycle.krylov_relax`` wraps a relaxation in a few such steps (Sec. 3.3.1);
* ``btp``    - the block-triangular comparison preconditioner (Sec. 4): SA
  V-cycles on A and on the scaled pressure mass matrix (or its exact
  block-diagonal inverse);
* ``search`` - the brute-force search of relaxation weights (Sec. 4);
* ``direct`` - sparse direct solves of the full Stokes system, used by the
  pins of the discretisation.

Its inputs come from the seeded problem generator (``problems``), which
holds no solve-phase arithmetic.
"""
