"""FP64 CPU oracle for the Neural Physics pressure-Poisson multigrid path.

This package is TEST INFRASTRUCTURE.  Only the test-suite, the smoke check of
``__graft_entry__`` and the CPU-baseline leg of ``bench.py`` may import it.
The GPU library never imports, links or calls anything here, and nothing here
imports the GPU library: the two share no code.  The only module both sides
read is the seeded input generator ``paper_2402_17913_gb300.inputs``, which
holds no arithmetic of the method.

Everything is plain numpy in float64, written so that each step can be
checked against the paper by eye:

* ``poisson``  -- the discrete operator (Sec. 2.1, Eq. A and App. A 5/7-point
  diffusion filters), weighted Jacobi (Eq. Jacobi-1-relax), restriction and
  prolongation (Sec. 2.2, 2x2 average / copy filters), the multigrid cycle
  (Sec. 2.2 step list, Fig. sawtooth), the Krylov wrapper and the iterative
  refinement loop, plus the dense direct solve that defines the answer.
* ``ns``       -- one projection time step of Algorithm 1 on a staggered
  (MAC) grid, with the predictor-corrector momentum update of Sec. 2.3
  (Eq. predictor-Burgers / Tn+1) and the solid-body absorption term sigma;
  optionally the finite-element 9/27-point filters of App. A.
* ``advdiff``  -- one implicit backward-Euler advection-diffusion step
  (Eq. BE-advection-concise, upwind or central advection) and its multigrid
  solution by V or sawtooth cycles as a stationary iteration (Sec. 3.2).
* ``convnet``  -- the learned initial-guess network and its training step.

Pins for every function live in ``tests/test_oracle_*.py`` (closed-form
eigenpairs, manufactured solutions, dense solves, invariants).  Functions that
have no such pin say "parity unpinned" in their docstring.
"""
