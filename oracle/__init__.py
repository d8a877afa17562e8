"""Plain, slow FP64 CPU oracle for the two-grid MLQMC level evaluation.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports, calls or runs
this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may use it.  It
shares no code with the CUDA library; the two meet only through the seeded
inputs of ``synthetic_inputs``.

What it computes (Gilbert & Scheichl, MLQMC for random elliptic eigenvalue
problems II):

* ``fem``      -- P1 finite elements on the uniform SW-NE triangulation of the
                  unit square, assembled by element loops (Sec. 2.3), and the
                  affine coefficient a = a0 + sum_j y_j psi_j at element centroids
                  (eq. coeff, truncated as in eq. coeff_s); the second test problem
                  of Sec. 5 (four islands, piecewise a0 and b0, a parametric reaction
                  b = b0 + sum_j y_j b_j and its reaction matrix); the integral of a
                  P1 function.
* ``lattice``  -- CBC generating vectors with product weights and randomly
                  shifted rank-1 lattice points (Sec. 2.5, eq. rqmc, eq. t_kl).
* ``twogrid``  -- exact smallest eigenpairs, P1 interpolation between nested
                  meshes and the two-grid-truncation step (Algorithm 1); the
                  eigenfunction functional G(u) = |integral of u| / ||u||_L2.
* ``mlqmc``    -- per-sample level differences (of the eigenvalue or of G(u)) and
                  the shift-averaged estimator
                  with its sample-variance error estimate (Algorithm 2,
                  eq. tg-mlqmc, eq. sample_var).

Every inner problem is solved exactly (dense LAPACK or sparse direct LU), so
the result does not depend on solver tolerances or warm starts.

Parity pins: every function is pinned by ``tests/test_oracle_*.py`` against
closed forms, invariants, library routines or brute force, except the
per-sample values at the full workloads, which the paper does not print
(parity of those is pinned only through the function-level checks).
"""
