"""Plain, slow FP64 CPU oracle for the Newton-GMRES-BDDC tangent solve.

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
baseline leg of the benchmark may import this package.  The CUDA library
never calls it, and it shares no code with the library: the only common
input is the seeded problem description from ``workloads``.

Modules and what they follow (section / equation of Barnafi, Pavarino,
Scacchi, "A comparative study of scalable multilevel preconditioners for
cardiac mechanics", arXiv 2208.06191):

* ``elements``  -- Q1/Q2 hexahedra, Gauss quadrature (Section 2,
  "Space discretization").
* ``material``  -- Guccione passive law and active stress (Section 2).
* ``assembly``  -- residual of Eq. (mechanics time discrete) without the
  inertia term, follower pressure of Eq. (bc endo), exact tangent of
  Eq. (tangent problem).
* ``bddc``      -- two-level BDDC of Section 3.2 (block factorization,
  spaces, counting scaling, coarse basis and coarse matrix).
* ``krylov``    -- restarted right-preconditioned GMRES and flexible GMRES.
* ``newton``    -- load-stepped Newton iteration of Eq. (tangent problem).

Parity status: every function is pinned by the CPU tests (finite
differences, closed forms, patch test, BDDC exactness and spectral
properties).  Absolute displacement values have no printed counterpart in
the paper and are pinned only through those properties.
"""
