"""Plain FP64 CPU oracle of the space-time GMG-preconditioned FGMRES solve.

THIS PACKAGE IS TEST INFRASTRUCTURE. Only the tests, the package smoke check and the benchmark's
CPU-baseline / reference legs may import, call or execute it. The GPU library never routes through
it and shares no code, table or helper with it; the only common input is the seeded generator in
`synth/`, which holds no discretisation or solver arithmetic.

The oracle follows Anselmann & Bause, "A geometric multigrid method for space-time finite element
discretizations of the Navier-Stokes equations and its application to 3d flow simulation"
(arXiv 2107.10561):
  * `fem`     -- Q2/P1^disc spaces, dG(k) Radau-Lagrange time basis, Nitsche forms and the Newton
                 Jacobian of one time slab (Sec. 2.3, 2.4, 3; Problem 3.1; Eqs. Def:Ah, Def:B_GamD,
                 linNewEq, totdofs, locdofs), intergrid transfer (Sec. 4.1);
  * `solvers` -- cell inverses (Sec. 4.3), the cell-based space-time Vanka smoother (Sec. 4.2,
                 Eq. LocVanka, damping of Sec. 5.3), the V-cycle (Algorithm 1) and flexible GMRES
                 (Sec. 3), plus the adjoint (transposed) solve.

Every function is pinned by tests in tests/test_oracle_*.py against closed forms, invariants,
manufactured solutions and brute-force dense solves.
"""
