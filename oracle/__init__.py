"""FP64 CPU oracle of the Enzo-P/Cello hydro hot path (arXiv:1810.01319).

TEST INFRASTRUCTURE ONLY.  Only tests/, the smoke check and the benchmark's
CPU-baseline leg may import this package; the product library never does,
and it shares no code with the CUDA path (the seeded initial conditions in
`workloads` are the only common input).

Modules: mesh (array-of-octrees leaf list, neighbour table, 2:1 balance,
build from flags), hydro (ghost refresh, PPM sweeps with the two-shock
Riemann flux, coarse-fine flux correction, CFL dt, conserved totals, refine
flags), exact (exact Riemann solver, Sedov-Taylor constant).

Parity pins: every function is pinned by tests/test_oracle_*.py against
closed forms, invariants, brute force or the exact reference solutions.
"""
