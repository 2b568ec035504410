"""CPU FP64 oracle for matrix-free finite-strain hyperelasticity (arXiv 1904.13131).

TEST INFRASTRUCTURE ONLY. Nothing in the product package imports this code;
only the tests, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline /
reference leg may use it. It shares no code with the CUDA path: it builds its
own basis tables, its own mesh connectivity, assembles the sparse tangent and
residual with full (non sum-factorised) shape-function tables, and solves with
scipy's sparse direct solver or a plain CG.

Modules
  basis     1D GLL nodes, Gauss rule, Lagrange basis, full tensor-product tables
  material  compressible neo-Hooke: psi, tau, J*C (Sec. 2.3)
  fem       lattice mesh, energy, residual (Eq. weak_form), tangent (Eq. algebraic_tangent),
            element-by-element operator action (Eq. mf_vmult), diagonal
  gmg       geometric transfers, displacement carried down to levels (Sec. 6),
            Chebyshev smoother, eigenvalue estimate, V-cycle, PCG
  newton    Newton-Raphson with load steps (Sec. 3, Sec. 7)
  rng       SplitMix64 counter-based generator (start vectors of the eigen estimate)

Every function states the passage of the paper it follows. Where the paper is
silent or ambiguous, the reading taken is stated where it is used (e.g. nodal
interpolation for carrying the displacement down, one Chebyshev sweep per
smoothing step, lifting of the prescribed increment into the first Newton solve).
Parity status: every function is pinned by tests in tests/test_oracle_*.py.
"""
