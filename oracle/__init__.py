"""Plain, slow FP64 CPU oracle for the SIPG discontinuous Galerkin elliptic
solver of Vincent, Pfeiffer & Fischer (arXiv:1907.01572).

This package is TEST INFRASTRUCTURE.  Only the tests, the smoke check in the
repository entry module and the CPU-baseline leg of the benchmark may import
it.  It shares no code, tables or helpers with the CUDA library: every
quantity here is computed from the paper's definitions with numpy / scipy
(dense basis matrices, brute-force quadrature, no sum factorisation).

Modules
-------
tables     1-D Legendre-Gauss-Lobatto / Gauss-Legendre rules, Lagrange basis (Sec. II.A.3, II.A.5)
mesh       single-block octree mesh, element maps, mortars (Sec. II.A.1)
blockmesh  multi-block meshes (hexahedral, cubed-sphere wedge and shell blocks), mortars across blocks
sipg       SIPG bilinear form and right-hand side by dense quadrature (Eqs. lh2, equationFh2)
multigrid  level meshes, prolongation, Chebyshev + CG-eigenvalue smoother, V-cycle (Sec. II.E, Algs. 3-5)
krylov     flexible CG (Alg. 2)
puncture   puncture initial-data source terms and Newton (Sec. III.D, Alg. 1)

Parity status of each function is stated in its module header.
"""
