"""Plain CPU oracle for the matrix-free Stokes / stabilised Navier--Stokes path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this
package: only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline``
leg of ``bench.py`` use it.  It shares no code with the CUDA library.

What it computes (all in float64, by straightforward quadrature and sparse
assembly, no sum factorisation):

* ``fe``        -- Gauss--Lobatto--Legendre support points, Gauss quadrature,
                   1D Lagrange polynomials (values and derivatives).
* ``mesh``      -- forests of axis-aligned squares/cubes: uniform meshes and a
                   ball refinement with 2:1 closure; node identification, DoF
                   numbering, Dirichlet and hanging-node constraints.
* ``forms``     -- element matrices of the weak forms: the vector Laplacian
                   (A block), Taylor--Hood Stokes (Eq. 1/5), the
                   Newton-linearised SUPG/PSPG-stabilised BDF2 Navier--Stokes
                   operator (Eq. 3 and the stabilisation terms of Section 5),
                   and the pressure mass matrix.
* ``assemble``  -- global sparse assembly, the constrained operator
                   A = C^T K C (+) I, its diagonal, and row sampling for large
                   meshes.
* ``transfer``  -- h- and p-prolongation by interpolation (Eq. 4); restriction
                   is the transpose.
* ``solvers``   -- Chebyshev--Jacobi and Jacobi smoothing, the V-cycle, FGMRES
                   with classical Gram--Schmidt (two passes) and the
                   block-triangular Stokes preconditioner (Eq. 5).
* ``ls``        -- local-smoothing multigrid (Section 2): level spaces on the
                   refined parts of the mesh with Dirichlet conditions on the
                   refinement edge, as a multiplicative subspace correction.
* ``spacetime`` -- space-time finite elements for transient Stokes (Section 4):
                   DG(r) in time on right Radau points, the stage-major
                   Kronecker operator G_Q (x) M + tau I_Q (x) A, time transfers.
* ``pdisc``     -- Stokes with a discontinuous pressure, Q_k / P^disc_{k-1}
                   (the spatial pair of Section 4), with its transfers.
* ``hp``        -- hp-adaptive continuous spaces (a degree per cell, h- and
                   p-hanging constraints), the vector Laplacian and Taylor--Hood
                   Stokes on them, hp transfers and the hp-multigrid hierarchy
                   (degrees lowered one by one, then h; Section 3).

Parity status: every function here is pinned by tests against closed forms,
textbook values, invariants or brute force (see ``tests/test_oracle_*.py``);
the eigenvalue estimate for the Chebyshev bounds is not part of the oracle:
parity tests pass the bounds explicitly.
"""
