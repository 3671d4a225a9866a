"""FP64 CPU oracle for the multiplicative vertex-patch smoother.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may use it.  It shares no code, no
tables and no constants with the CUDA library; the only module both sides
use is the seeded input generator ``paper_2407_02100_gb300.inputs``, which
holds none of the method's arithmetic.

What it computes, and where the paper defines it
-------------------------------------------------
* ``fe``        -- Q_k Lagrange basis on Gauss-Lobatto support points, Gauss
                   quadrature, cell stiffness by full d-dimensional
                   quadrature (Sec. 2, App. A.1/A.2).
* ``mesh``      -- node numbering of the uniform Cartesian mesh, vertex
                   patches with their closure and interior index maps
                   (Sec. 2.1 item 1, Sec. 3.1 "gather"), colours (Sec. 3.2).
* ``smoother``  -- the combined colourised smoother (Algorithm 4) with local
                   residuals (Sec. 3.1, gather/evaluate/solve/scatter) and
                   dense LU local solves, the naive global-residual loop
                   (Algorithm 1) and the single sequential combined loop
                   (Algorithm 2) as cross-checks.
* ``multigrid`` -- embedding prolongation and its transpose (Sec. 2),
                   dense coarse solve, V(1,1)-cycle, preconditioned CG.

Pins (tests/test_oracle_*.py): closed-form 1D matrices, polynomial
exactness of the quadrature, O(h^{k+1}) L2 convergence of the manufactured
solution, Galerkin identity P^T A_f P = A_c, prolongation reproducing coarse
polynomials, Algorithm 1 == Algorithm 4 on tiny meshes, Q1 sweep ==
hand-written multicolour Gauss-Seidel, zero local residual right after each
colour, monotone energy decrease, brute-force dense inverses.
"""
