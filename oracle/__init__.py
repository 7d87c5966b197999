"""CPU oracle for the matrix-full Vanka multigrid / FGMRES solver of Taylor-Hood Stokes.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  The product path (the C-ABI
library under ``paper_2409_14222_gb300/``) never imports, links or calls it, and this package never
imports the product.  The two share no code; only ``synthetic_inputs`` (seeded random inputs, no
arithmetic of the method) serves both.

Everything here is plain, slow, FP64 (or exact rational where the quantity is rational) and follows
the paper, arXiv 2409.14222 ("Achieving h- and p-robust monolithic multigrid solvers for the Stokes
equations"):

* ``exact``   -- P_k Lagrange basis on the reference triangle in exact rational arithmetic
                 (Sec. 2, Taylor-Hood pair (P_k, P_{k-1}), Case 1 of Sec. 3).
* ``fem``     -- structured mesh, DoF numbering, the bilinear forms a(.,.) and b(.,.) of Eqs.
                 (VariationalStokesa/b), the saddle-point block matrix of Sec. 3, Dirichlet
                 no-slip rows (Eq. StokesDirichletNoSlip), canonical transfers (Sec. 3, "grid
                 transfer operations"), manufactured solution (Eq. model_problem), error norms (Sec. 4.4).
* ``patches`` -- vertex / edge / cell ("composite", "topological") Vanka patches of Sec. 3.1.
* ``quad``    -- Taylor-Hood (Q_k, Q_{k-1}) on quadrilaterals (Case 2 of Sec. 3): exact tensor-product
                 element matrices, transfers, composite patches, manufactured data and error norms.
* ``bdm``     -- (BDM_k, dP_{k-1}) with the interior-penalty form of Eq. (DiscontBilinearForm) (Case 3):
                 exact reference basis and transfers, FP64 element and edge integrals, extended cell
                 patches (Sec. 3.1), manufactured data and broken error norms.
* ``solver``  -- additive subspace correction (Algorithm 1), Chebyshev acceleration with the
                 [lambda/4, 1.1 lambda] interval (Sec. 3, "Relaxation"), Arnoldi eigenvalue estimate,
                 multiplicative V-cycle, bordered coarse solve, FGMRES (Sec. 3 and Sec. 4).
* ``splitmix`` -- SplitMix64 counter-based generator (Steele, Lea and Flood, OOPSLA 2014) for the
                 start vector of the eigenvalue estimate.

Readings where the paper is silent are listed in each function's docstring.
"""
