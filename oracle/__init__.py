"""Plain, slow CPU oracle for the global-coarsening matrix-free multigrid
method of Munch, Heister, Prieto Saavedra & Kronbichler (arXiv:2203.12292).

THIS PACKAGE IS TEST INFRASTRUCTURE. Only ``tests/``, the ``smoke()`` entry
of ``__graft_entry__`` and the CPU-baseline leg of ``bench.py`` may import or
run it. The product (the CUDA library and its Python binding) never calls
into it and shares no code with it; the only shared module is ``synth``
(seeded inputs, no method arithmetic).

What it computes, each part a plain definition written out in fp64:

* ``mesh``      octree meshes, 2:1 closure, global-coarsening hierarchy
                (Sec. 2.2, Sec. 4 "Examples").
* ``fe``        Q_k on Gauss-Lobatto support points, Gauss quadrature,
                element matrices by full (k+1)^3-point quadrature (Sec. 3.2,
                Sec. 5 set-up).
* ``space``     support points, Dirichlet and hanging-node constraints as an
                explicit matrix C, assembled A = C^T (sum_e A_e) C (Sec. 3.1,
                Eq. 2 as its plain assembled definition), diagonal, RHS.
* ``transfer``  prolongation as the embedding of the coarse space into the
                fine one and restriction as its transpose (Sec. 3.5, Eq. 5).
* ``mg``        Chebyshev/point-Jacobi smoother (Sec. 3.3), exact coarse
                solve (Sec. 3.4), V-cycle (Algorithms 1-2), PCG (Sec. 2).
* ``dirichlet`` inhomogeneous Dirichlet data as constraints with b_i != 0:
                lifting u_g, right-hand side C^T (F - A_all u_g) (Sec. 3.1);
                the Gaussian manufactured solution of Table A.1 and
                polynomial ones.
* ``coefficient`` variable coefficient nu of -div(nu grad u): harmonic
                cell averages of Gauss-point values on the finest level,
                transfer to the coarser levels (Sec. 7, Sec. 3.5).
* ``ls``        geometric local smoothing, the paper's comparison variant:
                refinement levels, refinement-edge DoFs, the V-cycle with
                edge treatment and the copy to/from all active levels
                (Sec. 2.1, Algorithms 1-2).
* ``mapped``    non-Cartesian geometry: the cells mapped by a global
                non-affine map, element matrices with the Jacobian at every
                quadrature point (Sec. 3.2, Eq. 2 in its general form).
* ``mlp``       learned per-cell smoother, an extension outside the paper:
                network forward/backward, loss, Adam, cell features, owner-
                selected correction, optional bf16 operand rounding.

Parity status: every function is pinned by a test in ``tests/test_oracle_*``
against values the paper prints or closed forms; see the module headers.
"""
