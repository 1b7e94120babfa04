"""Transfer between two nested discrete spaces.

Test infrastructure (see ``oracle/__init__``).

Follows Sec. 3.5, Eq. 5: prolongation x_f = W P~ C_c x_c resolves the coarse
constraints, prolongates cell by cell on the discontinuous space and zeroes
the constrained fine values. For nested spaces (global coarsening: every fine
cell is a coarse leaf or lies inside one; polynomial coarsening: the same
mesh with k_c = floor(k_f / 2)) the element prolongation
P_e = M_f^{-1} (phi_f, phi_c) is interpolation, and the valence weights W
average equal values, so the prolongated vector is the plain definition used
here: the coarse finite-element function evaluated at the free fine support
points. Restriction is the transpose (Sec. 3.5: R = P^T).

Pins (tests/test_oracle_transfer.py): coarse polynomials are reproduced
exactly; Q1 uniform refinement gives the textbook trilinear weights;
R = P^T is checked by duality x^T (P y) = (R x)^T y against the evaluation
routine ``Space.evaluate`` (an independent code path).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import fe
from .mesh import ancestor_in
from .space import Space


def prolongation_matrix(fine: Space, coarse: Space) -> sp.csr_matrix:
    """P (n_free_fine x n_free_coarse)."""
    # one fine cell per free fine point
    nf = fine.n_free
    owner_cell = np.full(fine.n_points, -1, dtype=np.int64)
    owner_cell[fine.cell_nodes.ravel()[::-1]] = np.repeat(np.arange(fine.nc), fine.n3)[::-1]
    fp = fine.free_points
    fcell = owner_cell[fp]
    # coarse leaf containing each fine cell
    anc_cache = {}
    K = np.empty(nf, dtype=np.int64)
    for idx, fc in enumerate(fcell):
        if fc not in anc_cache:
            c = tuple(int(t) for t in fine.cells[fc])
            a = ancestor_in(coarse.mesh, c)
            anc_cache[fc] = int(coarse.find_cells(a[0], a[1], a[2], a[3]))
        K[idx] = anc_cache[fc]
    s = (fine.points[fp] - coarse.origin[K]) / coarse.h[K][:, None]
    phi = fe.basis_at(coarse.k, s)  # (nf, n3c)
    rows = np.repeat(np.arange(nf), coarse.n3)
    cols = coarse.cell_nodes[K].ravel()
    E = sp.csr_matrix((phi.ravel(), (rows, cols)), shape=(nf, coarse.n_points))
    E.eliminate_zeros()
    return (E @ coarse.C).tocsr()
