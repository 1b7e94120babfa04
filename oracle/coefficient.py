"""Variable coefficient nu of -div(nu grad u) on every multigrid level.

Test infrastructure (see ``oracle/__init__``).

Follows the set-up of the Stokes application (Sec. 7): the coefficient is
evaluated at the quadrature points of every cell of the finest level,
averaged harmonically on each cell, and carried to the coarser levels by
the transfer between levels (``interpolate_to_mg`` of the transfer
interface, Sec. 3.5).  Readings where the
text is silent:

* the harmonic average is weighted by the quadrature weights:
  nu_e = (sum_q w_q) / (sum_q w_q / nu_q) over the (k+1)^3 Gauss points;
* the transfer of a cell-wise constant field to a coarser level keeps the
  value of a cell that is not refined and gives a refined cell the
  arithmetic mean of its eight children (the L2 projection of a piecewise
  constant field onto the coarse cell); levels of the same mesh (polynomial
  coarsening) share the values.

The element matrix of a cell is then nu_e h_e A_ref (Space.element_matrices_scale).
"""
from __future__ import annotations

from typing import Callable, List

import numpy as np

from . import fe


def quadrature_points(space) -> np.ndarray:
    """Gauss points of every cell, (n_cells, (k+1)^3, 3), x fastest."""
    gq, _ = fe.gauss(space.k + 1)
    qa, qb, qc = fe.tensor_index(space.k)
    ref = np.stack([gq[qa], gq[qb], gq[qc]], axis=1)
    return space.origin[:, None, :] + space.h[:, None, None] * ref[None, :, :]


def quadrature_weights(k: int) -> np.ndarray:
    _, gw = fe.gauss(k + 1)
    qa, qb, qc = fe.tensor_index(k)
    return gw[qa] * gw[qb] * gw[qc]


def harmonic_cell_average(k: int, nu_q: np.ndarray) -> np.ndarray:
    """nu_e = (sum_q w_q) / (sum_q w_q / nu_q) for nu_q of shape (n_cells, (k+1)^3)."""
    w = quadrature_weights(k)
    return w.sum() / ((w[None, :] / nu_q).sum(axis=1))


def coarsen(fine, coarse, nu_fine: np.ndarray) -> np.ndarray:
    """Cell values of the coarse space from those of the fine one."""
    if fine.nc == coarse.nc and np.array_equal(fine.cells, coarse.cells):
        return nu_fine.copy()
    out = np.empty(coarse.nc)
    for c in range(coarse.nc):
        l, i, j, kk = coarse.cells[c]
        same = fine.find_cells(np.array([l]), np.array([i]), np.array([j]), np.array([kk]))[0]
        if same >= 0:
            out[c] = nu_fine[same]
            continue
        ch = [fine.find_cells(np.array([l + 1]), np.array([2 * i + a]), np.array([2 * j + b]),
                              np.array([2 * kk + e]))[0]
              for e in (0, 1) for b in (0, 1) for a in (0, 1)]
        if min(ch) < 0:
            raise RuntimeError("levels are not nested")
        out[c] = np.mean(nu_fine[ch])
    return out


def set_level_coefficients(spaces: List, nu: Callable[[np.ndarray], np.ndarray]) -> None:
    """spaces: coarsest first.  Harmonic averages of nu at the finest level's
    Gauss points, then the transfer down the hierarchy."""
    fine = spaces[-1]
    xq = quadrature_points(fine)
    nu_q = nu(xq.reshape(-1, 3)).reshape(fine.nc, -1)
    fine.nu = harmonic_cell_average(fine.k, nu_q)
    for l in range(len(spaces) - 2, -1, -1):
        spaces[l].nu = coarsen(spaces[l + 1], spaces[l], spaces[l + 1].nu)
