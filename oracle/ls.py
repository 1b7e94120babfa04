"""Geometric local smoothing (the paper's comparison variant).

Test infrastructure (see ``oracle/__init__``).

Follows Sec. 2.1 and Algorithms 1-2:

* level l holds every octree cell of refinement level l (active or refined);
  its Q_k space has no hanging nodes; Dirichlet values on the domain
  boundary are removed as on the active mesh;
* the DoFs of level l split into interior ones (S) and the ones on the
  refinement edges (E): support points on the boundary of the region that
  the level-l cells cover, inside the domain;
* the smoother sees A_SS only (homogeneous Dirichlet values on E); the
  residual passed to level l-1 is (b_S - A_SS x_S, -A_ES x_S) (the edge part
  of b already lives on a coarser level, Algorithm 1); after the
  prolongation the edge values are the prolongated coarse values and the
  postsmoother sees b_S - A_SE x_E (inhomogeneous Dirichlet values from the
  coarser level);
* Algorithm 1 copies the right-hand side to, and the solution from, every
  level with active cells.

Readings where the text is silent (the same as for global coarsening
otherwise: Chebyshev(3) around point Jacobi of A_SS, lambda_max by Lanczos
from 1 + seeded position-keyed values, exact coarse solve on level 0):

* a DoF of the active mesh is copied to the coarsest level among its active
  cells' levels; it is interior there, and an edge DoF on every finer level
  that holds it;
* the transfer between levels l-1 and l is the embedding of the level-(l-1)
  space (restricted to the parents of level-l cells) into the level-l space,
  evaluated at the S and E support points of level l; restriction is its
  transpose.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Callable, List, Optional

import numpy as np
import scipy.linalg as sla

import synth

from . import mesh as omesh
from .mg import EIG_SAFETY, chebyshev, lanczos_lambda_max, pcg, SolveResult
from .space import Space
from .transfer import prolongation_matrix


def level_mesh(fine: omesh.Mesh, l: int) -> omesh.Mesh:
    """The cells of refinement level l as a mesh (all of them leaves)."""
    m = omesh.Mesh(fine.lo, fine.hi)
    m.leaves = {c for c in fine.leaves | fine.internal if c[0] == l}
    m.internal = set()
    return m


def edge_points(space: Space) -> np.ndarray:
    """Bool mask over the free DoFs: support points on a refinement edge,
    i.e. next to a grid cell of the level that lies inside the domain but is
    not a cell of the level."""
    cells = set(map(tuple, space.cells.tolist()))
    l = int(space.level[0]) if space.nc else 0
    n = 1 << l
    h = (space.mesh.hi - space.mesh.lo) / n
    out = np.zeros(space.n_free, dtype=bool)
    for f, p in enumerate(space.free_points):
        t = (space.points[p] - space.mesh.lo) / h
        ranges = []
        for d in range(3):
            fl = int(np.floor(t[d] + 1e-9))
            on = abs(t[d] - round(t[d])) < 1e-9
            ranges.append((fl - 1, fl) if on else (fl,))
        for i in ranges[0]:
            for j in ranges[1]:
                for k in ranges[2]:
                    if 0 <= i < n and 0 <= j < n and 0 <= k < n and (l, i, j, k) not in cells:
                        out[f] = True
    return out


@dataclass
class LSLevel:
    space: Space
    edge: np.ndarray             # bool over the free DoFs
    A: object                    # assembled level matrix over S and E (sparse)
    diag: np.ndarray             # its diagonal
    lam_max: float = 1.0
    P: Optional[object] = None   # from level l-1 to level l (sparse)
    chol: object = None
    dtype: type = np.float64
    A32: object = None

    @property
    def dinv(self) -> np.ndarray:
        """point Jacobi of A_SS: zero on the edge DoFs, which the smoother never changes"""
        return np.where(self.edge, 0.0, 1.0 / self.diag)

    def apply64(self, x):
        return self.A @ x

    def apply(self, x):
        if self.dtype == np.float32:
            return self.A32 @ x
        return self.A @ x


@dataclass
class CopyMap:
    """Algorithm 1: active free DoF g <-> (level[g], index[g]) of that level."""
    level: np.ndarray
    index: np.ndarray


def build_ls_levels(fine: omesh.Mesh, k: int) -> List[LSLevel]:
    """Levels 0 (one cell) .. L (finest refinement level)."""
    L = fine.max_level
    levels: List[LSLevel] = []
    for l in range(L + 1):
        s = Space(level_mesh(fine, l), k)
        A = s.assemble()
        lev = LSLevel(s, edge_points(s), A, A.diagonal().copy())
        if l > 0:
            lev.P = prolongation_matrix(s, levels[-1].space)
        levels.append(lev)
    if np.any(levels[0].edge):
        raise RuntimeError("level 0 must cover the domain")
    if levels[0].space.n_free:
        levels[0].chol = sla.cho_factor(levels[0].A.toarray(), lower=True)
    for lev in levels[1:]:
        start = 1.0 + synth.point_values(lev.space.free_coordinates(), synth.LANCZOS_START_SEED)
        lev.lam_max = EIG_SAFETY * lanczos_lambda_max(lev.apply64, lev.dinv, start=start)
    return levels


def copy_map(active: Space, levels: List[LSLevel]) -> CopyMap:
    """Every free DoF of the active mesh goes to the coarsest level among the
    levels of the active cells that hold it."""
    n = active.n_free
    lvl = np.full(n, 1 << 30, dtype=np.int64)
    idx = np.full(n, -1, dtype=np.int64)
    for c in range(active.nc):
        l = int(active.level[c])
        lev = levels[l].space
        lc = int(lev.find_cells(np.array([l]), *[np.array([int(active.cells[c, d])]) for d in (1, 2, 3)])[0])
        for nd in range(active.n3):
            g = active.free_index[active.cell_nodes[c, nd]]
            if g < 0 or l >= lvl[g]:
                continue
            f = lev.free_index[lev.cell_nodes[lc, nd]]
            lvl[g], idx[g] = l, f
    if np.any(idx < 0):
        raise RuntimeError("a free DoF without a level")
    return CopyMap(lvl, idx)


def set_precision(levels: List[LSLevel], dtype) -> None:
    for lev in levels:
        lev.dtype = dtype
        if dtype == np.float32:
            lev.A32 = lev.A.astype(np.float32)


def vcycle(levels: List[LSLevel], l: int, b: List[np.ndarray], x: List[np.ndarray]) -> None:
    """The V-cycle with local smoothing (Sec. 2.2; Algorithm 2 with
    refinement edges) on level l, in residual-correction form.  Smoothing acts
    on A_SS of the level's own cells (b[l] has zero entries on the edge E).  The
    defect of the smoothed iterate, (b_S - A_SS x_S, -A_ES x_S), is restricted
    and added to the coarser level's right-hand side (which already holds that
    level's share of b).  The coarse solution interpolated back supplies x_E,
    and the second smoothing sees b_S - A_SE x_E.  Level 0 is solved exactly."""
    lev = levels[l]
    dt = b[l].dtype
    if l == 0:
        if lev.space.n_free:
            x[0] = sla.cho_solve(lev.chol, b[0].astype(np.float64)).astype(dt)
        return
    dinv = lev.dinv.astype(dt)
    P = lev.P.astype(dt) if dt == np.float32 else lev.P
    xs = chebyshev(lev.apply, dinv, b[l], None, lev.lam_max)
    b[l - 1] = b[l - 1] + P.T @ (b[l] - lev.apply(xs))
    vcycle(levels, l - 1, b, x)
    x[l] = chebyshev(lev.apply, dinv, b[l], xs + P @ x[l - 1], lev.lam_max)


def multigrid_vcycle(levels: List[LSLevel], cmap: CopyMap, b: np.ndarray, dtype=np.float64) -> np.ndarray:
    """Algorithm 1: copy to the levels, V-cycle from the finest level, copy back."""
    bl = [np.zeros(lev.space.n_free, dtype=dtype) for lev in levels]
    xl = [np.zeros(lev.space.n_free, dtype=dtype) for lev in levels]
    for l in range(len(levels)):
        sel = cmap.level == l
        bl[l][cmap.index[sel]] = b[sel].astype(dtype)
    vcycle(levels, len(levels) - 1, bl, xl)
    out = np.empty(len(b))
    for l in range(len(levels)):
        sel = cmap.level == l
        out[sel] = xl[l][cmap.index[sel]]
    return out


def solve(active: Space, levels: List[LSLevel], cmap: CopyMap, b: np.ndarray, rtol: float,
          mg_dtype=np.float64, maxit: int = 200) -> SolveResult:
    """CG on the active mesh (fp64) preconditioned by one local-smoothing V-cycle."""
    set_precision(levels, mg_dtype)
    return pcg(active.apply, b, lambda r: multigrid_vcycle(levels, cmap, r, mg_dtype), rtol, maxit)
