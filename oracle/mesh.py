"""Octree hexahedral meshes, 2:1 closure and the global-coarsening hierarchy.

Test infrastructure (see ``oracle/__init__``).

Follows:
* Sec. 4 "Examples": meshes obtained from one coarse cell by repeated
  refinement, each step completed by a closure "ensuring one-irregularity in
  the sense that two leaf cells may only differ by one level if they share a
  vertex".
* Sec. 2.2: global coarsening coarsens all cells simultaneously; the levels
  cover the whole domain and may contain hanging nodes.

A cell is the tuple (l, i, j, k): the box lo + h_l * [i, i+1] x [j, j+1] x
[k, k+1] with h_l = (hi - lo) / 2^l.

Pins (tests/test_oracle_mesh.py): the cell counts of Fig. 4 and the
per-level counts of the single-process workload figure of Sec. 4
(local smoothing 1, 8, 64, 216, ... and global coarsening 1, 8, 15, 120,
701, 4712, 34903, 269998, 2127189).
"""
from __future__ import annotations

import itertools
import math
from typing import Dict, List, Optional, Set, Tuple

import synth

Cell = Tuple[int, int, int, int]

NEIGHBOUR_DIRS = [d for d in itertools.product((-1, 0, 1), repeat=3) if d != (0, 0, 0)]


def children(c: Cell) -> List[Cell]:
    l, i, j, k = c
    return [(l + 1, 2 * i + a, 2 * j + b, 2 * k + cc)
            for cc in (0, 1) for b in (0, 1) for a in (0, 1)]


def parent(c: Cell) -> Cell:
    l, i, j, k = c
    return (l - 1, i >> 1, j >> 1, k >> 1)


class Mesh:
    """Leaves and refined (internal) cells of one octree."""

    def __init__(self, lo: float, hi: float):
        self.lo = lo
        self.hi = hi
        self.leaves: Set[Cell] = {(0, 0, 0, 0)}
        self.internal: Set[Cell] = set()

    # ---- geometry -------------------------------------------------------
    def h(self, l: int) -> float:
        return (self.hi - self.lo) / (1 << l)

    def box(self, c: Cell):
        l, i, j, k = c
        h = self.h(l)
        lo = (self.lo + i * h, self.lo + j * h, self.lo + k * h)
        return lo, (lo[0] + h, lo[1] + h, lo[2] + h)

    def centre(self, c: Cell):
        (a, b, cc), (d, e, f) = self.box(c)
        return ((a + d) / 2, (b + e) / 2, (cc + f) / 2)

    @property
    def max_level(self) -> int:
        return max(c[0] for c in self.leaves)

    def copy(self) -> "Mesh":
        m = Mesh(self.lo, self.hi)
        m.leaves = set(self.leaves)
        m.internal = set(self.internal)
        return m

    # ---- queries --------------------------------------------------------
    def leaf_containing(self, c: Cell) -> Optional[Cell]:
        """The leaf that contains the block c, or None if c is refined."""
        if c in self.internal:
            return None
        l, i, j, k = c
        while l >= 0:
            if (l, i, j, k) in self.leaves:
                return (l, i, j, k)
            l, i, j, k = l - 1, i >> 1, j >> 1, k >> 1
        return None

    def sorted_leaves(self) -> List[Cell]:
        """Leaves in a fixed order (by level, then lexicographic)."""
        return sorted(self.leaves)

    # ---- refinement -----------------------------------------------------
    def _split(self, c: Cell) -> None:
        self.leaves.remove(c)
        self.internal.add(c)
        self.leaves.update(children(c))

    def refine(self, marked) -> None:
        """Refine the marked leaves, then refine further leaves until every
        two leaves that share a vertex differ by at most one level.

        Refining a leaf of level l creates cells of level l+1, so only leaves
        of level <= l-1 that touch it can become unbalanced; they are found
        through the 26 same-size neighbour blocks of the refined leaf."""
        work = list(marked)
        while work:
            c = work.pop()
            if c not in self.leaves:
                continue
            self._split(c)
            l, i, j, k = c
            n = 1 << l
            for di, dj, dk in NEIGHBOUR_DIRS:
                ii, jj, kk = i + di, j + dj, k + dk
                if not (0 <= ii < n and 0 <= jj < n and 0 <= kk < n):
                    continue
                leaf = self.leaf_containing((l, ii, jj, kk))
                if leaf is not None and leaf[0] < l:
                    work.append(leaf)

    def refine_step(self, step: synth.RefineStep) -> None:
        self.refine([c for c in self.sorted_leaves() if self._predicate(step, c)])

    def _predicate(self, s: synth.RefineStep, c: Cell) -> bool:
        if s.pred == synth.PRED_ALL:
            return True
        lo, hi = self.box(c)
        if s.pred == synth.PRED_OCTANT_CENTRE:
            x = self.centre(c)
            return all(s.a <= t <= s.b for t in x)
        if s.pred == synth.PRED_OCTANT_STRICT:
            return all(t < s.b for t in hi) and all(t >= s.a for t in lo)
        if s.pred == synth.PRED_SHELL:
            r = math.sqrt(sum(t * t for t in self.centre(c)))
            return s.a <= r <= s.b
        if s.pred == synth.PRED_SPHERE:
            cen, rad = s.a, s.b
            dmin2 = sum(max(lo[d] - cen, 0.0, cen - hi[d]) ** 2 for d in range(3))
            dmax2 = sum(max(abs(lo[d] - cen), abs(hi[d] - cen)) ** 2 for d in range(3))
            return dmin2 <= rad * rad <= dmax2
        raise ValueError(f"unknown predicate {s.pred}")

    # ---- statistics -----------------------------------------------------
    def cells_per_refinement_level(self) -> List[int]:
        """Number of octree cells (leaf or refined) on each refinement level;
        the level meshes of local smoothing (Sec. 2.1)."""
        L = self.max_level
        cnt = [0] * (L + 1)
        for c in itertools.chain(self.leaves, self.internal):
            cnt[c[0]] += 1
        return cnt


def build_mesh(recipe: synth.MeshRecipe) -> Mesh:
    m = Mesh(recipe.lo, recipe.hi)
    for s in recipe.steps:
        m.refine_step(s)
    return m


def coarsen_global(fine: Mesh) -> Mesh:
    """One step of global coarsening (Sec. 2.2): every refined cell whose
    children are all leaves is coarsened, except where the coarsened cell
    would touch a leaf two or more levels finer; the exception is applied
    repeatedly until no coarsened cell violates the 2:1 condition."""
    cand: Set[Cell] = set()
    for c in fine.internal:
        if all(ch in fine.leaves for ch in children(c)):
            cand.add(c)

    def internal_new(c: Cell) -> bool:
        return c in fine.internal and c not in cand

    changed = True
    while changed:
        changed = False
        for p in sorted(cand):
            l, i, j, k = p
            n = 1 << l
            bad = False
            for di, dj, dk in NEIGHBOUR_DIRS:
                ii, jj, kk = i + di, j + dj, k + dk
                if not (0 <= ii < n and 0 <= jj < n and 0 <= kk < n):
                    continue
                nb = (l, ii, jj, kk)
                if not internal_new(nb):
                    continue
                # children of nb that touch p
                xs = (0, 1) if di == 0 else ((0,) if di > 0 else (1,))
                ys = (0, 1) if dj == 0 else ((0,) if dj > 0 else (1,))
                zs = (0, 1) if dk == 0 else ((0,) if dk > 0 else (1,))
                for a in xs:
                    for b in ys:
                        for cc in zs:
                            if internal_new((l + 1, 2 * ii + a, 2 * jj + b, 2 * kk + cc)):
                                bad = True
                if bad:
                    break
            if bad:
                cand.discard(p)
                changed = True
    coarse = Mesh(fine.lo, fine.hi)
    coarse.internal = {c for c in fine.internal if c not in cand}
    coarse.leaves = {c for c in fine.leaves if parent(c) not in cand or c[0] == 0}
    coarse.leaves |= cand
    return coarse


def gc_hierarchy(fine: Mesh) -> List[Mesh]:
    """Global-coarsening levels, coarsest (one cell) first."""
    levels = [fine]
    while len(levels[-1].leaves) > 1:
        levels.append(coarsen_global(levels[-1]))
    return levels[::-1]


def ancestor_in(mesh: Mesh, c: Cell) -> Cell:
    """The leaf of ``mesh`` that contains the cell c of a finer nested mesh."""
    while c not in mesh.leaves:
        c = parent(c)
        if c[0] < 0:
            raise ValueError("meshes are not nested")
    return c
