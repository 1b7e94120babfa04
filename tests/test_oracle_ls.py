"""Pins of the local-smoothing oracle (oracle/ls.py).

* without local refinement local smoothing is global coarsening: the two
  V-cycles agree to rounding;
* the V-cycle with refinement-edge treatment is a symmetric positive
  definite preconditioner (brute force, column by column);
* the refinement edges against a second definition: level-l support points
  in the closed box of an active cell of a coarser level;
* Algorithm 1's copy: every active DoF goes to the coarsest level among its
  active cells, to a level DoF at the same point that is not an edge DoF;
* the level sizes are the cells per refinement level of the workload figure;
* the iteration counts of Table 4 (octant, f = 1) and Table A.1 (Gaussian,
  inhomogeneous Dirichlet data) printed for local smoothing, and equal
  counts for fp32 and fp64 V-cycles.
"""
import numpy as np
import pytest

import synth
from golden_data import table
from oracle import dirichlet as od
from oracle import ls
from oracle import mesh as omesh
from oracle import mg
from oracle.space import Space


def _setup(rec, k):
    fine = omesh.build_mesh(rec)
    levels = ls.build_ls_levels(fine, k)
    act = Space(fine, k)
    return fine, levels, act, ls.copy_map(act, levels)


def test_uniform_mesh_local_smoothing_is_global_coarsening():
    fine, levels, act, cm = _setup(synth.uniform_cube(3), 2)
    assert not any(np.any(lev.edge) for lev in levels)
    glev = mg.build_levels(fine, 2)
    b = synth.point_values(act.free_coordinates(), 4)
    x1 = ls.multigrid_vcycle(levels, cm, b)
    x2 = mg.multigrid_vcycle(glev, b)
    assert np.abs(x1 - x2).max() <= 1e-13 * np.abs(x2).max()


def test_vcycle_is_symmetric_positive_definite():
    fine, levels, act, cm = _setup(synth.octant(3), 1)
    assert np.any(levels[-1].edge)
    n = act.n_free
    B = np.stack([ls.multigrid_vcycle(levels, cm, np.eye(n)[:, j]) for j in range(n)], axis=1)
    assert np.abs(B - B.T).max() <= 1e-13 * np.abs(B).max()
    assert np.linalg.eigvalsh(0.5 * (B + B.T)).min() > 0


@pytest.mark.parametrize("k", [1, 3])
def test_edges_lie_on_coarser_active_cells(k):
    """Second definition of the refinement edges: level-l support points in
    the closed box of an active cell of a coarser level."""
    fine, levels, act, cm = _setup(synth.octant(4), k)
    for l, lev in enumerate(levels):
        sel = act.level < l
        lo, hi = act.origin[sel], act.origin[sel] + act.h[sel][:, None]
        pts = lev.space.free_coordinates()
        inside = np.zeros(len(pts), dtype=bool)
        for a, b in zip(lo, hi):
            inside |= np.all((pts >= a - 1e-12) & (pts <= b + 1e-12), axis=1)
        assert np.array_equal(lev.edge, inside), l


def test_copy_map_brute_force():
    fine, levels, act, cm = _setup(synth.octant(4), 2)
    for g, p in enumerate(act.free_points):
        cells = np.nonzero(np.any(act.cell_nodes == p, axis=1))[0]
        m = int(act.level[cells].min())
        assert cm.level[g] == m
        lev = levels[m]
        assert np.allclose(lev.space.free_coordinates()[cm.index[g]], act.points[p], atol=1e-14)
        assert not lev.edge[cm.index[g]]


def test_level_sizes_are_the_refinement_levels():
    ref = [int(v) for v in table("workload_ls")[0]]
    fine = omesh.build_mesh(synth.octant(5))
    # levels below the finest one of the L = 5 mesh have the counts of the L = 8 figure
    assert [len(ls.level_mesh(fine, l).leaves) for l in range(5)] == ref[:5]
    assert len(ls.level_mesh(fine, 5).leaves) == sum(1 for c in fine.leaves if c[0] == 5)


@pytest.mark.parametrize("k,L", [(1, 3), (1, 4), (1, 5), (4, 3)])
def test_iterations_table_4(k, L):
    row = [r for r in table("octant_t4") if int(r[0]) == L][0]
    ref = row[1] if k == 1 else row[3]
    fine, levels, act, cm = _setup(synth.octant(L), k)
    b = act.rhs()
    r32 = ls.solve(act, levels, cm, b, 1e-4, np.float32)
    r64 = ls.solve(act, levels, cm, b, 1e-4, np.float64)
    assert np.linalg.norm(b - act.apply(r32.x)) <= 1e-4 * np.linalg.norm(b)
    assert ref - 1 <= r32.iterations <= ref and r32.iterations == r64.iterations


@pytest.mark.parametrize("k,L", [(1, 3), (1, 4), (4, 3)])
def test_iterations_table_a1(k, L):
    ref = [r for r in table("gaussian_gc") if int(r[0]) == L][0][1 if k == 1 else 3]
    u, f = od.gaussian(0.1, (-0.5, -0.5, -0.5))
    fine, levels, act, cm = _setup(synth.octant(L), k)
    b = od.rhs(act, f, u)
    r = ls.solve(act, levels, cm, b, 1e-4, np.float32)
    assert ref - 1 <= r.iterations <= ref
