"""Pins of oracle/mesh.py against the cell counts the paper prints."""
import pytest

import synth
from oracle import mesh as omesh
from golden_data import table


def _two_digits(x):
    return float(f"{x:.1e}")


@pytest.mark.parametrize("L", [3, 4, 5, 6])
def test_octant_cell_counts_fig4(L):
    row = [r for r in table("fig4_octant") if int(r[0]) == L][0]
    m = omesh.build_mesh(synth.octant(L))
    assert _two_digits(len(m.leaves)) == row[1]


def test_gc_hierarchy_matches_workload_figure():
    # octant L=7: its global-coarsening levels are the first 8 levels of the
    # printed L=8 hierarchy
    gc = table("workload_gc")[0]
    m = omesh.build_mesh(synth.octant(7))
    levels = omesh.gc_hierarchy(m)
    assert [len(x.leaves) for x in levels] == [int(v) for v in gc[:8]]


def test_ls_levels_match_workload_figure():
    ls = table("workload_ls")[0]
    m = omesh.build_mesh(synth.octant(7))
    assert m.cells_per_refinement_level()[:7] == [int(v) for v in ls[:7]]


@pytest.mark.parametrize("L", [5, 6, 7])
def test_shell_cell_counts_fig4(L):
    row = [r for r in table("fig4_shell") if int(r[0]) == L][0]
    m = omesh.build_mesh(synth.shell(L))
    assert _two_digits(len(m.leaves)) == row[1]


def test_two_to_one_balance_and_nesting():
    m = omesh.build_mesh(synth.octant(5))
    # every pair of leaves sharing a vertex differs by at most one level
    for c in m.leaves:
        l, i, j, k = c
        n = 1 << l
        for d in omesh.NEIGHBOUR_DIRS:
            ii, jj, kk = i + d[0], j + d[1], k + d[2]
            if 0 <= ii < n and 0 <= jj < n and 0 <= kk < n:
                leaf = m.leaf_containing((l, ii, jj, kk))
                if leaf is not None:
                    assert abs(leaf[0] - l) <= 1
                else:  # refined neighbour: its touching children must be leaves
                    xs = (0, 1) if d[0] == 0 else ((0,) if d[0] > 0 else (1,))
                    ys = (0, 1) if d[1] == 0 else ((0,) if d[1] > 0 else (1,))
                    zs = (0, 1) if d[2] == 0 else ((0,) if d[2] > 0 else (1,))
                    for a in xs:
                        for b in ys:
                            for cc in zs:
                                ch = (l + 1, 2 * ii + a, 2 * jj + b, 2 * kk + cc)
                                assert ch not in m.internal
    # levels are nested and the coarsest is one cell
    levels = omesh.gc_hierarchy(m)
    assert len(levels[0].leaves) == 1
    for coarse, fine in zip(levels[:-1], levels[1:]):
        for c in fine.leaves:
            omesh.ancestor_in(coarse, c)


def test_benchmark_workload_cell_counts():
    assert len(omesh.build_mesh(synth.WORKLOAD_Q2_OCTANT.recipe).leaves) == 960
    m = omesh.build_mesh(synth.WORKLOAD_Q4_OCTANT.recipe)
    assert len(m.leaves) == 296535
    assert len(omesh.build_mesh(synth.WORKLOAD_Q4_SPHERE.recipe).leaves) == 82776
