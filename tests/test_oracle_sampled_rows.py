"""The one-by-one row evaluator of the full-size GPU tests (tests/sampled.py)
against the oracle's global operator C^T A C on meshes it takes whole: on the
rows it selects the two agree to rounding, and the selection finds cells in
every level that has a one-level neighbourhood."""
import numpy as np
import pytest

import synth
from oracle import mesh as omesh
from oracle.space import Space
from parity import rel_err
from sampled import deep_cells, sampled_rows


@pytest.mark.parametrize("rec,k", [(synth.cube_octant(3, 2), 4), (synth.cube_octant(3, 1), 2),
                                   (synth.cube_octant(3, 2), 3)], ids=["cube3+2-Q4", "cube3+1-Q2", "cube3+2-Q3"])
def test_sampled_rows_equal_the_global_operator(rec, k):
    m = omesh.build_mesh(rec)
    s = Space(m, k)
    rng = np.random.default_rng(12)
    cells = deep_cells(m, rng, 6)
    assert {c[0] for c in cells} == {min(c[0] for c in m.leaves), m.max_level}
    pos, ref = sampled_rows(m, k, cells, rng, 9)
    xyz = s.free_coordinates()
    y = s.apply(synth.point_values(xyz, 9))
    near = [int(np.argmin(np.abs(xyz - p).sum(1))) for p in pos]
    assert np.abs(xyz[near] - pos).max() < 1e-12
    assert rel_err(ref, y[near]) < 1e-13


class _Node:
    """stands in for the generator: always the same local node"""

    def __init__(self, abc):
        self.abc = np.array(abc)

    def integers(self, lo, hi, n):
        return self.abc


def test_rows_touched_by_hanging_nodes_are_refused():
    """A point on the face of a coarse cell whose neighbour across the face
    is refined is a master of hanging nodes: its row holds terms of the fine
    cells, and the evaluator refuses it instead of returning the plain sum
    (this coarse cell is not one deep_cells would select)."""
    m = omesh.build_mesh(synth.cube_octant(2, 1))  # level-2 cells, the octant [0, 1/2]^3 at level 3
    c = (2, 2, 0, 0)  # x in [1/2, 3/4]: its face x = 1/2 touches the refined octant
    assert c in m.leaves and (2, 1, 0, 0) in m.internal
    with pytest.raises(AssertionError):
        sampled_rows(m, 2, [c], _Node((0, 1, 1)), 3)
    assert c not in deep_cells(m, np.random.default_rng(0), 100)
    # the interior node of the same cell is fine
    s = Space(m, 2)
    xyz = s.free_coordinates()
    y = s.apply(synth.point_values(xyz, 3))
    pos, ref = sampled_rows(m, 2, [c], _Node((1, 1, 1)), 3)
    i = int(np.argmin(np.abs(xyz - pos[0]).sum(1)))
    assert abs(ref[0] - y[i]) < 1e-13 * max(1.0, abs(y[i]))
