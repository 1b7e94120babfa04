"""The C-ABI library loads, exports every declared symbol, and its host-side
set-up (octree, global coarsening, DoF numbering) agrees with the oracle.
No GPU is used."""
import os
import re

import numpy as np
import pytest

import synth
from oracle import mesh as omesh, space as ospace
from golden_data import table
from parity import match

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "gcmg.h")


def declared_symbols():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:int|int64_t|void|const char\*)\s+(gcmg_\w+)\s*\(", src, re.M)))


def test_library_exports_every_declared_symbol(gcmg):
    lib = gcmg.lib()
    names = declared_symbols()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(gcmg.exported_symbols())


def test_gc_hierarchy_through_abi_matches_paper(gcmg):
    gc = [int(v) for v in table("workload_gc")[0]]
    m = gcmg.Mesh.from_recipe(synth.octant(7))
    assert [m.level_cells(l) for l in range(m.num_levels)] == gc[:8]


@pytest.mark.parametrize("rec", [synth.shell(5), synth.sphere(5), synth.cube_octant(3, 1), synth.cube_octant(5, 2)],
                         ids=lambda r: r.name)
def test_hierarchy_matches_oracle(gcmg, rec):
    m = gcmg.Mesh.from_recipe(rec)
    levels = omesh.gc_hierarchy(omesh.build_mesh(rec))
    assert [m.level_cells(l) for l in range(m.num_levels)] == [len(x.leaves) for x in levels]


@pytest.mark.parametrize("rec,k,level", [
    (synth.octant(3), 1, -1), (synth.octant(3), 4, -1), (synth.octant(4), 2, -1), (synth.octant(4), 3, -2),
    (synth.cube_octant(3, 1), 2, -1), (synth.sphere(4), 3, -1), (synth.cube_octant(2, 1), 4, -1),
    (synth.shell(5), 2, -1), (synth.cube_octant(2, 2), 1, -1)], ids=str)
def test_dof_support_points_match_oracle(gcmg, rec, k, level):
    m = gcmg.Mesh.from_recipe(rec)
    lv = m.num_levels + level if level < 0 else level
    xyz = m.dof_coords(lv, k)
    om = omesh.gc_hierarchy(omesh.build_mesh(rec))[lv]
    s = ospace.Space(om, k)
    match(xyz, s.free_coordinates())


def test_dof_numbering_independent_of_tile_size(gcmg):
    m = gcmg.Mesh.from_recipe(synth.octant(4))
    a = m.dof_coords(m.num_levels - 1, 2, 8)
    b = m.dof_coords(m.num_levels - 1, 2, 64)
    match(a, b)


def test_q4_octant_workload_size(gcmg):
    m = gcmg.Mesh.from_recipe(synth.WORKLOAD_Q4_OCTANT.recipe)
    assert m.num_levels == 8
    assert m.level_cells(7) == 296535
    xyz = m.dof_coords(7, 4)
    assert len(xyz) == 18740987
    assert np.all((xyz > 0) & (xyz < 1))


def test_bad_arguments_are_reported(gcmg):
    with pytest.raises(gcmg.GcmgError):
        gcmg.Mesh(1.0, 0.0, [])
    with pytest.raises(gcmg.GcmgError):
        gcmg.Mesh(0.0, 1.0, [(99, 0, 0)])
    m = gcmg.Mesh.from_recipe(synth.octant(2))
    with pytest.raises(gcmg.GcmgError):
        m.dof_coords(0, 7)
    with pytest.raises(gcmg.GcmgError):
        m.level_cells(99)


def test_point_values_are_numbering_independent():
    xyz = np.random.default_rng(0).random((1000, 3))
    v = synth.point_values(xyz, 5)
    p = np.random.default_rng(1).permutation(1000)
    assert np.array_equal(synth.point_values(xyz[p], 5), v[p])
    assert -1 <= v.min() and v.max() < 1 and abs(v.mean()) < 0.1


@pytest.mark.parametrize("rec,k,tc", [
    (synth.octant(3), 1, 0), (synth.octant(4), 2, 0), (synth.octant(4), 4, 0), (synth.octant(5), 3, 0),
    (synth.cube_octant(3, 1), 2, 0), (synth.sphere(5), 4, 0), (synth.shell(5), 2, 0), (synth.octant(4), 4, 3),
    (synth.octant(4), 1, 255), (synth.cube_octant(2, 2), 4, 17)], ids=str)
def test_tile_invariants_all_levels(gcmg, rec, k, tc):
    m = gcmg.Mesh.from_recipe(rec)
    for l in range(m.num_levels):
        m.check_level(l, k, tc)


@pytest.mark.slow
def test_tile_invariants_q4_octant_workload(gcmg):
    m = gcmg.Mesh.from_recipe(synth.WORKLOAD_Q4_OCTANT.recipe)
    m.check_level(m.num_levels - 1, 4)
