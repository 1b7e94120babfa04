"""Pins of oracle/transfer.py."""
import numpy as np
import pytest

import synth
from oracle import mesh as omesh, space as ospace, transfer


def _pair(recipe, kf, kc=None, p=False):
    fine_mesh = omesh.build_mesh(recipe)
    if p:
        return ospace.Space(fine_mesh, kf), ospace.Space(fine_mesh, kc)
    coarse_mesh = omesh.gc_hierarchy(fine_mesh)[-2]
    return ospace.Space(fine_mesh, kf), ospace.Space(coarse_mesh, kf)


def test_q1_uniform_refinement_textbook_weights():
    fine, coarse = _pair(synth.uniform_cube(3), 1)
    P = transfer.prolongation_matrix(fine, coarse)
    # rows: coinciding points 1; edge midpoints 1/2 x2; face centres 1/4 x4;
    # cell centres 1/8 x8 (entries of Dirichlet coarse points dropped)
    full = [tuple(np.round(np.sort(P[i].data), 14)) for i in range(fine.n_free)
            if abs(P[i].data.sum() - 1) < 1e-14]
    assert set(full) == {(1.0,), (0.5, 0.5), (0.25,) * 4, (0.125,) * 8}


@pytest.mark.parametrize("k", [1, 2, 4])
def test_prolongation_is_evaluation_of_coarse_function(k):
    # independent path: point location + evaluation in Space.evaluate
    fine, coarse = _pair(synth.octant(3), k)
    P = transfer.prolongation_matrix(fine, coarse)
    xc = synth.uniform_vector(coarse.n_free, 11)
    assert np.abs(P @ xc - coarse.evaluate(xc, fine.free_coordinates())).max() < 1e-12


@pytest.mark.parametrize("kf,kc", [(2, 1), (4, 2)])
def test_p_transfer_is_evaluation(kf, kc):
    fine, coarse = _pair(synth.octant(3), kf, kc, p=True)
    P = transfer.prolongation_matrix(fine, coarse)
    xc = synth.uniform_vector(coarse.n_free, 12)
    assert np.abs(P @ xc - coarse.evaluate(xc, fine.free_coordinates())).max() < 1e-12


@pytest.mark.parametrize("k", [2, 3])
def test_prolongation_reproduces_polynomials(k):
    u = lambda x: x[:, 0] * (1 - x[:, 0]) * x[:, 1] * (1 - x[:, 1]) * x[:, 2] * (1 - x[:, 2])
    fine, coarse = _pair(synth.cube_octant(2, 1), k)
    P = transfer.prolongation_matrix(fine, coarse)
    assert np.abs(P @ coarse.interpolate(u) - fine.interpolate(u)).max() < 1e-13


def test_restriction_is_transpose_duality():
    fine, coarse = _pair(synth.octant(3), 2)
    P = transfer.prolongation_matrix(fine, coarse)
    x = synth.uniform_vector(fine.n_free, 3)
    y = synth.uniform_vector(coarse.n_free, 4)
    # x^T (P y) with P y evaluated independently
    lhs = x @ coarse.evaluate(y, fine.free_coordinates())
    assert abs(lhs - (P.T @ x) @ y) < 1e-11 * abs(lhs)
