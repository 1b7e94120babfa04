"""Pins of oracle/mg.py: closed forms for the smoother and the eigenvalue
estimate, and the iteration counts the paper prints."""
import numpy as np
import pytest
import scipy.sparse as sp

import synth
from oracle import mesh as omesh, mg
from golden_data import table


def test_chebyshev_matches_polynomial_closed_form():
    # diagonal test matrix: error after the smoother equals the scaled
    # Chebyshev polynomial T_3((theta - lam)/delta) / T_3(theta/delta)
    lam = np.linspace(0.05, 2.0, 40)
    A = sp.diags(lam)
    xstar = synth.uniform_vector(40, 5)
    b = A @ xstar
    lmax = 2.0
    x = mg.chebyshev(lambda v: A @ v, np.ones(40), b, None, lmax, degree=3, smoothing_range=20.0)
    lmin = lmax / 20
    theta, delta = (lmax + lmin) / 2, (lmax - lmin) / 2
    T3 = lambda t: 4 * t ** 3 - 3 * t
    factor = T3((theta - lam) / delta) / T3(theta / delta)
    assert np.abs((x - xstar) - factor * (0 - xstar)).max() < 1e-13
    # from a non-zero start the same polynomial acts on the initial error
    x0 = synth.uniform_vector(40, 6)
    x = mg.chebyshev(lambda v: A @ v, np.ones(40), b, x0, lmax, degree=3, smoothing_range=20.0)
    assert np.abs((x - xstar) - factor * (x0 - xstar)).max() < 1e-13


def test_chebyshev_operator_counts():
    calls = []
    A = sp.identity(5)

    def apply(v):
        calls.append(1)
        return A @ v

    mg.chebyshev(apply, np.ones(5), np.ones(5), None, 1.2)
    assert len(calls) == 2  # from zero: 2 evaluations (Sec. 5.2 profile)
    calls.clear()
    mg.chebyshev(apply, np.ones(5), np.ones(5), np.ones(5), 1.2)
    assert len(calls) == 3


def test_lanczos_exact_for_small_diagonal():
    lam = np.array([0.5, 1.0, 3.0, 7.5])
    A = sp.diags(lam)
    est = mg.lanczos_lambda_max(lambda v: A @ v, np.ones(4), n_steps=12)
    assert abs(est - 7.5) < 1e-10


def test_pcg_solves_spd_system():
    rng = np.random.default_rng(0)
    B = rng.standard_normal((30, 30))
    A = B @ B.T + 30 * np.eye(30)
    b = rng.standard_normal(30)
    r = mg.pcg(lambda v: A @ v, b, lambda v: v, 1e-12)
    assert np.abs(r.x - np.linalg.solve(A, b)).max() < 1e-9


@pytest.mark.parametrize("L,k", [(3, 1), (4, 1), (5, 1), (3, 4), (4, 4)])
def test_iteration_counts_table_a4(L, k):
    row = [r for r in table("tol_gc") if int(r[0]) == L][0]
    it4, it8 = (row[1], row[3]) if k == 1 else (row[2], row[4])
    levels = mg.build_levels(omesh.build_mesh(synth.octant(L)), k, assembled=(k == 1 or L == 3))
    b = levels[-1].space.rhs()
    # the paper's coarse solver is inexact AMG; an exact coarse solve may save
    # at most one iteration
    assert it8 - 1 <= mg.solve(levels, b, 1e-8).iterations <= it8
    assert it4 - 1 <= mg.solve(levels, b, 1e-4).iterations <= it4


@pytest.mark.parametrize("L,k", [(3, 1), (4, 1), (3, 4)])
def test_float_vcycle_same_iterations_table_a3(L, k):
    row = [r for r in table("mgnumber_gc") if int(r[0]) == L][0]
    levels = mg.build_levels(omesh.build_mesh(synth.octant(L)), k)
    b = levels[-1].space.rhs()
    n64 = mg.solve(levels, b, 1e-4, np.float64).iterations
    n32 = mg.solve(levels, b, 1e-4, np.float32).iterations
    assert n64 == n32
    assert (row[1] if k == 1 else row[2]) - 1 <= n64 <= (row[1] if k == 1 else row[2])


@pytest.mark.parametrize("L,k", [(3, 1), (4, 1), (3, 4)])
def test_uniform_cube_table_a7(L, k):
    row = [r for r in table("hypercube_gc") if int(r[0]) == L][0]
    levels = mg.build_levels(omesh.build_mesh(synth.uniform_cube(L, -1.0, 1.0)), k)
    b = levels[-1].space.rhs()
    it = mg.solve(levels, b, 1e-4).iterations
    assert row[1 if k == 1 else 2] - 1 <= it <= row[1 if k == 1 else 2]
