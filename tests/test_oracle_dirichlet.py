"""Pins of the inhomogeneous-Dirichlet oracle (oracle/dirichlet.py).

* closed forms: -Lap u of the Gaussian and of polynomials against fourth-order
  finite differences; the Gaussian's peak value;
* Galerkin exactness: for u in Q_k the discrete solution is u's interpolant,
  at the free DoFs and (through the lifting) at every support point, hanging
  points with boundary masters included, on the octant mesh;
* g = 0 gives the homogeneous right-hand side; the lifting is g on the
  boundary and zero at free points;
* Table A.1: the GC solve of the Gaussian case needs the printed number of
  iterations (the paper's coarse solver is AMG, ours exact: one fewer is
  accepted).
"""
import numpy as np
import pytest
import scipy.sparse.linalg as sla

import synth
from golden_data import table
from oracle import dirichlet as od
from oracle import mesh as omesh
from oracle import mg
from oracle.space import Space

X0 = (-0.5, -0.5, -0.5)
ALPHA = 0.1


def _fd_laplacian(u, x, h):
    out = np.zeros(len(x))
    for d in range(3):
        e = np.zeros(3)
        e[d] = h
        out += (-u(x + 2 * e) + 16 * u(x + e) - 30 * u(x) + 16 * u(x - e) - u(x - 2 * e)) / (12 * h * h)
    return out


def _poly_terms(k):
    return [(1.0, k, 0, 0), (0.5, 1, k, 1), (-0.25, 0, 1, k), (2.0, k, k, k), (0.3, 0, 0, 0)]


def test_gaussian_laplacian_closed_form():
    u, f = od.gaussian(ALPHA, X0)
    rng = np.random.default_rng(1)
    x = np.asarray(X0) + 0.25 * rng.standard_normal((50, 3))
    fd = -_fd_laplacian(u, x, 1e-3)
    assert np.allclose(f(x), fd, rtol=1e-5, atol=1e-6 * np.abs(fd).max())
    assert np.isclose(u(np.array([X0]))[0], (ALPHA * np.sqrt(2 * np.pi)) ** -3, rtol=1e-15)


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_polynomial_laplacian_closed_form(k):
    u, f = od.polynomial(_poly_terms(k))
    x = np.random.default_rng(k).uniform(-1, 1, (40, 3))
    assert np.allclose(f(x), -_fd_laplacian(u, x, 1e-3), rtol=1e-6, atol=1e-6)


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_polynomial_solution_is_exact(k):
    u, f = od.polynomial(_poly_terms(k))
    s = Space(omesh.build_mesh(synth.octant(2)), k)
    lift = od.lifting(s, u)
    hp = s.hanging & ~s.on_boundary
    # the mesh has hanging points whose masters carry Dirichlet values
    assert np.count_nonzero(lift[hp]) > 0
    x = sla.spsolve(s.assemble().tocsc(), od.rhs(s, f, u))
    scale = np.abs(u(s.points)).max()
    assert np.abs(x - s.interpolate(u)).max() <= 1e-12 * scale
    assert np.abs(od.solution_all(s, x, u) - u(s.points)).max() <= 1e-12 * scale


def test_lifting_and_homogeneous_case():
    u, f = od.gaussian(ALPHA, X0)
    s = Space(omesh.build_mesh(synth.octant(2)), 2)
    lift = od.lifting(s, u)
    assert np.array_equal(lift[s.on_boundary], u(s.points[s.on_boundary]))
    assert not np.any(lift[s.free_points])
    zero = lambda x: np.zeros(len(x))
    assert np.array_equal(od.rhs(s, f, zero), s.rhs(f))


@pytest.mark.parametrize("k,L", [(1, 3), (1, 4), (1, 5), (4, 3)])
def test_gaussian_iterations_table_a1(k, L):
    ref = [r for r in table("gaussian_gc") if int(r[0]) == L][0][2 if k == 1 else 4]
    u, f = od.gaussian(ALPHA, X0)
    levels = mg.build_levels(omesh.build_mesh(synth.octant(L)), k)
    s = levels[-1].space
    b = od.rhs(s, f, u)
    res = mg.solve(levels, b, 1e-4, np.float32)
    assert res.iterations <= 50 and np.linalg.norm(b - s.apply(res.x)) <= 1e-4 * np.linalg.norm(b)
    assert ref - 1 <= res.iterations <= ref
