"""Pins of the mapped-geometry oracle (oracle/mapped.py).

* eps = 0 is the Cartesian space: operator, diagonal and right-hand side
  agree with oracle/space.py;
* element matrices are symmetric, positive semi-definite, annihilate
  constants;
* the quadrature of det J over all cells is the volume of Phi(cube) in
  closed form;
* patch test: a function linear in the physical coordinates, with its own
  Dirichlet values and f = 0, is reproduced exactly on a mesh with hanging
  nodes (it lies in the space; the quadrature is exact for it);
* the mapped Jacobian against central differences of Phi; it is not
  symmetric, so the patch test also catches a transposed J^-1;
* multigrid on the mapped levels converges like the Cartesian one.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as sla

import synth
from oracle import fe
from oracle import mapped as om
from oracle import mesh as omesh
from oracle import mg
from oracle.space import Space

EPS = 0.3


def test_eps_zero_is_cartesian():
    m = omesh.build_mesh(synth.octant(2))
    a, b = om.MappedSpace(m, 3, 0.0), Space(m, 3)
    x = synth.point_values(b.free_coordinates(), 3)
    assert np.allclose(a.apply(x), b.apply(x), rtol=0, atol=1e-13 * np.abs(b.apply(x)).max())
    assert np.allclose(a.diagonal(), b.diagonal(), rtol=1e-13)
    assert np.allclose(a.rhs(), b.rhs(), rtol=1e-13, atol=1e-16)


def test_element_matrices():
    s = om.MappedSpace(omesh.build_mesh(synth.octant(2)), 2, EPS)
    A = s._Ae
    assert np.allclose(A, np.transpose(A, (0, 2, 1)), atol=1e-14 * np.abs(A).max())
    assert np.abs(A.sum(axis=2)).max() <= 1e-13 * np.abs(A).max()
    ev = np.linalg.eigvalsh(A)
    assert ev.min() >= -1e-13 * ev.max()


def test_jacobian_against_differences():
    x = np.random.default_rng(2).uniform(-1, 1, (20, 3))
    J = om.warp_jacobian(x, EPS)
    h = 1e-6
    for b in range(3):
        e = np.zeros(3)
        e[b] = h
        fd = (om.warp(x + e, EPS) - om.warp(x - e, EPS)) / (2 * h)
        assert np.allclose(J[:, :, b], fd, atol=1e-9)


def test_volume_closed_form():
    lo, hi = -1.0, 1.0
    s = om.MappedSpace(omesh.build_mesh(synth.octant(2)), 1, EPS)
    ref, w = s._quadrature()
    xq = s.origin[:, None, :] + s.h[:, None, None] * ref[None, :, :]
    vol = np.sum(w[None, :] * np.linalg.det(s.h[:, None, None, None] * om.warp_jacobian(xq, EPS)))
    # det J_Phi = 1 - eps^2 (x^2 + y^2 / 2 + 2 z^2) + 2 eps^3 x y z
    L = hi - lo
    m2 = (hi ** 3 - lo ** 3) / 3          # integral of x^2 over [lo, hi]
    m1 = (hi ** 2 - lo ** 2) / 2
    exact = L ** 3 - EPS ** 2 * 3.5 * m2 * L ** 2 + 2 * EPS ** 3 * m1 ** 3
    assert np.isclose(vol, exact, rtol=1e-14)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_patch_test(k):
    s = om.MappedSpace(omesh.build_mesh(synth.octant(2)), k, EPS)
    assert s.n_hanging > 0
    a = np.array([0.7, -0.4, 1.3])
    u = lambda y: y @ a + 0.25
    zero = lambda y: np.zeros(len(y))
    b = om.rhs_dirichlet(s, zero, u)
    x = sla.spsolve(s.assemble().tocsc(), b)
    ref = u(s.physical_points()[s.free_points])
    assert np.abs(x - ref).max() <= 1e-12 * np.abs(ref).max()


def test_multigrid_on_mapped_levels():
    levels = mg.build_levels(omesh.build_mesh(synth.octant(3)), 2, warp_eps=EPS)
    s = levels[-1].space
    b = s.rhs()
    r = mg.solve(levels, b, 1e-8, np.float32)
    assert np.linalg.norm(b - s.apply(r.x)) <= 1e-8 * np.linalg.norm(b)
    cart = mg.solve(mg.build_levels(omesh.build_mesh(synth.octant(3)), 2), Space(omesh.build_mesh(synth.octant(3)), 2).rhs(),
                    1e-8, np.float32)
    assert r.iterations <= cart.iterations + 2
