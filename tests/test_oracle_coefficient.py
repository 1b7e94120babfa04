"""Pins of the variable-coefficient oracle (oracle/coefficient.py and the
per-cell scale nu_e of oracle/space.py).

* a constant coefficient c scales operator and diagonal by c and leaves the
  Jacobi-preconditioned spectrum (lambda_max) and the solve unchanged;
* the weighted harmonic average is exact in closed form for a coefficient
  whose reciprocal is linear, and lies between the minimum and the
  arithmetic mean;
* the transfer to coarser levels against brute force by geometric
  containment of cell centres;
* an exact solution: for a coefficient jumping across a plane of cell faces,
  the piecewise-linear u with continuous flux lies in the FE space and the
  Galerkin solution (Dirichlet data = u) reproduces it;
* the multigrid-preconditioned CG converges on a coefficient with contrast
  1e3.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as sla

import synth
from oracle import coefficient as oc
from oracle import dirichlet as od
from oracle import mesh as omesh
from oracle import mg
from oracle.space import Space


def test_constant_coefficient_scales():
    s = Space(omesh.build_mesh(synth.octant(2)), 3)
    x = synth.point_values(s.free_coordinates(), 5)
    y1, d1 = s.apply(x), s.diagonal()
    s.nu = np.full(s.nc, 7.5)
    assert np.allclose(s.apply(x), 7.5 * y1, rtol=1e-14, atol=1e-14 * np.abs(y1).max())
    assert np.allclose(s.diagonal(), 7.5 * d1, rtol=1e-14)
    lev1 = mg.build_levels(omesh.build_mesh(synth.octant(3)), 2)
    lev2 = mg.build_levels(omesh.build_mesh(synth.octant(3)), 2, coefficient=lambda p: np.full(len(p), 7.5))
    for a, b in zip(lev1[1:], lev2[1:]):
        assert np.isclose(a.lam_max, b.lam_max, rtol=1e-10)
    b = lev1[-1].space.rhs()
    r1 = mg.solve(lev1, b, 1e-8)
    r2 = mg.solve(lev2, 7.5 * b, 1e-8)
    assert r1.iterations == r2.iterations
    assert np.allclose(r1.x, r2.x, rtol=1e-8, atol=1e-10 * np.abs(r1.x).max())


def test_harmonic_average_closed_form():
    s = Space(omesh.build_mesh(synth.octant(2)), 2)
    nu = lambda p: 1.0 / (3.0 + 0.5 * p[:, 0] - 0.25 * p[:, 1] + 0.125 * p[:, 2])
    xq = oc.quadrature_points(s)
    nu_e = oc.harmonic_cell_average(2, nu(xq.reshape(-1, 3)).reshape(s.nc, -1))
    centre = s.origin + 0.5 * s.h[:, None]
    assert np.allclose(nu_e, nu(centre), rtol=1e-14)


def test_harmonic_average_bounds():
    v = 10.0 ** np.random.default_rng(3).uniform(-2, 2, (50, 27))
    h = oc.harmonic_cell_average(2, v)
    w = oc.quadrature_weights(2)
    assert np.all(h >= v.min(axis=1) * (1 - 1e-14))
    assert np.all(h <= (v * w).sum(axis=1) / w.sum() * (1 + 1e-14))
    assert np.isclose(w.sum(), 1.0, rtol=1e-14)


def test_coarsen_by_containment():
    meshes = omesh.gc_hierarchy(omesh.build_mesh(synth.octant(3)))
    spaces = [Space(m, 1) for m in meshes]
    oc.set_level_coefficients(spaces, synth.random_cells(11))
    for l in range(len(spaces) - 1):
        f, c = spaces[l + 1], spaces[l]
        fc = f.origin + 0.5 * f.h[:, None]
        for e in range(c.nc):
            inside = np.all((fc > c.origin[e]) & (fc < c.origin[e] + c.h[e]), axis=1)
            idx = np.nonzero(inside)[0]
            if len(idx) == 1:
                assert f.h[idx[0]] == c.h[e] and c.nu[e] == f.nu[idx[0]]
            else:
                assert len(idx) == 8 and np.all(f.h[idx] == c.h[e] / 2)
                assert np.isclose(c.nu[e], f.nu[idx].mean(), rtol=1e-15)


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_jump_coefficient_exact_solution(k):
    nu_lo, nu_hi = 10.0, 1.0
    s1 = 1.0
    s2 = nu_lo * s1 / nu_hi  # continuous normal flux across x = 0

    def u(p):
        p = np.asarray(p)
        return 1.0 + np.where(p[..., 0] < 0, s1, s2) * p[..., 0] + 0.5 * p[..., 1] + 0.25 * p[..., 2]

    zero = lambda p: np.zeros(np.asarray(p).shape[:-1])
    levels = mg.build_levels(omesh.build_mesh(synth.octant(2)), k, assembled=False,
                             coefficient=synth.step(0.0, nu_lo, nu_hi))
    s = levels[-1].space
    centre_x = s.origin[:, 0] + 0.5 * s.h
    assert np.allclose(s.nu, np.where(centre_x < 0, nu_lo, nu_hi), rtol=1e-14)
    b = od.rhs(s, zero, u)
    x = sla.spsolve(s.assemble().tocsc(), b)
    assert np.abs(x - s.interpolate(u)).max() <= 1e-12 * np.abs(u(s.points)).max()
    # a coefficient that is one everywhere does not reproduce it
    s.nu = np.ones(s.nc)
    x1 = sla.spsolve(s.assemble().tocsc(), od.rhs(s, zero, u))
    assert np.abs(x1 - s.interpolate(u)).max() > 1e-3


def test_multigrid_converges_with_contrast():
    nu = synth.inclusions(7, -1.0, 1.0, contrast=1e3)
    levels = mg.build_levels(omesh.build_mesh(synth.octant(3)), 2, coefficient=nu)
    s = levels[-1].space
    assert s.nu.max() / s.nu.min() > 100
    b = s.rhs()
    r = mg.solve(levels, b, 1e-8, np.float32)
    assert np.linalg.norm(b - s.apply(r.x)) <= 1e-8 * np.linalg.norm(b)
    assert r.iterations <= 25, r.iterations
