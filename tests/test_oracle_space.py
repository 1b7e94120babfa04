"""Pins of oracle/space.py: DoF counts of Fig. 4, hanging-node constraint
values, patch test, symmetry/definiteness, convergence order."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import synth
from oracle import fe, mesh as omesh, space as ospace
from golden_data import table


def _two_digits(x):
    return float(f"{x:.1e}")


@pytest.mark.parametrize("L", [3, 4, 5])
def test_dof_counts_and_hanging_share_fig4(L):
    row = [r for r in table("fig4_octant") if int(r[0]) == L][0]
    m = omesh.build_mesh(synth.octant(L))
    s1 = ospace.Space(m, 1)
    assert _two_digits(s1.n_points) == row[3]
    assert round(100 * s1.cell_has_hanging.mean()) == round(row[2])
    # for p = 1 the count is the number of distinct support points
    assert ospace.paper_dof_count(m, 1) == s1.n_points
    assert _two_digits(ospace.paper_dof_count(m, 4)) == row[4]


@pytest.mark.parametrize("L", [5, 6])
def test_shell_counts_fig4(L):
    row = [r for r in table("fig4_shell") if int(r[0]) == L][0]
    m = omesh.build_mesh(synth.shell(L))
    s1 = ospace.Space(m, 1)
    assert _two_digits(s1.n_points) == row[3]
    assert round(100 * s1.cell_has_hanging.mean()) == round(row[2])
    assert _two_digits(ospace.paper_dof_count(m, 4)) == row[4]


def test_support_points_vs_entity_count():
    # distinct GLL support points: coinciding midpoint nodes counted once
    m = omesh.build_mesh(synth.octant(3))
    s4 = ospace.Space(m, 4)
    assert s4.n_points == 9253 and ospace.paper_dof_count(m, 4) == 9295


def _two_cell_mesh():
    # the cube [0,1]^3 refined twice and the cells of the octant [0,1/2]^3
    # once more: hanging interfaces at x, y or z = 1/2
    return omesh.build_mesh(synth.cube_octant(2, 1))


def test_q1_constraint_weights():
    s = ospace.Space(_two_cell_mesh(), 1)
    C = s.C.tocsr()
    # hanging points whose constraining points are all free: coarse-edge
    # midpoints get weights 1/2, 1/2 and coarse-face centres 1/4 (x4)
    seen = set()
    for p in np.nonzero(s.hanging & ~s.on_boundary)[0]:
        row = C[p]
        if abs(row.data.sum() - 1.0) > 1e-14:  # a Dirichlet point was dropped
            continue
        seen.add(tuple(np.round(np.sort(row.data), 14)))
    assert seen == {(0.5, 0.5), (0.25, 0.25, 0.25, 0.25)}


def test_q2_constraint_weights_textbook():
    # Q2 on a coarse edge [a, a+H]: the value at a + H/4 is
    # 3/8 u(a) + 3/4 u(a + H/2) - 1/8 u(a + H)
    s = ospace.Space(_two_cell_mesh(), 2)
    C = s.C.tocsr()
    target = np.array([0.5, 0.25, 0.3125])
    p = int(np.nonzero(np.all(s.points == target, axis=1))[0][0])
    assert s.hanging[p]
    row = C[p]
    w = {tuple(s.free_coordinates()[c]): v for c, v in zip(row.indices, row.data)}
    assert set(w) == {(0.5, 0.25, 0.25), (0.5, 0.25, 0.375), (0.5, 0.25, 0.5)}
    assert np.isclose(w[(0.5, 0.25, 0.25)], 3 / 8, atol=1e-14)
    assert np.isclose(w[(0.5, 0.25, 0.375)], 3 / 4, atol=1e-14)
    assert np.isclose(w[(0.5, 0.25, 0.5)], -1 / 8, atol=1e-14)


def _patch(x):
    X, Y, Z = x[:, 0], x[:, 1], x[:, 2]
    return X * (1 - X) * Y * (1 - Y) * Z * (1 - Z)


def _patch_f(x):
    X, Y, Z = x[:, 0], x[:, 1], x[:, 2]
    return 2 * (Y * (1 - Y) * Z * (1 - Z) + X * (1 - X) * Z * (1 - Z) + X * (1 - X) * Y * (1 - Y))


@pytest.mark.parametrize("k", [2, 3, 4])
def test_patch_test_with_hanging_nodes(k):
    s = ospace.Space(omesh.build_mesh(synth.cube_octant(2, 1)), k)
    assert s.n_hanging > 0
    A = s.assemble()
    x = spla.spsolve(A.tocsc(), s.rhs(_patch_f))
    assert np.abs(x - s.interpolate(_patch)).max() < 1e-12


@pytest.mark.parametrize("k", [1, 2, 4])
def test_symmetric_positive_definite_and_paths_agree(k):
    s = ospace.Space(omesh.build_mesh(synth.octant(3)), k)
    A = s.assemble()
    assert abs(A - A.T).max() < 1e-13
    d = np.linalg.eigvalsh(A.toarray()) if s.n_free < 3000 else spla.eigsh(A, 1, which="SA")[0]
    assert d.min() > 0
    x = synth.uniform_vector(s.n_free, 7)
    assert np.abs(A @ x - s.apply(x)).max() < 1e-12 * np.abs(A @ x).max()
    assert np.abs(A.diagonal() - s.diagonal()).max() < 1e-12 * A.diagonal().max()


def _l2_error(s, x, u, nq=6):
    gq, gw = fe.gauss(nq)
    P = np.stack(np.meshgrid(gq, gq, gq, indexing="ij"), -1).reshape(-1, 3)
    W = np.prod(np.stack(np.meshgrid(gw, gw, gw, indexing="ij"), -1).reshape(-1, 3), axis=1)
    err = 0.0
    for e in range(s.nc):
        pts = s.origin[e] + s.h[e] * P
        # interior quadrature points lie in the cell: evaluate there
        v = s.evaluate(x, pts)
        err += np.sum(W * (v - u(pts)) ** 2) * s.h[e] ** 3
    return np.sqrt(err)


def _solve(s, b):
    """A x = b: sparse direct for small degrees; for Q3/Q4 (56 k unknowns)
    Jacobi-preconditioned CG on the oracle's cell-by-cell operator to a
    relative residual of 1e-13, far below the discretisation error."""
    if s.k <= 2:
        return spla.spsolve(s.assemble().tocsc(), b)
    d = s.diagonal()
    A = spla.LinearOperator((s.n_free, s.n_free), matvec=s.apply)
    M = spla.LinearOperator((s.n_free, s.n_free), matvec=lambda r: r / d)
    x, info = spla.cg(A, b, rtol=1e-13, atol=0.0, M=M, maxiter=5000)
    assert info == 0
    return x


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_convergence_order_k_plus_1(k):
    # L2 error O(h^{k+1}) for the smooth solution on octant meshes with hanging
    # nodes: a constraint or quadrature slip that keeps polynomial exactness
    # still lowers the order (measured rates: 4.0 for Q3, 5.0 for Q4)
    u = lambda x: np.sin(np.pi * x[:, 0]) * np.sin(np.pi * x[:, 1]) * np.sin(np.pi * x[:, 2])
    f = lambda x: 3 * np.pi ** 2 * u(x)
    errs = []
    for g in (1, 2, 3):
        s = ospace.Space(omesh.build_mesh(synth.cube_octant(g, 1)), k)
        x = _solve(s, s.rhs(f))
        errs.append(_l2_error(s, x, u))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert rates[-1] > k + 1 - 0.3, rates
