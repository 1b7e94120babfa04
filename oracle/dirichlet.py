"""Inhomogeneous Dirichlet values and manufactured solutions.

Test infrastructure (see ``oracle/__init__``).

Follows Sec. 3.1: constraints are x_i = sum_j c_ij x_j + b_i; with Dirichlet
values g the inhomogeneity b_i is g at boundary support points and, at a
hanging support point, the part of its constraint row that acts on
constraining values at boundary points.  Condensation moves the known values
to the right-hand side:

    b = C^T (F - A_all u_g),    u_all = C x + u_g,

with u_g the lifting (g at boundary points, the interpolated boundary values
at hanging points, zero at free points) and A_all the unconstrained matrix
sum_e P_e^T A_e P_e.

Manufactured solutions (appendix, Table A.1 set-up): a Gaussian bump
u(x) = (alpha sqrt(2 pi))^-3 exp(-|x - x0|^2 / alpha^2) — the paper prints
the norm without the square, read as the squared norm that a Gaussian has —
and polynomials sum_m c_m x^a y^b z^c; f = -Lap u in closed form.
"""
from __future__ import annotations

from typing import Callable, Sequence, Tuple

import numpy as np

from . import fe


# ---------------------------------------------------------------------------
# manufactured solutions
# ---------------------------------------------------------------------------
def gaussian(alpha: float, x0: Sequence[float]) -> Tuple[Callable, Callable]:
    """(u, f = -Lap u) of the Gaussian bump."""
    c = (alpha * np.sqrt(2.0 * np.pi)) ** -3
    a = alpha * alpha
    x0 = np.asarray(x0, dtype=np.float64)

    def u(x):
        s = np.sum((np.asarray(x) - x0) ** 2, axis=-1)
        return c * np.exp(-s / a)

    def f(x):
        s = np.sum((np.asarray(x) - x0) ** 2, axis=-1)
        return c * np.exp(-s / a) * (6.0 / a - 4.0 * s / (a * a))

    return u, f


def polynomial(terms: Sequence[Tuple[float, int, int, int]]) -> Tuple[Callable, Callable]:
    """(u, f = -Lap u) of u = sum c x^a y^b z^c over the terms (c, a, b, c)."""
    def mono(x, a, b, e):
        x = np.asarray(x)
        return x[..., 0] ** a * x[..., 1] ** b * x[..., 2] ** e

    def u(x):
        return sum(cf * mono(x, a, b, e) for cf, a, b, e in terms)

    def f(x):
        out = 0.0
        for cf, a, b, e in terms:
            if a >= 2:
                out = out - cf * a * (a - 1) * mono(x, a - 2, b, e)
            if b >= 2:
                out = out - cf * b * (b - 1) * mono(x, a, b - 2, e)
            if e >= 2:
                out = out - cf * e * (e - 1) * mono(x, a, b, e - 2)
        return out + 0.0 * mono(x, 0, 0, 0)

    return u, f


# ---------------------------------------------------------------------------
# lifting and condensed right-hand side
# ---------------------------------------------------------------------------
def lifting(space, g: Callable) -> np.ndarray:
    """u_g at every support point."""
    u = np.zeros(space.n_points)
    bnd = space.on_boundary
    u[bnd] = g(space.points[bnd])
    hp = np.nonzero(space.hanging & ~space.on_boundary)[0]
    if len(hp):
        K = space.hang_cell[hp]
        s = (space.points[hp] - space.origin[K]) / space.h[K][:, None]
        phi = fe.basis_at(space.k, s)  # (m, n3): the coarse cell's basis at the point
        masters = space.cell_nodes[K]   # (m, n3)
        vals = np.where(space.on_boundary[masters], u[masters], 0.0)
        u[hp] = np.sum(phi * vals, axis=1)
    return u


def apply_all(space, u_all: np.ndarray) -> np.ndarray:
    """A_all u_all = sum_e P_e^T A_e P_e u_all (all support points)."""
    Aref = fe.reference_laplace_matrix(space.k)
    U = u_all[space.cell_nodes]
    V = (U @ Aref.T) * space.element_matrices_scale()[:, None]
    return np.bincount(space.cell_nodes.ravel(), weights=V.ravel(), minlength=space.n_points)


def rhs(space, f: Callable, g: Callable) -> np.ndarray:
    """b = C^T (F - A_all u_g)."""
    return space.rhs(f) - space.C.T @ apply_all(space, lifting(space, g))


def solution_all(space, x: np.ndarray, g: Callable) -> np.ndarray:
    """Values at all support points: C x + u_g."""
    return space.C @ x + lifting(space, g)
