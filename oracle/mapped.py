"""Non-Cartesian geometry: the octree cells mapped by a global map Phi.

Test infrastructure (see ``oracle/__init__``).

Follows Sec. 3.2's operator evaluation with the geometry at the quadrature
points (the general case of Eq. 2, where Q_e holds the Jacobian of the cell's
map at every quadrature point).  The mesh lives in parameter space (the
octree on [lo, hi]^3); the physical cell is Phi(cell), so the map of a cell
is x = Phi(x0 + h xi) with Jacobian J = h J_Phi.  The element matrix by
(k+1)^3-point Gauss quadrature is

    A_e[i, j] = sum_q w_q det(J_q) (J_q^-T grad phi_i(xi_q)) . (J_q^-T grad phi_j(xi_q)),

and the right-hand side F_i = sum_q w_q det(J_q) f(Phi(x_q)) phi_i(xi_q).
Hanging-node constraints and the transfer between levels act on the
parameter-space coefficients and are unchanged.

The map of the tests (reading: the paper's curved meshes come from ASPECT's
spherical manifold, which needs a multi-patch coarse mesh; a single-patch
octree is mapped instead):

    Phi(x) = x + eps * (x_1 x_2, 2 x_2 x_0, x_0 x_1 / 2)

is of degree one in every variable, so every cell is a general trilinear
hexahedron, functions linear in the physical coordinates lie in Q_k for all
k >= 1 and the Gauss rule integrates the mapped Laplacian of such functions
exactly (the patch test); its Jacobian is not symmetric, so a transposed
J^-1 does not pass unnoticed.
"""
from __future__ import annotations

from typing import Callable

import numpy as np
import scipy.sparse as sp

from . import fe
from .space import Space


def warp(x: np.ndarray, eps: float) -> np.ndarray:
    """Phi(x), x of shape (..., 3)."""
    x = np.asarray(x, dtype=np.float64)
    return x + eps * np.stack([x[..., 1] * x[..., 2], 2.0 * x[..., 2] * x[..., 0], 0.5 * x[..., 0] * x[..., 1]],
                              axis=-1)


def warp_jacobian(x: np.ndarray, eps: float) -> np.ndarray:
    """J_Phi(x) of shape (..., 3, 3): d Phi_a / d x_b."""
    x = np.asarray(x, dtype=np.float64)
    J = np.zeros(x.shape[:-1] + (3, 3))
    J[..., 0, 0] = J[..., 1, 1] = J[..., 2, 2] = 1.0
    J[..., 0, 1], J[..., 0, 2] = eps * x[..., 2], eps * x[..., 1]
    J[..., 1, 0], J[..., 1, 2] = 2.0 * eps * x[..., 2], 2.0 * eps * x[..., 0]
    J[..., 2, 0], J[..., 2, 1] = 0.5 * eps * x[..., 1], 0.5 * eps * x[..., 0]
    return J


class MappedSpace(Space):
    """A Space whose cells are mapped by Phi; element matrices per cell."""

    def __init__(self, mesh, k: int, eps: float):
        super().__init__(mesh, k)
        self.eps = eps
        self._Ae = self._element_matrices()

    def physical_points(self) -> np.ndarray:
        return warp(self.points, self.eps)

    def _quadrature(self):
        gq, gw = fe.gauss(self.k + 1)
        qa, qb, qc = fe.tensor_index(self.k)
        ref = np.stack([gq[qa], gq[qb], gq[qc]], axis=1)
        w = gw[qa] * gw[qb] * gw[qc]
        return ref, w

    def _ref_gradients(self, ref):
        """(3, nq, n3): d phi_n / d xi_d at the Gauss points."""
        xi = fe.gll_nodes(self.k)
        a, b, c = fe.tensor_index(self.k)
        v = [fe.lagrange_values(xi, ref[:, d]) for d in range(3)]
        dv = [fe.lagrange_derivs(xi, ref[:, d]) for d in range(3)]
        gx = dv[0][:, a] * v[1][:, b] * v[2][:, c]
        gy = v[0][:, a] * dv[1][:, b] * v[2][:, c]
        gz = v[0][:, a] * v[1][:, b] * dv[2][:, c]
        return np.stack([gx, gy, gz])

    def _element_matrices(self) -> np.ndarray:
        """(nc, n3, n3) by the formula of the module docstring."""
        ref, w = self._quadrature()
        G = self._ref_gradients(ref)                          # (3, nq, n3)
        xq = self.origin[:, None, :] + self.h[:, None, None] * ref[None, :, :]   # (nc, nq, 3)
        J = self.h[:, None, None, None] * warp_jacobian(xq, self.eps)             # (nc, nq, 3, 3)
        det = np.linalg.det(J)
        Jinv = np.linalg.inv(J)
        # physical gradients: grad_x phi = J^-T grad_xi phi
        Pg = np.einsum("cqba,bqn->cqan", Jinv, G)             # (nc, nq, 3, n3)
        wd = (w[None, :] * det * self.nu[:, None])
        return np.einsum("cq,cqan,cqam->cnm", wd, Pg, Pg)

    def set_coefficient(self, nu):
        self.nu = np.asarray(nu, dtype=np.float64)
        self._Ae = self._element_matrices()

    # ---- the operations of Space with per-cell element matrices -----------
    def apply(self, x: np.ndarray) -> np.ndarray:
        dt = x.dtype
        C = self.C.astype(dt) if dt != np.float64 else self.C
        u = C @ x
        U = u[self.cell_nodes]
        V = np.einsum("cnm,cm->cn", self._Ae.astype(dt), U)
        v = np.bincount(self.cell_nodes.ravel(), weights=V.ravel(), minlength=self.n_points).astype(dt)
        return C.T @ v

    def apply_all(self, u_all: np.ndarray) -> np.ndarray:
        V = np.einsum("cnm,cm->cn", self._Ae, u_all[self.cell_nodes])
        return np.bincount(self.cell_nodes.ravel(), weights=V.ravel(), minlength=self.n_points)

    def assemble(self) -> sp.csr_matrix:
        n3 = self.n3
        r = np.repeat(self.cell_nodes, n3, axis=1).ravel()
        c = np.tile(self.cell_nodes, (1, n3)).ravel()
        Aall = sp.csr_matrix((self._Ae.ravel(), (r, c)), shape=(self.n_points, self.n_points))
        return (self.C.T @ Aall @ self.C).tocsr()

    def diagonal(self) -> np.ndarray:
        return self.assemble().diagonal().copy()

    def rhs(self, f: Callable = None) -> np.ndarray:
        ref, w = self._quadrature()
        V = fe.basis_at(self.k, ref)
        xq = self.origin[:, None, :] + self.h[:, None, None] * ref[None, :, :]
        det = np.linalg.det(self.h[:, None, None, None] * warp_jacobian(xq, self.eps))
        if f is None:
            fq = np.ones(det.shape)
        else:
            fq = f(warp(xq, self.eps).reshape(-1, 3)).reshape(det.shape)
        Fe = (fq * w[None, :] * det) @ V
        F = np.bincount(self.cell_nodes.ravel(), weights=Fe.ravel(), minlength=self.n_points)
        return self.C.T @ F


def lifting(space: MappedSpace, g: Callable) -> np.ndarray:
    """u_g with g evaluated at the physical support points (the constraint
    rows of hanging points act on parameter-space coefficients)."""
    u = np.zeros(space.n_points)
    bnd = space.on_boundary
    u[bnd] = g(space.physical_points()[bnd])
    hp = np.nonzero(space.hanging & ~space.on_boundary)[0]
    if len(hp):
        K = space.hang_cell[hp]
        s = (space.points[hp] - space.origin[K]) / space.h[K][:, None]
        phi = fe.basis_at(space.k, s)
        masters = space.cell_nodes[K]
        vals = np.where(space.on_boundary[masters], u[masters], 0.0)
        u[hp] = np.sum(phi * vals, axis=1)
    return u


def rhs_dirichlet(space: MappedSpace, f: Callable, g: Callable) -> np.ndarray:
    """b = C^T (F - A_all u_g) on the mapped mesh."""
    return space.rhs(f) - space.C.T @ space.apply_all(lifting(space, g))
