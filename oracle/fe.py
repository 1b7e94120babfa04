"""1D and 3D finite-element ingredients for Q_k on hexahedra.

Test infrastructure (see ``oracle/__init__``).

Follows Sec. 5 (set-up): a continuous Lagrange element defined as the tensor
product of 1D elements of degree k, integrated with the Gauss-Legendre rule of
(k+1)^3 points. The support points are the Gauss-Lobatto-Legendre (GLL)
points (reading of the paper's DoF counts: the p=4 count 9.3e3 of the octant
L=3 mesh in Fig. 4 is matched by GLL points, not by equidistant ones).

Local node numbering: n = a + (k+1) b + (k+1)^2 c with (a, b, c) the 1D node
indices along x, y, z.

Pins (tests/test_oracle_fe.py): closed-form GLL nodes, exactness of the
Gauss rule on monomials, Lagrange property, element matrix against the
closed form h (K x M x M + M x K x M + M x M x K) with exactly integrated 1D
matrices, zero row sums.
"""
from __future__ import annotations

import functools

import numpy as np
from numpy.polynomial import legendre as npleg


@functools.lru_cache(maxsize=None)
def gll_nodes(k: int) -> np.ndarray:
    """k+1 Gauss-Lobatto-Legendre points on [0,1]: the end points and the
    roots of P_k' (derivative of the Legendre polynomial of degree k)."""
    if k < 1:
        raise ValueError("degree must be >= 1")
    if k == 1:
        return np.array([0.0, 1.0])
    dP = npleg.Legendre.basis(k).deriv()
    r = np.sort(np.real(dP.roots()))
    x = np.concatenate([[-1.0], r, [1.0]])
    x = 0.5 * (x + 1.0)
    x = 0.5 * (x + (1.0 - x[::-1]))  # exact symmetry about 1/2
    if k % 2 == 0:
        x[k // 2] = 0.5
    return x


@functools.lru_cache(maxsize=None)
def gauss(n: int):
    """n-point Gauss-Legendre rule on [0,1]: points, weights."""
    x, w = npleg.leggauss(n)
    return 0.5 * (x + 1.0), 0.5 * w


def lagrange_values(nodes: np.ndarray, t) -> np.ndarray:
    """L_a(t_q) for all nodes a and points t_q: array (len(t), len(nodes)).
    L_a(t) = prod_{b != a} (t - x_b) / (x_a - x_b)."""
    t = np.atleast_1d(np.asarray(t, dtype=np.float64))
    n = len(nodes)
    out = np.ones((len(t), n))
    for a in range(n):
        for b in range(n):
            if b != a:
                out[:, a] *= (t - nodes[b]) / (nodes[a] - nodes[b])
    return out


def lagrange_derivs(nodes: np.ndarray, t) -> np.ndarray:
    """L_a'(t_q) by the product rule: sum_{c != a} 1/(x_a - x_c) *
    prod_{b != a, c} (t - x_b)/(x_a - x_b)."""
    t = np.atleast_1d(np.asarray(t, dtype=np.float64))
    n = len(nodes)
    out = np.zeros((len(t), n))
    for a in range(n):
        for c in range(n):
            if c == a:
                continue
            term = np.full(len(t), 1.0 / (nodes[a] - nodes[c]))
            for b in range(n):
                if b != a and b != c:
                    term *= (t - nodes[b]) / (nodes[a] - nodes[b])
            out[:, a] += term
    return out


def tensor_index(k: int):
    """(a, b, c) for every local node n = a + (k+1) b + (k+1)^2 c."""
    n1 = k + 1
    idx = np.arange(n1 ** 3)
    return idx % n1, (idx // n1) % n1, idx // (n1 * n1)


def basis_at(k: int, pts: np.ndarray) -> np.ndarray:
    """Values of all (k+1)^3 reference basis functions at reference points
    pts (m, 3) in [0,1]^3: array (m, (k+1)^3)."""
    xi = gll_nodes(k)
    vx = lagrange_values(xi, pts[:, 0])
    vy = lagrange_values(xi, pts[:, 1])
    vz = lagrange_values(xi, pts[:, 2])
    a, b, c = tensor_index(k)
    return vx[:, a] * vy[:, b] * vz[:, c]


@functools.lru_cache(maxsize=None)
def reference_laplace_matrix(k: int) -> np.ndarray:
    """Element Laplace matrix of the unit cube, by full Gauss quadrature with
    (k+1)^3 points: A_ij = sum_q w_q grad phi_i(x_q) . grad phi_j(x_q).
    For a cube of edge h the element matrix is h * this matrix
    (gradients scale with 1/h, the volume element with h^3)."""
    xi = gll_nodes(k)
    gq, gw = gauss(k + 1)
    n1 = k + 1
    # all 3D quadrature points and weights (x fastest)
    qa, qb, qc = tensor_index(k)  # same count of points per direction (k+1)
    px, py, pz = gq[qa], gq[qb], gq[qc]
    w = gw[qa] * gw[qb] * gw[qc]
    a, b, c = tensor_index(k)
    vx, vy, vz = lagrange_values(xi, px), lagrange_values(xi, py), lagrange_values(xi, pz)
    dx, dy, dz = lagrange_derivs(xi, px), lagrange_derivs(xi, py), lagrange_derivs(xi, pz)
    gx = dx[:, a] * vy[:, b] * vz[:, c]
    gy = vx[:, a] * dy[:, b] * vz[:, c]
    gz = vx[:, a] * vy[:, b] * dz[:, c]
    A = np.zeros((n1 ** 3, n1 ** 3))
    for g in (gx, gy, gz):
        A += g.T @ (w[:, None] * g)
    return A


@functools.lru_cache(maxsize=None)
def reference_mass_matrix(k: int) -> np.ndarray:
    """Element mass matrix of the unit cube by (k+1)^3-point Gauss quadrature."""
    gq, gw = gauss(k + 1)
    qa, qb, qc = tensor_index(k)
    pts = np.stack([gq[qa], gq[qb], gq[qc]], axis=1)
    w = gw[qa] * gw[qb] * gw[qc]
    V = basis_at(k, pts)
    return V.T @ (w[:, None] * V)
