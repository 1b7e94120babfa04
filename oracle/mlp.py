"""Learned per-cell smoother: network, loss, gradients, Adam, cell features
and the owner-selected correction.

Test infrastructure (see ``oracle/__init__``).

The paper's smoother is Chebyshev around point Jacobi (Sec. 3.3, Sec. 5);
this learned variant is an extension outside the paper, so every definition
below is stated here and followed literally:

network   y = W3 g(W2 g(W1 x + b1) + b2) + b3 with g the exact GELU,
          g(z) = z Phi(z) = z (1 + erf(z / sqrt 2)) / 2.  W1 is n_h x n_in,
          W2 n_h x n_h, W3 n_out x n_h (one row per output unit).  Packed
          parameter vector: W1, b1, W2, b2, W3, b3, matrices row-major.
loss      L = sum_b w_b ||y_b - t_b||^2 / (2 sum_b w_b) over a batch of B
          samples with weights w_b (all 1: the plain mean squared error).
Adam      Kingma & Ba (2015), Algorithm 1: beta1 0.9, beta2 0.999, eps 1e-8,
          bias-corrected moments.
features  for cell e with the cell values r_e = (C r)|_e of the residual and
          d_e = (C diag(A))|_e of the diagonal at its (k+1)^3 support points
          (lexicographic, x fastest): s_e = ||r_e||_2 and
          x_e = [r_e / s_e, d_e / (h_e a_k)], a_k the mean diagonal entry of
          the Laplace matrix of the unit cell (x_e = [0, ...] when s_e = 0).
target    t_e = e_e h_e a_k / s_e for the cell values e_e of the error, and
          weight w_e = (s_e / (h_e a_k))^2, so that w_e ||y - t_e||^2 =
          ||c_e - e_e||^2 is the squared error of the correction itself.
correction c_e = y(x_e) s_e / (h_e a_k): a positively 1-homogeneous map of
          the residual.  Free value i receives c_{o(i)} at its node in its
          owner cell o(i) (the weighting W_e of the transfer, realised as a
          selection).
owner     o(i) = the first cell in Morton order (bit-interleaved anchor on the
          finest lattice, x in the lowest bit) among the cells in which i is
          a regular support point, i.e. not on a closed face or closed edge of
          the cell that borders a coarser leaf.
bf16      with bf16=True the operands of every matrix product (features,
          weights, activations, backward signals) are rounded to bfloat16
          (round to nearest, ties to even) and the products accumulate in
          fp64: the extension fixes bf16 operands with wide accumulation.
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from typing import Dict, List, Tuple

import numpy as np
from scipy.special import erf

from . import fe

BETA1, BETA2, ADAM_EPS = 0.9, 0.999, 1e-8


# ---------------------------------------------------------------------------
# scalar pieces
# ---------------------------------------------------------------------------
def gelu(z):
    """g(z) = z Phi(z) with the standard normal distribution function Phi."""
    return 0.5 * z * (1.0 + erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    """g'(z) = Phi(z) + z phi(z)."""
    return 0.5 * (1.0 + erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def round_bf16(x) -> np.ndarray:
    """Round to the nearest bfloat16 (8 significand bits), ties to even, via
    the binary32 pattern (the value is first rounded to binary32)."""
    f = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    out = r.astype(np.uint32).view(np.float32).astype(np.float64)
    return out.reshape(np.shape(x))


# ---------------------------------------------------------------------------
# parameters
# ---------------------------------------------------------------------------
@dataclass
class Shape:
    n_in: int
    n_h: int
    n_out: int

    def sizes(self) -> List[Tuple[str, Tuple[int, ...]]]:
        return [("W1", (self.n_h, self.n_in)), ("b1", (self.n_h,)), ("W2", (self.n_h, self.n_h)),
                ("b2", (self.n_h,)), ("W3", (self.n_out, self.n_h)), ("b3", (self.n_out,))]

    def n_params(self) -> int:
        return sum(int(np.prod(s)) for _, s in self.sizes())


def unpack(shape: Shape, theta: np.ndarray) -> Dict[str, np.ndarray]:
    out, pos = {}, 0
    for name, s in shape.sizes():
        m = int(np.prod(s))
        out[name] = np.asarray(theta[pos:pos + m], dtype=np.float64).reshape(s)
        pos += m
    assert pos == len(theta)
    return out


def pack(shape: Shape, p: Dict[str, np.ndarray]) -> np.ndarray:
    return np.concatenate([np.asarray(p[name], dtype=np.float64).ravel() for name, _ in shape.sizes()])


# ---------------------------------------------------------------------------
# forward, loss, backward
# ---------------------------------------------------------------------------
def forward(shape: Shape, theta: np.ndarray, X: np.ndarray, bf16: bool = False):
    """Network outputs for the rows of X, and the intermediate values."""
    q = round_bf16 if bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    p = unpack(shape, theta)
    X = np.asarray(X, dtype=np.float64)
    Z1 = q(X) @ q(p["W1"]).T + p["b1"]
    H1 = gelu(Z1)
    Z2 = q(H1) @ q(p["W2"]).T + p["b2"]
    H2 = gelu(Z2)
    Y = q(H2) @ q(p["W3"]).T + p["b3"]
    return Y, dict(X=X, Z1=Z1, H1=H1, Z2=Z2, H2=H2)


def loss(Y: np.ndarray, T: np.ndarray, W=None) -> float:
    w = np.ones(Y.shape[0]) if W is None else np.asarray(W, dtype=np.float64)
    return float(0.5 * np.sum(w[:, None] * (Y - T) ** 2) / np.sum(w))


def loss_and_grad(shape: Shape, theta: np.ndarray, X: np.ndarray, T: np.ndarray, bf16: bool = False, W=None):
    """L and dL/dtheta (packed like theta), by the chain rule backwards
    through the three layers."""
    q = round_bf16 if bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    p = unpack(shape, theta)
    Y, c = forward(shape, theta, X, bf16)
    w = np.ones(Y.shape[0]) if W is None else np.asarray(W, dtype=np.float64)
    dY = w[:, None] * (Y - T) / np.sum(w)
    g = {}
    g["W3"] = q(dY).T @ q(c["H2"])
    g["b3"] = dY.sum(axis=0)
    dZ2 = (q(dY) @ q(p["W3"])) * gelu_grad(c["Z2"])
    g["W2"] = q(dZ2).T @ q(c["H1"])
    g["b2"] = dZ2.sum(axis=0)
    dZ1 = (q(dZ2) @ q(p["W2"])) * gelu_grad(c["Z1"])
    g["W1"] = q(dZ1).T @ q(c["X"])
    g["b1"] = dZ1.sum(axis=0)
    return loss(Y, T, w), pack(shape, g)


def adam_step(theta, grad, m, v, t: int, lr: float):
    """One Adam update (step number t >= 1); returns theta, m, v."""
    m = BETA1 * m + (1.0 - BETA1) * grad
    v = BETA2 * v + (1.0 - BETA2) * grad * grad
    mh = m / (1.0 - BETA1 ** t)
    vh = v / (1.0 - BETA2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + ADAM_EPS), m, v


def train(shape: Shape, theta: np.ndarray, X: np.ndarray, T: np.ndarray, order: np.ndarray, batch: int,
          lr: float, bf16: bool = False, W=None):
    """Adam on consecutive batches of the sample order; returns the final
    parameters and the loss of every step (before its update)."""
    theta = np.asarray(theta, dtype=np.float64).copy()
    m = np.zeros_like(theta)
    v = np.zeros_like(theta)
    losses = []
    for s in range(len(order) // batch):
        idx = order[s * batch:(s + 1) * batch]
        L, g = loss_and_grad(shape, theta, X[idx], T[idx], bf16, None if W is None else np.asarray(W)[idx])
        losses.append(L)
        theta, m, v = adam_step(theta, g, m, v, s + 1, lr)
    return theta, np.array(losses)


# ---------------------------------------------------------------------------
# cells: features, targets, owners, correction
# ---------------------------------------------------------------------------
def mean_reference_diagonal(k: int) -> float:
    """a_k: mean diagonal entry of the Laplace matrix of the unit cell."""
    return float(np.mean(np.diag(fe.reference_laplace_matrix(k))))


def cell_values(space, v: np.ndarray) -> np.ndarray:
    """(C v)|_e for every cell: values at the support points of each cell,
    hanging points interpolated from their constraining values, Dirichlet
    points zero."""
    return (space.C @ v)[space.cell_nodes]


def cell_features(space, r: np.ndarray, diag: np.ndarray):
    """x_e for every cell, and s_e."""
    a = mean_reference_diagonal(space.k)
    re = cell_values(space, r)
    de = cell_values(space, diag)
    s = np.linalg.norm(re, axis=1)
    safe = np.where(s > 0, s, 1.0)
    xr = np.where(s[:, None] > 0, re / safe[:, None], 0.0)
    X = np.concatenate([xr, de / (space.h[:, None] * a)], axis=1)
    return X, s


def cell_weights(space, r: np.ndarray) -> np.ndarray:
    """w_e = (s_e / (h_e a_k))^2."""
    a = mean_reference_diagonal(space.k)
    s = np.linalg.norm(cell_values(space, r), axis=1)
    return (s / (space.h * a)) ** 2


def cell_targets(space, r: np.ndarray, e: np.ndarray) -> np.ndarray:
    """t_e = e_e h_e a_k / s_e (zero where s_e = 0)."""
    a = mean_reference_diagonal(space.k)
    s = np.linalg.norm(cell_values(space, r), axis=1)
    ee = cell_values(space, e)
    safe = np.where(s > 0, s, 1.0)
    return np.where(s[:, None] > 0, ee * (space.h * a / safe)[:, None], 0.0)


def morton_key(cell, lmax: int) -> int:
    """Bit-interleaved anchor of (l, i, j, k) on the 2^lmax lattice, x in the
    lowest bit of every triple."""
    l, i, j, k = (int(c) for c in cell)
    sh = lmax - l
    X, Y, Z = i << sh, j << sh, k << sh
    key = 0
    for bit in range(lmax + 1):
        key |= ((X >> bit) & 1) << (3 * bit)
        key |= ((Y >> bit) & 1) << (3 * bit + 1)
        key |= ((Z >> bit) & 1) << (3 * bit + 2)
    return key


def _coarser_neighbour(mesh, cell, offs) -> bool:
    """Does the leaf containing the level-l block at cell + offs exist and lie
    on a coarser level than the cell?"""
    l, i, j, k = cell
    n = 1 << l
    q = (i + offs[0], j + offs[1], k + offs[2])
    if min(q) < 0 or max(q) >= n:
        return False
    leaf = mesh.leaf_containing((l,) + q)
    return leaf is not None and leaf[0] < l


def regular_nodes(space, ci: int) -> np.ndarray:
    """Boolean per local node of cell ci: not on a closed face or closed edge
    of the cell that borders a coarser leaf."""
    k = space.k
    cell = tuple(int(v) for v in space.cells[ci])
    a, b, c = fe.tensor_index(k)
    coord = np.stack([a, b, c], axis=1)
    ok = np.ones(len(a), dtype=bool)
    for d in range(3):
        for side in (0, 1):
            offs = [0, 0, 0]
            offs[d] = 1 if side else -1
            if _coarser_neighbour(space.mesh, cell, offs):
                ok &= coord[:, d] != side * k
    for d in range(3):
        t1, t2 = [x for x in range(3) if x != d]
        for s1 in (0, 1):
            for s2 in (0, 1):
                o1 = [0, 0, 0]
                o1[t1] = 1 if s1 else -1
                o2 = [0, 0, 0]
                o2[t2] = 1 if s2 else -1
                o12 = [o1[x] + o2[x] for x in range(3)]
                if any(_coarser_neighbour(space.mesh, cell, o) for o in (o1, o2, o12)):
                    ok &= ~((coord[:, t1] == s1 * k) & (coord[:, t2] == s2 * k))
    return ok


def owners(space) -> Tuple[np.ndarray, np.ndarray]:
    """Owner cell and local node of every free value."""
    lmax = int(space.level.max())
    keys = [morton_key(c, lmax) for c in space.cells]
    order = sorted(range(space.nc), key=lambda ci: keys[ci])
    own_cell = np.full(space.n_free, -1, dtype=np.int64)
    own_node = np.full(space.n_free, -1, dtype=np.int64)
    for ci in order:
        reg = regular_nodes(space, ci)
        fi = space.free_index[space.cell_nodes[ci]]
        for j in np.nonzero(reg & (fi >= 0))[0]:
            if own_cell[fi[j]] < 0:
                own_cell[fi[j]] = ci
                own_node[fi[j]] = j
    assert np.all(own_cell >= 0), "free value without a regular support point"
    return own_cell, own_node


def correction(space, shape: Shape, theta: np.ndarray, r: np.ndarray, diag: np.ndarray, bf16: bool = False,
               own=None) -> np.ndarray:
    """The learned correction of the free values for the residual r."""
    X, s = cell_features(space, r, diag)
    Y, _ = forward(shape, theta, X, bf16)
    a = mean_reference_diagonal(space.k)
    C = Y * (s / (space.h * a))[:, None]
    oc, on = own if own is not None else owners(space)
    return C[oc, on]
