"""The discrete space V_h on one octree mesh: support points, constraints,
assembled operator, diagonal and right-hand side.

Test infrastructure (see ``oracle/__init__``).

Follows:
* Sec. 3.1: Dirichlet values imposed strongly and hanging-node constraints,
  both written as x_i = sum_j c_ij x_j + b_i (here b_i = 0), handled by
  condensation. The constraint matrix C maps the free (unconstrained,
  non-Dirichlet) values to the values at all support points.
* Eq. 2: the operator v = sum_e G_e^T C_e^T S_e^T Q_e S_e C_e G_e x. Its plain
  assembled definition is A = C^T (sum_e P_e^T A_e P_e) C with A_e the full
  quadrature element matrix and P_e the cell's node selection; this module
  writes exactly that out (sparse matrix for small meshes, cell-by-cell dense
  products for large ones).
* Eqs. 3-4: the diagonal of A, i.e. diag(C^T A_all C).

Hanging nodes are found from their definition: a support point p is
constrained if some leaf K contains p in its closed box without p being one of
K's support points; its constraint row is the trace of K's polynomial space
at p, i.e. the values phi_j^K(p) of K's basis functions. On 2:1 meshes the
constraining values are never themselves constrained (asserted).

Vectors of the operator hold only the free values (reading of the vector
convention: constrained and Dirichlet entries are not stored, so A is SPD).
"""
from __future__ import annotations

from typing import Callable, Optional

import numpy as np
import scipy.sparse as sp

from . import fe
from .mesh import Mesh

_LSH, _ISH, _JSH = 57, 38, 19


def cell_code(l, i, j, k):
    l = np.asarray(l, dtype=np.int64)
    return (l << _LSH) | (np.asarray(i, np.int64) << _ISH) | (np.asarray(j, np.int64) << _JSH) | np.asarray(k, np.int64)


class Space:
    """Continuous Q_k on the leaves of ``mesh`` with homogeneous Dirichlet
    values on the boundary of the cube."""

    def __init__(self, mesh: Mesh, k: int):
        self.mesh = mesh
        self.k = k
        self.n1 = k + 1
        self.n3 = (k + 1) ** 3
        cells = np.array(mesh.sorted_leaves(), dtype=np.int64)
        self.cells = cells
        self.nc = len(cells)
        self.level = cells[:, 0]
        self.h = (mesh.hi - mesh.lo) / (2.0 ** self.level)
        self.origin = mesh.lo + self.h[:, None] * cells[:, 1:4]
        # per-cell coefficient nu_e of -div(nu grad u) (1 unless set)
        self.nu = np.ones(self.nc)
        self.codes = cell_code(cells[:, 0], cells[:, 1], cells[:, 2], cells[:, 3])
        self.code_order = np.argsort(self.codes)
        self.sorted_codes = self.codes[self.code_order]

        xi = fe.gll_nodes(k)
        a, b, c = fe.tensor_index(k)
        X = self.origin[:, None, 0] + self.h[:, None] * xi[a][None, :]
        Y = self.origin[:, None, 1] + self.h[:, None] * xi[b][None, :]
        Z = self.origin[:, None, 2] + self.h[:, None] * xi[c][None, :]
        pts = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
        self.points, inv = np.unique(pts, axis=0, return_inverse=True)
        self.cell_nodes = inv.reshape(self.nc, self.n3)
        self.n_points = len(self.points)

        lo, hi = mesh.lo, mesh.hi
        self.on_boundary = np.any((self.points == lo) | (self.points == hi), axis=1)
        self._find_hanging()
        self._build_C()

    # ------------------------------------------------------------------
    def find_cells(self, l, i, j, k):
        """Index of leaf (l,i,j,k) or -1."""
        code = cell_code(l, i, j, k)
        pos = np.searchsorted(self.sorted_codes, code)
        pos = np.minimum(pos, self.nc - 1)
        hit = self.sorted_codes[pos] == code
        return np.where(hit, self.code_order[pos], -1)

    def _find_hanging(self):
        mesh, k = self.mesh, self.k
        xi = fe.gll_nodes(k)
        # finest level among the cells that have p as a support point
        pl = np.zeros(self.n_points, dtype=np.int64)
        np.maximum.at(pl, self.cell_nodes.ravel(), np.repeat(self.level, self.n3))
        lmin = int(self.level.min())
        hang_cell = np.full(self.n_points, -1, dtype=np.int64)
        hang_level = np.full(self.n_points, 1 << 30, dtype=np.int64)
        for l in range(lmin, int(pl.max())):
            sel = np.nonzero(pl > l)[0]
            if len(sel) == 0:
                continue
            hl = (mesh.hi - mesh.lo) / (2.0 ** l)
            t = (self.points[sel] - mesh.lo) / hl
            fl = np.floor(t)
            integral = fl == t
            n = 1 << l
            for combo in range(8):
                idx = fl.copy()
                shift = np.array([(combo >> d) & 1 for d in range(3)], dtype=bool)
                # candidate -1 along axes where t is integral and the bit is set
                use = np.all(~shift[None, :] | integral, axis=1)
                idx = idx - (shift[None, :] & integral)
                ok = use & np.all((idx >= 0) & (idx < n), axis=1)
                if not np.any(ok):
                    continue
                ii = idx[ok].astype(np.int64)
                cid = self.find_cells(np.full(len(ii), l), ii[:, 0], ii[:, 1], ii[:, 2])
                hit = cid >= 0
                if not np.any(hit):
                    continue
                pidx = sel[ok][hit]
                s = t[ok][hit] - ii[hit]  # local coordinates in [0,1]
                dist = np.min(np.abs(s[:, :, None] - xi[None, None, :]), axis=2)
                is_node = np.all(dist < 1e-9, axis=1)
                cand = ~is_node
                better = cand & (l < hang_level[pidx])
                hang_cell[pidx[better]] = cid[hit][better]
                hang_level[pidx[better]] = l
        self.hanging = hang_cell >= 0
        self.hang_cell = hang_cell

    def _build_C(self):
        k = self.k
        free = ~self.hanging & ~self.on_boundary
        self.free_index = np.full(self.n_points, -1, dtype=np.int64)
        self.free_points = np.nonzero(free)[0]
        self.n_free = len(self.free_points)
        self.free_index[self.free_points] = np.arange(self.n_free)
        rows = list(self.free_points)
        cols = list(range(self.n_free))
        vals = [1.0] * self.n_free
        hp = np.nonzero(self.hanging & ~self.on_boundary)[0]
        self.n_hanging = int(np.count_nonzero(self.hanging))
        if len(hp):
            K = self.hang_cell[hp]
            s = (self.points[hp] - self.origin[K]) / self.h[K][:, None]
            phi = fe.basis_at(k, s)  # (m, n3)
            for r, p in enumerate(hp):
                nodes = self.cell_nodes[K[r]]
                for n in np.nonzero(np.abs(phi[r]) > 1e-13)[0]:
                    q = nodes[n]
                    if self.hanging[q] and not self.on_boundary[q]:
                        raise RuntimeError("constraint chain: a constraining value is itself constrained")
                    fq = self.free_index[q]
                    if fq >= 0:
                        rows.append(p)
                        cols.append(fq)
                        vals.append(phi[r, n])
        self.C = sp.csr_matrix((vals, (rows, cols)), shape=(self.n_points, self.n_free))
        # cells that carry at least one hanging support point
        self.cell_has_hanging = np.any(self.hanging[self.cell_nodes], axis=1)

    # ------------------------------------------------------------------
    def free_coordinates(self) -> np.ndarray:
        return self.points[self.free_points]

    def element_matrices_scale(self) -> np.ndarray:
        """A_e = nu_e h_e A_ref: the Laplace matrix of a cube of edge h times
        the cell's coefficient."""
        return self.h * self.nu

    def apply(self, x: np.ndarray) -> np.ndarray:
        """y = C^T sum_e P_e^T (nu_e h_e A_ref) P_e C x, cell by cell, in the
        precision of x (fp64, or fp32 with fp32 element products)."""
        dt = x.dtype
        Aref = fe.reference_laplace_matrix(self.k).astype(dt)
        C = self.C.astype(dt) if dt != np.float64 else self.C
        u = C @ x
        U = u[self.cell_nodes]
        V = (U @ Aref.T) * self.element_matrices_scale().astype(dt)[:, None]
        v = np.bincount(self.cell_nodes.ravel(), weights=V.ravel(), minlength=self.n_points).astype(dt)
        return C.T @ v

    def assemble(self) -> sp.csr_matrix:
        """Sparse A = C^T A_all C (small meshes)."""
        Aref = fe.reference_laplace_matrix(self.k)
        n3 = self.n3
        r = np.repeat(self.cell_nodes, n3, axis=1).ravel()
        c = np.tile(self.cell_nodes, (1, n3)).ravel()
        v = (self.element_matrices_scale()[:, None, None] * Aref[None, :, :]).ravel()
        Aall = sp.csr_matrix((v, (r, c)), shape=(self.n_points, self.n_points))
        return (self.C.T @ Aall @ self.C).tocsr()

    def diagonal(self) -> np.ndarray:
        """diag(C^T A_all C) = sum_e diag(C_e^T A_e C_e)  (Eq. 4)."""
        Aref = fe.reference_laplace_matrix(self.k)
        d = np.zeros(self.n_free)
        plain = ~self.cell_has_hanging
        # cells without constrained values: d_e(i) = A_e(i, i)
        nodes = self.cell_nodes[plain]
        fi = self.free_index[nodes]
        contrib = self.element_matrices_scale()[plain][:, None] * np.diag(Aref)[None, :]
        m = fi >= 0
        np.add.at(d, fi[m], contrib[m])
        C = self.C.tocsr()
        for e in np.nonzero(self.cell_has_hanging)[0]:
            Ce = C[self.cell_nodes[e], :]
            cols = np.unique(Ce.indices)
            if len(cols) == 0:
                continue
            Ced = Ce[:, cols].toarray()
            d[cols] += np.einsum("mi,mn,ni->i", Ced, self.element_matrices_scale()[e] * Aref, Ced)
        return d

    def rhs(self, f: Optional[Callable[[np.ndarray], np.ndarray]] = None) -> np.ndarray:
        """b = C^T F with F_p = sum_e sum_q h^3 w_q f(x_q) phi_p(x_q) over the
        (k+1)^3 Gauss points of each cell; f = 1 when not given."""
        gq, gw = fe.gauss(self.k + 1)
        qa, qb, qc = fe.tensor_index(self.k)
        ref = np.stack([gq[qa], gq[qb], gq[qc]], axis=1)
        w = gw[qa] * gw[qb] * gw[qc]
        V = fe.basis_at(self.k, ref)  # (nq, n3)
        if f is None:
            fq = np.ones((self.nc, len(w)))
        else:
            xq = self.origin[:, None, :] + self.h[:, None, None] * ref[None, :, :]
            fq = f(xq.reshape(-1, 3)).reshape(self.nc, len(w))
        Fe = (fq * w[None, :] * (self.h ** 3)[:, None]) @ V
        F = np.bincount(self.cell_nodes.ravel(), weights=Fe.ravel(), minlength=self.n_points)
        return self.C.T @ F

    def interpolate(self, u: Callable[[np.ndarray], np.ndarray]) -> np.ndarray:
        """Free values of the nodal interpolant of u."""
        return u(self.free_coordinates())

    def evaluate(self, x: np.ndarray, pts: np.ndarray) -> np.ndarray:
        """Evaluate the FE function with free values x at physical points."""
        u = self.C @ x
        out = np.empty(len(pts))
        mesh = self.mesh
        L = int(self.level.max())
        found = np.full(len(pts), -1)
        for l in range(int(self.level.min()), L + 1):
            hl = (mesh.hi - mesh.lo) / (2.0 ** l)
            ii = np.clip(np.floor((pts - mesh.lo) / hl).astype(np.int64), 0, (1 << l) - 1)
            cid = self.find_cells(np.full(len(pts), l), ii[:, 0], ii[:, 1], ii[:, 2])
            upd = (found < 0) & (cid >= 0)
            found[upd] = cid[upd]
        assert np.all(found >= 0)
        s = (pts - self.origin[found]) / self.h[found][:, None]
        phi = fe.basis_at(self.k, s)
        return np.sum(phi * u[self.cell_nodes[found]], axis=1)


def paper_dof_count(mesh: Mesh, k: int) -> int:
    """Number of DoFs in the counting convention of Fig. 4: every vertex,
    edge, face and cell of the active cells carries 1, k-1, (k-1)^2 and
    (k-1)^3 DoFs, and the entities of both sides of a hanging interface are
    counted (the fine-side entities carry the constrained DoFs). For even k
    this exceeds the number of distinct support points, because the midpoint
    node of a coarse edge or face coincides with a fine-side vertex."""
    L = mesh.max_level
    V, E, F = set(), set(), set()
    for (l, i, j, kk) in mesh.leaves:
        s = 1 << (L - l)
        x0 = (i * s, j * s, kk * s)
        for a in (0, 1):
            for b in (0, 1):
                for c in (0, 1):
                    V.add((x0[0] + a * s, x0[1] + b * s, x0[2] + c * s))
        for d in range(3):
            o1, o2 = (d + 1) % 3, (d + 2) % 3
            for a in (0, 1):
                for b in (0, 1):
                    p = list(x0)
                    p[o1] += a * s
                    p[o2] += b * s
                    E.add((d, tuple(p), s))
            for a in (0, 1):
                p = list(x0)
                p[d] += a * s
                F.add((d, tuple(p), s))
    return len(V) + len(E) * (k - 1) + len(F) * (k - 1) ** 2 + len(mesh.leaves) * (k - 1) ** 3


def fourier_function(rhs) -> Callable[[np.ndarray], np.ndarray]:
    """f(x) = amp * sum_m cos(2 pi kappa_m . x + phi_m)."""
    kap = np.asarray(rhs.kappa, dtype=np.float64)
    phi = np.asarray(rhs.phi)

    def f(x):
        arg = 2.0 * np.pi * (x @ kap.T) + phi[None, :]
        return rhs.amp * np.cos(arg).sum(axis=1)

    return f
