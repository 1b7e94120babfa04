"""Rows of the operator evaluated one by one from the oracle's element
matrix, for meshes too large for the oracle's global operator: at support
points whose neighbourhood is a single refinement level no hanging-node
constraint enters the row, so (A x)_i is a sum over the cells around the
point.  Pinned against the oracle's global operator on small meshes
(tests/test_oracle_sampled_rows.py)."""
import numpy as np

import synth
from oracle import fe


def deep_cells(m, rng, per_level):
    """Random leaves whose 5x5x5 block of same-level cells (inside the
    domain) consists of leaves only."""
    by_level = {}
    for c in m.sorted_leaves():
        by_level.setdefault(c[0], []).append(c)
    out = []
    for l, cells in sorted(by_level.items()):
        n = 1 << l
        found = 0
        for idx in rng.permutation(len(cells)):
            _, i, j, k = cells[idx]
            if all((l, a, b, c) in m.leaves
                   for a in range(i - 2, i + 3) for b in range(j - 2, j + 3) for c in range(k - 2, k + 3)
                   if 0 <= a < n and 0 <= b < n and 0 <= c < n):
                out.append(cells[idx])
                found += 1
                if found == per_level:
                    break
    return out


def sampled_rows(m, K, cells, rng, seed):
    """(positions, (A x) at them) for one random node of each cell that is
    not on the boundary, for Q_K, x = synth.point_values(., seed) at free
    points and 0 on the boundary: the sum over the cells around the point of
    h times the oracle's reference Laplace matrix (Eq. 2 on a cube of edge h)
    applied to x at the cells' nodes.  Valid where no hanging node touches
    the row: cells from deep_cells."""
    xi = fe.gll_nodes(K)
    Aref = fe.reference_laplace_matrix(K)
    ta, tb, tc = fe.tensor_index(K)
    n1 = K + 1
    pos, val = [], []
    for cell in cells:
        l, i, j, k = cell
        h = m.h(l)
        n_cells = 1 << l
        while True:
            a, b, c = (int(v) for v in rng.integers(0, n1, 3))
            p = np.array([m.lo + h * (i + xi[a]), m.lo + h * (j + xi[b]), m.lo + h * (k + xi[c])])
            if np.all(p > m.lo + 1e-12) and np.all(p < m.hi - 1e-12):
                break

        def axis(t):  # (cell offset, local index of the point in that cell)
            return [(0, 0), (-1, K)] if t == 0 else ([(0, K), (1, 0)] if t == K else [(0, t)])

        y = 0.0
        for dx, la in axis(a):
            for dy, lb in axis(b):
                for dz, lc in axis(c):
                    ci, cj, ck = i + dx, j + dy, k + dz
                    if not (0 <= ci < n_cells and 0 <= cj < n_cells and 0 <= ck < n_cells):
                        continue
                    assert (l, ci, cj, ck) in m.leaves
                    nodes = np.stack([m.lo + h * (ci + xi[ta]), m.lo + h * (cj + xi[tb]), m.lo + h * (ck + xi[tc])], 1)
                    bnd = np.any((nodes < m.lo + 1e-12) | (nodes > m.hi - 1e-12), axis=1)
                    xv = np.where(bnd, 0.0, synth.point_values(nodes, seed))
                    y += h * (Aref[la + n1 * lb + n1 * n1 * lc] @ xv)
        pos.append(p)
        val.append(y)
    return np.array(pos), np.array(val)
