"""Helpers of the parity tests: match two numberings of the same support
points by their coordinates."""
import numpy as np


def match(xyz_a: np.ndarray, xyz_b: np.ndarray, tol: float = 1e-10) -> np.ndarray:
    """perm such that xyz_a[i] == xyz_b[perm[i]] (within tol); asserts a
    bijection."""
    assert xyz_a.shape == xyz_b.shape, (xyz_a.shape, xyz_b.shape)
    if len(xyz_a) == 0:
        return np.zeros(0, dtype=np.int64)
    ka = np.round(xyz_a / tol).astype(np.int64)
    kb = np.round(xyz_b / tol).astype(np.int64)
    ia = np.lexsort(ka.T[::-1])
    ib = np.lexsort(kb.T[::-1])
    assert np.abs(xyz_a[ia] - xyz_b[ib]).max() < 10 * tol, "support points differ"
    perm = np.empty(len(xyz_a), dtype=np.int64)
    perm[ia] = ib
    return perm


def rel_err(a, b) -> float:
    a = np.asarray(a)
    b = np.asarray(b)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))
