"""Independent reference constructions used by the oracle pins.

Nothing here calls the oracle or the CUDA library: these are brute-force / dense restatements
(coordinates -> adjacency, dense Laplacians) used to check the oracle from outside.
"""
from __future__ import annotations

import numpy as np


def kept_coords(kept: np.ndarray) -> np.ndarray:
    """(n, 3) array of (z, y, x) coordinates of the True voxels, in raster order."""
    return np.argwhere(kept)


def dense_adjacency(kept: np.ndarray, weight=None) -> np.ndarray:
    """Dense adjacency of the 6-connected graph on the True voxels, from coordinates alone.
    `weight(a, b)` (node indices) gives an edge weight; default 1."""
    c = kept_coords(kept)
    n = c.shape[0]
    A = np.zeros((n, n))
    if n == 0:
        return A
    diff = np.abs(c[:, None, :] - c[None, :, :]).sum(axis=2)
    ii, jj = np.nonzero(diff == 1)
    for a, b in zip(ii, jj):
        A[a, b] = 1.0 if weight is None else weight(a, b)
    return A


def dense_laplacian(kept: np.ndarray, weight=None) -> np.ndarray:
    A = dense_adjacency(kept, weight)
    return np.diag(A.sum(axis=1)) - A


def brute_components(kept: np.ndarray):
    """Component id per True voxel (raster order), ids ordered by smallest member, by transitive
    closure of the dense adjacency (tiny inputs only)."""
    A = dense_adjacency(kept) > 0
    n = A.shape[0]
    R = A | np.eye(n, dtype=bool)
    while True:
        R2 = (R.astype(np.int64) @ R.astype(np.int64)) > 0
        if (R2 == R).all():
            break
        R = R2
    comp = -np.ones(n, dtype=np.int64)
    nxt = 0
    for i in range(n):
        if comp[i] < 0:
            comp[R[i]] = nxt
            nxt += 1
    return comp, nxt


def rel_l2(a, b) -> float:
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    if nb == 0:
        return float(np.abs(a - b).max()) if a.size else 0.0
    return float(np.linalg.norm(a - b) / nb)
