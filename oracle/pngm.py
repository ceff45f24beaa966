"""FP64 CPU restatement of the coarse primitive-graph (PNGM) diffusion model and of its
calibration from voxel data (Sec. V.A, Schemes 3 and 4, Objectives 1 and 2 and their gradients,
the normalised SGD update).

TEST INFRASTRUCTURE: only the test suite, the package's smoke check and the benchmark's CPU
baseline leg may import this module.  It shares nothing with the CUDA library.

Plain numpy, vectorised only where the formula is a sum over a set that numpy can express
directly (np.bincount, np.unique); Scheme 4 is a dense solve, so it is for small graphs only.

Readings of the paper applied here:
  P1  Primitives are given as a partition of the pore voxels (one primitive label per node); the
      maximal-ball extraction that defines them in the paper is a separate tool.  v_i = number of
      voxels of primitive i.  Two primitives are adjacent when a voxel face joins them.
  P2  The initial conductance S_ij / d_ij (Sec. V.B): S_ij = number of voxel faces between the two
      primitives (voxel^2), d_ij = distance between their voxel centroids (voxel).
  P3  Conductances are indexed by ordered pairs: the derivation of the gradient drops every
      residual but row i, which holds only when theta_ij and theta_ji are separate parameters.
      With tied=True the pair shares one value and its gradient is the sum of the two ordered
      terms (the derivative of the loss under the constraint theta_ij = theta_ji).
  P4  The objectives and gradients use x_j / v_j where the objective lines print x_i / v_j (the
      gradient lines have the corrected form).
  P5  The gradient of Objective 2 is the derivative of its residual, -c (y_i/v_i - y_j/v_j) times
      2 r_i / (l q); the printed formula lacks the minus sign, which would make the normalised
      update climb the loss.
  P6  Normalised SGD: theta <- theta - lr g / |g| per parameter; a parameter with g = 0 is left
      unchanged (g / |g| is undefined there).  An optional lower bound theta_min (the paper sets
      none) keeps conductances non-negative.
"""
from __future__ import annotations

import numpy as np


def coarse_graph(nbr: np.ndarray, voxel_of_node: np.ndarray, shape, labels: np.ndarray, q: int) -> dict:
    """Primitive graph of a node partition (readings P1, P2).

    nbr: (n, 6) node neighbours in the order -x, +x, -y, +y, -z, +z (-1 = none); voxel_of_node:
    raster index of every node in an image of shape (nz, ny, nx); labels: (n,) primitive of every
    node, values in [0, q).  Returns volumes v (q,), centroids (q, 3) as (x, y, z), and the ordered
    pairs in CSR form: row_ptr (q+1,), col (nslots,), S and d per slot, rev = slot of (j, i)."""
    nz, ny, nx = (int(s) for s in shape)
    labels = np.asarray(labels, dtype=np.int64)
    n = labels.shape[0]
    vol = np.bincount(labels, minlength=q).astype(np.float64)
    vox = np.asarray(voxel_of_node, dtype=np.int64)
    x, y, z = vox % nx, (vox // nx) % ny, vox // (nx * ny)
    cen = np.zeros((q, 3))
    with np.errstate(invalid="ignore", divide="ignore"):
        for a, coord in enumerate((x, y, z)):
            cen[:, a] = np.bincount(labels, weights=coord.astype(np.float64), minlength=q) / vol
    # voxel faces between different primitives, each face seen once from its lower node (+ slots)
    keys = []
    for d in (1, 3, 5):
        j = nbr[:, d]
        i = np.nonzero(j >= 0)[0]
        a, b = labels[i], labels[j[i]]
        cross = a != b
        lo, hi = np.minimum(a[cross], b[cross]), np.maximum(a[cross], b[cross])
        keys.append(lo * q + hi)
    keys = np.concatenate(keys) if keys else np.zeros(0, dtype=np.int64)
    pairs, faces = np.unique(keys, return_counts=True)
    lo, hi = pairs // q, pairs % q
    # ordered pairs (i, j) and (j, i), sorted by row then column
    rows = np.concatenate([lo, hi])
    cols = np.concatenate([hi, lo])
    S = np.concatenate([faces, faces]).astype(np.float64)
    order = np.lexsort((cols, rows))
    rows, cols, S = rows[order], cols[order], S[order]
    row_ptr = np.zeros(q + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=q), out=row_ptr[1:])
    dx = cen[rows, 0] - cen[cols, 0]
    dy = cen[rows, 1] - cen[cols, 1]
    dz = cen[rows, 2] - cen[cols, 2]
    dist = np.sqrt(dx * dx + dy * dy + dz * dz)
    slot_of = {(int(r), int(c)): s for s, (r, c) in enumerate(zip(rows, cols))}
    rev = np.array([slot_of[(int(c), int(r))] for r, c in zip(rows, cols)], dtype=np.int64)
    return dict(q=q, n=n, vol=vol, centroid=cen, row_ptr=row_ptr, row=rows.astype(np.int64),
                col=cols.astype(np.int64), S=S, dist=dist, rev=rev)


def initial_theta(cg: dict) -> np.ndarray:
    """theta_ij = S_ij / d_ij per ordered pair (Sec. V.B, reading P2)."""
    return cg["S"] / cg["dist"]


def restrict(labels: np.ndarray, q: int, m: np.ndarray) -> np.ndarray:
    """Mass of every primitive: the sum of its voxels' masses (the voxel-to-primitive mapping of
    Sec. V.A)."""
    return np.bincount(np.asarray(labels, dtype=np.int64), weights=np.asarray(m, dtype=np.float64), minlength=q)


def _flux_sum(cg: dict, theta: np.ndarray, m: np.ndarray) -> np.ndarray:
    """sum_{j in nb(i)} theta_ij (m_i / v_i - m_j / v_j) for every primitive i."""
    conc = m / cg["vol"]
    f = theta * (conc[cg["row"]] - conc[cg["col"]])
    return np.bincount(cg["row"], weights=f, minlength=cg["q"])


def scheme3(cg: dict, theta: np.ndarray, m: np.ndarray, c: float, nsteps: int = 1) -> np.ndarray:
    """Explicit PNGM step (Scheme 3): m_i <- m_i - c sum_j theta_ij (m_i/v_i - m_j/v_j), c = Dc dt."""
    m = np.asarray(m, dtype=np.float64).copy()
    for _ in range(nsteps):
        m = m - c * _flux_sum(cg, theta, m)
    return m


def scheme4_matrix(cg: dict, theta: np.ndarray, c: float) -> np.ndarray:
    """Dense B with Scheme 4 written as B m^{k+1} = m^k: B = I + c L_theta V^{-1}."""
    q = cg["q"]
    L = np.zeros((q, q))
    np.add.at(L, (cg["row"], cg["row"]), theta)
    np.add.at(L, (cg["row"], cg["col"]), -theta)
    return np.eye(q) + c * L / cg["vol"][None, :]


def scheme4(cg: dict, theta: np.ndarray, m: np.ndarray, c: float, nsteps: int = 1) -> np.ndarray:
    """Implicit PNGM step (Scheme 4) by a dense solve of B m^{k+1} = m^k."""
    B = scheme4_matrix(cg, theta, c)
    m = np.asarray(m, dtype=np.float64).copy()
    for _ in range(nsteps):
        m = np.linalg.solve(B, m)
    return m


def objective(kind: int, cg: dict, theta: np.ndarray, X: np.ndarray, Y: np.ndarray, c: float,
              tied: bool = False):
    """Objective 1 (kind=1) or 2 (kind=2) over the l pairs (X[p], Y[p]) and its gradient per slot
    (Sec. V.A; readings P3-P5).  Returns (loss, grad)."""
    X = np.atleast_2d(np.asarray(X, dtype=np.float64))
    Y = np.atleast_2d(np.asarray(Y, dtype=np.float64))
    l, q = X.shape
    row, col, v = cg["row"], cg["col"], cg["vol"]
    loss = 0.0
    grad = np.zeros_like(theta)
    for p in range(l):
        x, y = X[p], Y[p]
        if kind == 1:
            # r_i = y_i - x_i + c sum_j theta_ij (x_i/v_i - x_j/v_j); dr_i/dtheta_ij = c (x_i/v_i - x_j/v_j)
            r = y - x + c * _flux_sum(cg, theta, x)
            dr = c * (x[row] / v[row] - x[col] / v[col])
        elif kind == 2:
            # r_i = x_i - y_i - c sum_j theta_ij (y_i/v_i - y_j/v_j); dr_i/dtheta_ij = -c (y_i/v_i - y_j/v_j)
            r = x - y - c * _flux_sum(cg, theta, y)
            dr = -c * (y[row] / v[row] - y[col] / v[col])
        else:
            raise ValueError("objective must be 1 or 2")
        loss += np.sum(r * r) / (l * q)
        grad += 2.0 * dr * r[row] / (l * q)
    if tied:
        grad = grad + grad[cg["rev"]]
    return loss, grad


def sgd_step(kind: int, cg: dict, theta: np.ndarray, X: np.ndarray, Y: np.ndarray, c: float, lr: float,
             tied: bool = False, theta_min: float = -np.inf):
    """One normalised-gradient update (reading P6), bounded below by theta_min.  Returns (new
    theta, loss before the update)."""
    loss, g = objective(kind, cg, theta, X, Y, c, tied=tied)
    step = np.where(g > 0, 1.0, np.where(g < 0, -1.0, 0.0))
    return np.maximum(theta - lr * step, theta_min), loss
