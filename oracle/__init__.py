"""FP64 CPU oracle of the voxel-graph method (arXiv 2406.04177) -- TEST INFRASTRUCTURE.

Only the test suite, the package smoke check and the benchmark's CPU-baseline leg may import this
package.  It shares no code with the CUDA library: the arithmetic lives in `vga_oracle.c`
(plain C, FP64, adjacency lists), and this module only compiles it with gcc and marshals numpy
arrays through ctypes.

Functions and the passages they restate:
  graph_build          Sec. II.A (pore set V, 6-connected edges, Fig. 2), Sec. III
  transform_sync       Sec. II.C eq. 3 with the Appendix A clamps (synchronous)
  transform_async      Appendix A sequential listing (asynchronous)
  explicit_run         Scheme 1 (Sec. II.B.3a) after the transformation, per Sec. III
  implicit_run         Scheme 2 (Sec. II.B.3b) by Jacobi-PCG (Sec. III)
  pcg_solve            the PCG of Sec. III on B = I + D dt L_g
  totals               compartment masses (Sec. IV.C figures), Neumaier summation
  adjoint_run          reverse of the explicit synchronous step, gradients in the structure of
                       the Sec. V.A closed forms (weights) plus rates and D

Every function is pinned by `tests/test_oracle_*.py` against closed forms, dense linear algebra,
scipy routines, brute force and values fixed by the paper.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vga_oracle.c")
_LIB_PATH = os.path.join(_HERE, "libvga_oracle.so")
_lock = threading.Lock()
_lib = None

PARAM_NAMES = ("D", "dt", "rho", "mu", "beta", "v_som", "v_fom", "v_dom", "K_dom")
GRAD_NAMES = ("D", "rho", "mu", "beta", "v_som", "v_fom", "v_dom", "K_dom")


class _Params(C.Structure):
    _fields_ = [(k, C.c_double) for k in PARAM_NAMES]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP on).  Returns the library path."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"],
                       check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            P, I64, I32, D = C.c_void_p, C.c_int64, C.c_int32, C.c_double
            lib.vo_graph_build.restype = I64
            lib.vo_graph_build.argtypes = [P, C.c_int, C.c_int, C.c_int, C.c_int, P, P, P, P, P]
            lib.vo_transform_sync.argtypes = [P, P]
            lib.vo_transform_async.argtypes = [P, P]
            lib.vo_diffuse_explicit.argtypes = [I64, P, P, D, P, P]
            lib.vo_pcg_solve.restype = C.c_int
            lib.vo_pcg_solve.argtypes = [I64, P, P, D, P, P, D, C.c_int, P, P]
            lib.vo_explicit_run.restype = C.c_int
            lib.vo_explicit_run.argtypes = [I64, P, P, P, C.c_int, P, I64]
            lib.vo_implicit_run.restype = C.c_int
            lib.vo_implicit_run.argtypes = [I64, P, P, P, C.c_int, P, I64, D, C.c_int, P, P]
            lib.vo_totals.argtypes = [I64, P, P]
            lib.vo_adjoint_run.restype = C.c_int
            lib.vo_adjoint_run.argtypes = [I64, P, P, P, P, I64, I64, P, P, P, P, P]
            lib.vo_num_threads.restype = C.c_int
            lib.vo_set_num_threads.argtypes = [C.c_int]
            lib.vo_ticks_before.restype = I64
            lib.vo_ticks_before.argtypes = [I64, D, D]
            lib.vo_run_subcycled.restype = C.c_int
            lib.vo_run_subcycled.argtypes = [I64, P, P, P, C.c_int, C.c_int, P, I64, D, I64, D, C.c_int, P]
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _params(p: dict) -> _Params:
    return _Params(*[float(p[k]) for k in PARAM_NAMES])


def num_threads() -> int:
    """OpenMP threads the oracle's parallel loops use."""
    return int(_load().vo_num_threads())


def set_num_threads(k: int) -> None:
    """Thread count of the oracle's parallel loops from now on (k >= 1)."""
    _load().vo_set_num_threads(int(k))


class Graph:
    """Result of `graph_build`: node count, labels, raster index of each node, neighbour table."""

    def __init__(self, shape, labels, n_components, largest, voxel_of_node, nbr):
        self.shape = shape
        self.labels = labels
        self.n_components = n_components
        self.largest = largest
        self.voxel_of_node = voxel_of_node
        self.nbr = nbr

    @property
    def n(self) -> int:
        return int(self.voxel_of_node.size)


def graph_build(img: np.ndarray, keep_largest: bool = True) -> Graph:
    """Voxel graph of Sec. II.A: nodes = pore voxels (I == 0), edges = face neighbours."""
    img = np.ascontiguousarray(img, dtype=np.uint8)
    nz, ny, nx = img.shape
    nvox = img.size
    labels = np.empty(nvox, dtype=np.int32)
    von = np.empty(max(nvox, 1), dtype=np.int64)
    nbr = np.empty(max(6 * nvox, 6), dtype=np.int32)
    ncomp = np.zeros(1, dtype=np.int32)
    largest = np.zeros(1, dtype=np.int32)
    n = _load().vo_graph_build(_ptr(img), nx, ny, nz, int(bool(keep_largest)), _ptr(labels),
                               _ptr(ncomp), _ptr(largest), _ptr(von), _ptr(nbr))
    if n < 0:
        raise MemoryError("oracle graph build failed")
    return Graph((nz, ny, nx), labels.reshape(nz, ny, nx), int(ncomp[0]), int(largest[0]),
                 von[:n].copy(), nbr[: 6 * n].reshape(n, 6).copy())


def transform_sync(p: dict, x) -> np.ndarray:
    """One synchronous transformation of one voxel (5 masses)."""
    v = np.array(x, dtype=np.float64).copy()
    pp = _params(p)
    _load().vo_transform_sync(C.byref(pp), _ptr(v))
    return v


def transform_async(p: dict, x) -> np.ndarray:
    """One asynchronous transformation of one voxel (5 masses)."""
    v = np.array(x, dtype=np.float64).copy()
    pp = _params(p)
    _load().vo_transform_async(C.byref(pp), _ptr(v))
    return v


def _g6(g6, n):
    if g6 is None:
        return None
    g = np.ascontiguousarray(g6, dtype=np.float64).reshape(n, 6)
    return g


def explicit_run(nbr: np.ndarray, p: dict, X: np.ndarray, nsteps: int, g6=None,
                 transform: int = 0) -> np.ndarray:
    """`nsteps` steps of transformation + Scheme 1 from state X (5, n); returns the new state."""
    nbr = np.ascontiguousarray(nbr, dtype=np.int32)
    n = nbr.shape[0]
    Xo = np.ascontiguousarray(X, dtype=np.float64).reshape(5, n).copy()
    g = _g6(g6, n)
    pp = _params(p)
    if _load().vo_explicit_run(n, _ptr(nbr), _ptr(g), C.byref(pp), int(transform), _ptr(Xo), int(nsteps)):
        raise MemoryError("oracle explicit run failed")
    return Xo


def run_subcycled(nbr, p: dict, X: np.ndarray, nsteps: int, dt_transform: float, step0: int = 0,
                  g6=None, transform: int = 0, scheme: int = 0, rtol: float = 1e-10, maxit: int = 10000) -> np.ndarray:
    """Steps of p['dt'] (scheme 0: Scheme 1, scheme 1: Scheme 2 by PCG) with the transformation on
    its own step dt_transform (Sec. III, global-clock reading); step0 = diffusion steps already taken."""
    nbr = np.ascontiguousarray(nbr, dtype=np.int32)
    n = nbr.shape[0]
    Xo = np.ascontiguousarray(X, dtype=np.float64).reshape(5, n).copy()
    pp = _params(p)
    it = C.c_int64(0)
    st = _load().vo_run_subcycled(n, _ptr(nbr), _ptr(_g6(g6, n)), C.byref(pp), int(transform), int(scheme), _ptr(Xo),
                                  int(nsteps), float(dt_transform), int(step0), float(rtol), int(maxit), C.byref(it))
    if st < 0:
        raise MemoryError("oracle sub-cycled run failed")
    if st > 0:
        raise RuntimeError("oracle PCG did not converge")
    return Xo


def ticks_before(k: int, dt: float, dt_transform: float) -> int:
    """Transformation ticks in [0, k dt) under the global-clock reading."""
    return int(_load().vo_ticks_before(int(k), float(dt), float(dt_transform)))


def diffuse_explicit(nbr, c: float, m: np.ndarray, g6=None) -> np.ndarray:
    """One Scheme 1 diffusion step m <- Q_g m with D dt = c (no transformation)."""
    nbr = np.ascontiguousarray(nbr, dtype=np.int32)
    n = nbr.shape[0]
    m = np.ascontiguousarray(m, dtype=np.float64)
    out = np.empty_like(m)
    _load().vo_diffuse_explicit(n, _ptr(nbr), _ptr(_g6(g6, n)), float(c), _ptr(m), _ptr(out))
    return out


def pcg_solve(nbr, c: float, b: np.ndarray, x0=None, rtol: float = 1e-12, maxit: int = 10000,
              g6=None):
    """Solve (I + c L_g) x = b by Jacobi-PCG.  Returns (x, status, iterations, relres)."""
    nbr = np.ascontiguousarray(nbr, dtype=np.int32)
    n = nbr.shape[0]
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = (b.copy() if x0 is None else np.ascontiguousarray(x0, dtype=np.float64).copy())
    it = np.zeros(1, dtype=np.int32)
    rr = np.zeros(1, dtype=np.float64)
    s = _load().vo_pcg_solve(n, _ptr(nbr), _ptr(_g6(g6, n)), float(c), _ptr(b), _ptr(x),
                             float(rtol), int(maxit), _ptr(it), _ptr(rr))
    if s < 0:
        raise MemoryError("oracle pcg failed")
    return x, int(s), int(it[0]), float(rr[0])


def implicit_run(nbr, p: dict, X: np.ndarray, nsteps: int, rtol: float = 1e-12,
                 maxit: int = 10000, g6=None, transform: int = 0):
    """`nsteps` steps of transformation + Scheme 2.  Returns (X, status, total_iters, worst_relres)."""
    nbr = np.ascontiguousarray(nbr, dtype=np.int32)
    n = nbr.shape[0]
    Xo = np.ascontiguousarray(X, dtype=np.float64).reshape(5, n).copy()
    tot = np.zeros(1, dtype=np.int64)
    worst = np.zeros(1, dtype=np.float64)
    pp = _params(p)
    s = _load().vo_implicit_run(n, _ptr(nbr), _ptr(_g6(g6, n)), C.byref(pp), int(transform),
                                _ptr(Xo), int(nsteps), float(rtol), int(maxit), _ptr(tot), _ptr(worst))
    if s < 0:
        raise MemoryError("oracle implicit run failed")
    return Xo, int(s), int(tot[0]), float(worst[0])


def totals(X: np.ndarray) -> np.ndarray:
    """Per-compartment total masses of a (5, n) state."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    n = X.shape[1]
    out = np.zeros(5, dtype=np.float64)
    _load().vo_totals(n, _ptr(X), _ptr(out))
    return out


def adjoint_run(nbr, p: dict, X0: np.ndarray, nsteps: int, lamN: np.ndarray, ckpt: int = 100,
                g6=None, want_gface: bool = False):
    """Reverse of `nsteps` explicit synchronous steps.  Returns a dict with XN, lam0 (dL/dX0),
    grad (dict over GRAD_NAMES) and, if requested, gface (n, 6)."""
    nbr = np.ascontiguousarray(nbr, dtype=np.int32)
    n = nbr.shape[0]
    X0 = np.ascontiguousarray(X0, dtype=np.float64).reshape(5, n)
    lamN = np.ascontiguousarray(lamN, dtype=np.float64).reshape(5, n)
    XN = np.empty((5, n))
    lam0 = np.empty((5, n))
    grad = np.zeros(8)
    gface = np.zeros((n, 6)) if want_gface else None
    pp = _params(p)
    s = _load().vo_adjoint_run(n, _ptr(nbr), _ptr(_g6(g6, n)), C.byref(pp), _ptr(X0), int(nsteps),
                               int(ckpt), _ptr(lamN), _ptr(XN), _ptr(lam0), _ptr(grad), _ptr(gface))
    if s < 0:
        raise MemoryError("oracle adjoint failed")
    out = dict(XN=XN, lam0=lam0, grad=dict(zip(GRAD_NAMES, grad.tolist())))
    if want_gface:
        out["gface"] = gface
    return out


# ---------------------------------------------------------------------------------------------
# Block conductances (Sec. V.A weighted flux, voxel form) and the block-mass objective.
# ---------------------------------------------------------------------------------------------
def block_grid(shape, bs: int):
    """Number of blocks (nbz, nby, nbx) of side `bs` covering an image of `shape`."""
    return tuple(-(-int(s) // bs) for s in shape)


def interface_count(nb) -> int:
    nbz, nby, nbx = nb
    return nbz * nby * (nbx - 1) + nbz * (nby - 1) * nbx + (nbz - 1) * nby * nbx


def edge_interface(shape, bs: int, voxel_of_node, nbr):
    """For every (node, slot) pair, the index of the block interface the edge crosses, or -1 when
    the edge stays inside a block (or does not exist).  Interfaces are numbered x-normal first
    ((nbz, nby, nbx-1) in C order), then y-normal ((nbz, nby-1, nbx)), then z-normal
    ((nbz-1, nby, nbx)); an edge is attributed to the interface on the high side of its lower block.
    """
    nz, ny, nx = shape
    nbz, nby, nbx = block_grid(shape, bs)
    v = np.asarray(voxel_of_node, dtype=np.int64)
    x, y, z = v % nx, (v // nx) % ny, v // (nx * ny)
    bx, by, bz = x // bs, y // bs, z // bs
    offx = 0
    offy = nbz * nby * (nbx - 1)
    offz = offy + nbz * (nby - 1) * nbx
    out = np.full((v.size, 6), -1, dtype=np.int64)
    exists = np.asarray(nbr) >= 0
    # slot 0 (-x): crosses when x % bs == 0 and x > 0; lower block is bx-1
    m = exists[:, 0] & (x % bs == 0)
    out[m, 0] = offx + (bz[m] * nby + by[m]) * (nbx - 1) + (bx[m] - 1)
    m = exists[:, 1] & ((x + 1) % bs == 0)
    out[m, 1] = offx + (bz[m] * nby + by[m]) * (nbx - 1) + bx[m]
    m = exists[:, 2] & (y % bs == 0)
    out[m, 2] = offy + (bz[m] * (nby - 1) + (by[m] - 1)) * nbx + bx[m]
    m = exists[:, 3] & ((y + 1) % bs == 0)
    out[m, 3] = offy + (bz[m] * (nby - 1) + by[m]) * nbx + bx[m]
    m = exists[:, 4] & (z % bs == 0)
    out[m, 4] = offz + ((bz[m] - 1) * nby + by[m]) * nbx + bx[m]
    m = exists[:, 5] & ((z + 1) % bs == 0)
    out[m, 5] = offz + (bz[m] * nby + by[m]) * nbx + bx[m]
    return out


def block_face_weights(shape, bs: int, voxel_of_node, nbr, theta) -> np.ndarray:
    """Per-slot edge conductances g (n, 6): theta of the crossed interface, 1 inside a block."""
    ei = edge_interface(shape, bs, voxel_of_node, nbr)
    g = np.ones(ei.shape, dtype=np.float64)
    m = ei >= 0
    g[m] = np.asarray(theta, dtype=np.float64)[ei[m]]
    return g


def block_theta_grad(shape, bs: int, voxel_of_node, nbr, gface, n_interfaces: int) -> np.ndarray:
    """dL/dtheta from per-edge gradients: each edge is counted once (from its lower node)."""
    ei = edge_interface(shape, bs, voxel_of_node, nbr)
    own = np.zeros(ei.shape, dtype=bool)
    own[:, 1] = own[:, 3] = own[:, 5] = True  # the +x/+y/+z slot holds each edge exactly once
    m = (ei >= 0) & own
    out = np.zeros(n_interfaces)
    np.add.at(out, ei[m], np.asarray(gface)[m])
    return out


def node_block(shape, bs: int, voxel_of_node) -> np.ndarray:
    """Block index (C order over (nbz, nby, nbx)) of every node."""
    nz, ny, nx = shape
    nbz, nby, nbx = block_grid(shape, bs)
    v = np.asarray(voxel_of_node, dtype=np.int64)
    x, y, z = v % nx, (v // nx) % ny, v // (nx * ny)
    return ((z // bs) * nby + (y // bs)) * nbx + (x // bs)


def block_mass_loss(shape, bs: int, voxel_of_node, X, target, comps=(1, 4)):
    """L = sum over blocks and the listed compartments (default DOM, CO2) of
    (block mass - target)^2, and dL/dX (5, n).  target has shape (len(comps), n_blocks)."""
    nb = block_grid(shape, bs)
    nblk = nb[0] * nb[1] * nb[2]
    b = node_block(shape, bs, voxel_of_node)
    X = np.asarray(X, dtype=np.float64)
    lam = np.zeros_like(X)
    L = 0.0
    for t, c in enumerate(comps):
        M = np.bincount(b, weights=X[c], minlength=nblk)
        r = M - target[t]
        L += float(np.sum(r * r))
        lam[c] = 2.0 * r[b]
    return L, lam


def block_masses(shape, bs: int, voxel_of_node, X, comps=(1, 4)) -> np.ndarray:
    """Block masses (len(comps), n_blocks) of the listed compartments."""
    nb = block_grid(shape, bs)
    nblk = nb[0] * nb[1] * nb[2]
    b = node_block(shape, bs, voxel_of_node)
    X = np.asarray(X, dtype=np.float64)
    return np.stack([np.bincount(b, weights=X[c], minlength=nblk) for c in comps])
