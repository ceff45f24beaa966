"""Seeded synthetic inputs shared by the FP64 oracle tests, the GPU tests and the benchmark.

This module builds INPUTS only (pore images, initial masses, parameter sets). It holds none of
the method's arithmetic: no graph construction, no transformation, no diffusion. Both sides of
every parity check receive identical arrays from here.

Stand-in for the paper's data (Sec. IV.A): the Bullion Field sandy-loam micro-CT image (512^3
voxels of 24 um, 17% visible porosity, indicator-kriging segmentation) is not available, so a
pore image with the same size and porosity is drawn from a Gaussian-smoothed white-noise field.

Units: masses in micrograms of carbon, time in days, lengths in voxels (Sec. IV.C parameter list).
"""
from __future__ import annotations

import numpy as np

# --- Sec. IV.C parameter list (Arthrobacter sp. 9R); rates are per day ------------------------
RHO = 0.2        # relative respiration rate
MU = 0.5         # relative mortality rate
BETA = 0.55      # fraction of dead biomass returned to DOM
V_SOM = 0.01     # SOM hydrolysis rate
V_FOM = 0.3      # FOM hydrolysis rate
V_DOM = 9.6      # maximum relative growth rate of MB
D_DOM = 100950.0  # DOM diffusion coefficient, voxel^2 per day
# K_DOM = 0.001 gC per g of water.  The state is a mass per voxel, so the half-saturation
# constant is expressed per voxel of water: (24e-4 cm)^3 * 1 g/cm^3 * 1e-3 gC/g = 1.3824e-11 gC
# = 1.3824e-5 ug C.
VOXEL_CM = 24e-4
K_DOM_VOXEL = VOXEL_CM ** 3 * 1.0 * 1e-3 * 1e6

# Sec. IV.C initial condition: 289.5 ug of DOM and 2.8132 ug of MB carbon over the pore space of
# the 512^3 image at 17% porosity.
M_DOM_TOTAL = 289.5
M_MB_TOTAL = 2.8132
N_PORE_PAPER = 22817014  # round(0.17 * 512^3)

SCHEME_EXPLICIT = 0
SCHEME_IMPLICIT_PCG = 1
TRANSFORM_SYNC = 0
TRANSFORM_ASYNC = 1


def explicit_dt(D: float = D_DOM, safety: float = 0.9) -> float:
    """Time step (days) at `safety` times the positivity limit D*dt*6 <= 1 of Scheme 1 on a
    6-connected voxel graph (Sec. II.B.3a: the diagonal 1 - D dt deg(i) of Q must stay >= 0)."""
    return safety / (6.0 * D)


def paper_params(dt: float | None = None, scheme: int = SCHEME_EXPLICIT,
                 transform: int = TRANSFORM_SYNC, cg_rtol: float = 1e-8, cg_maxit: int = 500,
                 scale: dict | None = None) -> dict:
    """Parameter dictionary with the Sec. IV.C values.  `scale` multiplies named rates (used by
    the batched workload, which draws per-instance rates around these values)."""
    p = dict(D=D_DOM, dt=explicit_dt() if dt is None else dt, rho=RHO, mu=MU, beta=BETA,
             v_som=V_SOM, v_fom=V_FOM, v_dom=V_DOM, K_dom=K_DOM_VOXEL, scheme=scheme,
             transform=transform, cg_rtol=cg_rtol, cg_maxit=cg_maxit)
    if scale:
        for k, s in scale.items():
            p[k] = p[k] * s
    return p


def pore_mask(shape, porosity: float, seed: int, sigma: float = 2.0) -> np.ndarray:
    """Binary image I with 0 = pore and 1 = solid (Sec. II.A), C order [z][y][x].

    Field = i.i.d. N(0,1) float32 from PCG64(seed), smoothed by a separable Gaussian of width
    `sigma` voxels (truncated at 4 sigma, reflecting border).  The round(porosity * size) lowest
    field values become pore; ties at the threshold go to the lowest raster indices, so the pore
    count is exact.  Keeping the largest 6-connected component is NOT done here: it is part of the
    graph construction under test.
    """
    from scipy import ndimage

    nz, ny, nx = (int(s) for s in shape)
    size = nx * ny * nz
    rng = np.random.Generator(np.random.PCG64(seed))
    f = rng.standard_normal((nz, ny, nx), dtype=np.float32)
    if sigma > 0:
        f = ndimage.gaussian_filter(f, sigma=sigma, mode="reflect", truncate=4.0)
    flat = f.ravel()
    k = int(round(porosity * size))
    img = np.ones(size, dtype=np.uint8)
    if k <= 0:
        return img.reshape(nz, ny, nx)
    if k >= size:
        return np.zeros((nz, ny, nx), dtype=np.uint8)
    thr = np.partition(flat, k - 1)[k - 1]  # k-th smallest value
    below = flat < thr
    img[below] = 0
    need = k - int(below.sum())
    if need > 0:
        ties = np.flatnonzero(flat == thr)[:need]
        img[ties] = 0
    return img.reshape(nz, ny, nx)


def kept_mask_from_nodes(shape, voxel_of_node: np.ndarray) -> np.ndarray:
    """Dense boolean image of the graph's nodes, from the exported raster index of each node."""
    nz, ny, nx = shape
    kept = np.zeros(nx * ny * nz, dtype=bool)
    kept[np.asarray(voxel_of_node, dtype=np.int64)] = True
    return kept.reshape(nz, ny, nx)


def _face_neighbour_count(kept: np.ndarray) -> np.ndarray:
    """Number of face neighbours of each voxel that are in `kept` (inputs only: used to find pore
    voxels touching solid or the image border, where the paper seeds its bacterial spots)."""
    k = kept.astype(np.int8)
    c = np.zeros(kept.shape, dtype=np.int8)
    c[:, :, 1:] += k[:, :, :-1]
    c[:, :, :-1] += k[:, :, 1:]
    c[:, 1:, :] += k[:, :-1, :]
    c[:, :-1, :] += k[:, 1:, :]
    c[1:, :, :] += k[:-1, :, :]
    c[:-1, :, :] += k[1:, :, :]
    return c


def initial_masses(kept: np.ndarray, seed: int, dom_fraction: float = 0.05,
                   mb_fraction: float = 0.01, with_organic_matter: bool = False) -> np.ndarray:
    """Initial state X(0) as a (5, n) float64 array in node order (raster order of kept pores).

    Rows are (MB, DOM, SOM, FOM, CO2) = (x1..x5) of Sec. II.A.  Every value is exactly
    representable in float32, so an FP32 device state and an FP64 host state start identical.

    * DOM: `dom_fraction` of the nodes, drawn without replacement, each U(0, 2*mbar) with
      mbar = 289.5 ug / (dom_fraction * 22817014): the paper's mean DOM density (Sec. IV.C).
    * MB: round(mb_fraction * n) nodes drawn without replacement among the nodes with fewer than
      6 pore face neighbours (touching solid or the border), each U(0, 2 * 2.8132 ug /
      (mb_fraction * 22817014)).
    * SOM = FOM = CO2 = 0 (Sec. IV.C), unless `with_organic_matter`: then FOM = DOM in the same
      nodes and SOM = 0.1 * DOM, so that the FOM and SOM hydrolysis rates influence the outcome.
    """
    kept = np.asarray(kept, dtype=bool)
    flat = kept.ravel()
    n = int(flat.sum())
    X = np.zeros((5, n), dtype=np.float64)
    if n == 0:
        return X
    rng = np.random.Generator(np.random.PCG64(seed))
    n_dom = min(n, max(1, int(round(dom_fraction * n))))
    dom_nodes = rng.choice(n, size=n_dom, replace=False)
    mbar = M_DOM_TOTAL / (dom_fraction * N_PORE_PAPER)
    X[1, dom_nodes] = rng.uniform(0.0, 2.0 * mbar, size=n_dom)
    deg = _face_neighbour_count(kept).ravel()[flat]
    border = np.flatnonzero(deg < 6)
    n_mb = min(border.size, max(1, int(round(mb_fraction * n)))) if border.size else 0
    if n_mb:
        mb_nodes = rng.choice(border, size=n_mb, replace=False)
        mb_mean = M_MB_TOTAL / (mb_fraction * N_PORE_PAPER)
        X[0, mb_nodes] = rng.uniform(0.0, 2.0 * mb_mean, size=n_mb)
    if with_organic_matter:
        X[3] = X[1]
        X[2] = 0.1 * X[1]
    return X.astype(np.float32).astype(np.float64)


def random_masses(n: int, seed: int, scale: float = 1e-4, density: float = 0.3) -> np.ndarray:
    """Generic (5, n) float32-representable state for small tests: each compartment nonzero on a
    random `density` fraction of the nodes, U(0, 2*scale)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    X = rng.uniform(0.0, 2.0 * scale, size=(5, n))
    X *= rng.random((5, n)) < density
    return X.astype(np.float32).astype(np.float64)


def block_conductances(nb: tuple, seed: int, spread: float = 0.5) -> np.ndarray:
    """Target block-interface conductances theta* for the adjoint workload: one value per face
    between face-adjacent blocks, log-uniform in [1-spread, 1+spread].  Layout: three
    arrays concatenated, for interfaces normal to x ((nbz,nby,nbx-1)), y ((nbz,nby-1,nbx)) and z
    ((nbz-1,nby,nbx)), each in C order."""
    nbz, nby, nbx = nb
    count = nbz * nby * (nbx - 1) + nbz * (nby - 1) * nbx + (nbz - 1) * nby * nbx
    rng = np.random.Generator(np.random.PCG64(seed))
    lo, hi = np.log(1.0 - spread), np.log(1.0 + spread)
    return np.exp(rng.uniform(lo, hi, size=count)).astype(np.float32).astype(np.float64)


def batch_instances(count: int, seed: int, side_lo: int = 64, side_hi: int = 192,
                    por_lo: float = 0.10, por_hi: float = 0.35, rate_spread: float = 0.5):
    """Per-instance recipe of the batched workload: side lengths U{side_lo..side_hi}, porosities
    U(por_lo, por_hi), and each rate constant log-uniform in [1-rate_spread, 1+rate_spread] times
    the paper's value.  Returns a list of dicts (shape, porosity, mask seed, mass seed, params)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(count):
        side = int(rng.integers(side_lo, side_hi + 1))
        por = float(rng.uniform(por_lo, por_hi))
        lo, hi = np.log(1.0 - rate_spread), np.log(1.0 + rate_spread)
        scale = {k: float(np.exp(rng.uniform(lo, hi)))
                 for k in ("rho", "mu", "v_som", "v_fom", "v_dom")}
        out.append(dict(shape=(side, side, side), porosity=por, mask_seed=100 + i,
                        mass_seed=1000 + i, params=paper_params(scale=scale)))
    return out


def block_primitives(shape, voxel_of_node: np.ndarray, block_side: int):
    """Synthetic primitive partition for the coarse model: every node belongs to the cube of
    `block_side` voxels that contains it; non-empty cubes are numbered in raster order of the cube
    grid.  Returns (labels int32 per node, q)."""
    nz, ny, nx = (int(s) for s in shape)
    bs = int(block_side)
    nbx, nby = -(-nx // bs), -(-ny // bs)
    v = np.asarray(voxel_of_node, dtype=np.int64)
    x, y, z = v % nx, (v // nx) % ny, v // (nx * ny)
    blk = ((z // bs) * nby + y // bs) * nbx + x // bs
    used, labels = np.unique(blk, return_inverse=True)
    return labels.astype(np.int32), int(used.size)


def diffusion_params(dt_seconds: float = 0.1) -> dict:
    """Pure DOM diffusion (every transformation rate 0) with the Sec. IV.C coefficient and a step
    given in seconds (the coarse-model data of Sec. V.B use 0.1 s)."""
    p = paper_params(dt=dt_seconds / 86400.0)
    p.update(rho=0.0, mu=0.0, v_som=0.0, v_fom=0.0, v_dom=0.0)
    return p


def dom_scenario(n: int, seed: int, total: float = M_DOM_TOTAL, fraction: float = 0.05) -> np.ndarray:
    """One data scenario of Sec. V.B: a random total mass M0 ~ U(0.5, 1.5) * total spread over a
    random `fraction` of the nodes with U(0, 1) weights; DOM only.  Returns (5, n) float64."""
    rng = np.random.Generator(np.random.PCG64(seed))
    m0 = total * rng.uniform(0.5, 1.5)
    k = max(1, int(round(fraction * n)))
    idx = rng.choice(n, size=k, replace=False)
    w = rng.random(k)
    X = np.zeros((5, n))
    X[1, idx] = m0 * w / w.sum()
    return X
