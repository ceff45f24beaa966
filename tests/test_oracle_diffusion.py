"""Pins of the oracle's Scheme 1 / Scheme 2 diffusion (Sec. II.B) against dense linear algebra,
the matrix exponential of Sec. II.B.2, conservation, per-component steady states, the 1D slab
reduction and its reflected-erfc continuum solution, and the positivity limit of Sec. IV.C."""
import math

import numpy as np
import pytest
from scipy.linalg import expm
from scipy.special import erfc

from tests.helpers import dense_laplacian, rel_l2

ZERO_RATES = dict(rho=0.0, mu=0.0, beta=0.5, v_som=0.0, v_fom=0.0, v_dom=0.0, K_dom=1.0)


def _diff_params(D, dt):
    return dict(D=D, dt=dt, **ZERO_RATES)


def _tiny_mask(seed, shape=(3, 4, 5), por=0.55):
    rng = np.random.default_rng(seed)
    return (rng.random(shape) >= por).astype(np.uint8)


def _state_with_dom(m):
    X = np.zeros((5, m.size))
    X[1] = m
    return X


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_scheme1_equals_dense_Q_power(oracle_lib, seed):
    img = _tiny_mask(seed)
    g = oracle_lib.graph_build(img, keep_largest=False)
    L = dense_laplacian(img == 0)
    D, dt, k = 2.0, 0.05, 37
    Q = np.eye(g.n) - D * dt * L  # Scheme 1 matrix
    m0 = np.random.default_rng(seed).random(g.n)
    X = oracle_lib.explicit_run(g.nbr, _diff_params(D, dt), _state_with_dom(m0), k)
    ref = np.linalg.matrix_power(Q, k) @ m0
    assert rel_l2(X[1], ref) < 1e-13


def test_weighted_scheme1_equals_dense(oracle_lib):
    img = _tiny_mask(9, shape=(4, 4, 4), por=0.4)
    g = oracle_lib.graph_build(img, keep_largest=False)
    rng = np.random.default_rng(4)
    # symmetric random conductance per edge
    n = g.n
    W = np.zeros((n, n))
    for i in range(n):
        for d in (1, 3, 5):
            j = g.nbr[i, d]
            if j >= 0:
                W[i, j] = W[j, i] = rng.uniform(0.2, 1.8)
    g6 = np.array([[W[i, g.nbr[i, d]] if g.nbr[i, d] >= 0 else 0.0 for d in range(6)] for i in range(n)])
    L = np.diag(W.sum(1)) - W
    D, dt, k = 1.0, 0.08, 25
    m0 = rng.random(n)
    X = oracle_lib.explicit_run(g.nbr, _diff_params(D, dt), _state_with_dom(m0), k, g6=g6)
    assert rel_l2(X[1], np.linalg.matrix_power(np.eye(n) - D * dt * L, k) @ m0) < 1e-13
    Xi, s, it, rr = oracle_lib.implicit_run(g.nbr, _diff_params(D, dt), _state_with_dom(m0), k, g6=g6)
    B = np.eye(n) + D * dt * L
    ref = m0.copy()
    for _ in range(k):
        ref = np.linalg.solve(B, ref)
    assert s == 0 and rel_l2(Xi[1], ref) < 1e-10


@pytest.mark.parametrize("seed", [4, 5])
def test_scheme2_equals_dense_solve(oracle_lib, seed):
    img = _tiny_mask(seed)
    g = oracle_lib.graph_build(img, keep_largest=False)
    L = dense_laplacian(img == 0)
    D, dt, k = 3.0, 0.5, 6  # D dt far above the explicit limit: Scheme 2 is unconditionally stable
    B = np.eye(g.n) + D * dt * L
    m0 = np.random.default_rng(seed).random(g.n)
    X, s, it, rr = oracle_lib.implicit_run(g.nbr, _diff_params(D, dt), _state_with_dom(m0), k, rtol=1e-14)
    ref = m0.copy()
    for _ in range(k):
        ref = np.linalg.solve(B, ref)
    assert s == 0
    assert rel_l2(X[1], ref) < 1e-12
    assert np.all(X[1] >= -1e-15)


def test_schemes_converge_first_order_to_expm(oracle_lib):
    """M(t) = exp(-D L t) M(0) (Sec. II.B.2); forward and backward Euler are first order in dt."""
    img = _tiny_mask(7, shape=(2, 4, 4), por=0.3)
    g = oracle_lib.graph_build(img, keep_largest=True)
    L = dense_laplacian(np.isin(np.arange(img.size), g.voxel_of_node).reshape(img.shape))
    m0 = np.random.default_rng(7).random(g.n)
    D, T = 1.0, 0.4
    exact = expm(-D * L * T) @ m0
    errs_e, errs_i = [], []
    for nsteps in (40, 80, 160):
        p = _diff_params(D, T / nsteps)
        Xe = oracle_lib.explicit_run(g.nbr, p, _state_with_dom(m0), nsteps)
        Xi, _, _, _ = oracle_lib.implicit_run(g.nbr, p, _state_with_dom(m0), nsteps, rtol=1e-14)
        errs_e.append(np.linalg.norm(Xe[1] - exact))
        errs_i.append(np.linalg.norm(Xi[1] - exact))
    for errs in (errs_e, errs_i):
        r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
        assert 1.85 < r1 < 2.15 and 1.9 < r2 < 2.1
    # the two Euler schemes bracket the exact solution from opposite sides at leading order
    assert errs_e[-1] < 0.02 * np.linalg.norm(exact)


def test_conservation_and_component_steady_state(oracle_lib):
    """The Laplacian has zero row and column sums, so Scheme 1 and Scheme 2 conserve mass exactly;
    on each connected component the state relaxes to the component mean (Sec. II.B.2)."""
    import synth

    img = synth.pore_mask((10, 10, 10), 0.22, 3)
    g = oracle_lib.graph_build(img, keep_largest=False)
    assert g.n_components >= 3
    lab = g.labels.ravel()[g.voxel_of_node]
    m0 = np.random.default_rng(3).random(g.n)
    p = _diff_params(1.0, 0.16)
    X = oracle_lib.explicit_run(g.nbr, p, _state_with_dom(m0), 200)
    assert abs(X[1].sum() - m0.sum()) <= 1e-12 * m0.sum()
    Xi, s, _, _ = oracle_lib.implicit_run(g.nbr, _diff_params(1.0, 2.0), _state_with_dom(m0), 50)
    assert abs(Xi[1].sum() - m0.sum()) <= 1e-11 * m0.sum()
    Xl = oracle_lib.explicit_run(g.nbr, p, _state_with_dom(m0), 20000)
    for c in range(g.n_components):
        sel = lab == c
        assert np.allclose(Xl[1][sel], m0[sel].mean(), rtol=1e-9, atol=0)


def _path_scheme1(m, c, k):
    """Scheme 1 on a path graph, written as an explicit 1D loop (independent of the oracle)."""
    m = m.copy()
    for _ in range(k):
        new = m.copy()
        for i in range(m.size):
            acc = 0.0
            if i > 0:
                acc += m[i] - m[i - 1]
            if i < m.size - 1:
                acc += m[i] - m[i + 1]
            new[i] = m[i] - c * acc
        m = new
    return m


def test_slab_reduces_to_1d_path(oracle_lib):
    """Sec. IV.B experiment set-up: all pore voxels of layers z = 0, 1 hold the same mass.  In an
    open box every layer stays uniform, so the 3D graph evolves like a path graph along z."""
    img = np.zeros((24, 5, 6), dtype=np.uint8)
    g = oracle_lib.graph_build(img)
    nlay = 5 * 6
    m0 = np.zeros(g.n)
    m0[: 2 * nlay] = 1.0 / (2 * nlay)
    c, k = 0.15, 120
    X = oracle_lib.explicit_run(g.nbr, _diff_params(c, 1.0), _state_with_dom(m0), k)
    layers = X[1].reshape(24, nlay)
    assert np.allclose(layers, layers[:, :1], rtol=1e-12, atol=1e-300)  # layers stay uniform
    ref = _path_scheme1(np.repeat([1.0 / (2 * nlay), 0.0], [2, 22]), c, k)
    assert rel_l2(layers[:, 0], ref) < 1e-12


def _reflected_slab(z, t, D, a, Lz, nimg=6):
    """Continuum solution of dC/dt = D d2C/dz2 on [0, Lz] with no-flux walls and C(z,0) = 1 on
    [0, a): the erfc slab solution with its images in both walls."""
    s = 2.0 * math.sqrt(D * t)
    out = np.zeros_like(z)
    for k in range(-nimg, nimg + 1):
        # source [2kLz - a, 2kLz + a) is the slab and its mirror, repeated with period 2Lz
        lo, hi = 2 * k * Lz - a, 2 * k * Lz + a
        out += 0.5 * (erfc((lo - z) / s) - erfc((hi - z) / s))
    return out


def test_slab_matches_reflected_erfc(oracle_lib):
    """Layer profile of the slab experiment (Sec. IV.B set-up) against the continuum solution.
    Layer centres at z + 1/2 and a slab of a layers.  Refining h -> h/2 at fixed D dt / h^2 (so dt
    shrinks like h^2) must shrink the gap like h^2: the scheme is O(dt + h^2)."""
    errs = []
    for nz, a, T in ((48, 2, 60.0), (96, 4, 240.0)):
        img = np.zeros((nz, 2, 2), dtype=np.uint8)
        g = oracle_lib.graph_build(img)
        m0 = np.zeros(g.n)
        m0[: a * 4] = 1.0
        c = 0.05
        k = int(round(T / c))
        X = oracle_lib.explicit_run(g.nbr, _diff_params(1.0, c), _state_with_dom(m0), k)
        prof = X[1].reshape(nz, 4)[:, 0]
        exact = _reflected_slab(np.arange(nz) + 0.5, T, 1.0, float(a), float(nz))
        errs.append(np.abs(prof - exact).max())
        assert abs(X[1].sum() - 4.0 * a) < 1e-12 * a
    assert errs[0] < 5e-4
    assert 0.2 < errs[1] / errs[0] < 0.3


def test_positivity_limit(oracle_lib):
    """Q has nonnegative entries iff D dt deg(i) <= 1 (Sec. II.B.3a).  At the paper's 0.1 s step
    (Sec. IV.C, with D = 100950 voxel^2/day) a spike stays nonnegative; above 1/(6D) an interior
    spike turns negative after one step."""
    img = np.zeros((5, 5, 5), dtype=np.uint8)
    g = oracle_lib.graph_build(img)
    centre = 2 * 25 + 2 * 5 + 2
    m0 = np.zeros(g.n)
    m0[centre] = 1.0
    D = 100950.0
    dt_paper = 0.1 / 86400.0
    X = oracle_lib.explicit_run(g.nbr, _diff_params(D, dt_paper), _state_with_dom(m0), 50)
    assert X[1].min() >= 0.0
    dt_bad = 1.1 / (6 * D)
    X = oracle_lib.explicit_run(g.nbr, _diff_params(D, dt_bad), _state_with_dom(m0), 1)
    assert X[1][centre] < 0.0
    assert math.isclose(X[1][centre], 1.0 - 6 * 1.1 / 6, rel_tol=1e-12)


def test_pcg_status_zero_rhs_and_preconditioner(oracle_lib):
    """PCG of Sec. III: zero right-hand side gives zero; an iteration cap reports non-convergence;
    the Jacobi preconditioner makes a graph whose B is diagonal converge in one iteration."""
    img = _tiny_mask(3)
    g = oracle_lib.graph_build(img, keep_largest=False)
    x, s, it, rr = oracle_lib.pcg_solve(g.nbr, 1.5, np.zeros(g.n))
    assert s == 0 and np.all(x == 0)
    b = np.random.default_rng(1).random(g.n)
    x, s, it, rr = oracle_lib.pcg_solve(g.nbr, 1.5, b, x0=np.zeros(g.n), rtol=1e-14, maxit=1)
    assert s == 1 and it == 1 and rr > 1e-14
    iso = -np.ones((5, 6), dtype=np.int32)  # five isolated nodes: B = I
    x, s, it, rr = oracle_lib.pcg_solve(iso, 1.5, np.arange(1.0, 6.0), x0=np.zeros(5), rtol=1e-14)
    assert s == 0 and it == 1 and np.allclose(x, np.arange(1.0, 6.0), rtol=1e-15)
