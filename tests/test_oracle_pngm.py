"""Pins of the oracle's coarse primitive-graph model (Sec. V.A): the graph against brute force and
a hand-worked case, Schemes 3 and 4 against the pinned voxel schemes when every voxel is its own
primitive, conservation and steady states, the objectives' zeros, and the closed-form gradients
against central finite differences."""
import itertools

import numpy as np
import pytest

import synth
from oracle import pngm


def _graph(oracle_lib, shape, por, seed):
    img = synth.pore_mask(shape, por, seed)
    g = oracle_lib.graph_build(img, keep_largest=True)
    return img, g


def _random_labels(n, q, seed):
    rng = np.random.default_rng(seed)
    lab = rng.integers(0, q, n)
    lab[:q] = np.arange(q)  # every primitive non-empty
    return lab


def test_hand_worked_two_halves(oracle_lib):
    """A 2x2x2 all-pore image cut at x: two primitives of 4 voxels, 4 shared faces, centroids at
    x = 0 and x = 1, so S = 4, d = 1 and theta = 4."""
    img = np.zeros((2, 2, 2), dtype=np.uint8)
    g = oracle_lib.graph_build(img)
    x = g.voxel_of_node % 2
    cg = pngm.coarse_graph(g.nbr, g.voxel_of_node, img.shape, x, 2)
    assert list(cg["vol"]) == [4.0, 4.0]
    assert list(cg["row_ptr"]) == [0, 1, 2]
    assert list(cg["col"]) == [1, 0]
    assert list(cg["S"]) == [4.0, 4.0] and list(cg["dist"]) == [1.0, 1.0]
    assert list(pngm.initial_theta(cg)) == [4.0, 4.0]
    assert list(cg["rev"]) == [1, 0]


def test_graph_brute_force(oracle_lib):
    """Face counts and centroids by a double loop over node pairs on a small random case."""
    img, g = _graph(oracle_lib, (7, 6, 8), 0.6, 3)
    q = 9
    lab = _random_labels(g.n, q, 4)
    cg = pngm.coarse_graph(g.nbr, g.voxel_of_node, img.shape, lab, q)
    nz, ny, nx = img.shape
    coords = [(v % nx, (v // nx) % ny, v // (nx * ny)) for v in g.voxel_of_node]
    S = {}
    for i in range(g.n):
        for j in range(g.n):
            if i < j and sum(abs(a - b) for a, b in zip(coords[i], coords[j])) == 1 and lab[i] != lab[j]:
                key = (lab[i], lab[j])
                S[key] = S.get(key, 0) + 1
                S[(lab[j], lab[i])] = S.get((lab[j], lab[i]), 0) + 1
    got = {(int(r), int(c)): s for r, c, s in zip(cg["row"], cg["col"], cg["S"])}
    assert got == {k: float(v) for k, v in S.items()}
    for k in range(q):
        members = [coords[i] for i in range(g.n) if lab[i] == k]
        assert cg["vol"][k] == len(members)
        assert np.allclose(cg["centroid"][k], np.mean(members, axis=0), rtol=0, atol=1e-12)
    for s in range(len(cg["row"])):
        a, b = cg["row"][s], cg["col"][s]
        assert np.isclose(cg["dist"][s], np.linalg.norm(cg["centroid"][a] - cg["centroid"][b]), rtol=1e-15)
        assert cg["row"][cg["rev"][s]] == b and cg["col"][cg["rev"][s]] == a
    # CSR rows sorted by column
    for i in range(q):
        cols = cg["col"][cg["row_ptr"][i]:cg["row_ptr"][i + 1]]
        assert np.all(np.diff(cols) > 0)


def test_singleton_primitives_reduce_to_voxel_schemes(oracle_lib):
    """Every voxel its own primitive: v = 1, S = 1, d = 1, theta = 1, and Scheme 3 / Scheme 4 are
    Scheme 1 / Scheme 2 of the voxel graph."""
    img, g = _graph(oracle_lib, (9, 8, 10), 0.35, 5)
    cg = pngm.coarse_graph(g.nbr, g.voxel_of_node, img.shape, np.arange(g.n), g.n)
    th = pngm.initial_theta(cg)
    assert np.all(th == 1.0) and np.all(cg["vol"] == 1.0)
    m = np.random.default_rng(6).random(g.n)
    c = 0.15
    a = pngm.scheme3(cg, th, m, c, nsteps=3)
    b = m.copy()
    for _ in range(3):
        b = oracle_lib.diffuse_explicit(g.nbr, c, b)
    assert np.allclose(a, b, rtol=1e-14, atol=1e-16)
    if g.n <= 800:
        a4 = pngm.scheme4(cg, th, m, 1.5)
        b4 = oracle_lib.pcg_solve(g.nbr, 1.5, m, rtol=1e-14)[0]
        assert np.allclose(a4, b4, rtol=1e-11, atol=1e-14)


def test_conservation_and_steady_state(oracle_lib):
    """With tied conductances both schemes conserve total mass; equal concentrations m_i = k v_i
    are a fixed point of both."""
    img, g = _graph(oracle_lib, (10, 10, 10), 0.4, 7)
    q = 12
    lab = _random_labels(g.n, q, 8)
    cg = pngm.coarse_graph(g.nbr, g.voxel_of_node, img.shape, lab, q)
    th = pngm.initial_theta(cg)
    m = np.random.default_rng(9).random(q)
    c = 0.2 / max(np.bincount(cg["row"], weights=th, minlength=q) / cg["vol"])
    assert np.isclose(pngm.scheme3(cg, th, m, c, 5).sum(), m.sum(), rtol=1e-14)
    assert np.isclose(pngm.scheme4(cg, th, m, 10 * c, 5).sum(), m.sum(), rtol=1e-13)
    ss = 0.3 * cg["vol"]
    assert np.allclose(pngm.scheme3(cg, th, ss, c), ss, rtol=1e-15)
    assert np.allclose(pngm.scheme4(cg, th, ss, 10 * c), ss, rtol=1e-13)


def test_restriction_sums():
    lab = np.array([2, 0, 2, 1, 0])
    m = np.array([1.0, 2.0, 4.0, 8.0, 16.0])
    assert list(pngm.restrict(lab, 4, m)) == [18.0, 8.0, 5.0, 0.0]


def _setup_pairs(oracle_lib, q=10, seed=11):
    img, g = _graph(oracle_lib, (9, 9, 9), 0.45, seed)
    lab = _random_labels(g.n, q, seed + 1)
    cg = pngm.coarse_graph(g.nbr, g.voxel_of_node, img.shape, lab, q)
    rng = np.random.default_rng(seed + 2)
    th = pngm.initial_theta(cg) * rng.uniform(0.5, 1.5, len(cg["row"]))
    X = rng.random((3, q)) * cg["vol"]
    c = 0.1 / max(np.bincount(cg["row"], weights=th, minlength=q) / cg["vol"])
    return cg, th, X, c


@pytest.mark.parametrize("kind", [1, 2])
def test_objective_zero_at_truth(oracle_lib, kind):
    """Objective 1 vanishes on pairs made by Scheme 3 with the same conductances, Objective 2 on
    pairs made by Scheme 4; the gradients vanish with them."""
    cg, th, X, c = _setup_pairs(oracle_lib)
    step = pngm.scheme3 if kind == 1 else pngm.scheme4
    Y = np.stack([step(cg, th, x, c) for x in X])
    loss, grad = pngm.objective(kind, cg, th, X, Y, c)
    assert loss < 1e-28 * np.mean(X ** 2)
    assert np.max(np.abs(grad)) < 1e-12 * c * np.max(X)
    loss2, _ = pngm.objective(kind, cg, th * 1.1, X, Y, c)
    assert loss2 > 1e-6 * np.mean(X ** 2) * c * c


@pytest.mark.parametrize("kind,tied", list(itertools.product([1, 2], [False, True])))
def test_gradient_matches_finite_differences(oracle_lib, kind, tied):
    """The closed-form gradients (Sec. V.A, readings P3-P5) against central differences of the
    objective; tied parameters move both ordered slots together."""
    cg, th, X, c = _setup_pairs(oracle_lib)
    th = (th + th[cg["rev"]]) / 2 if tied else th
    Y = np.stack([pngm.scheme3(cg, th * 0.8, x, c) for x in X])
    _, grad = pngm.objective(kind, cg, th, X, Y, c, tied=tied)
    rng = np.random.default_rng(3)
    for s in rng.choice(len(th), size=12, replace=False):
        e = np.zeros_like(th)
        e[s] = 1.0
        if tied:
            e[cg["rev"][s]] = 1.0
        h = 1e-4 * th[s]
        lp, _ = pngm.objective(kind, cg, th + h * e, X, Y, c)
        lm, _ = pngm.objective(kind, cg, th - h * e, X, Y, c)
        fd = (lp - lm) / (2 * h)
        assert np.isclose(grad[s], fd, rtol=1e-6, atol=1e-12 * abs(lp)), (s, grad[s], fd)


def test_sign_sgd_recovers_conductances(oracle_lib):
    """Normalised SGD on Objective 1 with data from Scheme 3 at known tied conductances drives
    the conductances to them and the loss down by orders of magnitude."""
    cg, th_true, X, c = _setup_pairs(oracle_lib, q=6, seed=21)
    th_true = (th_true + th_true[cg["rev"]]) / 2
    rng = np.random.default_rng(4)
    Xs = rng.random((40, cg["q"])) * cg["vol"]
    Ys = np.stack([pngm.scheme3(cg, th_true, x, c) for x in Xs])
    th = pngm.initial_theta(cg)
    lr = 0.05 * np.mean(th_true)
    first = None
    for epoch in range(600):
        idx = rng.choice(len(Xs), 4, replace=False)
        th, loss = pngm.sgd_step(1, cg, th, Xs[idx], Ys[idx], c, lr, tied=True)
        first = loss if first is None else first
        if epoch % 50 == 49:
            lr *= 0.5
    final, _ = pngm.objective(1, cg, th, Xs, Ys, c)
    assert final < 1e-4 * first
    assert np.allclose(th, th_true, rtol=2e-2)
    assert np.array_equal(th, th[cg["rev"]])


def test_sgd_lower_bound(oracle_lib):
    """theta_min bounds the update from below and changes nothing above it."""
    cg, th, X, c = _setup_pairs(oracle_lib)
    Y = np.stack([pngm.scheme3(cg, th * 0.8, x, c) for x in X])
    free, _ = pngm.sgd_step(1, cg, th, X, Y, c, lr=10.0)
    low, _ = pngm.sgd_step(1, cg, th, X, Y, c, lr=10.0, theta_min=0.0)
    assert np.array_equal(low, np.where(free < 0.0, 0.0, free))
    assert free.min() < 0.0 <= low.min()
