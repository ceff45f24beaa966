"""Pins of three oracle functions every GPU totals and gradient check rests on:

- `totals` (compensated summation of the compartment masses tracked in Sec. IV.C) against the
  exactly rounded sum `math.fsum`, on inputs built so that a plain or a sign-slipped compensated
  sum visibly fails;
- `block_mass_loss` (the block-mass objective of the adjoint workload, the voxel analogue of the
  least-squares objectives of Sec. V.A): L against a per-block loop over the definition, dL/dX
  against central differences (exact for a quadratic);
- `block_theta_grad` (dL/dtheta of block-face conductances, the Sec. V.A weighted flux on voxel
  edges): the interface numbering against hand-worked cases and against the block pair every edge
  joins, and the whole chain loss -> explicit run -> theta against central differences per
  interface, so a double count over the six slots or a wrong interface on one axis fails.
"""
import math

import numpy as np
import pytest

import synth

U = 2.0 ** -53  # unit roundoff of FP64


def _naive(v):
    s = 0.0
    for x in v:
        s += x
    return s


def test_totals_exact_on_cancelling_inputs(oracle_lib):
    """Neumaier's compensated sum is exact on these classic cancellations, where a plain sum (and
    Kahan's) returns 0 or loses the small terms.  Each compartment gets a different vector, so a
    transposed (n, 5) reading fails too."""
    rows = [
        [1.0, 1e100, 1.0, -1e100],
        [1e16, 1.0, -1e16, 1.0, 1e16, 1.0, -1e16],
        [3.0, 1e20, 7.0, -1e20, 0.5],
        [1e-3, 2.0 ** 60, 1e-3, -(2.0 ** 60), 1e-3, 0.0],
        [-1e300, 2.5, 1e300, -4.0],
    ]
    n = max(len(r) for r in rows)
    X = np.zeros((5, n))
    for c, r in enumerate(rows):
        X[c, : len(r)] = r
    got = oracle_lib.totals(X)
    want = np.array([math.fsum(X[c]) for c in range(5)])
    assert np.array_equal(got, want), (got, want)
    # the inputs do discriminate: a plain running sum misses every one of them
    assert all(_naive(X[c]) != want[c] for c in range(5))


def test_totals_within_compensated_bound_on_random_inputs(oracle_lib):
    """|sum - exact| <= 2u|exact| + 4 n u^2 sum|x| (Neumaier's bound with slack) on wide-range
    signed values, where a plain sum errs by ~n u sum|x|."""
    rng = np.random.default_rng(11)
    n = 20000
    X = rng.standard_normal((5, n)) * 10.0 ** rng.uniform(-8, 8, (5, n))
    got = oracle_lib.totals(X)
    for c in range(5):
        exact = math.fsum(X[c])
        bound = 2 * U * abs(exact) + 4 * n * U * U * float(np.abs(X[c]).sum())
        assert abs(got[c] - exact) <= bound, (c, got[c], exact)
    assert oracle_lib.totals(np.zeros((5, 0))).tolist() == [0.0] * 5


def _loss_setup(oracle_lib, shape=(16, 16, 16), bs=8, seed=4, porosity=0.55):
    img = synth.pore_mask(shape, porosity, seed, sigma=1.0)
    g = oracle_lib.graph_build(img, keep_largest=True)
    nb = oracle_lib.block_grid(shape, bs)
    return img, g, nb


def test_block_mass_loss_value_and_gradient(oracle_lib):
    shape, bs = (16, 16, 16), 8
    img, g, nb = _loss_setup(oracle_lib, shape, bs)
    n = g.n
    rng = np.random.default_rng(3)
    X = rng.uniform(0, 1e-3, (5, n))
    nblk = nb[0] * nb[1] * nb[2]
    target = rng.uniform(0, 0.3, (2, nblk))
    L, lam = oracle_lib.block_mass_loss(shape, bs, g.voxel_of_node, X, target)
    # the definition, one block at a time from voxel coordinates
    z, y, x = np.unravel_index(g.voxel_of_node, shape)
    Lref = 0.0
    for t, c in enumerate((1, 4)):
        for bz in range(nb[0]):
            for by in range(nb[1]):
                for bx in range(nb[2]):
                    sel = (z // bs == bz) & (y // bs == by) & (x // bs == bx)
                    b = (bz * nb[1] + by) * nb[2] + bx
                    Lref += (X[c, sel].sum() - target[t, b]) ** 2
    assert L == pytest.approx(Lref, rel=1e-13)
    # dL/dX by central differences (L is quadratic in X: the difference quotient is exact up to
    # rounding); compartments outside the loss get zero
    for c in range(5):
        for i in rng.choice(n, 6, replace=False):
            h = 1e-4

            def Lx(d, c=c, i=i):
                Xp = X.copy()
                Xp[c, i] += d
                return oracle_lib.block_mass_loss(shape, bs, g.voxel_of_node, Xp, target)[0]

            num = (Lx(h) - Lx(-h)) / (2 * h)
            assert lam[c, i] == pytest.approx(num, rel=1e-7, abs=1e-12), (c, i, lam[c, i], num)
            if c not in (1, 4):
                assert lam[c, i] == 0.0


def test_interface_numbering_hand_worked(oracle_lib):
    """16^3 image of 8^3 blocks (2 x 2 x 2 blocks): x-normal interfaces 0..3 at (bz*2 + by),
    y-normal 4..7 at 4 + bz*2 + bx, z-normal 8..11 at 8 + by*2 + bx (the documented order)."""
    shape, bs = (16, 16, 16), 8
    img = np.zeros(shape, dtype=np.uint8)
    g = oracle_lib.graph_build(img)
    assert oracle_lib.interface_count(oracle_lib.block_grid(shape, bs)) == 12
    ei = oracle_lib.edge_interface(shape, bs, g.voxel_of_node, g.nbr)

    def node(z, y, x):
        return (z * 16 + y) * 16 + x  # full box: node = raster index

    cases = [  # (z, y, x), slot, interface
        ((0, 0, 7), 1, 0), ((0, 0, 8), 0, 0), ((9, 3, 7), 1, 2), ((3, 12, 8), 0, 1), ((15, 15, 7), 1, 3),
        ((0, 7, 12), 3, 5), ((0, 8, 12), 2, 5), ((10, 7, 2), 3, 6), ((15, 8, 9), 2, 7),
        ((7, 12, 3), 5, 10), ((8, 12, 3), 4, 10), ((7, 0, 0), 5, 8), ((8, 15, 15), 4, 11),
        ((3, 3, 3), 1, -1), ((3, 3, 3), 5, -1), ((0, 0, 0), 0, -1), ((15, 15, 15), 5, -1),
    ]
    for (z, y, x), slot, want in cases:
        assert ei[node(z, y, x), slot] == want, ((z, y, x), slot, ei[node(z, y, x), slot], want)


def test_interfaces_join_one_block_pair_each(oracle_lib):
    """On a random mask with 4^3 blocks: an edge has an interface iff its ends lie in different
    blocks, both slots of an edge carry the same interface, and every interface joins exactly one
    unordered pair of face-adjacent blocks (distinct interfaces, distinct pairs)."""
    shape, bs = (12, 16, 20), 4
    img, g, nb = _loss_setup(oracle_lib, shape, bs, seed=9, porosity=0.6)
    ei = oracle_lib.edge_interface(shape, bs, g.voxel_of_node, g.nbr)
    z, y, x = np.unravel_index(g.voxel_of_node, shape)
    blk = np.stack([z // bs, y // bs, x // bs], axis=1)
    opp = [1, 0, 3, 2, 5, 4]
    pair_of = {}
    for i in range(g.n):
        for d in range(6):
            j = g.nbr[i, d]
            if j < 0:
                assert ei[i, d] == -1
                continue
            same = bool((blk[i] == blk[j]).all())
            assert (ei[i, d] == -1) == same
            assert ei[j, opp[d]] == ei[i, d]
            if not same:
                pr = tuple(sorted((tuple(blk[i]), tuple(blk[j]))))
                assert int(np.abs(blk[i] - blk[j]).sum()) == 1
                assert pair_of.setdefault(int(ei[i, d]), pr) == pr
    assert len(set(pair_of.values())) == len(pair_of)
    assert all(0 <= k < oracle_lib.interface_count(nb) for k in pair_of)


def test_block_theta_grad_matches_central_differences(oracle_lib):
    """The chain theta -> per-edge weights -> explicit run -> block-mass loss, differentiated by
    adjoint_run + block_theta_grad, against central differences of the FP64 forward in every one
    of the 12 interfaces of a 16^3 mask with 8^3 blocks."""
    shape, bs = (16, 16, 16), 8
    img, g, nb = _loss_setup(oracle_lib, shape, bs)
    n = g.n
    nI = oracle_lib.interface_count(nb)
    rng = np.random.default_rng(6)
    X0 = np.zeros((5, n))
    X0[0] = rng.uniform(0, 5e-4, n) * (rng.random(n) < 0.2)
    X0[1] = rng.uniform(0, 2e-3, n) * (rng.random(n) < 0.4)
    X0[3] = X0[1] * rng.uniform(0.5, 1.0, n)
    X0[2] = 0.1 * X0[1]
    p = synth.paper_params()
    p["dt"] = 0.5 * synth.explicit_dt()
    nsteps = 15
    theta = rng.uniform(0.6, 1.4, nI)
    theta_star = rng.uniform(0.6, 1.4, nI)

    def forward(th):
        g6 = oracle_lib.block_face_weights(shape, bs, g.voxel_of_node, g.nbr, th)
        return g6, oracle_lib.explicit_run(g.nbr, p, X0, nsteps, g6=g6)

    target = oracle_lib.block_masses(shape, bs, g.voxel_of_node, forward(theta_star)[1])

    def loss(th):
        return oracle_lib.block_mass_loss(shape, bs, g.voxel_of_node, forward(th)[1], target)[0]

    g6, XN = forward(theta)
    L, lamN = oracle_lib.block_mass_loss(shape, bs, g.voxel_of_node, XN, target)
    res = oracle_lib.adjoint_run(g.nbr, p, X0, nsteps, lamN, ckpt=4, g6=g6, want_gface=True)
    grad = oracle_lib.block_theta_grad(shape, bs, g.voxel_of_node, g.nbr, res["gface"], nI)
    num = np.empty(nI)
    for k in range(nI):
        h = 1e-5 * theta[k]
        tp, tm = theta.copy(), theta.copy()
        tp[k] += h
        tm[k] -= h
        num[k] = (loss(tp) - loss(tm)) / (2 * h)
    scale = float(np.abs(num).max())
    assert scale > 0 and np.count_nonzero(np.abs(num) > 1e-3 * scale) >= 8  # the pin sees most interfaces
    assert np.allclose(grad, num, rtol=1e-6, atol=1e-7 * scale), np.stack([grad, num])
