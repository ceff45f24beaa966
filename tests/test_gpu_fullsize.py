"""Parity at the benchmark's full size: the 512^3 workload (17% porosity, largest component, Sec.
IV.C rates and masses) in the launch configuration the benchmark times (autotuned explicit kernel).

The oracle cannot run 20.8 M nodes in a test, so it computes sampled outputs one by one: after R
explicit steps a node depends only on the nodes within graph distance R (one hop per step), so the
oracle runs the ball of radius R around each sampled node as a graph of its own and the centre's
value is exact.  The implicit and adjoint paths are checked through properties that hold at any
size (mass conservation and the true residual; finite differences of the loss)."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

SIDE, POR, SEED = 512, 0.17, 3
R = 12  # explicit steps of the sampled check


@pytest.fixture(scope="module")
def full(vga, oracle_lib):
    img = synth.pore_mask((SIDE, SIDE, SIDE), POR, SEED)
    og = oracle_lib.graph_build(img, keep_largest=True)
    g = vga.Graph(img)
    assert g.n == og.n
    X0 = synth.initial_masses(synth.kept_mask_from_nodes(img.shape, og.voxel_of_node), SEED)
    return img, og, g, X0


def _ball(nbr, center, radius):
    """Nodes within graph distance `radius` of `center` (breadth-first), in discovery order."""
    seen = {int(center): 0}
    frontier = [int(center)]
    order = [int(center)]
    for d in range(radius):
        nxt = []
        for u in frontier:
            for v in nbr[u]:
                v = int(v)
                if v >= 0 and v not in seen:
                    seen[v] = d + 1
                    nxt.append(v)
                    order.append(v)
        frontier = nxt
    return np.array(order, dtype=np.int64)


def test_explicit_sampled_nodes_512(vga, oracle_lib, full):
    img, og, g, X0 = full
    p = synth.paper_params()
    sim = vga.Sim(g, p)
    sim.set_masses(X0)
    sim.autotune(20)  # the benchmark's configuration
    sim.step(R)
    got = sim.get_masses()
    rng = np.random.default_rng(11)
    # sample nodes that carry mass in their neighbourhood: DOM and MB sources, and random nodes
    cand = np.concatenate([np.nonzero(X0[1])[0][:2000], np.nonzero(X0[0])[0][:2000]])
    samples = np.concatenate([rng.choice(cand, 6, replace=False), rng.choice(og.n, 4, replace=False)])
    for c0 in samples:
        nodes = _ball(og.nbr, c0, R)
        local = -np.ones(og.n, dtype=np.int64)
        local[nodes] = np.arange(nodes.size)
        sub = og.nbr[nodes]
        sub = np.where(sub >= 0, local[np.maximum(sub, 0)], -1).astype(np.int32)
        ref = oracle_lib.explicit_run(sub, p, X0[:, nodes], R)[:, 0]
        for c in range(5):
            scale = max(abs(ref[c]), 1e-6 * np.abs(X0[c]).max(), 1e-30)
            assert abs(got[c, c0] - ref[c]) <= 1e-6 * scale, (int(c0), c, got[c, c0], ref[c])
    tot = sim.totals()
    assert abs(tot.sum() - X0.sum()) <= 1e-7 * X0.sum()


def test_implicit_properties_512(vga, full):
    """Scheme 2 at 10x the explicit limit with rtol 1e-8 (the benchmark's implicit configuration):
    the reported residual is the true one and below rtol, and the solve conserves mass (B has unit
    column sums) to about rtol."""
    img, og, g, X0 = full
    p = synth.paper_params(dt=10 * 0.9 / (6 * synth.D_DOM), scheme=1, cg_rtol=1e-8, cg_maxit=500)
    sim = vga.Sim(g, p)
    sim.set_masses(X0)
    sim.step(2)
    st = sim.stats()
    assert st["cg_last_relres"] <= 1e-8
    assert 0 < st["cg_iterations"] <= 2 * 200
    assert abs(sim.totals().sum() - X0.sum()) <= 1e-7 * X0.sum()


def test_adjoint_gradient_matches_finite_difference_512(vga, full):
    """dL/dD of the block-mass loss after 20 steps (checkpoints every 10, 8^3 blocks) against a
    central difference of the loss computed by two forward runs."""
    import torch

    img, og, g, X0 = full
    X0 = synth.initial_masses(synth.kept_mask_from_nodes(img.shape, og.voxel_of_node), SEED,
                              with_organic_matter=True)
    bs, N = 8, 20
    nb = tuple(-(-s // bs) for s in img.shape)
    target = np.zeros((2, nb[0] * nb[1] * nb[2]))
    mask = (1 << 1) | (1 << 4)
    p = synth.paper_params(dt=0.9 / (6 * synth.D_DOM * 1.05))
    dldx = torch.empty((5, og.n), dtype=torch.float64, device="cuda")

    def loss(D):
        s = vga.Sim(g, dict(p, D=D))
        s.set_masses(X0)
        s.step(N)
        L, _ = s.loss_block_mass(bs, mask, target)
        s.close()
        return L

    sim = vga.Sim(g, p)
    sim.set_masses(X0)
    sim.adjoint_forward(N, 10)
    L0, _ = sim.loss_block_mass(bs, mask, target, dL_dX=dldx)
    grad, _ = sim.adjoint_backward(dldx)
    h = 1e-2 * p["D"]
    fd = (loss(p["D"] + h) - loss(p["D"] - h)) / (2 * h)
    assert np.isclose(loss(p["D"]), L0, rtol=1e-9)
    assert np.isclose(grad["D"], fd, rtol=2e-3), (grad["D"], fd)
