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
    # the totals (float-float per thread over about 80 nodes each at this size, FP64 across
    # threads) against the FP64 sum of the state as stored
    exact = np.array([np.sum(got[c], dtype=np.float64) for c in range(5)])
    assert np.allclose(tot, exact, rtol=1e-12, atol=0), (tot, exact)


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


def test_implicit_every_node_512(vga, oracle_lib, full):
    """One Scheme 2 step at the benchmark's implicit configuration (10x the explicit limit, rtol
    1e-8, default solver) against the oracle's FP64 PCG solved to 1e-11, every node: relative L2 per
    compartment, and per-node relative error on the nodes holding mass."""
    from tests.helpers import rel_l2

    img, og, g, X0 = full
    p = synth.paper_params(dt=10 * 0.9 / (6 * synth.D_DOM), scheme=1, cg_rtol=1e-8, cg_maxit=500)
    sim = vga.Sim(g, p)
    sim.set_masses(X0)
    sim.step(1)
    got = sim.get_masses()
    sim.close()
    ref, status, iters, worst = oracle_lib.implicit_run(og.nbr, p, X0, 1, rtol=1e-11)
    assert status == 0
    for c in range(5):
        if np.abs(ref[c]).max() > 0:
            assert rel_l2(got[c], ref[c]) <= 1e-6, (c, rel_l2(got[c], ref[c]))
    # B x = b spreads every source over its neighbourhood: nodes above 1e-3 of the largest DOM value
    big = np.abs(ref[1]) > 1e-3 * np.abs(ref[1]).max()
    assert big.sum() > 1000
    assert np.max(np.abs(got[1, big] - ref[1, big]) / np.abs(ref[1, big])) <= 1e-5
    marked = X0[0] != 0
    assert np.max(np.abs(got[0, marked] - ref[0, marked]) / np.abs(ref[0, marked])) <= 1e-6


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


def test_config_256_ten_thousand_steps(vga, oracle_lib):
    """The FP32-state forward configuration: 256^3 at 20% porosity, 10^4 explicit steps, relative L2
    and total-mass drift against the FP64 oracle every 2000 steps."""
    from tests.helpers import rel_l2

    img = synth.pore_mask((256, 256, 256), 0.20, 7)
    og = oracle_lib.graph_build(img, keep_largest=True)
    g = vga.Graph(img)
    X0 = synth.initial_masses(synth.kept_mask_from_nodes(img.shape, og.voxel_of_node), 7)
    p = synth.paper_params()
    sim = vga.Sim(g, p)
    sim.set_masses(X0)
    sim.autotune(20)
    marked = (X0[[0, 2, 3, 4]] != 0).any(axis=0)
    assert marked.sum() > 1000
    ref = X0.copy()
    for _ in range(5):
        sim.step(2000)
        ref = oracle_lib.explicit_run(og.nbr, p, ref, 2000)
        got = sim.get_masses()
        for c in range(5):
            if np.abs(ref[c]).max() > 0:
                assert rel_l2(got[c], ref[c]) <= 1e-5, c
        assert abs(sim.totals().sum() - X0.sum()) <= 1e-7 * X0.sum()
        # the 1% marked nodes node by node: an error confined to them would be diluted about 100x in
        # the relative L2 over every node
        for c in range(5):
            r, m = ref[c, marked], got[c, marked]
            keep = np.abs(r) > 1e-6 * np.abs(ref[c]).max()
            if keep.any():
                assert np.max(np.abs(m[keep] - r[keep]) / np.abs(r[keep])) <= 1e-5, c


def test_config_batched_full(vga, oracle_lib):
    """The batched configuration: 64 subvolumes (sides 64..192, porosity 10..35%, rates within
    +-50%), 5000 steps in persistent launches; a size-stratified sample of instances against the
    FP64 oracle (the two smallest, the two largest, and four between, where tile and instance
    boundaries differ most), every instance's total mass conserved."""
    from tests.helpers import rel_l2

    specs = synth.batch_instances(64, 7)
    graphs, params, masses, imgs = [], [], [], []
    ogs = []
    for sp in specs:
        img = synth.pore_mask(sp["shape"], sp["porosity"], sp["mask_seed"])
        og = oracle_lib.graph_build(img, keep_largest=True)  # inputs come from the oracle side only
        graphs.append(vga.Graph(img))
        params.append(sp["params"])
        masses.append(synth.initial_masses(synth.kept_mask_from_nodes(img.shape, og.voxel_of_node), sp["mass_seed"]))
        imgs.append(img)
        ogs.append(og)
    b = vga.Batch(graphs, params)
    for k, X in enumerate(masses):
        b.set_masses(k, X)
    b.autotune(20)
    b.step(5000)
    by_size = np.argsort([gk.n for gk in graphs])
    sample = set(by_size[[0, 1, 13, 26, 39, 52, 62, 63]].tolist())
    for k in range(64):
        got = b.get_masses(k)
        assert abs(got.sum() - masses[k].sum()) <= 1e-7 * masses[k].sum(), k
        if k in sample:
            ref = oracle_lib.explicit_run(ogs[k].nbr, params[k], masses[k], 5000)
            for c in range(5):
                if np.abs(ref[c]).max() > 0:
                    assert rel_l2(got[c], ref[c]) <= 1e-5, (k, c)


def test_config_adjoint_128(vga, oracle_lib):
    """The adjoint configuration: 128^3 at 17% porosity, 2000 explicit steps, loss = squared error of
    the final 8^3-block DOM and CO2 masses against a seeded target run, 16^3 block-to-block
    conductances, checkpoints every 100: gradients against the oracle's FP64 adjoint."""
    import torch

    from tests.helpers import rel_l2

    img = synth.pore_mask((128, 128, 128), 0.17, 5)
    og = oracle_lib.graph_build(img)
    g = vga.Graph(img)
    X0 = synth.initial_masses(synth.kept_mask_from_nodes(img.shape, og.voxel_of_node), 5,
                              with_organic_matter=True)
    bs, N = 8, 2000
    nb = oracle_lib.block_grid(img.shape, bs)
    theta_star = synth.block_conductances(nb, 5)
    p = synth.paper_params(dt=0.9 / (6 * synth.D_DOM * 1.5))
    g6s = oracle_lib.block_face_weights(img.shape, bs, og.voxel_of_node, og.nbr, theta_star)
    target = oracle_lib.block_masses(img.shape, bs, og.voxel_of_node, oracle_lib.explicit_run(og.nbr, p, X0, N, g6=g6s))
    theta = np.ones(theta_star.size)
    g6 = oracle_lib.block_face_weights(img.shape, bs, og.voxel_of_node, og.nbr, theta)
    XN = oracle_lib.explicit_run(og.nbr, p, X0, N, g6=g6)
    L_ref, lamN = oracle_lib.block_mass_loss(img.shape, bs, og.voxel_of_node, XN, target)
    ref = oracle_lib.adjoint_run(og.nbr, p, X0, N, lamN, ckpt=100, g6=g6, want_gface=True)
    gref = oracle_lib.block_theta_grad(img.shape, bs, og.voxel_of_node, og.nbr, ref["gface"], theta.size)
    sim = vga.Sim(g, p)
    sim.set_block_conductances(bs, theta.astype(np.float32))
    sim.set_masses(X0)
    sim.adjoint_forward(N, 100)
    dldx = torch.empty((5, og.n), dtype=torch.float64, device="cuda")
    L, _ = sim.loss_block_mass(bs, (1 << 1) | (1 << 4), target, dL_dX=dldx)
    assert np.isclose(L, L_ref, rtol=1e-4)
    grad, gth = sim.adjoint_backward(dldx, n_theta=theta.size)
    assert rel_l2(gth, gref) <= 1e-4
    for name in oracle_lib.GRAD_NAMES:  # D and all seven rate constants
        assert np.isclose(grad[name], ref["grad"][name], rtol=1e-4), (name, grad[name], ref["grad"][name])
    # central differences of the GPU forward loss, relative step 1e-4, for every parameter.  The loss
    # of the FP32 forward carries noise of about 1e-9 of L, so a parameter whose step changes L by less
    # than 1e-5 of L (K_dom: the Monod half-saturation barely enters at these DOM levels) gets the step
    # that does, up to 1e-2 relative (truncation then stays below 1e-4)
    for name in oracle_lib.GRAD_NAMES:
        h = 1e-4 * p[name]
        if 2 * h * abs(grad[name]) < 1e-5 * L:
            h = min(1e-2 * p[name], 1e-5 * L / (2 * abs(grad[name])))

        def loss(v, name=name):
            s2 = vga.Sim(g, dict(p, **{name: v}))
            s2.set_block_conductances(bs, theta.astype(np.float32))
            s2.set_masses(X0)
            s2.step(N)
            Lv, _ = s2.loss_block_mass(bs, (1 << 1) | (1 << 4), target)
            s2.close()
            return Lv

        fd = (loss(p[name] + h) - loss(p[name] - h)) / (2 * h)
        assert np.isclose(grad[name], fd, rtol=2e-3), (name, grad[name], fd)
