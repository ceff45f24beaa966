"""Discrete adjoint on the GPU against the oracle's FP64 adjoint and central finite differences."""
import numpy as np
import pytest

import synth
from tests.helpers import rel_l2

pytestmark = pytest.mark.gpu

GRAD_TOL = 1e-4  # gradients within 1e-4 (relative) of the FP64 adjoint


def _setup(vga, oracle_lib, shape=(24, 24, 24), por=0.25, seed=3):
    img = synth.pore_mask(shape, por, seed)
    og = oracle_lib.graph_build(img)
    g = vga.Graph(img)
    X0 = synth.initial_masses(synth.kept_mask_from_nodes(img.shape, og.voxel_of_node), seed,
                              with_organic_matter=True)
    # biomass everywhere DOM sits, so the growth terms carry gradient
    X0[0] = np.where(X0[1] > 0, 0.3 * X0[1], X0[0]).astype(np.float32)
    return img, og, g, X0


def _close(a, b, tol):
    return abs(a - b) <= tol * max(abs(b), 1e-300)


def test_adjoint_forward_equals_plain_steps(vga, oracle_lib):
    img, og, g, X0 = _setup(vga, oracle_lib)
    p = synth.paper_params()
    a = vga.Sim(g, p)
    a.set_masses(X0)
    a.adjoint_forward(37, 5)
    b = vga.Sim(g, p)
    b.set_masses(X0)
    b.step(37)
    assert a.save_state() == b.save_state()


@pytest.mark.parametrize("block", [False, True])
@pytest.mark.parametrize("nsteps,ckpt", [(37, 5), (20, 20)])
def test_backward_twice_and_recorded_segment(vga, oracle_lib, block, nsteps, ckpt):
    """The forward sweep records the last segment and the backward sweep skips recomputing it.
    Two backward sweeps over one forward (after the first, the records hold another segment when
    there are several) and those of a second simulation run through the same calls give the same
    bits (the block-face gradients, sums of FP64 atomics, up to the order of those sums); agreement
    with the oracle is test_adjoint_matches_oracle's."""
    img, og, g, X0 = _setup(vga, oracle_lib)
    bs = 8
    theta = synth.block_conductances(oracle_lib.block_grid(img.shape, bs), 4) if block else None
    p = synth.paper_params(dt=0.9 / (6 * synth.D_DOM * (theta.max() if block else 1.0)))
    lamN = np.random.default_rng(9).standard_normal((5, og.n))
    runs = []
    for _ in range(2):
        sim = vga.Sim(g, p)
        if block:
            sim.set_block_conductances(bs, theta.astype(np.float32))
        sim.set_masses(X0)
        sim.adjoint_forward(nsteps, ckpt)
        for _ in range(2):
            lam0 = np.empty((5, og.n))
            grad, gth = sim.adjoint_backward(lamN, lam0, n_theta=0 if theta is None else theta.size)
            runs.append((lam0, grad, gth))
        sim.close()
    for lam0, grad, gth in runs[1:]:
        assert np.array_equal(lam0, runs[0][0])
        assert grad == runs[0][1]
        if block:
            assert np.allclose(gth, runs[0][2], rtol=1e-12, atol=1e-15 * np.abs(runs[0][2]).max())


@pytest.mark.parametrize("block", [False, True])
def test_adjoint_matches_oracle(vga, oracle_lib, block):
    img, og, g, X0 = _setup(vga, oracle_lib)
    nsteps, ckpt, bs = 60, 7, 8
    g6 = theta = None
    if block:
        nb = oracle_lib.block_grid(img.shape, bs)
        theta = synth.block_conductances(nb, 11)
        p = synth.paper_params(dt=0.9 / (6 * synth.D_DOM * theta.max()))
        g6 = oracle_lib.block_face_weights(img.shape, bs, og.voxel_of_node, og.nbr, theta)
    else:
        p = synth.paper_params()
    lamN = np.random.default_rng(5).standard_normal((5, og.n))
    ref = oracle_lib.adjoint_run(og.nbr, p, X0, nsteps, lamN, ckpt=ckpt, g6=g6, want_gface=block)
    sim = vga.Sim(g, p)
    if block:
        sim.set_block_conductances(bs, theta.astype(np.float32))
    sim.set_masses(X0)
    sim.adjoint_forward(nsteps, ckpt)
    assert rel_l2(sim.get_masses(), ref["XN"]) < 1e-7
    lam0 = np.empty((5, og.n))
    grad, gth = sim.adjoint_backward(lamN, lam0, n_theta=0 if theta is None else theta.size)
    for c in range(5):
        assert rel_l2(lam0[c], ref["lam0"][c]) <= GRAD_TOL, (c, rel_l2(lam0[c], ref["lam0"][c]))
    for name, v in ref["grad"].items():
        assert _close(grad[name], v, GRAD_TOL), (name, grad[name], v)
    if block:
        nI = theta.size
        gref = oracle_lib.block_theta_grad(img.shape, bs, og.voxel_of_node, og.nbr, ref["gface"], nI)
        assert rel_l2(gth, gref) <= GRAD_TOL
        big = np.abs(gref) > 1e-3 * np.abs(gref).max()
        assert np.all(np.abs(gth[big] - gref[big]) <= GRAD_TOL * np.abs(gref[big]) + 1e-12 * np.abs(gref).max())


def test_adjoint_central_differences_on_gpu(vga, oracle_lib):
    """Central differences of the GPU forward itself against the GPU adjoint, for D and a block
    conductance.  The forward's own rounding noise (~1e-10 of the loss) must stay well below the
    loss change, so the step is 1e-2 (truncation error ~1e-4 of the derivative).  The rate
    constants move the loss by less than that noise on this workload; they are checked by FP64
    central differences on the oracle, whose adjoint the GPU adjoint matches to 1e-4."""
    img, og, g, X0 = _setup(vga, oracle_lib, shape=(20, 20, 20), seed=4)
    bs = 5
    nb = oracle_lib.block_grid(img.shape, bs)
    theta = synth.block_conductances(nb, 2)
    p = synth.paper_params(dt=0.9 / (6 * synth.D_DOM * theta.max() * 1.02))
    nsteps = 40
    lamN = np.random.default_rng(9).standard_normal((5, og.n))

    def L(params, th):
        s = vga.Sim(g, params)
        s.set_block_conductances(bs, th.astype(np.float32))
        s.set_masses(X0)
        s.step(nsteps)
        return float(np.sum(lamN * s.get_masses()))

    sim = vga.Sim(g, p)
    sim.set_block_conductances(bs, theta.astype(np.float32))
    sim.set_masses(X0)
    sim.adjoint_forward(nsteps, 16)
    grad, gth = sim.adjoint_backward(lamN, n_theta=theta.size)
    for name in ("D",):
        # The kernels see FP32 constants (rate * dt, beta, 1 - beta): divide by the perturbation
        # they actually receive.  For beta a power-of-two step moves beta and 1 - beta exactly.
        if name == "beta":
            h = 2.0 ** -13
            two_h = 2 * h
        else:
            h = 1e-2 * p[name]
            dt = p["dt"]
            two_h = (float(np.float32((p[name] + h) * dt)) - float(np.float32((p[name] - h) * dt))) / dt
        num = (L(dict(p, **{name: p[name] + h}), theta) - L(dict(p, **{name: p[name] - h}), theta)) / two_h
        assert _close(grad[name], num, 2e-3), (name, grad[name], num)
    k = int(np.argmax(np.abs(gth)))
    # theta is rounded to FP32 inside: perturb by a representable step
    t0 = np.float32(theta[k])
    h = float(np.float32(t0 * 1.01) - t0)
    tp, tm = theta.copy(), theta.copy()
    tp[k] = t0 + h
    tm[k] = t0 - h
    num = (L(p, tp) - L(p, tm)) / (2 * h)
    assert _close(gth[k], num, 2e-3), (gth[k], num)


def test_block_mass_loss(vga, oracle_lib):
    img, og, g, X0 = _setup(vga, oracle_lib, shape=(32, 24, 40), seed=6)
    bs = 8
    nb = oracle_lib.block_grid(img.shape, bs)
    target = np.random.default_rng(2).uniform(0, 1e-3, size=(2, nb[0] * nb[1] * nb[2]))
    import torch

    sim = vga.Sim(g, synth.paper_params())
    sim.set_masses(X0)
    sim.step(25)
    X = sim.get_masses()
    L_ref, lam_ref = oracle_lib.block_mass_loss(img.shape, bs, og.voxel_of_node, X, target)
    dldx = torch.empty((5, og.n), dtype=torch.float64, device="cuda")
    L, mass = sim.loss_block_mass(bs, (1 << 1) | (1 << 4), target, dL_dX=dldx, want_mass=True)
    torch.cuda.synchronize()
    assert abs(L - L_ref) <= 1e-12 * L_ref
    assert np.allclose(mass, oracle_lib.block_masses(img.shape, bs, og.voxel_of_node, X), rtol=1e-12, atol=0)
    assert np.allclose(dldx.cpu().numpy(), lam_ref, rtol=1e-12, atol=1e-300)


def test_adjoint_error_paths(vga, oracle_lib):
    img, og, g, X0 = _setup(vga, oracle_lib, shape=(12, 12, 12))
    sim = vga.Sim(g, synth.paper_params())
    with pytest.raises(vga.VgaError):
        sim.adjoint_backward(np.zeros((5, og.n)))  # no forward pass yet
    sim.set_masses(X0)
    sim.adjoint_forward(5, 2)
    sim.set_params(dict(synth.paper_params(), mu=0.4))
    with pytest.raises(vga.VgaError):
        sim.adjoint_backward(np.zeros((5, og.n)))  # parameters changed
    asim = vga.Sim(g, synth.paper_params(transform=1))
    with pytest.raises(vga.VgaError) as e:
        asim.adjoint_forward(5, 2)
    assert e.value.name == "VGA_ERR_UNSUPPORTED"


def test_block_fit_reduced_config(vga, oracle_lib):
    """The adjoint workload at reduced size (64^3, 8^3 blocks, 200 steps, checkpoints every 100):
    block-mass loss gradient against the oracle's FP64 adjoint."""
    img = synth.pore_mask((64, 64, 64), 0.17, 5)
    og = oracle_lib.graph_build(img)
    g = vga.Graph(img)
    X0 = synth.initial_masses(synth.kept_mask_from_nodes(img.shape, og.voxel_of_node), 5,
                              with_organic_matter=True)
    bs = 8
    nb = oracle_lib.block_grid(img.shape, bs)
    theta_star = synth.block_conductances(nb, 5)
    p = synth.paper_params(dt=0.9 / (6 * synth.D_DOM * 1.5))
    g6s = oracle_lib.block_face_weights(img.shape, bs, og.voxel_of_node, og.nbr, theta_star)
    Xt = oracle_lib.explicit_run(og.nbr, p, X0, 200, g6=g6s)
    target = oracle_lib.block_masses(img.shape, bs, og.voxel_of_node, Xt)
    theta = np.ones(theta_star.size)
    g6 = oracle_lib.block_face_weights(img.shape, bs, og.voxel_of_node, og.nbr, theta)
    XN = oracle_lib.explicit_run(og.nbr, p, X0, 200, g6=g6)
    L_ref, lamN = oracle_lib.block_mass_loss(img.shape, bs, og.voxel_of_node, XN, target)
    ref = oracle_lib.adjoint_run(og.nbr, p, X0, 200, lamN, ckpt=100, g6=g6, want_gface=True)
    gref = oracle_lib.block_theta_grad(img.shape, bs, og.voxel_of_node, og.nbr, ref["gface"], theta.size)

    import torch

    sim = vga.Sim(g, p)
    sim.set_block_conductances(bs, theta.astype(np.float32))
    sim.set_masses(X0)
    sim.adjoint_forward(200, 100)
    dldx = torch.empty((5, og.n), dtype=torch.float64, device="cuda")
    L, _ = sim.loss_block_mass(bs, (1 << 1) | (1 << 4), target, dL_dX=dldx)
    assert _close(L, L_ref, 1e-4)
    grad, gth = sim.adjoint_backward(dldx, n_theta=theta.size)
    assert rel_l2(gth, gref) <= GRAD_TOL
    assert _close(grad["D"], ref["grad"]["D"], GRAD_TOL)


@pytest.mark.parametrize("block", [False, True])
@pytest.mark.parametrize("marked", ["paper", "organic", "none"])
def test_sparse_reverse_matches_dense(vga, oracle_lib, block, marked):
    """Records of the marked nodes only and reverse steps that skip the rate-gradient terms at the
    unmarked nodes (activity mask of X^0) give the bits of the dense records and reverse steps:
    dL/dX^0 and the eight parameter gradients exactly, the block-face gradients up to the order of
    their FP64 atomic sums.  Marked sets: the Sec. IV.C state (biomass on 1% of the nodes), biomass
    and organic matter wherever DOM sits, and none (DOM only: every node unmarked)."""
    img = synth.pore_mask((40, 36, 44), 0.25, 7)
    og = oracle_lib.graph_build(img)
    g = vga.Graph(img)
    kept = synth.kept_mask_from_nodes(img.shape, og.voxel_of_node)
    X0 = synth.initial_masses(kept, 7, with_organic_matter=(marked == "organic"))
    if marked == "organic":
        X0[0] = np.where(X0[1] > 0, 0.3 * X0[1], X0[0]).astype(np.float32)
    if marked == "none":
        X0[[0, 2, 3, 4]] = 0.0
    bs = 8
    theta = synth.block_conductances(oracle_lib.block_grid(img.shape, bs), 4) if block else None
    p = synth.paper_params(dt=0.9 / (6 * synth.D_DOM * (theta.max() if block else 1.0)))
    lamN = np.random.default_rng(19).standard_normal((5, og.n))
    out = []
    for skip in (True, False):
        sim = vga.Sim(g, p)
        sim.set_activity_skip(skip)
        if block:
            sim.set_block_conductances(bs, theta.astype(np.float32))
        sim.set_masses(X0)
        sim.adjoint_forward(45, 8)  # six recomputed segments and the recorded last one (5 steps)
        lam0 = np.empty((5, og.n))
        grad, gth = sim.adjoint_backward(lamN, lam0, n_theta=0 if theta is None else theta.size)
        out.append((lam0, grad, gth, sim.save_state()))
        sim.close()
    (l_s, g_s, t_s, x_s), (l_d, g_d, t_d, x_d) = out
    assert x_s == x_d
    assert np.array_equal(l_s, l_d)
    assert g_s == g_d
    if block:
        assert np.allclose(t_s, t_d, rtol=1e-12, atol=1e-15 * np.abs(t_d).max())


def test_device_conductances_and_device_gradient(vga, oracle_lib):
    """vga_sim_set_block_conductances_device gives the run of the host form (same bits); a NaN or
    negative device value is rejected and leaves the previous conductances in place; the stability
    check sees the device maximum; vga_adjoint_grad_theta copies the last backward's conductance
    gradient to device or host memory, equal to the one vga_adjoint_backward returns."""
    import torch

    img, og, g, X0 = _setup(vga, oracle_lib)
    bs = 8
    theta = synth.block_conductances(oracle_lib.block_grid(img.shape, bs), 4).astype(np.float32)
    p = synth.paper_params(dt=0.9 / (6 * synth.D_DOM * theta.max()))
    lamN = np.random.default_rng(3).standard_normal((5, og.n))
    runs = []
    for dev in (False, True):
        sim = vga.Sim(g, p)
        sim.set_block_conductances(bs, torch.from_numpy(theta).cuda() if dev else theta)
        sim.set_masses(X0)
        sim.adjoint_forward(25, 6)
        lam0 = np.empty((5, og.n))
        grad, gth = sim.adjoint_backward(lamN, lam0, n_theta=theta.size)
        d = torch.zeros(theta.size, dtype=torch.float64, device="cuda")
        sim.adjoint_grad_theta(d)
        h = sim.adjoint_grad_theta(np.zeros(theta.size))
        assert np.array_equal(d.cpu().numpy(), gth) and np.array_equal(h, gth)
        runs.append((sim.save_state(), lam0, grad, gth))
        if dev:
            bad = torch.from_numpy(theta).cuda()
            bad[3] = float("nan")
            with pytest.raises(vga.VgaError) as e:
                sim.set_block_conductances(bs, bad)
            assert e.value.name == "VGA_ERR_INVALID_ARG"
            bad[3] = -1.0
            with pytest.raises(vga.VgaError) as e:
                sim.set_block_conductances(bs, bad)
            assert e.value.name == "VGA_ERR_INVALID_ARG"
            with pytest.raises(vga.VgaError) as e:  # 6 D dt max theta > 1 at this time step
                sim.set_block_conductances(bs, torch.from_numpy(theta * 3).cuda())
            assert e.value.name == "VGA_ERR_UNSTABLE_DT"
            with pytest.raises(vga.VgaError):  # wrong count
                sim.set_block_conductances(bs, torch.from_numpy(theta[:-1]).cuda())
            assert np.array_equal(sim.get_block_conductances(theta.size), theta)
            with pytest.raises(vga.VgaError):  # wrong gradient size
                sim.adjoint_grad_theta(np.zeros(theta.size + 1))
        sim.close()
    assert runs[0][0] == runs[1][0]
    assert np.array_equal(runs[0][1], runs[1][1])
    assert runs[0][2] == runs[1][2]
    assert np.allclose(runs[0][3], runs[1][3], rtol=1e-12, atol=1e-15 * np.abs(runs[0][3]).max())
    sim = vga.Sim(g, p)
    sim.set_block_conductances(bs, theta)
    sim.set_masses(X0)
    sim.adjoint_forward(5, 5)
    with pytest.raises(vga.VgaError):  # no backward sweep yet
        sim.adjoint_grad_theta(np.zeros(theta.size))
    sim.close()
