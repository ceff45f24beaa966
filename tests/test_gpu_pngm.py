"""Coarse primitive-graph model on the GPU (Sec. V.A) against the FP64 oracle: the coarse graph
bit for bit, the restriction of voxel masses, Schemes 3 and 4, Objectives 1 and 2 with their
gradients, the normalised SGD update, and the whole calibration pipeline on voxel data."""
import numpy as np
import pytest

import synth
from oracle import pngm as opn
from tests.helpers import rel_l2

pytestmark = pytest.mark.gpu


def _torch():
    import torch

    return torch


def _case(vga, oracle_lib, shape=(40, 36, 44), por=0.25, seed=3, bs=8, labels="blocks"):
    img = synth.pore_mask(shape, por, seed)
    og = oracle_lib.graph_build(img, keep_largest=True)
    g = vga.Graph(img)
    assert g.n == og.n
    if labels == "blocks":
        lab, q = synth.block_primitives(img.shape, og.voxel_of_node, bs)
    elif labels == "random":
        q = 37
        rng = np.random.default_rng(seed)
        lab = rng.integers(0, q, og.n).astype(np.int32)
        lab[:q] = np.arange(q)
    else:
        lab, q = np.arange(og.n, dtype=np.int32), og.n
    cg = opn.coarse_graph(og.nbr, og.voxel_of_node, img.shape, lab, q)
    pg = vga.Pngm(g, lab, q)
    return img, og, g, lab, q, cg, pg


@pytest.mark.parametrize("labels", ["blocks", "random", "singletons"])
def test_coarse_graph_bit_exact(vga, oracle_lib, labels):
    shape = (20, 18, 22) if labels == "singletons" else (40, 36, 44)
    img, og, g, lab, q, cg, pg = _case(vga, oracle_lib, shape=shape, labels=labels)
    ex = pg.export()
    info = pg.info()
    assert info["q"] == q and info["n_slots"] == len(cg["row"]) and info["symmetric"] == 1
    assert np.array_equal(ex["vol"], cg["vol"])
    assert np.array_equal(ex["centroid"], cg["centroid"])
    assert np.array_equal(ex["row_ptr"], cg["row_ptr"])
    assert np.array_equal(ex["col"], cg["col"])
    assert np.array_equal(ex["rev"], cg["rev"])
    assert np.array_equal(ex["S"], cg["S"])
    assert np.array_equal(ex["dist"], cg["dist"])
    assert np.array_equal(pg.get_theta(), opn.initial_theta(cg))
    assert info["cross_faces"] == int(cg["S"].sum()) // 2


def test_restriction(vga, oracle_lib):
    torch = _torch()
    img, og, g, lab, q, cg, pg = _case(vga, oracle_lib)
    X0 = synth.initial_masses(synth.kept_mask_from_nodes(img.shape, og.voxel_of_node), 3)
    sim = vga.Sim(g, synth.paper_params())
    sim.set_masses(X0)
    sim.step(17)
    X = sim.get_masses()
    for comp in (0, 1):
        out = torch.empty(q, dtype=torch.float64, device="cuda")
        pg.restrict(sim, comp, out)
        ref = opn.restrict(lab, q, X[comp])
        assert np.allclose(out.cpu().numpy(), ref, rtol=1e-13, atol=1e-13 * np.abs(ref).max())


@pytest.mark.parametrize("labels", ["blocks", "random"])
def test_restriction_signed_tiny_and_zero_values(vga, oracle_lib, labels):
    """The fixed-point restriction on values of both signs spread over 46 decades (down into the FP32
    subnormal range, plus exact zeros), with block labels (runs of several nodes) and random labels
    (runs of one).  Every node's pair is rounded to a multiple of the unit u = 2^(e - 61), sum |m|
    < 2^e (e within one binade of the FP64 bound, as the device bound is an FP32 sum), so a
    primitive's sum is within (its node count) x 2u of the exact sum, plus the FP64 rounding of the
    oracle's own sum."""
    torch = _torch()
    img, og, g, lab, q, cg, pg = _case(vga, oracle_lib, labels=labels)
    rng = np.random.default_rng(11)
    n = og.n
    X = np.zeros((5, n))
    X[1] = rng.choice([-1.0, 1.0], n) * 10.0 ** rng.uniform(-44.0, 2.0, n)
    X[1][rng.random(n) < 0.1] = 0.0
    sim = vga.Sim(g, synth.paper_params())
    sim.set_masses(X)
    m = sim.get_masses()[1]  # the stored pairs, h + l, exactly in FP64
    out = torch.empty(q, dtype=torch.float64, device="cuda")
    pg.restrict(sim, 1, out)
    ref = opn.restrict(lab, q, m)
    S = np.abs(m).sum()
    unit = 2.0 ** (np.floor(np.log2(S)) + 2 - 61)  # the larger of the two possible units
    cnt = np.bincount(lab, minlength=q)
    absum = np.bincount(lab, weights=np.abs(m), minlength=q)
    err = np.abs(out.cpu().numpy() - ref)
    assert np.all(err <= 2 * cnt * unit + 1e-13 * absum), float((err - 2 * cnt * unit).max())


def test_scheme3_bit_exact_and_scheme4(vga, oracle_lib):
    torch = _torch()
    img, og, g, lab, q, cg, pg = _case(vga, oracle_lib)
    th = opn.initial_theta(cg)
    m0 = np.random.default_rng(1).random(q) * cg["vol"]
    c = 0.5 / max(np.bincount(cg["row"], weights=th, minlength=q) / cg["vol"])
    m = torch.from_numpy(m0.copy()).cuda()
    pg.step(m, 25, 0, c, 1.0)
    assert np.array_equal(m.cpu().numpy(), opn.scheme3(cg, th, m0, c, 25))
    m = torch.from_numpy(m0.copy()).cuda()
    pg.step(m, 4, 1, 20 * c, 1.0, cg_rtol=1e-13)
    ref = opn.scheme4(cg, th, m0, 20 * c, 4)
    assert rel_l2(m.cpu().numpy(), ref) <= 1e-11
    assert abs(m.sum().item() - m0.sum()) <= 1e-12 * m0.sum()
    assert pg.info()["last_cg_iterations"] > 0
    with pytest.raises(vga.VgaError) as e:
        pg.step(torch.from_numpy(m0.copy()).cuda(), 1, 1, 20 * c, 1.0, cg_rtol=1e-15, cg_maxit=1)
    assert e.value.name == "VGA_ERR_NOT_CONVERGED"
    th2 = th.copy()
    th2[0] *= 1.5
    pg.set_theta(th2)
    assert pg.info()["symmetric"] == 0
    with pytest.raises(vga.VgaError) as e:
        pg.step(torch.from_numpy(m0.copy()).cuda(), 1, 1, c, 1.0)
    assert e.value.name == "VGA_ERR_UNSUPPORTED"
    m = torch.from_numpy(m0.copy()).cuda()
    pg.step(m, 3, 0, c, 1.0)  # Scheme 3 takes ordered-pair conductances as they are
    assert np.array_equal(m.cpu().numpy(), opn.scheme3(cg, th2, m0, c, 3))


@pytest.mark.parametrize("kind", [1, 2])
@pytest.mark.parametrize("tied", [False, True])
def test_objective_and_gradient(vga, oracle_lib, kind, tied):
    torch = _torch()
    img, og, g, lab, q, cg, pg = _case(vga, oracle_lib, labels="random")
    rng = np.random.default_rng(7)
    th = opn.initial_theta(cg) * rng.uniform(0.6, 1.4, len(cg["row"]))
    th = (th + th[cg["rev"]]) / 2
    pg.set_theta(th)
    c = 0.2 / max(np.bincount(cg["row"], weights=th, minlength=q) / cg["vol"])
    X = rng.random((6, q)) * cg["vol"]
    Y = np.stack([opn.scheme3(cg, th * 0.7, x, c) for x in X])
    data = torch.from_numpy(np.concatenate([X, Y])).cuda()
    pairs = np.array([[0, 6], [2, 8], [5, 11], [1, 7]], dtype=np.int32)
    grad = torch.empty(pg.n_slots, dtype=torch.float64, device="cuda")
    loss = pg.objective(kind, data, pairs, c, 1.0, tied=tied, grad=grad)
    ref_loss, ref_grad = opn.objective(kind, cg, th, X[pairs[:, 0]], Y[pairs[:, 1] - 6], c, tied=tied)
    assert np.isclose(loss, ref_loss, rtol=1e-12)
    assert rel_l2(grad.cpu().numpy(), ref_grad) <= 1e-12
    # one normalised update: same signs, so the same new conductances wherever |g| is not tiny
    before = pg.sgd_step(kind, data, pairs, c, 1.0, 0.01, tied=tied)
    assert np.isclose(before, ref_loss, rtol=1e-12)
    new_ref, _ = opn.sgd_step(kind, cg, th, X[pairs[:, 0]], Y[pairs[:, 1] - 6], c, 0.01, tied=tied)
    got = pg.get_theta()
    big = np.abs(ref_grad) > 1e-9 * np.abs(ref_grad).max()
    assert np.array_equal(got[big], new_ref[big])
    if tied:
        assert np.array_equal(got, got[cg["rev"]])


def test_calibration_pipeline(vga, oracle_lib):
    """Sec. V.B on a small synthetic case: DOM scenarios diffused by the voxel scheme at 0.1 s,
    recorded every 10 s as primitive masses, and Objective 2 minimised by normalised SGD (4 pairs
    per epoch, lr halved every 10 epochs).  The records match the oracle's voxel run restricted to
    the primitives; the SGD trajectory matches the oracle's on the same data and draws; the loss
    over all pairs falls."""
    torch = _torch()
    from paper_2406_04177_gb300 import fit

    img, og, g, lab, q, cg, pg = _case(vga, oracle_lib, shape=(32, 32, 32), por=0.3, seed=4, bs=8)
    p = synth.diffusion_params(0.1)
    scen = [synth.dom_scenario(og.n, 100 + s) for s in range(3)]
    data, pairs = fit.pngm_dataset(g, pg, p, scen, steps_per_record=100, records=6)
    assert data.shape == (3 * 7, q) and pairs.shape == (18, 2)
    X = scen[1].copy()
    for r in range(3):
        X = oracle_lib.explicit_run(og.nbr, p, X, 100)
    ref = opn.restrict(lab, q, X[1])
    assert rel_l2(data[7 + 3].cpu().numpy(), ref) <= 1e-6
    c = p["D"] * (10.0 / 86400.0)
    th0 = opn.initial_theta(cg)
    lr0 = 0.05 * float(np.mean(th0))
    out = fit.fit_pngm(pg, data, pairs, p["D"], 10.0 / 86400.0, objective=2, epochs=40, lr0=lr0, halve_every=10, seed=1)
    # the same epochs in the oracle on the same data
    d = data.cpu().numpy()
    rng = np.random.Generator(np.random.PCG64(1))
    th, lr, hist = th0.copy(), lr0, []
    for epoch in range(40):
        if epoch > 0 and epoch % 10 == 0:
            lr *= 0.5
        idx = rng.choice(len(pairs), size=4, replace=False)
        th, loss = opn.sgd_step(2, cg, th, d[pairs[idx, 0]], d[pairs[idx, 1]], c, lr, tied=True, theta_min=0.0)
        hist.append(loss)
    assert np.allclose(out["loss"], hist, rtol=1e-9)
    assert np.mean(out["theta"] == th) >= 0.99
    assert np.array_equal(out["theta"], out["theta"][cg["rev"]])
    full0 = opn.objective(2, cg, th0, d[pairs[:, 0]], d[pairs[:, 1]], c)[0]
    full1 = opn.objective(2, cg, out["theta"], d[pairs[:, 0]], d[pairs[:, 1]], c)[0]
    assert full1 < full0


def test_invalid_partitions(vga, oracle_lib):
    img = synth.pore_mask((16, 16, 16), 0.4, 2)
    g = vga.Graph(img)
    lab = np.zeros(g.n, dtype=np.int32)
    with pytest.raises(vga.VgaError) as e:
        vga.Pngm(g, lab, 2)  # primitive 1 is empty
    assert e.value.name == "VGA_ERR_INVALID_ARG"
    lab[0] = 5
    with pytest.raises(vga.VgaError) as e:
        vga.Pngm(g, lab, 2)  # label outside [0, q)
    assert e.value.name == "VGA_ERR_INVALID_ARG"
    one = vga.Pngm(g, np.zeros(g.n, dtype=np.int32), 1)  # one primitive: no pairs
    assert one.info()["n_slots"] == 0


def test_buffers_survive_pair_growth_and_close_cleanly(vga, oracle_lib):
    """Growing the pair buffer (more than 64 pairs) between two restrictions leaves the restriction
    scratch intact, and every release call of the handles succeeds (close() reports a failed free)."""
    torch = _torch()
    img, og, g, lab, q, cg, pg = _case(vga, oracle_lib, shape=(24, 24, 24), bs=8)
    X0 = synth.initial_masses(synth.kept_mask_from_nodes(img.shape, og.voxel_of_node), 5)
    sim = vga.Sim(g, synth.paper_params())
    sim.set_masses(X0)
    out = torch.empty(q, dtype=torch.float64, device="cuda")
    pg.restrict(sim, 1, out)
    data = torch.rand((200, q), dtype=torch.float64, device="cuda")
    pairs = np.stack([np.arange(100), np.arange(100, 200)], axis=1).astype(np.int32)
    pg.objective(1, data, pairs, 1.0, 1e-3)
    sim.step(3)
    pg.restrict(sim, 1, out)
    ref = opn.restrict(lab, q, sim.get_masses()[1])
    assert np.allclose(out.cpu().numpy(), ref, rtol=1e-13, atol=1e-13 * np.abs(ref).max())
    pg.close()
    sim.close()
    g.close()
