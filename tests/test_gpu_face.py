"""Per-face conductances (the weighted flux of Sec. V.A on every voxel edge) through the explicit
scheme (every kernel variant), the implicit scheme and the discrete adjoint, against the FP64
oracle run with the same per-edge conductances."""
import numpy as np
import pytest

import synth
from tests.helpers import rel_l2

pytestmark = pytest.mark.gpu

OPP = [1, 0, 3, 2, 5, 4]


def _setup(vga, oracle_lib, shape=(24, 28, 20), por=0.3, seed=17):
    img = synth.pore_mask(shape, por, seed)
    og = oracle_lib.graph_build(img)
    g = vga.Graph(img)
    X0 = synth.initial_masses(synth.kept_mask_from_nodes(img.shape, og.voxel_of_node), seed, with_organic_matter=True)
    X0[0] = np.where(X0[1] > 0, 0.3 * X0[1], X0[0]).astype(np.float32)
    return img, og, g, X0


def _faces(og, seed, junk=7.0):
    """Symmetric conductances in [0.5, 1.5] on every edge (float32 values); slots without an edge get
    `junk`, which must be ignored."""
    rng = np.random.default_rng(seed)
    g6 = np.full((og.n, 6), junk, dtype=np.float32)
    for i in range(og.n):
        for d in (1, 3, 5):
            j = og.nbr[i, d]
            if j >= 0:
                v = np.float32(rng.uniform(0.5, 1.5))
                g6[i, d] = v
                g6[j, OPP[d]] = v
    return g6


def _oracle_g6(og, g6):
    g = g6.astype(np.float64).copy()
    g[og.nbr < 0] = 0.0
    return g


@pytest.mark.parametrize("variant", [5, 2, 0, 1])
def test_face_explicit_matches_oracle(vga, oracle_lib, variant):
    img, og, g, X0 = _setup(vga, oracle_lib)
    g6 = _faces(og, 3)
    p = synth.paper_params(dt=0.9 / (6 * synth.D_DOM * 1.5))
    sim = vga.Sim(g, p)
    sim.set_kernel(variant, 1024)
    sim.set_face_conductances(g6)
    sim.set_masses(X0)
    sim.step(150)
    got = sim.get_masses()
    ref = oracle_lib.explicit_run(og.nbr, p, X0, 150, g6=_oracle_g6(og, g6))
    for c in range(5):
        assert rel_l2(got[c], ref[c]) <= 1e-5, (variant, c, rel_l2(got[c], ref[c]))
    assert abs(sim.totals().sum() - X0.sum()) <= 1e-7 * X0.sum()


def test_face_variants_bit_identical(vga, oracle_lib):
    """The table kernels (one, two and four nodes per thread, sparse and dense) give the same bits with
    per-face conductances."""
    img, og, g, X0 = _setup(vga, oracle_lib, (30, 22, 37), 0.28, 19)
    g6 = _faces(og, 4)
    p = synth.paper_params(dt=0.9 / (6 * synth.D_DOM * 1.5))
    outs = []
    for variant, skip in ((2, False), (4, False), (5, False), (5, True)):
        sim = vga.Sim(g, p)
        sim.set_kernel(variant, 1024)
        sim.set_activity_skip(skip)
        sim.set_face_conductances(g6)
        sim.set_masses(X0)
        sim.step(23)
        outs.append(sim.save_state())
        sim.close()
    assert all(o == outs[0] for o in outs[1:])


def test_face_implicit_matches_oracle(vga, oracle_lib):
    img, og, g, X0 = _setup(vga, oracle_lib)
    g6 = _faces(og, 5)
    p = synth.paper_params(dt=5 * 0.9 / (6 * synth.D_DOM), scheme=1, cg_rtol=1e-10, cg_maxit=2000)
    sim = vga.Sim(g, p)
    sim.set_face_conductances(g6)
    sim.set_masses(X0)
    sim.step(6)
    got = sim.get_masses()
    ref, status, _, _ = oracle_lib.implicit_run(og.nbr, p, X0, 6, rtol=1e-13, g6=_oracle_g6(og, g6))
    assert status == 0
    for c in range(5):
        assert rel_l2(got[c], ref[c]) <= 1e-5, (c, rel_l2(got[c], ref[c]))


def test_face_adjoint_gradients_match_oracle(vga, oracle_lib):
    """dL/dg of every edge (both slots), dL/dD and the rate gradients of L = sum w X^N after 30 steps,
    against the oracle's FP64 adjoint with the same conductances."""
    img, og, g, X0 = _setup(vga, oracle_lib)
    g6 = _faces(og, 6)
    p = synth.paper_params(dt=0.9 / (6 * synth.D_DOM * 1.5))
    n, N = og.n, 30
    w = np.random.default_rng(2).standard_normal((5, n))
    sim = vga.Sim(g, p)
    sim.set_face_conductances(g6)
    sim.set_masses(X0)
    sim.adjoint_forward(N, 7)
    grad, gth = sim.adjoint_backward(w.copy(), n_theta=6 * n)
    ref = oracle_lib.adjoint_run(og.nbr, p, X0, N, w, ckpt=7, g6=_oracle_g6(og, g6), want_gface=True)
    exist = og.nbr >= 0
    gf = gth.reshape(n, 6)
    assert rel_l2(gf[exist], ref["gface"][exist]) <= 1e-4, rel_l2(gf[exist], ref["gface"][exist])
    assert np.all(gf[~exist] == 0.0)
    for name in ("D", "rho", "mu", "beta", "v_som", "v_fom", "v_dom", "K_dom"):
        v = ref["grad"][name]
        assert abs(grad[name] - v) <= 1e-4 * abs(v) + 1e-30, (name, grad[name], v)


def test_face_conductances_rejected(vga, oracle_lib):
    img, og, g, X0 = _setup(vga, oracle_lib, (12, 12, 12), 0.4, 23)
    p = synth.paper_params()
    sim = vga.Sim(g, p)
    g6 = _faces(og, 7, junk=0.0) * np.float32(0.6)  # D dt sum_j g_ij <= 0.15 * 6 * 0.9 < 1
    i = int(np.argmax(og.nbr[:, 1] >= 0))
    bad = g6.copy()
    bad[i, 1] *= np.float32(1.1)  # g_ij != g_ji
    with pytest.raises(vga.VgaError) as e:
        sim.set_face_conductances(bad)
    assert e.value.name == "VGA_ERR_INVALID_ARG"
    bad = g6.copy()
    bad[i, 1] = np.nan
    with pytest.raises(vga.VgaError) as e:
        sim.set_face_conductances(bad)
    assert e.value.name == "VGA_ERR_INVALID_ARG"
    with pytest.raises(vga.VgaError) as e:  # D dt sum_j g_ij > 1 at the paper's time step
        sim.set_face_conductances(_faces(og, 7, junk=0.0) * np.float32(5.0))
    assert e.value.name == "VGA_ERR_UNSTABLE_DT"
    sim.set_face_conductances(g6)  # accepted; block calls refuse while it is set
    with pytest.raises(vga.VgaError):
        sim.get_block_conductances(6 * og.n)
