"""Implicit scheme (Scheme 2 by Jacobi-PCG) on the GPU against the FP64 oracle."""
import numpy as np
import pytest

import synth
from tests.helpers import rel_l2

pytestmark = pytest.mark.gpu


def _setup(vga, oracle_lib, shape, por, seed):
    img = synth.pore_mask(shape, por, seed)
    og = oracle_lib.graph_build(img)
    g = vga.Graph(img)
    X0 = synth.initial_masses(synth.kept_mask_from_nodes(img.shape, og.voxel_of_node), seed,
                              with_organic_matter=True)
    return img, og, g, X0


def test_implicit_ten_times_explicit_limit(vga, oracle_lib):
    """dt = 10 x the explicit limit (D dt = 1.5), rtol 1e-8: the configuration of the paper-scale run."""
    img, og, g, X0 = _setup(vga, oracle_lib, (48, 48, 48), 0.17, 1)
    p = synth.paper_params(dt=10 * 0.9 / (6 * synth.D_DOM), scheme=1, cg_rtol=1e-8, cg_maxit=500)
    sim = vga.Sim(g, p)
    sim.set_masses(X0)
    sim.step(20)
    got = sim.get_masses()
    ref, status, iters, worst = oracle_lib.implicit_run(og.nbr, p, X0, 20, rtol=1e-12)
    assert status == 0
    for c in range(5):
        assert rel_l2(got[c], ref[c]) <= 1e-5, c
    st = sim.stats()
    assert 0 < st["cg_iterations"] <= 20 * 100
    assert st["cg_last_relres"] <= 1e-8
    assert abs(sim.totals().sum() - X0.sum()) <= 1e-7 * X0.sum()


def test_implicit_block_weights_and_async(vga, oracle_lib):
    img, og, g, X0 = _setup(vga, oracle_lib, (24, 32, 24), 0.25, 2)
    bs = 8
    nb = oracle_lib.block_grid(img.shape, bs)
    theta = synth.block_conductances(nb, 3)
    p = synth.paper_params(dt=5 * 0.9 / (6 * synth.D_DOM), scheme=1, transform=1, cg_rtol=1e-10)
    sim = vga.Sim(g, p)
    sim.set_block_conductances(bs, theta.astype(np.float32))
    sim.set_masses(X0)
    sim.step(8)
    g6 = oracle_lib.block_face_weights(img.shape, bs, og.voxel_of_node, og.nbr, theta)
    ref, status, _, _ = oracle_lib.implicit_run(og.nbr, p, X0, 8, rtol=1e-13, g6=g6, transform=1)
    got = sim.get_masses()
    for c in range(5):
        assert rel_l2(got[c], ref[c]) <= 1e-5, c


@pytest.mark.parametrize("solver", [1, 2, 0])
def test_not_converged_reported(vga, oracle_lib, solver):
    """cg_maxit reached before cg_rtol: every solver, including the graph-driven loops, stops and
    reports it."""
    img, og, g, X0 = _setup(vga, oracle_lib, (24, 24, 24), 0.25, 3)
    p = synth.paper_params(dt=50 * 0.9 / (6 * synth.D_DOM), scheme=1, cg_rtol=1e-14, cg_maxit=2)
    sim = vga.Sim(g, p)
    sim.set_solver(solver)
    sim.set_masses(X0)
    with pytest.raises(vga.VgaError) as e:
        sim.step(1)
    assert e.value.name == "VGA_ERR_NOT_CONVERGED"


def test_zero_dom(vga):
    g = vga.Graph(np.zeros((6, 6, 6), dtype=np.uint8))
    X = np.zeros((5, g.n))
    X[0] = 1e-4
    p = synth.paper_params(dt=1e-4, scheme=1)
    sim = vga.Sim(g, p)
    sim.set_masses(X)
    sim.step(3)
    assert np.isfinite(sim.get_masses()).all()


@pytest.mark.parametrize("rtol", [1e-6, 1e-8, 1e-10])
def test_mixed_refinement_matches_fp64_pcg(vga, oracle_lib, rtol):
    """The default implicit solver (float-float refinement around FP32 PCG) and the FP64 PCG both land
    within the requested tolerance of the oracle's solution; the mixed solver's reported residual
    is the true one, so it is at most rtol."""
    img, og, g, X0 = _setup(vga, oracle_lib, (40, 40, 40), 0.2, 7)
    p = synth.paper_params(dt=10 * 0.9 / (6 * synth.D_DOM), scheme=1, cg_rtol=rtol, cg_maxit=2000)
    ref, status, _, _ = oracle_lib.implicit_run(og.nbr, p, X0, 5, rtol=1e-13)
    assert status == 0
    out = {}
    for solver in (vga.VGA_SOLVER_MIXED_REFINEMENT, vga.VGA_SOLVER_FP64_PCG):
        sim = vga.Sim(g, p)
        sim.set_solver(solver)
        sim.set_masses(X0)
        sim.step(5)
        out[solver] = sim.get_masses()
        st = sim.stats()
        if solver == vga.VGA_SOLVER_MIXED_REFINEMENT:
            assert st["cg_last_relres"] <= rtol
        # a solve stops within rtol of the exact one; 5 steps accumulate at most ~5 rtol (x cond)
        assert rel_l2(out[solver][1], ref[1]) <= max(100 * rtol, 2e-7), (solver, rel_l2(out[solver][1], ref[1]))
        # B conserves mass exactly, so a solve stopped at rtol conserves it to about rtol
        assert abs(sim.totals().sum() - X0.sum()) <= max(1e-7, 10 * rtol) * X0.sum()
    for c in (0, 2, 3, 4):  # compartments the solve does not touch agree closely
        assert rel_l2(out[0][c], out[1][c]) <= 1e-6


def test_unknown_solver_rejected(vga):
    g = vga.Graph(np.zeros((4, 4, 4), dtype=np.uint8))
    sim = vga.Sim(g, synth.paper_params(scheme=1))
    with pytest.raises(vga.VgaError):
        sim.set_solver(7)


def test_mixed_graph_loop_matches_host_loop(vga, oracle_lib):
    """The mixed solve as one CUDA graph (device-side while loops) and driven from the host run the
    same kernels in the same order: the same bits and iteration counts, over an odd number of steps
    (both DOM buffer parities, cached graphs reused), and one graph launch per step."""
    img, og, g, X0 = _setup(vga, oracle_lib, (40, 36, 44), 0.2, 11)
    p = synth.paper_params(dt=10 * 0.9 / (6 * synth.D_DOM), scheme=1, cg_rtol=1e-9, cg_maxit=2000)
    out, stats = {}, {}
    for solver in (vga.VGA_SOLVER_MIXED_REFINEMENT, vga.VGA_SOLVER_MIXED_HOST_LOOP):
        sim = vga.Sim(g, p)
        sim.set_solver(solver)
        sim.set_masses(X0)
        for k in (1, 2, 4):
            sim.step(k)
        out[solver] = sim.save_state()
        stats[solver] = sim.stats()
        sim.close()
    assert out[1] == out[2]
    assert stats[1]["cg_iterations"] == stats[2]["cg_iterations"] > 0
    assert stats[1]["cg_last_relres"] == stats[2]["cg_last_relres"] <= 1e-9
    assert stats[1]["graph_launches"] == 7
    assert stats[2]["graph_launches"] == 0
    ref, status, _, _ = oracle_lib.implicit_run(og.nbr, p, X0, 7, rtol=1e-13)
    assert status == 0
    last = vga.Sim(g, p)
    last.load_state(out[1])
    got = last.get_masses()
    for c in range(5):
        assert rel_l2(got[c], ref[c]) <= 1e-5, c


@pytest.mark.parametrize("solver", [1, 2])
def test_mixed_solve_does_not_depend_on_the_mass_unit(vga, oracle_lib, solver):
    """The FP32 inner solve squares residuals; in a small mass unit (masses x 2^-40, e.g. grams
    instead of micrograms) those squares would underflow and the solve would stop at once on a
    zero residual norm.  The solve runs on a power-of-two scaled right-hand side, so with masses and
    K_DOM both x 2^-40 every result is the unscaled one x 2^-40 bit for bit, with the same iteration
    count and residual; with a factor 1e-12 (not a power of two) it still converges to rtol."""
    img, og, g, X0 = _setup(vga, oracle_lib, (32, 36, 28), 0.22, 13)
    p = synth.paper_params(dt=10 * 0.9 / (6 * synth.D_DOM), scheme=1, cg_rtol=1e-8, cg_maxit=2000)
    runs = {}
    for name, f in (("one", 1.0), ("pow2", 2.0 ** -40), ("1e-12", 1e-12)):
        q = dict(p)
        q["K_dom"] = p["K_dom"] * f
        sim = vga.Sim(g, q)
        sim.set_solver(solver)
        sim.set_masses(X0 * f)
        sim.step(3)
        runs[name] = (sim.get_masses(), sim.stats())
        sim.close()
    (x1, s1), (x2, s2), (x3, s3) = runs["one"], runs["pow2"], runs["1e-12"]
    assert s1["cg_iterations"] > 0
    assert np.array_equal(x2 * 2.0 ** 40, x1)
    assert s2["cg_iterations"] == s1["cg_iterations"]
    assert s2["cg_last_relres"] == s1["cg_last_relres"]
    assert s3["cg_last_relres"] <= 1e-8
    assert abs(s3["cg_iterations"] - s1["cg_iterations"]) <= 3
    for c in range(5):
        assert rel_l2(x3[c] / 1e-12, x1[c]) <= 1e-6, c
