"""Wavefront execution of the explicit time loop (several fused passes in one persistent launch)
gives bit-identical results to one launch per pass, for every chunk size, depth and grid size,
both state precisions, both transformations and block conductances."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def _setup(vga, oracle_lib, shape=(48, 44, 52), por=0.22, seed=5):
    img = synth.pore_mask(shape, por, seed)
    og = oracle_lib.graph_build(img, keep_largest=True)
    g = vga.Graph(img)
    X0 = synth.initial_masses(synth.kept_mask_from_nodes(img.shape, og.voxel_of_node), seed, with_organic_matter=True)
    return img, g, X0


def _run(vga, g, p, X0, steps, wave=None, blocks=None):
    sim = vga.Sim(g, p)
    if blocks is not None:
        sim.set_block_conductances(*blocks)
    if wave is not None:
        sim.set_wavefront(*wave)
    sim.set_masses(X0)
    for k in steps:
        sim.step(k)
    out = sim.get_masses()
    st = sim.stats()
    sim.close()
    return out, st


@pytest.mark.parametrize("wave", [(256, 1, 0), (256, 4, 0), (512, 2, 1), (256, 8, 2), (1024, 3, 0), (8192, 4, 0)])
def test_bit_identical_to_one_launch_per_pass(vga, oracle_lib, wave):
    img, g, X0 = _setup(vga, oracle_lib)
    p = synth.paper_params()
    steps = (2, 3, 7, 50)
    ref, _ = _run(vga, g, p, X0, steps)
    got, st = _run(vga, g, p, X0, steps, wave=wave)
    assert np.array_equal(got, ref)
    assert st["steps_done"] == sum(steps)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("transform", [0, 1])
def test_precisions_and_transforms(vga, oracle_lib, precision, transform):
    img, g, X0 = _setup(vga, oracle_lib, shape=(40, 40, 40))
    p = synth.paper_params(transform=transform)
    p["state_precision"] = precision
    ref, _ = _run(vga, g, p, X0, (31,))
    got, _ = _run(vga, g, p, X0, (31,), wave=(256, 4, 0))
    assert np.array_equal(got, ref)


def test_block_conductances(vga, oracle_lib):
    img, g, X0 = _setup(vga, oracle_lib, shape=(40, 40, 40))
    bs = 8
    nb = (5, 5, 5)
    theta = synth.block_conductances(nb, 3, spread=0.1).astype(np.float32)  # 6 D dt max theta <= 1
    p = synth.paper_params()
    ref, _ = _run(vga, g, p, X0, (25,), blocks=(bs, theta))
    got, _ = _run(vga, g, p, X0, (25,), wave=(512, 4, 0), blocks=(bs, theta))
    assert np.array_equal(got, ref)


def test_subcycled_runs_one_pass_per_launch(vga, oracle_lib):
    """Different transformation and diffusion steps use the per-pass launches (same result)."""
    img, g, X0 = _setup(vga, oracle_lib, shape=(32, 32, 32))
    p = synth.paper_params()
    p["dt_transform"] = 4.3 * p["dt"]
    ref, _ = _run(vga, g, p, X0, (20,))
    got, _ = _run(vga, g, p, X0, (20,), wave=(256, 4, 0))
    assert np.array_equal(got, ref)


def test_autotune_times_wavefront_candidates(vga, oracle_lib):
    img, g, X0 = _setup(vga, oracle_lib, shape=(40, 40, 40))
    sim = vga.Sim(g, synth.paper_params())
    sim.set_masses(X0)
    before = sim.get_masses()
    r = sim.autotune(10)
    assert any(e["variant"] == 3 and e["depth"] > 0 for e in r["entries"])
    assert np.array_equal(sim.get_masses(), before)
    sim.step(12)
    ref, _ = _run(vga, g, synth.paper_params(), X0, (12,))
    assert np.array_equal(sim.get_masses(), ref)


def test_invalid_wavefront_parameters(vga, oracle_lib):
    img, g, X0 = _setup(vga, oracle_lib, shape=(16, 16, 16))
    sim = vga.Sim(g, synth.paper_params())
    for bad in [(100, 4, 0), (256, 0, 0), (256, 65, 0), (9216, 4, 0), (256, 4, -1)]:
        with pytest.raises(vga.VgaError):
            sim.set_wavefront(*bad)


@pytest.mark.parametrize("wave", [(256, 4, 0), (1024, 3, 0), (512, 2, 1)])
def test_wavefront_against_oracle(vga, oracle_lib, wave):
    """The wavefront loop (variant 3) against the FP64 oracle at the 64^3 configuration (Sec. IV.C
    initial state, 400 steps in calls of 1, 9, 90 and 300): relative L2 per compartment within
    1e-5, the marked nodes' per-node relative error within 1e-5 on their own (diluted ~100x in the
    norm over all nodes), and the total mass within 1e-7."""
    from tests.helpers import rel_l2

    img = synth.pore_mask((64, 64, 64), 0.17, 1)
    og = oracle_lib.graph_build(img, keep_largest=True)
    g = vga.Graph(img)
    X0 = synth.initial_masses(synth.kept_mask_from_nodes(img.shape, og.voxel_of_node), 1)
    p = synth.paper_params()
    got, st = _run(vga, g, p, X0, (1, 9, 90, 300), wave=wave)
    assert st["steps_done"] == 400
    ref = oracle_lib.explicit_run(og.nbr, p, X0, 400)
    for c in range(5):
        assert rel_l2(got[c], ref[c]) <= 1e-5, (c, rel_l2(got[c], ref[c]))
    marked = (X0[[0, 2, 3, 4]] != 0).any(axis=0)
    assert marked.sum() > 10
    for c in range(5):
        r, m = ref[c, marked], got[c, marked]
        big = np.abs(r) > 1e-6 * np.abs(ref[c]).max()
        if big.any():
            assert np.max(np.abs(m[big] - r[big]) / np.abs(r[big])) <= 1e-5, c
    assert abs(got.sum() - X0.sum()) <= 1e-7 * X0.sum()
