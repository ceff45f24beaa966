"""Batched persistent path: several uneven instances with their own rates in one cooperative
launch sequence, against the FP64 oracle per instance and bit-identical to single simulations."""
import numpy as np
import pytest

import synth
from tests.helpers import rel_l2

pytestmark = pytest.mark.gpu


def _instances(oracle_lib, count=5, seed=41, lo=12, hi=40):
    specs = synth.batch_instances(count, seed, side_lo=lo, side_hi=hi)
    out = []
    for k, sp in enumerate(specs):
        img = synth.pore_mask(sp["shape"], sp["porosity"], sp["mask_seed"])
        og = oracle_lib.graph_build(img)
        X0 = synth.initial_masses(synth.kept_mask_from_nodes(img.shape, og.voxel_of_node), sp["mass_seed"],
                                  with_organic_matter=True)
        out.append((img, og, X0, sp["params"]))
    return out


def test_batch_matches_oracle_and_single_sims(vga, oracle_lib):
    inst = _instances(oracle_lib)
    graphs = [vga.Graph(img) for img, _, _, _ in inst]
    b = vga.Batch(graphs, [p for _, _, _, p in inst])
    for k, (_, _, X0, _) in enumerate(inst):
        b.set_masses(k, X0)
    b.step(150)
    b.step(1)
    st = b.stats()
    assert st["steps_done"] == 151 and st["instances"] == len(inst)
    for k, (img, og, X0, p) in enumerate(inst):
        got = b.get_masses(k)
        ref = oracle_lib.explicit_run(og.nbr, p, X0, 151)
        for c in range(5):
            assert rel_l2(got[c], ref[c]) <= 1e-5, (k, c)
        sim = vga.Sim(graphs[k], p)
        sim.set_kernel(2, 1024)
        sim.set_masses(X0)
        sim.step(150)
        sim.step(1)
        assert np.array_equal(sim.get_masses(), got)


@pytest.mark.parametrize("spl,bps,graph", [(1, 0, True), (7, 2, True), (1000, 0, False), (3, 1, False)])
def test_launch_shapes_bit_identical(vga, oracle_lib, spl, bps, graph):
    inst = _instances(oracle_lib, count=3, seed=43)
    graphs = [vga.Graph(img) for img, _, _, _ in inst]
    ref = vga.Batch(graphs, [p for _, _, _, p in inst])
    other = vga.Batch(graphs, [p for _, _, _, p in inst])
    other.set_launch(spl, bps, graph)
    for b in (ref, other):
        for k, (_, _, X0, _) in enumerate(inst):
            b.set_masses(k, X0)
        b.step(40)
        b.step(40)
    for k in range(len(inst)):
        assert np.array_equal(ref.get_masses(k), other.get_masses(k))


def test_batch_autotune_and_empty_instance(vga, oracle_lib):
    inst = _instances(oracle_lib, count=3, seed=47)
    graphs = [vga.Graph(img) for img, _, _, _ in inst]
    empty = vga.Graph(np.ones((4, 4, 4), dtype=np.uint8))
    params = [p for _, _, _, p in inst] + [synth.paper_params()]
    b = vga.Batch(graphs + [empty], params)
    for k, (_, _, X0, _) in enumerate(inst):
        b.set_masses(k, X0)
    before = [b.get_masses(k) for k in range(len(inst))]
    res = b.autotune(10)
    assert res["best"] is not None and len(res["entries"]) == 9
    assert all(np.array_equal(b.get_masses(k), before[k]) for k in range(len(inst)))
    b.step(20)
    assert b.get_masses(len(inst)).shape == (5, 0)


@pytest.mark.parametrize("organic", [False, True])
def test_batch_sparse_equals_dense(vga, oracle_lib, organic):
    """The batch's sparse fused passes (nodes with MB = SOM = FOM = CO2 = 0 only diffuse DOM) give
    the bits of the dense passes and of single simulations with the sparse pass off, over calls of
    several lengths and a second upload of the masses."""
    specs = synth.batch_instances(6, 77, side_lo=16, side_hi=44)
    inst = []
    for sp in specs:
        img = synth.pore_mask(sp["shape"], sp["porosity"], sp["mask_seed"])
        og = oracle_lib.graph_build(img)
        X0 = synth.initial_masses(synth.kept_mask_from_nodes(img.shape, og.voxel_of_node), sp["mass_seed"],
                                  with_organic_matter=organic)
        inst.append((img, og, X0, sp["params"]))
    graphs = [vga.Graph(img) for img, _, _, _ in inst]
    params = [p for _, _, _, p in inst]
    outs = []
    for skip in (True, False):
        b = vga.Batch(graphs, params)
        b.set_activity_skip(skip)
        for k, (_, _, X0, _) in enumerate(inst):
            b.set_masses(k, X0)
        b.step(40)
        b.step(1)
        b.step(7)
        mid = [b.get_masses(k) for k in range(len(inst))]
        for k, (_, _, X0, _) in enumerate(inst):
            b.set_masses(k, 0.5 * X0)
        b.step(23)
        outs.append((mid, [b.get_masses(k) for k in range(len(inst))]))
        b.close()
    for a, c in zip(outs[0][0] + outs[0][1], outs[1][0] + outs[1][1]):
        assert np.array_equal(a, c)
    for k, (_, _, X0, p) in enumerate(inst):
        sim = vga.Sim(graphs[k], p)
        sim.set_activity_skip(False)
        sim.set_masses(X0)
        sim.step(40)
        sim.step(1)
        sim.step(7)
        assert np.array_equal(sim.get_masses(), outs[0][0][k])


@pytest.mark.parametrize("skip", [0, 5])
def test_barrier_wait_runs_out_and_batch_recovers(vga, oracle_lib, skip):
    """Bounded waits: one block of every launch leaves before its first grid-barrier arrival, so the
    others' waits run out after 4096 polls; the step returns VGA_ERR_TIMEOUT (no fault, no hang).
    With the hook off, the same batch handle, given its masses again, runs bit-identical to a fresh
    batch and matches the oracle."""
    inst = _instances(oracle_lib, count=3, seed=47)
    graphs = [vga.Graph(img) for img, _, _, _ in inst]
    params = [p for _, _, _, p in inst]
    b = vga.Batch(graphs, params)
    fresh = vga.Batch(graphs, params)
    for k, (_, _, X0, _) in enumerate(inst):
        b.set_masses(k, X0)
        fresh.set_masses(k, X0)
    b.set_wait_test(skip, 4096)
    with pytest.raises(vga.VgaError) as e:
        b.step(20)
    assert e.value.name == "VGA_ERR_TIMEOUT"
    b.set_wait_test(-1, 0)
    for k, (_, _, X0, _) in enumerate(inst):
        b.set_masses(k, X0)
    b.step(20)
    fresh.step(20)
    for k, (img, og, X0, p) in enumerate(inst):
        got = b.get_masses(k)
        assert np.array_equal(got, fresh.get_masses(k)), k
        ref = oracle_lib.explicit_run(og.nbr, p, X0, 20)
        for c in range(5):
            assert rel_l2(got[c], ref[c]) <= 1e-5, (k, c)
