"""Transformation and diffusion on different time steps (Sec. III; Table 1 test 3 uses 0.1 s for
diffusion and 0.43 s for the transformation) on the GPU against the FP64 oracle's global-clock
runner."""
import numpy as np
import pytest

import synth
from tests.helpers import rel_l2

pytestmark = pytest.mark.gpu

TOL_L2 = 1e-5
TOL_DRIFT = 1e-7


def _setup(vga, oracle_lib, shape=(40, 36, 44), por=0.2, seed=11):
    img = synth.pore_mask(shape, por, seed)
    og = oracle_lib.graph_build(img, keep_largest=True)
    g = vga.Graph(img)
    assert g.n == og.n
    X0 = synth.initial_masses(synth.kept_mask_from_nodes(img.shape, og.voxel_of_node), seed,
                              with_organic_matter=True)
    return og, g, X0


def _close(got, ref, tol=TOL_L2):
    for c in range(5):
        assert rel_l2(got[c], ref[c]) <= tol, (c, rel_l2(got[c], ref[c]))


@pytest.mark.parametrize("transform", [0, 1])
@pytest.mark.parametrize("ratio", [4.3, 1.0 / 2.5])
def test_explicit_subcycled_parity(vga, oracle_lib, transform, ratio):
    """dt_transform = 4.3 dt (the 0.1 s / 0.43 s pair: one transformation every 4 or 5 steps) and
    dt_transform = dt / 2.5 (two or three per step); the run is split over calls of 1, 7 and 92
    steps so the clock must carry across calls and across the pipelined passes."""
    og, g, X0 = _setup(vga, oracle_lib)
    p = synth.paper_params(transform=transform)
    # scale the rates so that the transformation moves mass visibly within 100 steps
    p.update(v_dom=p["v_dom"] * 2000, rho=p["rho"] * 2000, mu=p["mu"] * 2000, v_fom=p["v_fom"] * 2000,
             v_som=p["v_som"] * 2000)
    p["dt_transform"] = ratio * p["dt"]
    sim = vga.Sim(g, p)
    sim.set_masses(X0)
    for k in (1, 7, 92):
        sim.step(k)
    got = sim.get_masses()
    ref = oracle_lib.run_subcycled(og.nbr, p, X0, 100, dt_transform=p["dt_transform"], transform=transform)
    _close(got, ref)
    plain = oracle_lib.explicit_run(og.nbr, dict(p, dt_transform=0.0), X0, 100, transform=transform)
    assert max(rel_l2(plain[c], ref[c]) for c in (0, 2, 4)) > 10 * TOL_L2  # the clock matters
    assert abs(sim.totals().sum() - X0.sum()) <= TOL_DRIFT * X0.sum()


def test_equal_steps_bit_identical(vga, oracle_lib):
    """dt_transform = dt and dt_transform = 0 run the same kernels on the same values."""
    og, g, X0 = _setup(vga, oracle_lib, shape=(24, 20, 28))
    p = synth.paper_params()
    a = vga.Sim(g, p)
    b = vga.Sim(g, dict(p, dt_transform=p["dt"]))
    for s in (a, b):
        s.set_masses(X0)
        s.step(33)
    assert np.array_equal(a.get_masses(), b.get_masses())


def test_implicit_subcycled_parity(vga, oracle_lib):
    """Scheme 2 with a 1 s diffusion step and a 0.43 s transformation step (two or three
    transformations per solve)."""
    og, g, X0 = _setup(vga, oracle_lib, shape=(32, 32, 32))
    s = 1.0 / 86400.0
    p = synth.paper_params(dt=1.0 * s, scheme=synth.SCHEME_IMPLICIT_PCG, cg_rtol=1e-10, cg_maxit=2000)
    p.update(v_dom=p["v_dom"] * 200, rho=p["rho"] * 200, mu=p["mu"] * 200)
    p["dt_transform"] = 0.43 * s
    sim = vga.Sim(g, p)
    sim.set_masses(X0)
    sim.step(4)
    sim.step(6)
    got = sim.get_masses()
    ref = oracle_lib.run_subcycled(og.nbr, p, X0, 10, dt_transform=p["dt_transform"], scheme=1, rtol=1e-12)
    _close(got, ref)


def test_clock_survives_save_load(vga, oracle_lib):
    """The step counter is part of the saved state, so a resumed run keeps the transformation clock."""
    og, g, X0 = _setup(vga, oracle_lib, shape=(24, 20, 28))
    p = synth.paper_params()
    p["dt_transform"] = 4.3 * p["dt"]
    a = vga.Sim(g, p)
    a.set_masses(X0)
    a.step(13)
    blob = a.save_state()
    a.step(20)
    b = vga.Sim(g, p)
    b.load_state(blob)
    b.step(20)
    assert b.stats()["steps_done"] == 33
    assert np.array_equal(a.get_masses(), b.get_masses())


def test_adjoint_and_batch_reject_subcycling(vga, oracle_lib):
    og, g, X0 = _setup(vga, oracle_lib, shape=(16, 16, 16))
    p = synth.paper_params()
    p["dt_transform"] = 2 * p["dt"]
    sim = vga.Sim(g, p)
    with pytest.raises(vga.VgaError) as e:
        sim.adjoint_forward(4, 2)
    assert e.value.name == "VGA_ERR_UNSUPPORTED"
    with pytest.raises(vga.VgaError) as e:
        vga.Batch([g], [p])
    assert e.value.name == "VGA_ERR_UNSUPPORTED"
    with pytest.raises(vga.VgaError) as e:
        vga.Sim(g, dict(p, dt_transform=-1.0))
    assert e.value.name == "VGA_ERR_INVALID_ARG"
