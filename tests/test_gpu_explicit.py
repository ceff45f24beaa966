"""Explicit synchronous/asynchronous stepping on the GPU (FP32 state) against the FP64 oracle."""
import numpy as np
import pytest

import synth
from tests.helpers import rel_l2

pytestmark = pytest.mark.gpu

TOL_L2 = 1e-5     # relative L2 per compartment against FP64
TOL_DRIFT = 1e-7  # relative total-mass drift


def _setup(vga, oracle_lib, shape, por, seed, keep=True, organic=False):
    img = synth.pore_mask(shape, por, seed)
    og = oracle_lib.graph_build(img, keep_largest=keep)
    g = vga.Graph(img, keep_largest=keep)
    assert g.n == og.n
    X0 = synth.initial_masses(synth.kept_mask_from_nodes(img.shape, og.voxel_of_node), seed,
                              with_organic_matter=organic)
    return img, og, g, X0


def _assert_close(got, ref, tol=TOL_L2):
    for c in range(5):
        assert rel_l2(got[c], ref[c]) <= tol, (c, rel_l2(got[c], ref[c]))


def test_c1_64cubed_1000_steps(vga, oracle_lib):
    """64^3, 17% porosity, largest component, paper parameters, dt = 0.9 h^2/(6D), 1000 steps."""
    img, og, g, X0 = _setup(vga, oracle_lib, (64, 64, 64), 0.17, 1)
    p = synth.paper_params()
    sim = vga.Sim(g, p)
    sim.set_masses(X0)
    sim.step(1000)
    got = sim.get_masses()
    ref = oracle_lib.explicit_run(og.nbr, p, X0, 1000)
    _assert_close(got, ref)
    tot = sim.totals()
    assert abs(tot.sum() - X0.sum()) <= TOL_DRIFT * X0.sum()
    assert np.allclose(tot, oracle_lib.totals(ref), rtol=1e-6, atol=1e-12)
    assert got.min() >= 0.0


def test_ten_thousand_steps_drift_and_error(vga, oracle_lib):
    """10^4 steps (the long-run configuration) on a 48^3 mask: relative L2 and drift every 2000."""
    img, og, g, X0 = _setup(vga, oracle_lib, (48, 48, 48), 0.2, 2, organic=True)
    p = synth.paper_params()
    sim = vga.Sim(g, p)
    sim.set_masses(X0)
    ref = X0.copy()
    for _ in range(5):
        sim.step(2000)
        ref = oracle_lib.explicit_run(og.nbr, p, ref, 2000)
        got = sim.get_masses()
        _assert_close(got, ref)
        assert abs(sim.totals().sum() - X0.sum()) <= TOL_DRIFT * X0.sum()


@pytest.mark.parametrize("transform", [0, 1])
def test_transform_variants(vga, oracle_lib, transform):
    img, og, g, X0 = _setup(vga, oracle_lib, (40, 36, 44), 0.22, 3, organic=True)
    p = synth.paper_params(transform=transform)
    sim = vga.Sim(g, p)
    sim.set_masses(X0)
    sim.step(300)
    _assert_close(sim.get_masses(), oracle_lib.explicit_run(og.nbr, p, X0, 300, transform=transform))


def test_clamps_active(vga, oracle_lib):
    """Rates large enough that every clamp of the synchronous listing fires (dyadic-free values)."""
    img, og, g, X0 = _setup(vga, oracle_lib, (20, 24, 28), 0.3, 4, organic=True)
    X0[0] = np.where(X0[1] > 0, X0[1] * 3.0, X0[0]).astype(np.float32)
    p = dict(D=1.0, dt=0.12, rho=3.0, mu=6.0, beta=0.55, v_som=9.0, v_fom=11.0, v_dom=40.0, K_dom=1e-5,
             scheme=0, transform=0)
    sim = vga.Sim(g, p)
    sim.set_masses(X0)
    sim.step(50)
    _assert_close(sim.get_masses(), oracle_lib.explicit_run(og.nbr, p, X0, 50), tol=2e-5)


def test_block_conductances(vga, oracle_lib):
    img, og, g, X0 = _setup(vga, oracle_lib, (32, 32, 32), 0.22, 5, organic=True)
    bs = 8
    nb = oracle_lib.block_grid(img.shape, bs)
    theta = synth.block_conductances(nb, 7)
    p = synth.paper_params(dt=0.9 / (6 * synth.D_DOM * theta.max()))
    sim = vga.Sim(g, p)
    sim.set_block_conductances(bs, theta.astype(np.float32))
    sim.set_masses(X0)
    sim.step(400)
    g6 = oracle_lib.block_face_weights(img.shape, bs, og.voxel_of_node, og.nbr, theta)
    _assert_close(sim.get_masses(), oracle_lib.explicit_run(og.nbr, p, X0, 400, g6=g6))


@pytest.mark.parametrize("shape,por", [((1, 1, 1), 0.0), ((1, 1, 3000), 0.0), ((3, 2, 5), 0.5),
                                       ((5, 40, 45), 0.55), ((2, 3, 1100), 0.1)])
def test_small_and_ragged(vga, oracle_lib, shape, por):
    """Single voxel, a long 1D path (several chunks, ragged tail), tiny graphs, several components."""
    rng = np.random.default_rng(11)
    img = (rng.random(shape) < por).astype(np.uint8)
    for keep in (True, False):
        og = oracle_lib.graph_build(img, keep_largest=keep)
        g = vga.Graph(img, keep_largest=keep)
        X0 = synth.random_masses(og.n, 3, scale=1e-3, density=0.5)
        p = synth.paper_params()
        sim = vga.Sim(g, p)
        sim.set_masses(X0)
        sim.step(37)
        _assert_close(sim.get_masses(), oracle_lib.explicit_run(og.nbr, p, X0, 37))


def test_empty_graph(vga):
    g = vga.Graph(np.ones((4, 4, 4), dtype=np.uint8))
    assert g.n == 0
    sim = vga.Sim(g, synth.paper_params())
    sim.set_masses(np.zeros((5, 0)))
    sim.step(10)
    assert np.all(sim.totals() == 0.0)
    assert sim.get_masses().shape == (5, 0)


def test_zero_and_one_step(vga, oracle_lib):
    img, og, g, X0 = _setup(vga, oracle_lib, (16, 16, 16), 0.3, 6)
    p = synth.paper_params()
    sim = vga.Sim(g, p)
    sim.set_masses(X0)
    sim.step(0)
    assert np.array_equal(sim.get_masses(), X0)
    sim.step(1)
    _assert_close(sim.get_masses(), oracle_lib.explicit_run(og.nbr, p, X0, 1), tol=1e-6)


def test_unstable_dt_rejected(vga):
    g = vga.Graph(np.zeros((3, 3, 3), dtype=np.uint8))
    p = synth.paper_params(dt=1.01 / (6 * synth.D_DOM))
    with pytest.raises(vga.VgaError) as e:
        vga.Sim(g, p)
    assert e.value.name == "VGA_ERR_UNSTABLE_DT"
    bad = synth.paper_params()
    bad["K_dom"] = 0.0
    with pytest.raises(vga.VgaError) as e:
        vga.Sim(g, bad)
    assert e.value.name == "VGA_ERR_INVALID_ARG"
    sim = vga.Sim(g, synth.paper_params())
    X = np.zeros((5, g.n))
    X[1, 0] = np.nan
    with pytest.raises(vga.VgaError) as e:
        sim.set_masses(X)
    assert e.value.name == "VGA_ERR_NONFINITE"


@pytest.mark.parametrize("precision", [0, 1])
def test_resume_is_bit_exact(vga, oracle_lib, precision):
    """N steps equal N/2 steps, checkpoint, restore into a new simulation, N/2 steps, bit for bit."""
    img, og, g, X0 = _setup(vga, oracle_lib, (30, 34, 38), 0.25, 8, organic=True)
    p = synth.paper_params()
    p["state_precision"] = precision
    a = vga.Sim(g, p)
    a.set_masses(X0)
    a.step(120)
    full = a.save_state()
    b = vga.Sim(g, p)
    b.set_masses(X0)
    b.step(60)
    saved = b.save_state()
    c = vga.Sim(g, p)
    c.load_state(saved)
    c.step(60)
    assert c.save_state() == full
    assert np.array_equal(c.get_masses(), a.get_masses())
    assert c.stats()["steps_done"] == 120
    bad = vga.Sim(g, dict(p, state_precision=1 - precision))
    with pytest.raises(vga.VgaError):
        bad.load_state(saved)


def test_plain_fp32_state_drifts(vga, oracle_lib):
    """The FP32-only storage mode runs, but its error grows with the step count: SOM hydrolysis
    (v_SOM dt = 1.5e-8 per step) is below half an FP32 ulp and never happens, while the compensated
    default tracks it."""
    img = np.zeros((6, 6, 6), dtype=np.uint8)
    og = oracle_lib.graph_build(img)
    g = vga.Graph(img)
    X0 = np.zeros((5, og.n))
    X0[2] = 1e-3
    ref = oracle_lib.explicit_run(og.nbr, synth.paper_params(), X0, 3000)
    errs = {}
    for prec in (0, 1):
        sim = vga.Sim(g, dict(synth.paper_params(), state_precision=prec))
        sim.set_masses(X0)
        sim.step(3000)
        errs[prec] = rel_l2(sim.get_masses()[2], ref[2])
    assert errs[0] < 1e-7
    assert errs[1] > 1e-5


def test_device_state_io(vga, oracle_lib):
    import torch

    img, og, g, X0 = _setup(vga, oracle_lib, (24, 24, 24), 0.25, 9)
    p = synth.paper_params()
    sim = vga.Sim(g, p)
    sim.set_masses(torch.from_numpy(X0).cuda())
    sim.step(25)
    out = torch.empty((5, g.n), dtype=torch.float64, device="cuda")
    sim.get_masses(out)
    torch.cuda.synchronize()
    _assert_close(out.cpu().numpy(), oracle_lib.explicit_run(og.nbr, p, X0, 25))
    f32 = torch.empty((5, g.n), dtype=torch.float32, device="cuda")
    sim.get_state_f32(f32)
    torch.cuda.synchronize()
    assert np.array_equal(f32.cpu().numpy(), out.cpu().numpy().astype(np.float32))
    host = sim.get_state_f32()
    assert np.array_equal(host, f32.cpu().numpy())


@pytest.mark.parametrize("block,transform,precision", [(False, 0, 0), (True, 0, 0), (False, 1, 0), (False, 0, 1)])
def test_kernel_variants_bit_identical(vga, oracle_lib, block, transform, precision):
    """Decode, staged and table stencil kernels (one and two nodes per thread), every chunk size:
    the same bits after 50 steps."""
    img, og, g, X0 = _setup(vga, oracle_lib, (40, 48, 36), 0.24, 12, organic=True)
    p = synth.paper_params(transform=transform)
    p["state_precision"] = precision
    bs = 8
    theta = synth.block_conductances(oracle_lib.block_grid(img.shape, bs), 4) if block else None
    if block:
        p["dt"] = 0.9 / (6 * synth.D_DOM * theta.max())
    states = []
    for variant, chunk in [(0, 1024), (1, 1024), (1, 512), (1, 2048), (0, 512), (0, 96), (2, 1024), (4, 1024), (5, 1024)]:
        sim = vga.Sim(g, p)
        sim.set_kernel(variant, chunk)
        if block:
            sim.set_block_conductances(bs, theta.astype(np.float32))
        sim.set_masses(X0)
        sim.step(50)
        states.append(sim.save_state())
    assert all(st == states[0] for st in states[1:])
    ref = oracle_lib.explicit_run(og.nbr, p, X0, 50, transform=transform,
                                  g6=oracle_lib.block_face_weights(img.shape, bs, og.voxel_of_node, og.nbr, theta)
                                  if block else None)
    last = vga.Sim(g, p)
    last.load_state(states[0])
    _assert_close(last.get_masses(), ref, tol=1e-5 if precision == 0 else 1e-4)


def test_autotune_keeps_state(vga, oracle_lib):
    img, og, g, X0 = _setup(vga, oracle_lib, (64, 64, 64), 0.2, 13)
    sim = vga.Sim(g, synth.paper_params())
    sim.set_masses(X0)
    sim.step(3)
    before = sim.save_state()
    res = sim.autotune(4)
    assert res["best"] is not None and len(res["entries"]) == 13
    assert sorted({e["variant"] for e in res["entries"]}) == [0, 1, 2, 3, 4, 5, 6]
    assert all(e["ms_per_step"] > 0 for e in res["entries"])
    assert sim.save_state() == before
    with pytest.raises(vga.VgaError):
        sim.set_kernel(1, 768)


def test_wide_z_offsets(vga, oracle_lib):
    """Planes of more than 65535 nodes need the 32-bit z offsets (the compact table applies only
    below that); both table forms and the decode kernel agree bit for bit and with the oracle."""
    img = np.zeros((4, 270, 260), dtype=np.uint8)  # 70,200 nodes per plane
    img[:, 100:110, 30:40] = 1
    og = oracle_lib.graph_build(img, keep_largest=True)
    g = vga.Graph(img)
    X0 = synth.random_masses(g.n, 9, scale=1e-3, density=0.5)
    p = synth.paper_params()
    outs = []
    for variant in (2, 4, 5, 0):
        sim = vga.Sim(g, p)
        sim.set_kernel(variant, 1024)
        sim.set_masses(X0)
        sim.step(12)
        outs.append(sim.get_masses())
    assert all(np.array_equal(outs[0], o) for o in outs[1:])
    _assert_close(outs[0], oracle_lib.explicit_run(og.nbr, p, X0, 12))


@pytest.mark.parametrize("nx", [1, 2, 3, 31, 63, 64, 65, 97])
def test_pair_kernel_ragged_rows(vga, oracle_lib, nx):
    """Two and four nodes per thread: a single x-row of nx nodes (a chain along x, so +-x
    neighbours cross group and warp boundaries, and counts that are not a multiple of the group
    leave a partial last group) plus a plane of scattered voxels; the same bits as one node per
    thread, and the oracle's values."""
    img = np.ones((3, 5, nx), dtype=np.uint8)  # 0 = pore
    img[1, 2, :] = 0
    rng = np.random.default_rng(nx)
    img[2] = rng.random((5, nx)) >= 0.5
    og = oracle_lib.graph_build(img, keep_largest=False)
    g = vga.Graph(img, keep_largest=False)
    assert g.n == og.n
    X0 = synth.random_masses(g.n, nx, scale=1e-3, density=0.7)
    p = synth.paper_params()
    outs = []
    for variant in (2, 4, 5):
        sim = vga.Sim(g, p)
        sim.set_kernel(variant, 1024)
        sim.set_masses(X0)
        sim.step(7)
        outs.append(sim.save_state())
    assert outs[0] == outs[1] and outs[0] == outs[2]
    last = vga.Sim(g, p)
    last.load_state(outs[1])
    _assert_close(last.get_masses(), oracle_lib.explicit_run(og.nbr, p, X0, 7))


@pytest.mark.parametrize("block,transform,precision,organic", [(False, 0, 0, False), (False, 0, 0, True),
                                                               (True, 0, 0, False), (False, 1, 0, False),
                                                               (False, 0, 1, False)])
def test_activity_skip_bit_identical(vga, oracle_lib, block, transform, precision, organic):
    """The sparse fused pass (groups of four nodes with MB = SOM = FOM = CO2 = 0 only diffuse DOM)
    gives the bits of the dense pass and of the one-node-per-thread kernel; the mask is rebuilt
    after each state upload (set_masses, set_state_f32, load_state), including states with negative
    zeros, and counts the nodes with any nonzero bit in MB, SOM, FOM or CO2."""
    img, og, g, X0 = _setup(vga, oracle_lib, (40, 48, 37), 0.24, 21, organic=organic)
    p = synth.paper_params(transform=transform)
    p["state_precision"] = precision
    bs = 8
    theta = synth.block_conductances(oracle_lib.block_grid(img.shape, bs), 4) if block else None
    if block:
        p["dt"] = 0.9 / (6 * synth.D_DOM * theta.max())
    X1 = X0.copy()
    rng = np.random.default_rng(3)
    X1[0, rng.choice(g.n, 40, replace=False)] = -0.0  # negative zeros mark a node as well
    X1[1, rng.choice(g.n, 40, replace=False)] = -0.0
    X1[0, rng.choice(g.n, 200, replace=False)] = 1e-4  # more biomass: a second, denser mask

    def run(variant, skip):
        sim = vga.Sim(g, p)
        sim.set_kernel(variant, 1024)
        sim.set_activity_skip(skip)
        if block:
            sim.set_block_conductances(bs, theta.astype(np.float32))
        sim.set_masses(X0)
        sim.step(30)
        a = sim.save_state()
        n0 = sim.stats()["active_nodes"]
        sim.set_masses(X1)
        sim.step(17)
        b = sim.save_state()
        n1 = sim.stats()["active_nodes"]
        sim.load_state(a)
        sim.step(5)
        c = sim.save_state()
        sim.set_state_f32(X0.astype(np.float32))
        sim.step(3)
        d = sim.save_state()
        sim.close()
        return (a, b, c, d), (n0, n1)

    ref, _ = run(2, False)
    dense, nd = run(5, False)
    sparse, ns = run(5, True)
    assert dense == ref
    assert sparse == ref
    assert nd == (-1, -1)
    marked = lambda X: int(np.count_nonzero((np.signbit(X[[0, 2, 3, 4]]) | (X[[0, 2, 3, 4]] != 0)).any(axis=0)
                                            | (np.signbit(X[1]) & (X[1] == 0))))
    assert ns == (marked(X0), marked(X1))
    assert 0 < ns[0] < g.n


@pytest.mark.parametrize("shape,por,transform,precision,organic", [
    ((40, 48, 37), 0.24, 0, 0, False),   # ragged in every axis (tiles of 32 x 16 x 16 cut at the borders)
    ((64, 64, 64), 0.17, 0, 0, True),    # every DOM node also holds SOM and FOM: 5% of nodes marked
    ((33, 20, 100), 0.3, 1, 0, False),   # asynchronous transformation, four tile columns in x
    ((50, 17, 31), 0.2, 0, 1, False),    # plain FP32 state, one tile column narrower than a word
])
def test_blocked_passes_bit_identical(vga, oracle_lib, shape, por, transform, precision, organic):
    """Variant 6 runs the fused passes of a sparse step call temporally blocked (3 passes per launch
    over tiles with a 3-voxel halo in shared memory).  Its state is the bits of variant 5 after every
    step count (1, 2, 3, 4 and 11 fused passes: every remainder of the 3-pass launches), after a
    state upload that rebuilds the mask, and across a save/load; the blocked path really ran."""
    img, og, g, X0 = _setup(vga, oracle_lib, shape, por, 31, organic=organic)
    p = synth.paper_params(transform=transform)
    p["state_precision"] = precision
    X1 = X0.copy()
    X1[0, np.random.default_rng(5).choice(g.n, 60, replace=False)] = 2e-4

    def run(variant):
        sim = vga.Sim(g, p)
        sim.set_kernel(variant, 1024)
        sim.set_masses(X0)
        out = []
        for k in (2, 3, 4, 5, 12):
            sim.step(k)
            out.append(sim.save_state())
        sim.set_masses(X1)
        sim.step(9)
        out.append(sim.save_state())
        sim.load_state(out[2])
        sim.step(6)
        out.append(sim.save_state())
        st = sim.stats()
        sim.close()
        return out, st

    ref, st5 = run(5)
    got, st6 = run(6)
    assert st5["blocked_passes"] == 0
    assert st6["blocked_passes"] == (1 + 2 + 3 + 4 + 11) + 8 + 5
    for k, (a, b) in enumerate(zip(ref, got)):
        assert a == b, k
    last = vga.Sim(g, p)
    last.load_state(got[-1])
    n_steps = 2 + 3 + 4 + 6
    _assert_close(last.get_masses(), oracle_lib.explicit_run(og.nbr, p, X0, n_steps, transform=transform),
                  tol=TOL_L2 if precision == 0 else 1e-4)


def test_blocked_passes_fall_back_when_marked_nodes_overflow(vga, oracle_lib):
    """With biomass in most nodes the marked nodes of a tile's region exceed its shared-memory list:
    the call runs unblocked (variant 5's passes) and the state is still the same bits."""
    img, og, g, X0 = _setup(vga, oracle_lib, (32, 32, 64), 0.3, 8)
    X0[0] = np.where(np.arange(g.n) % 2 == 0, 1e-5, 0.0)
    p = synth.paper_params()
    outs = []
    for variant in (5, 6):
        sim = vga.Sim(g, p)
        sim.set_kernel(variant, 1024)
        sim.set_masses(X0)
        sim.step(10)
        outs.append(sim.save_state())
        assert sim.stats()["blocked_passes"] == 0
        sim.close()
    assert outs[0] == outs[1]


def test_blocked_c1_against_oracle(vga, oracle_lib):
    """Variant 6 at the 64^3 reference configuration (1000 steps) against the FP64 oracle, with the
    per-node relative error of the marked nodes checked on its own (their DOM error would be diluted
    about 100x in the relative L2 over all nodes)."""
    img, og, g, X0 = _setup(vga, oracle_lib, (64, 64, 64), 0.17, 1)
    p = synth.paper_params()
    sim = vga.Sim(g, p)
    sim.set_kernel(6, 1024)
    sim.set_masses(X0)
    sim.step(1000)
    assert sim.stats()["blocked_passes"] == 999
    got = sim.get_masses()
    ref = oracle_lib.explicit_run(og.nbr, p, X0, 1000)
    _assert_close(got, ref)
    marked = (X0[[0, 2, 3, 4]] != 0).any(axis=0)
    assert marked.sum() > 10
    for c in range(5):
        r, m = ref[c, marked], got[c, marked]
        big = np.abs(r) > 1e-6 * np.abs(ref[c]).max()
        if big.any():
            assert np.max(np.abs(m[big] - r[big]) / np.abs(r[big])) <= 1e-5, c
    assert abs(sim.totals().sum() - X0.sum()) <= TOL_DRIFT * X0.sum()


def test_totals_scan_reports_nonfinite_and_negative(vga):
    """The totals pass scans the state: a negative mass is counted in the stats, a non-finite one
    (uploaded from device memory, which the host cannot check) makes vga_sim_totals return
    VGA_ERR_NONFINITE; the flags are cleared, so a clean state passes again."""
    import torch

    g = vga.Graph(np.zeros((8, 8, 8), dtype=np.uint8))
    sim = vga.Sim(g, synth.paper_params())
    X = np.zeros((5, g.n))
    X[1] = 1e-5
    X[0, ::7] = 2e-6
    sim.set_masses(X)
    sim.totals()
    assert sim.stats()["negative_reports"] == 0
    Xn = X.copy()
    Xn[3, 7] = -1e-9
    sim.set_masses(Xn)
    sim.totals()
    assert sim.stats()["negative_reports"] == 1
    Xd = torch.from_numpy(X).cuda()
    Xd[1, 3] = float("nan")
    sim.set_masses(Xd)
    with pytest.raises(vga.VgaError) as e:
        sim.totals()
    assert e.value.name == "VGA_ERR_NONFINITE"
    sim.set_masses(X)
    sim.step(5)
    assert np.isfinite(sim.totals()).all()
    assert sim.stats()["negative_reports"] == 1


@pytest.mark.parametrize("variant", [5, 2, 6])
def test_kernel_timing_spans_the_fused_passes(vga, oracle_lib, variant):
    """With timing on, a step call's fused passes count as n_steps - 1 timed launches of the fused
    kind and the first and last passes as one each; the state is the same bits as without timing."""
    img, og, g, X0 = _setup(vga, oracle_lib, (40, 36, 44), 0.2, 9)
    p = synth.paper_params()
    out = []
    for timing in (False, True):
        sim = vga.Sim(g, p)
        sim.set_kernel(variant, 1024)
        sim.set_masses(X0)
        sim.enable_timing(timing)
        sim.read_timing(reset=True)
        sim.step(37)
        sim.step(1)
        kt = sim.read_timing(reset=True)
        if timing:
            assert kt["fused_step"][1] == 36
            assert kt["fused_step"][0] > 0.0
            assert kt["transform"][1] == 2 and kt["diffuse"][1] == 2
        out.append(sim.save_state())
        sim.close()
    assert out[0] == out[1]


def test_rows_of_very_different_length(vga, oracle_lib):
    """Rows alternating between full pore rows and rows with a few pores: neighbouring nodes of one
    warp have +-y and +-z offsets hundreds apart. The sparse pass on the offset table matches the
    dense one-node kernel bit for bit, and the oracle."""
    nz, ny, nx = 6, 10, 600
    img = np.ones((nz, ny, nx), dtype=np.uint8)
    img[:, 0::2, :] = 0            # full pore rows
    img[:, 1::2, ::97] = 0         # a few pores between them, joining the full rows
    og = oracle_lib.graph_build(img)
    g = vga.Graph(img)
    X0 = synth.initial_masses(synth.kept_mask_from_nodes(img.shape, og.voxel_of_node), 3, with_organic_matter=True)
    p = synth.paper_params()
    out = []
    for variant in (5, 0):
        sim = vga.Sim(g, p)
        sim.set_kernel(variant, 1024)
        sim.set_masses(X0)
        sim.step(40)
        out.append((sim.save_state(), sim.get_masses()))
        sim.close()
    assert out[0][0] == out[1][0]
    ref = oracle_lib.explicit_run(og.nbr, p, X0, 40)
    _assert_close(out[0][1], ref)


@pytest.mark.parametrize("variant", [5, 2, 0])
def test_step_graphs_replay_bit_identical(vga, oracle_lib, variant):
    """On a small graph, a step call of a shape seen before is captured as a CUDA graph and later ones
    replay it (with the state-buffer parity and step count carried on the host); interleaved shapes,
    a parameter change and a new state between calls all give the bits of the same calls run
    launch by launch (kernel timing on turns the graphs off)."""
    img, og, g, X0 = _setup(vga, oracle_lib, (40, 36, 44), 0.2, 9)
    p = synth.paper_params()
    p2 = dict(p, rho=p["rho"] * 1.3)
    out = []
    for timing in (True, False):
        sim = vga.Sim(g, p)
        sim.set_kernel(variant, 1024)
        sim.enable_timing(timing)
        sim.set_masses(X0)
        for k in (7, 7, 7, 6, 7, 6, 7, 7):
            sim.step(k)
        mid = sim.save_state()
        sim.set_params(p2)
        for k in (7, 7, 7):
            sim.step(k)
        sim.set_masses(X0)
        for k in (9, 9, 9, 9):
            sim.step(k)
        out.append((mid, sim.save_state(), sim.stats()["steps_done"]))
        sim.close()
    assert out[0][0] == out[1][0]
    assert out[0][1] == out[1][1]
    assert out[0][2] == out[1][2]
