"""Pins of the oracle's microbial transformation (Sec. II.C eq. 3; Appendix A listings).

Hand-worked single-voxel cases use dyadic numbers so every intermediate value is exact in binary
floating point; each expected value is derived in the comment from the listing's steps.
"""
import numpy as np
import pytest

import synth

BASE = dict(D=0.0, dt=1.0, rho=0.25, mu=0.5, beta=0.5, v_som=0.125, v_fom=0.25, v_dom=0.5, K_dom=1.0)


def _p(**kw):
    p = dict(BASE)
    p.update(kw)
    return p


# Synchronous transformation (Appendix A, the listing computing every flux from the old state).
SYNC_CASES = [
    # no clamp: uptake = 0.5*1/(1+1)*0.25 = 0.0625; resp = 0.0625; morta = 0.125 (sum 0.1875 <= 0.25)
    # mortaDOM = mortaSOM = 0.0625; turnFOM = 0.25*1 = 0.25; turnSOM = 0.125*1 = 0.125
    (_p(), [0.25, 1.0, 1.0, 1.0, 0.0], [0.125, 1.375, 0.9375, 0.75, 0.0625]),
    # uptake clamp: 16*1/2*1 = 8 > x2 = 1 -> uptake = 1; resp 0.25, morta 0.5 (sum 0.75 <= 1)
    (_p(v_dom=16.0), [1.0, 1.0, 0.0, 0.0, 0.0], [1.25, 0.25, 0.25, 0.0, 0.25]),
    # resp + morta = 0.75 + 0.5 > x1 = 1, morta <= x1 -> resp = 1 - 0.5 = 0.5; v_dom = 0
    (_p(rho=0.75, v_dom=0.0), [1.0, 0.5, 0.0, 0.0, 0.0], [0.0, 0.75, 0.25, 0.0, 0.5]),
    # morta = 2 > x1 = 1 -> morta = 1, resp = 0
    (_p(rho=0.25, mu=2.0, v_dom=0.0), [1.0, 0.0, 0.0, 0.0, 0.125], [0.0, 0.5, 0.5, 0.0, 0.125]),
    # hydrolysis clamps: turnFOM = 2*1 > 1 -> 1; turnSOM = 4*0.5 > 0.5 -> 0.5; MB = 0
    (_p(v_fom=2.0, v_som=4.0), [0.0, 0.0, 0.5, 1.0, 0.0], [0.0, 1.5, 0.0, 0.0, 0.0]),
    # empty voxel stays empty
    (_p(), [0.0, 0.0, 0.0, 0.0, 0.0], [0.0, 0.0, 0.0, 0.0, 0.0]),
]

# Asynchronous transformation (Appendix A sequential listing, readings: SOM/FOM branches test their
# own turnover, add-then-zero in the exhaustion branches, MB reset when mortality exceeds it).
ASYNC_CASES = [
    # x1 = 0.25, x2 = 1: uptake 0.0625 < 1 -> x1 = 0.3125, x2 = 0.9375
    # morta = 0.5*0.3125 = 0.15625 < x1 -> x1 = 0.15625, x2 += 0.078125, x3 += 0.078125
    # resp = 0.25*0.15625 = 0.0390625 -> x1 = 0.1171875, x5 = 0.0390625
    # SOM: x3 = 1.078125, turnSOM = 0.125*1.078125 = 0.134765625 -> x3 = 0.943359375, x2 += it
    # FOM: turnFOM = 0.25 -> x4 = 0.75, x2 += 0.25
    (_p(), [0.25, 1.0, 1.0, 1.0, 0.0],
     [0.1171875, 0.9375 + 0.078125 + 0.134765625 + 0.25, 0.943359375, 0.75, 0.0390625]),
    # uptake 8 >= x2 = 1 -> x1 = 2, x2 = 0; morta = 1 < 2 -> x1 = 1, x2 = 0.5, x3 = 0.5;
    # resp = 0.25 -> x1 = 0.75, x5 = 0.25; SOM: turnSOM = 0.0625 -> x3 = 0.4375, x2 = 0.5625
    (_p(v_dom=16.0), [1.0, 1.0, 0.0, 0.0, 0.0], [0.75, 0.5625, 0.4375, 0.0, 0.25]),
    # mortality exhausts MB: morta = 2*1 >= 1 -> x2 += 0.5, x3 += 0.5, x1 = 0; resp = 0
    # then SOM: turnSOM = 0.125*0.5 = 0.0625 -> x3 = 0.4375, x2 = 0.5625
    (_p(mu=2.0, v_dom=0.0), [1.0, 0.0, 0.0, 0.0, 0.0], [0.0, 0.5625, 0.4375, 0.0, 0.0]),
    # respiration exhausts MB: morta = 0.25 < 1 -> x1 = 0.75; resp = 2*0.75 >= 0.75 -> x5 = 0.75, x1 = 0
    (_p(mu=0.25, rho=2.0, v_dom=0.0, beta=0.5, v_som=0.0), [1.0, 0.0, 0.0, 0.0, 0.0],
     [0.0, 0.125, 0.125, 0.0, 0.75]),
    # hydrolysis exhaustion: turnSOM = 4*0.5 >= 0.5 -> x2 += 0.5, x3 = 0; turnFOM = 2 >= 1 -> x2 += 1
    (_p(v_fom=2.0, v_som=4.0), [0.0, 0.25, 0.5, 1.0, 0.0], [0.0, 1.75, 0.0, 0.0, 0.0]),
]


@pytest.mark.parametrize("p,x,expect", SYNC_CASES)
def test_sync_hand_cases(oracle_lib, p, x, expect):
    assert np.array_equal(oracle_lib.transform_sync(p, x), np.array(expect))


@pytest.mark.parametrize("p,x,expect", ASYNC_CASES)
def test_async_hand_cases(oracle_lib, p, x, expect):
    assert np.array_equal(oracle_lib.transform_async(p, x), np.array(expect))


def _eq3(p, x):
    """Eq. (3) of Sec. II.C, the paper's forward-Euler statement of the transformation."""
    x1, x2, x3, x4, x5 = x
    dt = p["dt"]
    g = p["v_dom"] * x2 / (p["K_dom"] + x2) * x1 * dt
    return np.array([
        x1 + g - (p["rho"] * x1 + p["mu"] * x1) * dt,
        x2 - g + (p["v_som"] * x3 + p["v_fom"] * x4 + p["beta"] * p["mu"] * x1) * dt,
        x3 + ((1 - p["beta"]) * p["mu"] * x1 - p["v_som"] * x3) * dt,
        x4 - p["v_fom"] * x4 * dt,
        x5 + p["rho"] * x1 * dt,
    ])


def test_sync_equals_eq3_without_clamps(oracle_lib):
    """With the paper's parameters no clamp fires, and the synchronous listing equals eq. (3)."""
    p = synth.paper_params()
    rng = np.random.default_rng(1)
    for _ in range(200):
        x = rng.uniform(0, 1e-3, 5) * (rng.random(5) < 0.7)
        got = oracle_lib.transform_sync(p, x)
        ref = _eq3(p, x)
        assert np.allclose(got, ref, rtol=1e-14, atol=1e-22)


@pytest.mark.parametrize("kind", ["sync", "async"])
def test_total_carbon_conserved(oracle_lib, kind):
    """Every flux leaves one compartment and enters another (Fig. 1), so sum_c x^c is invariant,
    including when clamps fire."""
    f = oracle_lib.transform_sync if kind == "sync" else oracle_lib.transform_async
    rng = np.random.default_rng(2)
    for _ in range(300):
        p = _p(dt=float(rng.uniform(0.01, 3.0)), rho=float(rng.uniform(0, 2)), mu=float(rng.uniform(0, 2)),
               beta=float(rng.uniform(0, 1)), v_som=float(rng.uniform(0, 2)), v_fom=float(rng.uniform(0, 2)),
               v_dom=float(rng.uniform(0, 20)), K_dom=float(rng.uniform(0.01, 2)))
        x = rng.uniform(0, 1, 5) * (rng.random(5) < 0.8)
        y = f(p, x)
        assert abs(y.sum() - x.sum()) <= 4e-16 * max(1.0, x.sum())
        assert np.all(y >= -1e-15)


def _isolated_voxel_run(oracle_lib, p, x0, k):
    nbr = -np.ones((1, 6), dtype=np.int32)
    return oracle_lib.explicit_run(nbr, p, np.array(x0, dtype=float).reshape(5, 1), k)[:, 0]


def test_closed_form_hydrolysis_without_biomass(oracle_lib):
    """MB = 0: FOM and SOM decay geometrically, x4_k = x4_0 (1 - v_FOM dt)^k (eq. 3), and the
    hydrolysed carbon accumulates in DOM."""
    p = synth.paper_params(dt=0.01)
    k = 300
    x = _isolated_voxel_run(oracle_lib, p, [0.0, 0.0, 2.0, 3.0, 0.0], k)
    x3 = 2.0 * (1 - p["v_som"] * p["dt"]) ** k
    x4 = 3.0 * (1 - p["v_fom"] * p["dt"]) ** k
    assert np.isclose(x[2], x3, rtol=1e-13) and np.isclose(x[3], x4, rtol=1e-13)
    assert np.isclose(x[1], 5.0 - x3 - x4, rtol=1e-13)
    assert x[0] == 0.0 and x[4] == 0.0


def test_closed_form_biomass_decay(oracle_lib):
    """No substrate and no growth (v_DOM = 0, v_SOM = 0): x1_k = x1_0 (1 - (rho+mu) dt)^k,
    CO2 = rho/(rho+mu) of the lost biomass, DOM = beta mu/(rho+mu), SOM = (1-beta) mu/(rho+mu)."""
    p = synth.paper_params(dt=0.02)
    p.update(v_dom=0.0, v_som=0.0)
    k = 250
    x = _isolated_voxel_run(oracle_lib, p, [1.5, 0.0, 0.0, 0.0, 0.0], k)
    q = 1 - (p["rho"] + p["mu"]) * p["dt"]
    x1 = 1.5 * q ** k
    lost = 1.5 - x1
    s = p["rho"] + p["mu"]
    assert np.isclose(x[0], x1, rtol=1e-13)
    assert np.isclose(x[4], lost * p["rho"] / s, rtol=1e-12)
    assert np.isclose(x[1], lost * p["beta"] * p["mu"] / s, rtol=1e-12)
    assert np.isclose(x[2], lost * (1 - p["beta"]) * p["mu"] / s, rtol=1e-12)


def test_monod_saturation(oracle_lib):
    """Monod uptake (Sec. II.C): half the maximum rate at x2 = K_DOM, the maximum as x2 >> K."""
    p = _p(rho=0.0, mu=0.0, v_som=0.0, v_fom=0.0, v_dom=1.0, K_dom=0.25, dt=0.125)
    y = oracle_lib.transform_sync(p, [2.0, 0.25, 0.0, 0.0, 0.0])
    assert y[0] - 2.0 == 0.5 * 1.0 * 2.0 * 0.125
    y = oracle_lib.transform_sync(p, [1e-3, 1e9, 0.0, 0.0, 0.0])
    assert np.isclose(y[0] - 1e-3, 1.0 * 1e-3 * 0.125, rtol=1e-9)


def test_paper_constants(oracle_lib):
    """The parameter values and masses printed in Sec. IV.C (fixture tests/golden/paper_constants.json)."""
    import json
    import os

    path = os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")
    gold = json.load(open(path))
    v = gold["values"]
    assert synth.RHO == v["rho_per_day"] and synth.MU == v["mu_per_day"] and synth.BETA == v["beta"]
    assert synth.V_SOM == v["v_som_per_day"] and synth.V_FOM == v["v_fom_per_day"]
    assert synth.V_DOM == v["v_dom_per_day"] and synth.D_DOM == v["D_dom_voxel2_per_day"]
    assert synth.M_DOM_TOTAL == v["initial_dom_ug"]
    # 5.2e7 cells of 5.41e-8 ug C each make the printed 2.8132 ug of MB
    assert np.isclose(v["cells"] * v["ug_per_cell"], v["initial_mb_ug"], rtol=1e-12)
    assert synth.M_MB_TOTAL == v["initial_mb_ug"]
    # 99.0376 % DOM and 0.962 % MB of the initial carbon (printed to 4 and 3 decimals)
    tot = v["initial_dom_ug"] + v["initial_mb_ug"]
    assert round(100 * v["initial_dom_ug"] / tot, 4) == v["dom_percent"]
    assert round(100 * v["initial_mb_ug"] / tot, 3) == v["mb_percent"]
    # the largest stable explicit step of Sec. IV.C (0.1 s) lies below the positivity limit 1/(6D)
    assert v["largest_explicit_dt_s"] < 86400.0 / (6 * v["D_dom_voxel2_per_day"])


def test_subcycling_reading(oracle_lib):
    """Different transformation and diffusion steps (Sec. III, Table 1): equal steps reproduce the
    plain run exactly; the tick count follows the global clock (0.1 s diffusion, 0.43 s
    transformation: ticks at 0, 0.43, 0.86, ... s); with only FOM hydrolysis active, FOM after N
    steps is x4_0 (1 - v_FOM dt_T)^(ticks before N dt)."""
    import numpy as np

    img = np.zeros((3, 4, 5), dtype=np.uint8)
    g = oracle_lib.graph_build(img)
    X0 = synth.random_masses(g.n, 5, scale=1e-3, density=0.8)
    p = synth.paper_params()
    a = oracle_lib.explicit_run(g.nbr, p, X0, 37)
    b = oracle_lib.run_subcycled(g.nbr, p, X0, 37, dt_transform=p["dt"])
    assert np.array_equal(a, b)
    s = 1.0 / 86400.0
    ticks = [oracle_lib.ticks_before(k, 0.1 * s, 0.43 * s) for k in range(10)]
    assert ticks == [0, 1, 1, 1, 1, 2, 2, 2, 2, 3]  # multiples of 0.43 below 0, 0.1, ..., 0.9 s
    assert [oracle_lib.ticks_before(k, 2.0, 1.0) for k in range(4)] == [0, 2, 4, 6]
    q = dict(p, rho=0.0, mu=0.0, v_som=0.0, v_dom=0.0, D=0.0, v_fom=3e3, dt=0.1 * s)
    X = np.zeros((5, g.n))
    X[3] = 1.0
    out = oracle_lib.run_subcycled(g.nbr, q, X, 50, dt_transform=0.43 * s)
    nt = oracle_lib.ticks_before(50, 0.1 * s, 0.43 * s)
    assert nt == 12
    assert np.allclose(out[3], (1 - 3e3 * 0.43 * s) ** nt, rtol=1e-13)
    # splitting the run keeps the clock
    dtt = 4.3 * p["dt"]
    half = oracle_lib.run_subcycled(g.nbr, p, X0, 20, dt_transform=dtt)
    rest = oracle_lib.run_subcycled(g.nbr, p, half, 17, dt_transform=dtt, step0=20)
    full = oracle_lib.run_subcycled(g.nbr, p, X0, 37, dt_transform=dtt)
    assert np.array_equal(rest, full)
    # the implicit scheme with equal steps reproduces the plain implicit run
    ai = oracle_lib.implicit_run(g.nbr, synth.paper_params(dt=1.0 / 86400), X0, 5, rtol=1e-12)[0]
    bi = oracle_lib.run_subcycled(g.nbr, synth.paper_params(dt=1.0 / 86400), X0, 5, dt_transform=1.0 / 86400,
                                  scheme=1, rtol=1e-12)
    assert np.allclose(ai, bi, rtol=1e-11, atol=0)  # PCG dot products may sum in another order
