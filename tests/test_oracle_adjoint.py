"""Pins of the oracle's discrete adjoint: central finite differences of the FP64 forward, the
closed-form one-step gradient of Objective 1 (Sec. V.A), and invariance to the checkpoint spacing."""
import numpy as np
import pytest

import synth

OPP = [1, 0, 3, 2, 5, 4]


def _setup(oracle_lib, seed=1, shape=(3, 4, 5)):
    rng = np.random.default_rng(seed)
    img = (rng.random(shape) >= 0.6).astype(np.uint8)
    g = oracle_lib.graph_build(img, keep_largest=True)
    n = g.n
    X0 = np.zeros((5, n))
    X0[0] = rng.uniform(0.2e-3, 1e-3, n)
    X0[1] = rng.uniform(0.1e-3, 2e-3, n)
    X0[2] = rng.uniform(0, 1e-3, n)
    X0[3] = rng.uniform(0, 1e-3, n)
    X0[4] = rng.uniform(0, 1e-4, n)
    # symmetric per-edge conductances
    g6 = np.zeros((n, 6))
    for i in range(n):
        for d in (1, 3, 5):
            j = g.nbr[i, d]
            if j >= 0:
                g6[i, d] = g6[j, OPP[d]] = rng.uniform(0.5, 1.5)
    lamN = rng.standard_normal((5, n))
    return g, X0, g6, lamN


def _loss(oracle_lib, g, p, X0, g6, lamN, nsteps):
    return float(np.sum(lamN * oracle_lib.explicit_run(g.nbr, p, X0, nsteps, g6=g6)))


PARAMS_SMOOTH = dict(D=1.0, dt=0.1, rho=0.2, mu=0.5, beta=0.55, v_som=0.3, v_fom=0.6, v_dom=2.0, K_dom=1e-3)
# large dt: the uptake, respiration+mortality and hydrolysis clamps all fire somewhere
PARAMS_CLAMPED = dict(D=1.0, dt=0.12, rho=3.0, mu=6.0, beta=0.55, v_som=9.0, v_fom=11.0, v_dom=40.0, K_dom=1e-3)


@pytest.mark.parametrize("params", [PARAMS_SMOOTH, PARAMS_CLAMPED])
def test_adjoint_matches_central_differences(oracle_lib, params):
    g, X0, g6, lamN = _setup(oracle_lib)
    nsteps = 12
    res = oracle_lib.adjoint_run(g.nbr, params, X0, nsteps, lamN, ckpt=5, g6=g6, want_gface=True)
    # forward state agrees with the plain forward run
    assert np.array_equal(res["XN"], oracle_lib.explicit_run(g.nbr, params, X0, nsteps, g6=g6))

    def fd(fn, x, h):
        return (fn(x + h) - fn(x - h)) / (2 * h)

    # parameters
    for name in oracle_lib.GRAD_NAMES:
        base = params[name]
        h = 1e-5 * abs(base)

        def L(v, name=name):
            q = dict(params)
            q[name] = v
            return _loss(oracle_lib, g, q, X0, g6, lamN, nsteps)

        num = fd(L, base, h)
        ana = res["grad"][name]
        assert abs(num - ana) <= 1e-5 * max(abs(num), 1e-6 * abs(base)), (name, num, ana)
    # initial state, along random directions
    rng = np.random.default_rng(5)
    for _ in range(3):
        v = rng.standard_normal(X0.shape) * X0 * 1e-3 + 1e-9 * rng.standard_normal(X0.shape) * (X0 > 0)

        def L(t):
            return _loss(oracle_lib, g, params, X0 + t * v, g6, lamN, nsteps)

        num = fd(L, 0.0, 1.0)
        ana = float(np.sum(res["lam0"] * v))
        assert abs(num - ana) <= 1e-6 * abs(num) + 1e-12
    # a few edge conductances (perturbing both slots of the edge together)
    for i in range(0, g.n, max(1, g.n // 5)):
        for d in (1, 3, 5):
            j = g.nbr[i, d]
            if j < 0:
                continue

            def L(t, i=i, d=d, j=j):
                gg = g6.copy()
                gg[i, d] += t
                gg[j, OPP[d]] += t
                return _loss(oracle_lib, g, params, X0, gg, lamN, nsteps)

            num = fd(L, 0.0, 1e-5)
            ana = res["gface"][i, d]
            assert abs(num - ana) <= 1e-5 * abs(num) + 1e-12, (i, d, num, ana)
            assert res["gface"][j, OPP[d]] == ana


def test_clamps_fire_in_clamped_case(oracle_lib):
    g, X0, g6, lamN = _setup(oracle_lib)
    p = PARAMS_CLAMPED
    fired = set()
    for i in range(g.n):
        x1, x2, x3, x4 = X0[0, i], X0[1, i], X0[2, i], X0[3, i]
        if p["v_dom"] * x2 / (p["K_dom"] + x2) * x1 * p["dt"] > x2:
            fired.add("uptake")
        if (p["rho"] + p["mu"]) * x1 * p["dt"] > x1:
            fired.add("mort+resp")
        if p["v_fom"] * x4 * p["dt"] > x4:
            fired.add("fom")
        if p["v_som"] * x3 * p["dt"] > x3:
            fired.add("som")
    assert fired == {"uptake", "mort+resp", "fom", "som"}


def test_one_step_matches_objective1_closed_form(oracle_lib):
    """Sec. V.A: for one explicit diffusion step with v_i = 1 and the loss
    L1 = (1/q) sum_i (y_i - x_i + D dt sum_f theta_if (x_i - x_f))^2, the paper's closed form is
    dL1/dtheta_ij = (2/q) D dt (x_i - x_j) r_i with r_i the bracket.  The conductance of an
    undirected edge enters rows i and j, so its derivative is the sum of the two directed forms."""
    g, X0, g6, _ = _setup(oracle_lib, seed=3, shape=(4, 4, 3))
    n = g.n
    p = dict(D=2.0, dt=0.05, rho=0.0, mu=0.0, beta=0.5, v_som=0.0, v_fom=0.0, v_dom=0.0, K_dom=1.0)
    x = X0[1]
    Y = np.random.default_rng(8).uniform(0, 2e-3, n)
    c = p["D"] * p["dt"]
    r = np.array([Y[i] - x[i] + c * sum(g6[i, d] * (x[i] - x[g.nbr[i, d]]) for d in range(6) if g.nbr[i, d] >= 0)
                  for i in range(n)])
    X1 = oracle_lib.explicit_run(g.nbr, p, X0, 1, g6=g6)
    assert np.allclose(Y - X1[1], r, rtol=0, atol=1e-15)  # the bracket is y - (Q x)
    lamN = np.zeros((5, n))
    lamN[1] = (2.0 / n) * (X1[1] - Y)  # dL1/dX^1
    res = oracle_lib.adjoint_run(g.nbr, p, X0, 1, lamN, ckpt=1, g6=g6, want_gface=True)
    for i in range(n):
        for d in range(6):
            j = g.nbr[i, d]
            if j < 0:
                continue
            directed_ij = (2.0 / n) * c * (x[i] - x[j]) * r[i]
            directed_ji = (2.0 / n) * c * (x[j] - x[i]) * r[j]
            assert np.isclose(res["gface"][i, d], directed_ij + directed_ji, rtol=1e-12, atol=1e-22)


def test_checkpoint_spacing_does_not_change_result(oracle_lib):
    g, X0, g6, lamN = _setup(oracle_lib, seed=2)
    p = synth.paper_params(dt=0.05)
    p["D"] = 2.0
    outs = [oracle_lib.adjoint_run(g.nbr, p, X0, 23, lamN, ckpt=k, g6=g6, want_gface=True) for k in (1, 4, 23, 100)]
    for o in outs[1:]:
        assert np.array_equal(o["lam0"], outs[0]["lam0"])
        assert o["grad"] == outs[0]["grad"]
        assert np.array_equal(o["gface"], outs[0]["gface"])
