"""Pin of the normalised-gradient SGD rule of Sec. V.A on a 2-block toy: one conductance between two
8^3 blocks of an open box, data from a target run with theta* = 0.6.  The objective is monotone in
theta on each side of theta*, so sign steps with a halving learning rate must converge to it."""
import numpy as np

import synth

THETA_STAR = 0.6


def toy(oracle_lib):
    img = np.zeros((8, 8, 16), dtype=np.uint8)  # (nz, ny, nx): two 8^3 blocks side by side in x
    g = oracle_lib.graph_build(img)
    X0 = np.zeros((5, g.n))
    x = g.voxel_of_node % 16
    X0[1, x < 8] = 1e-3  # DOM in the left block only
    p = synth.paper_params()
    p.update(rho=0.0, mu=0.0, v_som=0.0, v_fom=0.0, v_dom=0.0)
    return img, g, X0, p


def oracle_fit(oracle_lib, img, g, X0, p, epochs, nsteps=40, bs=8):
    nb = oracle_lib.block_grid(img.shape, bs)
    nI = oracle_lib.interface_count(nb)
    g6s = oracle_lib.block_face_weights(img.shape, bs, g.voxel_of_node, g.nbr, np.full(nI, THETA_STAR))
    target = oracle_lib.block_masses(img.shape, bs, g.voxel_of_node, oracle_lib.explicit_run(g.nbr, p, X0, nsteps, g6=g6s))
    theta = np.ones(nI)
    losses = []
    for ep in range(epochs):
        g6 = oracle_lib.block_face_weights(img.shape, bs, g.voxel_of_node, g.nbr, theta)
        XN = oracle_lib.explicit_run(g.nbr, p, X0, nsteps, g6=g6)
        L, lamN = oracle_lib.block_mass_loss(img.shape, bs, g.voxel_of_node, XN, target)
        res = oracle_lib.adjoint_run(g.nbr, p, X0, nsteps, lamN, ckpt=16, g6=g6, want_gface=True)
        gth = oracle_lib.block_theta_grad(img.shape, bs, g.voxel_of_node, g.nbr, res["gface"], nI)
        lr = 0.1 * 0.5 ** (ep // 10)
        theta = theta - lr * np.sign(gth)
        losses.append(L)
    return theta, np.array(losses), target


def test_sign_sgd_recovers_two_block_conductance(oracle_lib):
    img, g, X0, p = toy(oracle_lib)
    theta, losses, _ = oracle_fit(oracle_lib, img, g, X0, p, epochs=60)
    assert theta.shape == (1,)
    assert abs(theta[0] - THETA_STAR) < 0.01
    assert losses[-1] < 1e-6 * losses[0]
