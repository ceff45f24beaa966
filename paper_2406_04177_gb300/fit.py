"""Fitting block-to-block diffusional conductances to voxel-simulation data (Sec. V: the use of the
voxel graph to calibrate a coarse pore network).

The coarse model here is the voxel graph itself with one conductance theta per face between
face-adjacent cubic blocks; the data are the block masses of DOM and CO2 after N explicit steps of
a target run.  Each epoch runs the checkpointed forward pass, evaluates the block-mass objective
and its gradient with respect to the final state, back-propagates it with the discrete adjoint, and
takes the normalised gradient step of Sec. V.A (theta <- theta - lr * g/|g| element-wise) on the
device.  The learning rate starts at lr0 and halves every `halve_every` epochs (Sec. V.B uses 0.1
and 10).  Every numerical step runs in the library's kernels; this module only sequences calls.
"""
from __future__ import annotations

import numpy as np

from . import Sim

COMP_DOM_CO2 = (1 << 1) | (1 << 4)


def stability_bound(params: dict) -> float:
    """Largest conductance the explicit scheme tolerates: 6 D dt theta <= 1."""
    return 1.0 / (6.0 * params["D"] * params["dt"])


def fit_block_conductances(graph, params: dict, X0, block_side: int, target: np.ndarray, n_theta: int,
                           n_steps: int = 2000, ckpt: int = 100, epochs: int = 200, lr0: float = 0.1,
                           halve_every: int = 10, theta0=None, theta_min: float = 0.0, theta_max=None,
                           comp_mask: int = COMP_DOM_CO2, stream=None, callback=None) -> dict:
    """Returns dict(theta (final, float32), loss (per epoch, before its update), lr (per epoch))."""
    import torch

    theta_max = stability_bound(params) if theta_max is None else theta_max
    theta = np.ones(n_theta, dtype=np.float32) if theta0 is None else np.asarray(theta0, dtype=np.float32)
    sim = Sim(graph, params, stream=stream)
    sim.set_block_conductances(block_side, theta)
    x0 = X0 if isinstance(X0, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(X0, dtype=np.float64)).cuda()
    dldx = torch.empty((5, graph.n), dtype=torch.float64, device=x0.device)
    losses, lrs = [], []
    for epoch in range(epochs):
        sim.set_masses(x0)
        sim.adjoint_forward(n_steps, ckpt)
        loss, _ = sim.loss_block_mass(block_side, comp_mask, target, dL_dX=dldx)
        sim.adjoint_backward(dldx, n_theta=n_theta)
        lr = lr0 * 0.5 ** (epoch // halve_every)
        sim.sgd_block_conductances(lr, theta_min, theta_max)
        losses.append(loss)
        lrs.append(lr)
        if callback is not None:
            callback(epoch, loss)
    theta = sim.get_block_conductances(n_theta)
    sim.close()
    return dict(theta=theta, loss=np.array(losses), lr=np.array(lrs))
