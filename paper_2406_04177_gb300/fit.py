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


# ---- coarse primitive-graph model (Sec. V.A, V.B) ----------------------------------------------
def pngm_dataset(graph, pngm, params: dict, scenarios, steps_per_record: int, records: int, stream=None):
    """Voxel-graph data for the coarse model (Sec. V.B): for every initial state in `scenarios`
    ((5, n) float64 arrays or CUDA tensors), run the voxel simulation and store the primitive
    masses of DOM every `steps_per_record` steps, `records` + 1 times (t = 0 included).  Returns
    (data (S*(records+1), q) CUDA float64 tensor, pairs (S*records, 2) int32 array of consecutive
    records of one scenario)."""
    import torch

    q = pngm.q
    S = len(scenarios)
    data = torch.empty((S * (records + 1), q), dtype=torch.float64, device="cuda")
    pairs = []
    sim = Sim(graph, params, stream=stream)
    for s, X0 in enumerate(scenarios):
        sim.set_masses(X0)
        base = s * (records + 1)
        pngm.restrict(sim, 1, data[base])
        for r in range(records):
            sim.step(steps_per_record)
            pngm.restrict(sim, 1, data[base + r + 1])
            pairs.append((base + r, base + r + 1))
    sim.sync()
    sim.close()
    return data, np.asarray(pairs, dtype=np.int32)


def fit_pngm(pngm, data, pairs: np.ndarray, D: float, dt: float, objective: int = 2, epochs: int = 1000,
             batch: int = 4, lr0: float = 0.1, halve_every: int = 10, tied: bool = True, seed: int = 0,
             theta_min: float = 0.0, callback=None) -> dict:
    """Normalised SGD on Objective 1 or 2 (Sec. V.B: 1000 epochs of 4 random data pairs, lr 0.1
    halved every 10 epochs).  dt is the coarse step (the spacing of consecutive records).  The
    pairs of each epoch are drawn without replacement from a PCG64(seed) stream.  Conductances are
    kept >= theta_min (non-negative by default, so Scheme 4 stays positive definite).  Returns
    dict(loss (per epoch, before its update), lr, theta (final))."""
    rng = np.random.Generator(np.random.PCG64(seed))
    losses, lrs = [], []
    lr = lr0
    for epoch in range(epochs):
        if epoch > 0 and halve_every > 0 and epoch % halve_every == 0:
            lr *= 0.5
        idx = rng.choice(len(pairs), size=min(batch, len(pairs)), replace=False)
        loss = pngm.sgd_step(objective, data, pairs[idx], D, dt, lr, tied=tied, theta_min=theta_min)
        losses.append(loss)
        lrs.append(lr)
        if callback is not None:
            callback(epoch, loss, lr)
    return dict(loss=np.asarray(losses), lr=np.asarray(lrs), theta=pngm.get_theta())
