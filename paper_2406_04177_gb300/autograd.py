"""torch.autograd.Function over the discrete adjoint (explicit synchronous scheme).

    XN = VoxelGraphRun.apply(theta, rates, X0, sim, n_steps, ckpt, block_side)

theta: block conductances (CUDA tensor, or an empty tensor for unit conductances; it stays on the
device: the library checks and copies it there, and the gradient comes back there);
rates: CPU float64 tensor (D, rho, mu, beta, v_som, v_fom, v_dom, K_dom); X0: CUDA float64 (5, n).
The forward runs the checkpointed forward pass of the library; the backward runs its discrete
adjoint and returns dL/dtheta, dL/drates and dL/dX0.  The simulation object must not be used in
between (its checkpoints belong to the pending backward).
"""
from __future__ import annotations

import torch

from . import GRAD_NAMES

RATE_NAMES = GRAD_NAMES  # D, rho, mu, beta, v_som, v_fom, v_dom, K_dom


class VoxelGraphRun(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, rates, X0, sim, n_steps: int, ckpt: int, block_side: int):
        base = dict(sim._base_params) if hasattr(sim, "_base_params") else {}
        params = dict(base, **{k: float(v) for k, v in zip(RATE_NAMES, rates.tolist())})
        sim.set_params(params)
        if theta.numel() > 0:
            sim.set_block_conductances(block_side, theta.detach().to(torch.float32).contiguous())
        else:
            sim.clear_conductances()
        sim.set_masses(X0.detach().contiguous())
        sim.adjoint_forward(int(n_steps), int(ckpt))
        XN = torch.empty((5, sim.n), dtype=torch.float64, device=X0.device)
        sim.get_masses(XN)
        torch.cuda.current_stream(X0.device).synchronize()
        ctx.sim = sim
        ctx.n_theta = theta.numel()
        ctx.theta_device = theta.device
        return XN

    @staticmethod
    def backward(ctx, grad_XN):
        sim = ctx.sim
        g = grad_XN.detach().contiguous().to(torch.float64)
        dX0 = torch.empty_like(g)
        torch.cuda.current_stream(g.device).synchronize()
        grad, _ = sim.adjoint_backward(g, dX0)
        gtheta = torch.zeros(ctx.n_theta, dtype=torch.float64, device=g.device)
        if ctx.n_theta > 0:
            sim.adjoint_grad_theta(gtheta)
        gtheta = gtheta.to(ctx.theta_device)
        grates = torch.tensor([grad[k] for k in RATE_NAMES], dtype=torch.float64)
        return gtheta, grates, dX0, None, None, None, None


def run(sim, theta, rates, X0, n_steps: int, ckpt: int = 100, block_side: int = 8):
    return VoxelGraphRun.apply(theta, rates, X0, sim, n_steps, ckpt, block_side)
