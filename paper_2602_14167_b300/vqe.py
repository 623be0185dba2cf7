"""Batched VQE on the C ABI: an autograd Function, and a device-side Adam loop.

The paper's Sec. I.B pipeline is value_and_grad -> vmap -> jit of the TFIM
energy, optimised with Adam; its Sec. III.A wraps such a function as a native
differentiable PyTorch operator (torch_interface).  Here:
  * ``EnergyGrad`` is a ``torch.autograd.Function`` whose forward calls
    ``tcng_energy_grad`` (energy and adjoint gradient in one persistent launch)
    and whose backward returns grad_out * dE/dtheta;
  * ``VQEBatch.optimize`` runs energy+gradient and ``tcng_adam_step`` on the
    device for many steps, optionally replayed from one CUDA graph per circuit
    structure.
All arithmetic runs in the library's kernels; this module only marshals.
"""
from __future__ import annotations

import numpy as np
import torch

from . import tcng as T
from .state import StateBatch


class VQEBatch:
    """B parameter sets of one circuit structure with per-item Hamiltonian coefficients."""

    def __init__(self, n, gates, pool, terms, batch, coeffs=None, dtype="c64", device="cuda"):
        self.n, self.batch = int(n), int(batch)
        self.gates, self.pool, self.terms = gates, pool, terms
        self.P = int(max((int(g["param"]) for g in gates), default=-1) + 1)
        self.device = torch.device(device)
        if self.device.type == "cuda" and self.device.index is None:
            self.device = torch.device("cuda", torch.cuda.current_device())
        self.state = StateBatch(n, batch=batch, dtype=dtype, device=self.device)
        self.coeffs = None
        if coeffs is not None:
            self.coeffs = torch.as_tensor(np.asarray(coeffs, dtype=np.float64)).to(self.device).contiguous()
        self.energy = torch.empty(batch, dtype=torch.float64, device=self.device)
        self.grad = torch.empty((batch, self.P), dtype=torch.float64, device=self.device)

    def energy_and_grad(self, theta: torch.Tensor):
        """(E [B], dE/dtheta [B, P]) for theta [B, P] (float64, on this device)."""
        if theta.dtype != torch.float64 or not theta.is_contiguous() or theta.device != self.device:
            raise TypeError("theta must be a contiguous float64 tensor on the batch's device")
        if tuple(theta.shape) != (self.batch, self.P):
            raise ValueError(f"theta must have shape {(self.batch, self.P)}")
        T.tcng_energy_grad(self.state.handle, self.gates, self.pool, theta, self.P, self.terms,
                           self.coeffs, self.energy, self.grad)
        return self.energy, self.grad

    def optimize(self, theta0, steps=500, lr=2e-2, b1=0.9, b2=0.999, eps=1e-8, use_graph=True,
                 record_every=1):
        """Adam on the device.  Returns (theta [B,P], energies [n_records, B])."""
        theta = torch.as_tensor(theta0, dtype=torch.float64).to(self.device).contiguous().clone()
        m = torch.zeros_like(theta)
        v = torch.zeros_like(theta)
        step = torch.zeros(1, dtype=torch.int32, device=self.device)
        hist = []

        def one_step():
            self.energy_and_grad(theta)
            T.tcng_adam_step(theta, m, v, self.grad, theta.numel(), lr, b1, b2, eps, step)

        graph = None
        stream = torch.cuda.Stream(self.device)
        with torch.cuda.stream(stream):
            if use_graph and steps > 1:
                one_step()                       # warm-up builds plans and scratch
                hist.append(self.energy.clone())
                stream.synchronize()
                graph = torch.cuda.CUDAGraph()
                with torch.cuda.graph(graph, stream=stream):
                    one_step()
                done = 1
            else:
                done = 0
            for i in range(done, steps):
                if graph is not None:
                    graph.replay()
                else:
                    one_step()
                if record_every and (i % record_every == 0 or i == steps - 1):
                    hist.append(self.energy.clone())
        torch.cuda.current_stream(self.device).wait_stream(stream)
        return theta, (torch.stack(hist) if hist else None)


class EnergyGrad(torch.autograd.Function):
    """E(theta) of a VQEBatch as a differentiable torch op (adjoint gradient)."""

    @staticmethod
    def forward(ctx, theta, batch: VQEBatch):
        e, g = batch.energy_and_grad(theta.detach().contiguous())
        ctx.save_for_backward(g.clone())
        return e.clone()

    @staticmethod
    def backward(ctx, grad_out):
        (g,) = ctx.saved_tensors
        return grad_out.to(g.dtype)[:, None] * g, None


def energy(theta: torch.Tensor, batch: VQEBatch) -> torch.Tensor:
    return EnergyGrad.apply(theta, batch)
