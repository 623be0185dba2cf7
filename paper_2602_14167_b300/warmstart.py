"""Learned warm start for batched VQE (no counterpart in the paper).

A BF16 MLP (``tcng_mlp_forward``/``tcng_mlp_backward``, FP32 master weights,
device Adam) maps Hamiltonian couplings to initial ansatz angles.  Training
targets are converged angles produced by the batched adjoint simulator itself
(``tcng_energy_grad_ragged`` + ``tcng_adam_step`` for many steps).  The network
is measured by the exact simulated energy: how many Adam steps a warm-started
run needs against random initialisation.

Chains are dicts {kind: 0 TFIM / 1 XXZ, n, J[n-1], delta, g}; the ansatz is the
ring ansatz of ``hea_ring`` layout (RX, RY per qubit, RZZ ring per layer), whose
parameter (layer l, kind k, qubit q) sits at l*3n + k*n + q for n qubits and at
l*3*n_max + k*n_max + q in the network output.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import tcng as T

OPS_RX, OPS_RY, OPS_RZZ = 7, 8, 14


def features(chain, n_max=20):
    """[J_1..J_{n_max-1} zero-padded, delta (XXZ), g, n/n_max, one-hot kind]."""
    f = np.zeros(n_max - 1 + 5, dtype=np.float32)
    f[: chain["n"] - 1] = chain["J"]
    f[n_max - 1] = chain["delta"] if chain["kind"] == 1 else 0.0
    f[n_max] = chain["g"]
    f[n_max + 1] = chain["n"] / n_max
    f[n_max + 2 + chain["kind"]] = 1.0
    return f


def ring_ansatz(n, layers):
    """Gate list of the ring ansatz (same layout as the benchmark's VQE batches)."""
    g = np.zeros(3 * n * layers, dtype=T.GATE_DTYPE)
    k = 0
    for l in range(layers):
        base = l * 3 * n
        for q in range(n):
            g[k] = (OPS_RX, 1, 0, (q, -1, -1, -1, -1), base + q, 1.0, 0.0, -1); k += 1
        for q in range(n):
            g[k] = (OPS_RY, 1, 0, (q, -1, -1, -1, -1), base + n + q, 1.0, 0.0, -1); k += 1
        for i in range(n):
            g[k] = (OPS_RZZ, 2, 0, (i, (i + 1) % n, -1, -1, -1), base + 2 * n + i, 1.0, 0.0, -1); k += 1
    return g


def param_slots(n, layers, n_max):
    """Network-output index of each of the 3*n*layers parameters."""
    idx = []
    for l in range(layers):
        for k in range(3):
            for q in range(n):
                idx.append(l * 3 * n_max + k * n_max + q)
    return np.asarray(idx, dtype=np.int64)


class RaggedVQE:
    """Many chains (different n and Hamiltonians) optimised together on the device."""

    def __init__(self, chains, terms_of, layers=12, device="cuda"):
        self.layers = layers
        self.device = torch.device(device)
        self.chains = chains
        structs, self.problems = {}, []
        self.item_problem = []
        coeffs = []
        for ch in chains:
            terms = terms_of(ch)
            key = (ch["n"], ch["kind"])
            if key not in structs:
                structs[key] = len(self.problems)
                self.problems.append(dict(n=ch["n"], gates=ring_ansatz(ch["n"], layers), pool=None,
                                          P=3 * ch["n"] * layers, terms=terms))
            self.item_problem.append(structs[key])
            coeffs.append(np.asarray(terms["coeff"], dtype=np.float64))
        self.P = [self.problems[s]["P"] for s in self.item_problem]
        self.offsets = np.concatenate([[0], np.cumsum(self.P)])
        self.coeffs = torch.tensor(np.concatenate(coeffs), device=self.device)
        self.B = len(chains)
        self.energy = torch.empty(self.B, dtype=torch.float64, device=self.device)
        self.grad = torch.empty(int(self.offsets[-1]), dtype=torch.float64, device=self.device)

    def pack(self, thetas):
        return torch.tensor(np.concatenate(thetas), dtype=torch.float64, device=self.device)

    def unpack(self, packed):
        p = packed.detach().cpu().numpy()
        return [p[self.offsets[i]:self.offsets[i + 1]] for i in range(self.B)]

    def energy_and_grad(self, theta):
        T.tcng_energy_grad_ragged(self.problems, self.item_problem, theta, self.coeffs, self.energy,
                                  self.grad)
        return self.energy, self.grad

    def optimize(self, theta_packed, steps=500, lr=2e-2):
        """Adam from theta_packed; returns (theta, energies [steps+1, B]) (energy before each step)."""
        theta = theta_packed.clone()
        m = torch.zeros_like(theta)
        v = torch.zeros_like(theta)
        step = torch.zeros(1, dtype=torch.int32, device=self.device)
        hist = torch.empty((steps + 1, self.B), dtype=torch.float64, device=self.device)
        for s in range(steps):
            self.energy_and_grad(theta)
            hist[s].copy_(self.energy)
            T.tcng_adam_step(theta, m, v, self.grad, theta.numel(), lr, 0.9, 0.999, 1e-8, step)
        self.energy_and_grad(theta)
        hist[steps].copy_(self.energy)
        return theta, hist


class MLP:
    """F -> H -> H -> O network with BF16 GEMMs on the tensor cores."""

    def __init__(self, F, H, O, seed=0, device="cuda"):
        self.F, self.H, self.O = F, H, O
        self.device = torch.device(device)
        g = torch.Generator().manual_seed(seed)
        sizes = [F * H, H, H * H, H, H * O, O]
        self.flat = torch.zeros(sum(sizes), dtype=torch.float32)
        views, off = [], 0
        for s in sizes:
            views.append((off, s))
            off += s
        w1 = torch.randn(F, H, generator=g) * math.sqrt(2.0 / F)
        w2 = torch.randn(H, H, generator=g) * math.sqrt(2.0 / H)
        w3 = torch.randn(H, O, generator=g) * math.sqrt(1.0 / H)
        self.flat[views[0][0]:views[0][0] + views[0][1]] = w1.reshape(-1)
        self.flat[views[2][0]:views[2][0] + views[2][1]] = w2.reshape(-1)
        self.flat[views[4][0]:views[4][0] + views[4][1]] = w3.reshape(-1)
        self.flat = self.flat.to(self.device)
        self.views = views
        self.grads = torch.zeros_like(self.flat)
        self.m = torch.zeros_like(self.flat)
        self.v = torch.zeros_like(self.flat)
        self.step = torch.zeros(1, dtype=torch.int32, device=self.device)
        self.loss = torch.zeros(1, dtype=torch.float64, device=self.device)

    def p(self, i):
        o, s = self.views[i]
        return self.flat[o:o + s]

    def forward(self, x):
        N = x.shape[0]
        self.act = torch.empty((2, N, self.H), dtype=torch.float32, device=self.device)
        y = torch.empty((N, self.O), dtype=torch.float32, device=self.device)
        T.tcng_mlp_forward(x, N, self.F, self.H, self.O, self.p(0), self.p(1), self.p(2), self.p(3),
                           self.p(4), self.p(5), self.act, y)
        return y

    def backward(self, x, y, target, mask):
        N = x.shape[0]
        T.tcng_mlp_backward(x, N, self.F, self.H, self.O, self.p(0), self.p(2), self.p(4), self.act, y,
                            target, mask, self.grads, self.loss)
        return self.loss

    def train(self, x, target, mask, steps=500, lr=1e-3):
        hist = []
        for s in range(steps):
            y = self.forward(x)
            self.backward(x, y, target, mask)
            T.tcng_adam_step_f32(self.flat, self.m, self.v, self.grads, self.flat.numel(), lr, 0.9,
                                 0.999, 1e-8, self.step)
            if s % 50 == 0 or s == steps - 1:
                hist.append(float(self.loss.item()))
        return hist


def targets_for(chains, thetas, layers, n_max):
    """Pad converged angles into the network's output layout (+ validity mask)."""
    O = 3 * layers * n_max
    tgt = np.zeros((len(chains), O), dtype=np.float32)
    mask = np.zeros((len(chains), O), dtype=np.float32)
    for i, (ch, th) in enumerate(zip(chains, thetas)):
        sl = param_slots(ch["n"], layers, n_max)
        tgt[i, sl] = th
        mask[i, sl] = 1.0
    return tgt, mask


def predict_init(mlp, chains, layers, n_max):
    x = torch.tensor(np.stack([features(c, n_max) for c in chains]), device=mlp.device)
    y = mlp.forward(x).detach().cpu().numpy().astype(np.float64)
    return [y[i, param_slots(c["n"], layers, n_max)] for i, c in enumerate(chains)]


def steps_to_reach(hist, threshold):
    """First step index whose energy is <= threshold (per item); len(hist) if never."""
    h = hist.detach().cpu().numpy()
    out = np.full(h.shape[1], h.shape[0], dtype=np.int64)
    for b in range(h.shape[1]):
        idx = np.nonzero(h[:, b] <= threshold[b])[0]
        if idx.size:
            out[b] = idx[0]
    return out
