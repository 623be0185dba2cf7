"""Measurement trajectories and shadow snapshots on the C ABI (marshalling only).

* ``MIPTBatch.run`` evolves B trajectories of the paper's measurement-induced
  phase transition study (Sec. VII.C): per time step one call applying every
  trajectory's own Haar gates (``tcng_apply_circuit_pooled``) and one call
  measuring the selected qubits by the Born rule (``tcng_measure``); returns the
  outcomes and each trajectory's log-probability.
* ``shadow_snapshots`` rotates copies of a state into random Pauli bases and
  measures every qubit (the classical-shadow data of Sec. VII.A).
All arithmetic runs in the library's kernels.
"""
from __future__ import annotations

import numpy as np
import torch

from . import tcng as T
from .state import StateBatch


class MIPTBatch:
    """B trajectories of n qubits (complex64 by default)."""

    def __init__(self, n, batch, dtype="c64", device="cuda"):
        self.n, self.batch = int(n), int(batch)
        self.state = StateBatch(n, batch=batch, dtype=dtype, device=device)
        self.device = self.state.buf.device

    def run(self, gates, pool, pools_dev, masks_dev, u_dev):
        """gates/pool: one time step's gate list and a representative host pool;
        pools_dev: device complex128 [D][B][S] per-item matrices of every step;
        masks_dev: device int64 [D][B] measured-qubit masks; u_dev: device float64
        [D][B][n].  Returns (outcomes int8 [D][B][n], -1 = not measured;
        logp float64 [B])."""
        D = pools_dev.shape[0]
        S = pools_dev.shape[2]
        out = torch.full((D, self.batch, self.n), -1, dtype=torch.int8, device=self.device)
        logp = torch.zeros(self.batch, dtype=torch.float64, device=self.device)
        self.state.reset()
        for t in range(D):
            T.tcng_apply_circuit_pooled(self.state.handle, gates, pool, pools_dev[t], S)
            T.tcng_measure(self.state.handle, masks_dev[t], u_dev[t], out[t], logp)
        return out, logp


# op codes of tcng_op (include/tcng.h)
_RX, _RY = 7, 8


def shadow_rotation(n):
    """Gate list rotating each qubit's Pauli basis onto Z before a Z measurement:
    RY(theta[q]) then RX(theta[n + q]) on qubit q; the X basis takes
    RY(-pi/2) (|+> -> |0>), the Y basis RX(pi/2) (|+i> -> |0>), Z no rotation.
    Returns (gates, angles(bases) -> float64 [S][2n])."""
    g = np.zeros(2 * n, dtype=T.GATE_DTYPE)
    for q in range(n):
        for k, (op, prm) in enumerate(((_RY, q), (_RX, n + q))):
            r = g[k * n + q]
            r["op"], r["nq"], r["param"], r["scale"], r["mat_off"] = op, 1, prm, 1.0, -1
            r["q"] = [q, -1, -1, -1, -1]

    def angles(bases):
        bases = np.asarray(bases)
        th = np.zeros((bases.shape[0], 2 * n))
        th[:, :n][bases == 1] = -np.pi / 2
        th[:, n:][bases == 2] = np.pi / 2
        return th
    return g, angles


def shadow_snapshots(psi, bases, u_dev, dtype="c64"):
    """psi: device [2^n] state; bases: host int [S][n] (1 = X, 2 = Y, 3 = Z, the
    paper's pauli_strings); u_dev: device float64 [S][n] Born uniforms.  Returns
    device int8 [S][n] outcome bits (0 = eigenvalue +1 of the basis Pauli)."""
    bases = np.asarray(bases)
    S, n = bases.shape
    st = StateBatch(n, batch=S, dtype=dtype, device=psi.device)
    st.batch_view().copy_(psi.reshape(1, -1).expand(S, -1))
    g, angles = shadow_rotation(n)
    th = torch.tensor(angles(bases), dtype=torch.float64, device=psi.device)
    st.apply(g, None, th)
    masks = torch.full((S,), (1 << n) - 1, dtype=torch.int64, device=psi.device)
    out = torch.full((S, n), -1, dtype=torch.int8, device=psi.device)
    T.tcng_measure(st.handle, masks, u_dev, out, None)
    st.free()
    return out
