"""StateBatch: a batch of state vectors in a torch-owned CUDA buffer."""
from __future__ import annotations

import numpy as np
import torch

from . import tcng as T


class StateBatch:
    """``batch`` state vectors |0..0> of ``n_qubits`` (int or per-item list)."""

    def __init__(self, n_qubits, batch: int = 1, dtype: str = "c64", device="cuda"):
        if np.isscalar(n_qubits):
            n_qubits = [int(n_qubits)] * batch
        self.n = [int(v) for v in n_qubits]
        self.batch = len(self.n)
        self.dt = T.C64 if dtype in ("c64", "complex64", torch.complex64) else T.C128
        self.cdtype = torch.complex64 if self.dt == T.C64 else torch.complex128
        nbytes = T.tcng_state_bytes(self.dt, self.n)
        # torch's caching allocator returns 512-byte aligned blocks
        self.buf = torch.empty(nbytes, dtype=torch.uint8, device=device)
        if self.buf.data_ptr() % 256:
            raise RuntimeError("device buffer is not 256-byte aligned")
        self.handle = T.tcng_state_init(self.dt, self.n, self.buf, nbytes)
        self._elem = 8 if self.dt == T.C64 else 16

    def amplitudes(self, item: int = 0) -> torch.Tensor:
        """A complex view (no copy) of item ``item``."""
        ptr, nb = T.tcng_state_ptr(self.handle, item)
        off = ptr - self.buf.data_ptr()
        return self.buf[off:off + nb].view(self.cdtype)

    def batch_view(self) -> torch.Tensor:
        """A [batch, 2^n] complex view (no copy) when every item has the same n and
        the items lie back to back (2^n amplitudes >= 256 bytes)."""
        if len(set(self.n)) != 1:
            raise ValueError("ragged batch")
        n = self.n[0]
        ptr0, nb = T.tcng_state_ptr(self.handle, 0)
        if self.batch > 1:
            ptr1, _ = T.tcng_state_ptr(self.handle, 1)
            if ptr1 - ptr0 != nb:
                raise ValueError("items are not back to back")
        off = ptr0 - self.buf.data_ptr()
        return self.buf[off:off + nb * self.batch].view(self.cdtype).view(self.batch, 1 << n)

    def probs(self, qubits) -> torch.Tensor:
        """Born probabilities of ``qubits`` per item (qubits[0] most significant)."""
        out = torch.empty((self.batch, 1 << len(qubits)), dtype=torch.float64, device=self.buf.device)
        T.tcng_marginal_probs(self.handle, list(qubits), out)
        return out

    def reset(self):
        T.tcng_state_reset(self.handle)

    def apply(self, gates, pool=None, params=None):
        P = 0 if params is None else int(params.shape[-1])
        T.tcng_apply_circuit(self.handle, gates, pool, params, P)

    def expect(self, terms) -> torch.Tensor:
        out = torch.empty((self.batch, len(terms)), dtype=torch.float64, device=self.buf.device)
        T.tcng_expect_pauli(self.handle, terms, out)
        return out

    def energy(self, terms, coeffs=None) -> torch.Tensor:
        out = torch.empty(self.batch, dtype=torch.float64, device=self.buf.device)
        T.tcng_energy(self.handle, terms, coeffs, out)
        return out

    def free(self):
        if getattr(self, "handle", None):
            T.tcng_state_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass
