"""B300 (sm_103a) state-vector simulator: Python side of the C ABI.

``tcng`` is the one-to-one ctypes binding of ``include/tcng.h``; ``StateBatch``
is a convenience owner of a batch of state vectors living in a torch CUDA
buffer.  All arithmetic runs in the library's CUDA kernels.
"""
from __future__ import annotations

from . import tcng  # noqa: F401
from .tcng import C64, C128, GATE_DTYPE, PAULI_DTYPE, TcngError  # noqa: F401
from .state import StateBatch  # noqa: F401
