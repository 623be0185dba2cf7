"""Seeded synthetic inputs in the flat gate-list format (no simulation arithmetic).

Both the oracle (``oracle/``) and the CUDA library's tests and benchmark draw
their inputs from here; nothing in this package computes a state, an
expectation or a gradient.
"""
from .ir import GATE_DTYPE, PAULI_DTYPE, OPS, OP_NAMES, NQ, PARAMETRIC, Circuit, pauli_terms  # noqa: F401
from . import generators  # noqa: F401
