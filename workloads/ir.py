"""Flat gate-list input format shared by the oracle and the CUDA path.

This module defines only the data layout of a circuit and of a Pauli-sum
observable (no simulation arithmetic).  The circuit/observable statement it
encodes follows the paper's circuit primitives (Sec. I.B "Primitives":
``Circuit(n)`` with ``rx``/``ry``/``rzz``/``h``/``cx``/``su4`` gates and
``expectation_ps`` over Pauli strings).

Conventions (the paper is silent on them):
  * qubit q is bit q of the amplitude index (little-endian);
  * a gate's angle is ``angle0 + scale * params[param]`` (``param < 0``: no
    parameter, the angle is ``angle0``);
  * R_P(t) = exp(-i t P / 2) for RX, RY, RZ and RZZ;
  * the local row/column index of a k-qubit gate matrix is
    ``sum_j bit(q[j]) << (k-1-j)``, i.e. ``q[0]`` is the most significant;
  * CX lists (control, target); CP(phi) = diag(1, 1, 1, e^{i phi});
  * a Pauli string is (xmask, zmask): X on bits of xmask only, Z on bits of
    zmask only, Y where both are set.
"""
from __future__ import annotations

import numpy as np

OPS = {
    "I": 0, "X": 1, "Y": 2, "Z": 3, "H": 4, "S": 5, "T": 6,
    "RX": 7, "RY": 8, "RZ": 9, "CX": 10, "CZ": 11, "CP": 12, "SWAP": 13,
    "RZZ": 14, "U1": 15, "U2": 16, "UK": 17, "RP": 18,
}
OP_NAMES = {v: k for k, v in OPS.items()}
NQ = {"I": 1, "X": 1, "Y": 1, "Z": 1, "H": 1, "S": 1, "T": 1, "RX": 1, "RY": 1,
      "RZ": 1, "CX": 2, "CZ": 2, "CP": 2, "SWAP": 2, "RZZ": 2, "U1": 1, "U2": 2}
PARAMETRIC = {"RX", "RY", "RZ", "RZZ", "CP", "RP"}
PAULI_DIGIT = {"I": 0, "X": 1, "Y": 2, "Z": 3}

# struct tcng_gate { uint16 op; uint8 nq; uint8 pad; int32 q[5]; int32 param;
#                    double scale; double angle0; int64 mat_off; }  -> 56 bytes
GATE_DTYPE = np.dtype(
    [("op", "<u2"), ("nq", "u1"), ("pad", "u1"), ("q", "<i4", (5,)),
     ("param", "<i4"), ("scale", "<f8"), ("angle0", "<f8"), ("mat_off", "<i8")],
    align=True)
# struct tcng_pauli { uint64 xmask; uint64 zmask; double coeff; } -> 24 bytes
PAULI_DTYPE = np.dtype([("xmask", "<u8"), ("zmask", "<u8"), ("coeff", "<f8")],
                       align=True)

assert GATE_DTYPE.itemsize == 56 and GATE_DTYPE.fields["scale"][1] == 32
assert PAULI_DTYPE.itemsize == 24


class Circuit:
    """Builder for the flat gate list.  Matrices go to a complex128 pool."""

    def __init__(self, n: int):
        self.n = int(n)
        self.ops: list[tuple] = []      # (op, qubits, param, scale, angle0, mat)
        self.n_params = 0

    # -- generic ---------------------------------------------------------
    def add(self, name, qubits, param=-1, scale=1.0, angle0=0.0, matrix=None):
        qubits = tuple(int(q) for q in qubits)
        if name in NQ and len(qubits) != NQ[name]:
            raise ValueError(f"{name} takes {NQ[name]} qubits")
        if name == "RP":   # `matrix` carries the Pauli word: digit j (2 bits) on qubits[j]
            word = int(matrix)
            if not 0 <= word < 4 ** len(qubits):
                raise ValueError("Pauli word out of range")
            matrix = word
        elif matrix is not None:
            matrix = np.asarray(matrix, dtype=np.complex128)
            d = 1 << len(qubits)
            if matrix.shape != (d, d):
                raise ValueError("matrix shape does not match qubit count")
        if param is not None and param >= 0:
            self.n_params = max(self.n_params, int(param) + 1)
        self.ops.append((name, qubits, -1 if param is None else int(param),
                         float(scale), float(angle0), matrix))
        return self

    def __len__(self):
        return len(self.ops)

    # -- named gates -----------------------------------------------------
    def _rot(self, name, qubits, param, angle, scale):
        return self.add(name, qubits, param=-1 if param is None else param,
                        scale=scale, angle0=angle)

    def i(self, q): return self.add("I", (q,))
    def x(self, q): return self.add("X", (q,))
    def y(self, q): return self.add("Y", (q,))
    def z(self, q): return self.add("Z", (q,))
    def h(self, q): return self.add("H", (q,))
    def s(self, q): return self.add("S", (q,))
    def t(self, q): return self.add("T", (q,))
    def cx(self, c, t): return self.add("CX", (c, t))
    def cz(self, a, b): return self.add("CZ", (a, b))
    def swap(self, a, b): return self.add("SWAP", (a, b))

    def rx(self, q, param=None, angle=0.0, scale=1.0):
        return self._rot("RX", (q,), param, angle, scale)

    def ry(self, q, param=None, angle=0.0, scale=1.0):
        return self._rot("RY", (q,), param, angle, scale)

    def rz(self, q, param=None, angle=0.0, scale=1.0):
        return self._rot("RZ", (q,), param, angle, scale)

    def rzz(self, a, b, param=None, angle=0.0, scale=1.0):
        return self._rot("RZZ", (a, b), param, angle, scale)

    def cp(self, a, b, param=None, angle=0.0, scale=1.0):
        return self._rot("CP", (a, b), param, angle, scale)

    def rp(self, qubits, paulis, param=None, angle=0.0, scale=1.0):
        """exp(-i t P / 2) with P = paulis[0] on qubits[0] (x) paulis[1] on qubits[1] ...,
        paulis a string over I, X, Y, Z; t = angle + scale * params[param]."""
        word = sum(PAULI_DIGIT[c] << (2 * j) for j, c in enumerate(paulis))
        return self.add("RP", qubits, param=-1 if param is None else param, scale=scale,
                        angle0=angle, matrix=word)

    def unitary(self, qubits, matrix):
        qubits = tuple(qubits)
        name = {1: "U1", 2: "U2"}.get(len(qubits), "UK")
        return self.add(name, qubits, matrix=matrix)

    # -- serialisation ---------------------------------------------------
    def to_ir(self):
        """Return (gates[GATE_DTYPE], pool float64[2*n_mat]) (pool: re,im pairs)."""
        gates = np.zeros(len(self.ops), dtype=GATE_DTYPE)
        pool = []
        off = 0
        for i, (name, qubits, param, scale, angle0, mat) in enumerate(self.ops):
            g = gates[i]
            g["op"] = OPS[name]
            g["nq"] = len(qubits)
            q = np.full(5, -1, dtype=np.int32)
            q[:len(qubits)] = qubits
            g["q"] = q
            g["param"] = param
            g["scale"] = scale
            g["angle0"] = angle0
            if name == "RP":
                g["mat_off"] = mat
            elif mat is not None:
                g["mat_off"] = off
                pool.append(mat.reshape(-1))
                off += mat.size
            else:
                g["mat_off"] = -1
        if pool:
            flat = np.concatenate(pool)
            pool_arr = np.empty(2 * flat.size, dtype=np.float64)
            pool_arr[0::2] = flat.real
            pool_arr[1::2] = flat.imag
        else:
            pool_arr = np.zeros(0, dtype=np.float64)
        return gates, pool_arr


def pauli_terms(strings, coeffs=None):
    """Build a PAULI_DTYPE array from [{qubit: 'X'|'Y'|'Z'}, ...] dicts."""
    out = np.zeros(len(strings), dtype=PAULI_DTYPE)
    for i, s in enumerate(strings):
        xm = zm = 0
        for q, p in s.items():
            if p in ("X", "Y"):
                xm |= 1 << int(q)
            if p in ("Z", "Y"):
                zm |= 1 << int(q)
        out[i]["xmask"] = xm
        out[i]["zmask"] = zm
        out[i]["coeff"] = 1.0 if coeffs is None else float(coeffs[i])
    return out
