"""Dense-matrix checkers for small registers (n <= 10).

TEST INFRASTRUCTURE ONLY.  An independent second route to the same results as
``oracle/sv.c``: every gate is built as a full 2^n x 2^n operator from Pauli
matrices, projectors and ``scipy.linalg.expm`` of its generator (not from the
closed-form entries the C oracle uses), and composed by Kronecker products.
Also holds the exact ground energies used as pins:
  * dense exact diagonalisation of a Pauli-sum Hamiltonian (numpy ``eigh``);
  * the free-fermion closed form of the open-chain TFIM ground energy
    (Jordan-Wigner to a Majorana chain; the covariance-matrix formalism of the
    paper's fermion Gaussian state section, Sec. IV.C).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.linalg import expm

I2 = np.eye(2, dtype=np.complex128)
PX = np.array([[0, 1], [1, 0]], dtype=np.complex128)
PY = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
PZ = np.array([[1, 0], [0, -1]], dtype=np.complex128)
P0 = (I2 + PZ) / 2          # |0><0|
P1 = (I2 - PZ) / 2          # |1><1|

OPN = {0: "I", 1: "X", 2: "Y", 3: "Z", 4: "H", 5: "S", 6: "T", 7: "RX", 8: "RY", 9: "RZ",
       10: "CX", 11: "CZ", 12: "CP", 13: "SWAP", 14: "RZZ", 15: "U1", 16: "U2", 17: "UK", 18: "RP"}


def embed(n: int, factors: dict) -> np.ndarray:
    """kron of per-qubit 2x2 factors; qubit q is bit q (qubit n-1 leftmost)."""
    out = np.ones((1, 1), dtype=np.complex128)
    for q in range(n - 1, -1, -1):
        out = np.kron(out, factors.get(q, I2))
    return out


def embed_matrix(n: int, qubits, U: np.ndarray) -> np.ndarray:
    """Full operator of a k-qubit matrix whose local index is sum_j bit(q_j) << (k-1-j).

    Expands U = sum_{r,s} U[r,s] (x)_j |r_j><s_j| on qubit q_j.
    """
    k = len(qubits)
    full = np.zeros((1 << n, 1 << n), dtype=np.complex128)
    E = [[P0, np.array([[0, 1], [0, 0]], np.complex128)],
         [np.array([[0, 0], [1, 0]], np.complex128), P1]]
    for r in range(1 << k):
        for s in range(1 << k):
            if U[r, s] == 0:
                continue
            f = {}
            for j, q in enumerate(qubits):
                rj = (r >> (k - 1 - j)) & 1
                sj = (s >> (k - 1 - j)) & 1
                f[q] = E[rj][sj]
            full += U[r, s] * embed(n, f)
    return full


def gate_operator(n: int, g, pool, params) -> np.ndarray:
    """Full 2^n operator of one IR record, built from generators/projectors."""
    name = OPN[int(g["op"])]
    k = int(g["nq"]) if name in ("UK", "RP") else (2 if name in ("CX", "CZ", "CP", "SWAP", "RZZ", "U2") else 1)
    q = [int(v) for v in g["q"][:k]]
    ang = float(g["angle0"])
    if int(g["param"]) >= 0:
        ang += float(g["scale"]) * float(params[int(g["param"])])
    one = lambda A: embed(n, {q[0]: A})  # noqa: E731
    if name == "I":
        return np.eye(1 << n, dtype=np.complex128)
    if name == "X":
        return one(PX)
    if name == "Y":
        return one(PY)
    if name == "Z":
        return one(PZ)
    if name == "H":
        return one((PX + PZ) / math.sqrt(2))
    if name == "S":    # S = e^{i pi/4} exp(-i (pi/4) Z)
        return one(np.exp(1j * math.pi / 4) * expm(-1j * math.pi / 4 * PZ))
    if name == "T":    # T = e^{i pi/8} exp(-i (pi/8) Z)
        return one(np.exp(1j * math.pi / 8) * expm(-1j * math.pi / 8 * PZ))
    if name in ("RX", "RY", "RZ"):
        P = {"RX": PX, "RY": PY, "RZ": PZ}[name]
        return one(expm(-0.5j * ang * P))
    if name == "CX":
        return embed(n, {q[0]: P0}) + embed(n, {q[0]: P1, q[1]: PX})
    if name == "CZ":
        return embed(n, {q[0]: P0}) + embed(n, {q[0]: P1, q[1]: PZ})
    if name == "CP":
        p11 = embed(n, {q[0]: P1, q[1]: P1})
        return np.eye(1 << n) - p11 + np.exp(1j * ang) * p11
    if name == "SWAP":
        return 0.5 * (np.eye(1 << n) + embed(n, {q[0]: PX, q[1]: PX})
                      + embed(n, {q[0]: PY, q[1]: PY}) + embed(n, {q[0]: PZ, q[1]: PZ}))
    if name == "RZZ":
        return expm(-0.5j * ang * embed(n, {q[0]: PZ, q[1]: PZ}))
    if name == "RP":   # exp(-i ang P / 2), P = (x)_j sigma_{word digit j} on q[j]
        word = int(g["mat_off"])
        paulis = [I2, PX, PY, PZ]
        P = embed(n, {q[j]: paulis[(word >> (2 * j)) & 3] for j in range(k)})
        return expm(-0.5j * ang * P)
    off = int(g["mat_off"])
    d = 1 << k
    flat = pool[2 * off: 2 * (off + d * d)]
    U = (flat[0::2] + 1j * flat[1::2]).reshape(d, d)
    return embed_matrix(n, q, U)


def circuit_unitary(n: int, gates, pool, params) -> np.ndarray:
    U = np.eye(1 << n, dtype=np.complex128)
    for g in gates:
        U = gate_operator(n, g, pool, params) @ U
    return U


def run(n: int, gates, pool, params, psi0=None) -> np.ndarray:
    psi = np.zeros(1 << n, dtype=np.complex128)
    psi[0] = 1
    if psi0 is not None:
        psi = np.array(psi0, dtype=np.complex128)
    for g in gates:
        psi = gate_operator(n, g, pool, params) @ psi
    return psi


def pauli_operator(n: int, xmask: int, zmask: int) -> np.ndarray:
    f = {}
    for q in range(n):
        xb = (int(xmask) >> q) & 1
        zb = (int(zmask) >> q) & 1
        if xb and zb:
            f[q] = PY
        elif xb:
            f[q] = PX
        elif zb:
            f[q] = PZ
    return embed(n, f)


def hamiltonian_matrix(n: int, terms, coeffs=None) -> np.ndarray:
    c = terms["coeff"] if coeffs is None else coeffs
    H = np.zeros((1 << n, 1 << n), dtype=np.complex128)
    for t, ci in zip(terms, c):
        H += float(ci) * pauli_operator(n, int(t["xmask"]), int(t["zmask"]))
    return H


def ground_energy_ed(n: int, terms, coeffs=None) -> float:
    H = hamiltonian_matrix(n, terms, coeffs)
    return float(np.linalg.eigvalsh(H)[0])


def tfim_ground_energy_free_fermion(J, g) -> float:
    """Open-chain H = -sum J_i Z_i Z_{i+1} - sum g_i X_i (any real J_i, g_i).

    Jordan-Wigner maps H to i sum_{jk} M_jk a_j b_k over Majorana pairs with M
    upper-bidiagonal (M_ii = g_i, M_{i,i+1} = J_i); its ground energy is minus
    the sum of the singular values of M.
    """
    g = np.atleast_1d(np.asarray(g, dtype=np.float64))
    n = g.size
    J = np.broadcast_to(np.asarray(J, dtype=np.float64), (max(n - 1, 0),))
    M = np.diag(g)
    for i in range(n - 1):
        M[i, i + 1] = J[i]
    return float(-np.linalg.svd(M, compute_uv=False).sum())
