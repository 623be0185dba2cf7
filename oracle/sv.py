"""ctypes wrapper around the oracle's C simulator (``oracle/sv.c``).

TEST INFRASTRUCTURE ONLY: only the tests, the smoke check and the benchmark's
CPU-baseline leg use this module.  It builds ``liboracle.so`` with gcc on first
use (plain C99 + OpenMP) and exposes numpy-friendly functions.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sv.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile liboracle.so (gcc -O2 -fopenmp).  Returns the library path."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu99", "-fopenmp", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB)
            dp = C.POINTER(C.c_double)
            vp = C.c_void_p
            u64p = C.POINTER(C.c_uint64)
            i64 = C.c_int64
            L.orc_apply.argtypes = [C.c_int, dp, vp, i64, dp, i64, dp, C.c_int]
            L.orc_gate_matrix.argtypes = [vp, dp, dp, dp]
            L.orc_expect.argtypes = [C.c_int, dp, u64p, u64p, i64, dp, dp]
            L.orc_hamiltonian_apply.argtypes = [C.c_int, dp, u64p, u64p, dp, i64, dp]
            L.orc_energy.argtypes = [C.c_int, vp, i64, dp, i64, dp, C.c_int, u64p, u64p, dp, i64, dp]
            L.orc_grad_param_shift.argtypes = [C.c_int, vp, i64, dp, i64, dp, C.c_int, u64p, u64p,
                                               dp, i64, dp]
            L.orc_grad_fd.argtypes = [C.c_int, vp, i64, dp, i64, dp, C.c_int, u64p, u64p, dp, i64,
                                      C.c_double, dp]
            L.orc_marginal_probs.argtypes = [C.c_int, dp, C.POINTER(C.c_int32), C.c_int, dp]
            L.orc_measure_qubit.argtypes = [C.c_int, dp, C.c_int, C.c_double, C.c_int, dp, dp]
            for f in ("orc_marginal_probs", "orc_measure_qubit", "orc_apply", "orc_gate_matrix", "orc_expect", "orc_hamiltonian_apply",
                      "orc_energy", "orc_grad_param_shift", "orc_grad_fd"):
                getattr(L, f).restype = C.c_int
            L.orc_num_threads.restype = C.c_int
            _lib = L
    return _lib


def _d(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _u(a):
    return a.ctypes.data_as(C.POINTER(C.c_uint64))


def _prep(gates, pool, params):
    gates = np.ascontiguousarray(gates)
    pool = np.ascontiguousarray(pool if pool is not None else np.zeros(0), dtype=np.float64)
    params = np.ascontiguousarray(params if params is not None else np.zeros(0), dtype=np.float64)
    if pool.size == 0:
        pool = np.zeros(2, dtype=np.float64)
    P = params.size
    if params.size == 0:
        params = np.zeros(1, dtype=np.float64)
    return gates, pool, params, P


def _terms(terms, coeffs=None):
    xm = np.ascontiguousarray(terms["xmask"], dtype=np.uint64)
    zm = np.ascontiguousarray(terms["zmask"], dtype=np.uint64)
    c = np.ascontiguousarray(terms["coeff"] if coeffs is None else coeffs, dtype=np.float64)
    if xm.size == 0:
        xm = np.zeros(1, np.uint64); zm = np.zeros(1, np.uint64); c = np.zeros(1)
        return xm, zm, c, 0
    return xm, zm, c, xm.size


def zero_state(n: int) -> np.ndarray:
    psi = np.zeros(1 << n, dtype=np.complex128)
    psi[0] = 1.0
    return psi


def apply(n, gates, pool, params, psi=None) -> np.ndarray:
    """Apply the gate list (unfused, in order) to psi (default |0..0>)."""
    gates, pool, params, P = _prep(gates, pool, params)
    psi = zero_state(n) if psi is None else np.array(psi, dtype=np.complex128, copy=True)
    pf = psi.view(np.float64)
    rc = lib().orc_apply(n, _d(pf), gates.ctypes.data, len(gates), _d(pool), pool.size // 2,
                         _d(params), P)
    if rc:
        raise ValueError("oracle rejected the gate list")
    return psi


def gate_matrix(gate, pool=None, params=None) -> np.ndarray:
    g = np.ascontiguousarray(np.atleast_1d(gate))
    _, pool, params, _ = _prep(g, pool, params)
    k = int(g[0]["nq"])
    out = np.zeros((1 << k) ** 2, dtype=np.complex128)
    rc = lib().orc_gate_matrix(g.ctypes.data, _d(pool), _d(params), _d(out.view(np.float64)))
    if rc:
        raise ValueError("bad gate")
    return out.reshape(1 << k, 1 << k)


def expect(n, psi, terms) -> np.ndarray:
    """Complex <psi|P_t|psi> per term (coefficients are not applied)."""
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    xm, zm, _, T = _terms(terms)
    re = np.zeros(max(T, 1)); im = np.zeros(max(T, 1))
    rc = lib().orc_expect(n, _d(psi.view(np.float64)), _u(xm), _u(zm), T, _d(re), _d(im))
    if rc:
        raise ValueError("mask outside the register")
    return (re + 1j * im)[:T]


def hamiltonian_apply(n, psi, terms, coeffs=None) -> np.ndarray:
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    xm, zm, c, T = _terms(terms, coeffs)
    out = np.zeros_like(psi)
    lib().orc_hamiltonian_apply(n, _d(psi.view(np.float64)), _u(xm), _u(zm), _d(c), T,
                                _d(out.view(np.float64)))
    return out


def energy(n, gates, pool, params, terms, coeffs=None) -> float:
    gates, pool, params, P = _prep(gates, pool, params)
    xm, zm, c, T = _terms(terms, coeffs)
    e = np.zeros(1)
    rc = lib().orc_energy(n, gates.ctypes.data, len(gates), _d(pool), pool.size // 2, _d(params),
                          P, _u(xm), _u(zm), _d(c), T, _d(e))
    if rc:
        raise ValueError("oracle rejected the input")
    return float(e[0])


def grad_param_shift(n, gates, pool, params, terms, coeffs=None) -> np.ndarray:
    gates, pool, params, P = _prep(gates, pool, params)
    xm, zm, c, T = _terms(terms, coeffs)
    g = np.zeros(max(P, 1))
    rc = lib().orc_grad_param_shift(n, gates.ctypes.data, len(gates), _d(pool), pool.size // 2,
                                    _d(params), P, _u(xm), _u(zm), _d(c), T, _d(g))
    if rc:
        raise ValueError("oracle rejected the input")
    return g[:P]


def grad_fd(n, gates, pool, params, terms, coeffs=None, h=1e-5) -> np.ndarray:
    gates, pool, params, P = _prep(gates, pool, params)
    xm, zm, c, T = _terms(terms, coeffs)
    g = np.zeros(max(P, 1))
    rc = lib().orc_grad_fd(n, gates.ctypes.data, len(gates), _d(pool), pool.size // 2, _d(params),
                           P, _u(xm), _u(zm), _d(c), T, float(h), _d(g))
    if rc:
        raise ValueError("oracle rejected the input")
    return g[:P]


def marginal_probs(n, psi, qubits) -> np.ndarray:
    """Born probabilities of measuring ``qubits`` (qubits[0] most significant bit
    of the outcome index)."""
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    q = np.ascontiguousarray(qubits, dtype=np.int32)
    out = np.zeros(1 << q.size)
    rc = lib().orc_marginal_probs(n, _d(psi.view(np.float64)), q.ctypes.data_as(C.POINTER(C.c_int32)),
                                  int(q.size), _d(out))
    if rc:
        raise ValueError("bad qubit list")
    return out


def measure_qubit(n, psi, q, u, forced=-1):
    """Measure qubit q of psi in place (Born rule with uniform u, or the forced
    outcome).  Returns (outcome, probability of the outcome, p0)."""
    assert psi.dtype == np.complex128 and psi.flags.c_contiguous
    prob = np.zeros(1)
    p0 = np.zeros(1)
    out = lib().orc_measure_qubit(n, _d(psi.view(np.float64)), int(q), float(u), int(forced), _d(prob), _d(p0))
    if out < 0:
        raise ValueError("bad qubit")
    return out, float(prob[0]), float(p0[0])


def num_threads() -> int:
    return int(lib().orc_num_threads())
