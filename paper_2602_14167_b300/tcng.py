"""Thin Python binding of the C ABI in ``include/tcng.h`` (ctypes).

Argument marshalling only: every step of the simulation runs in the CUDA
kernels of ``libtcng.so``.  Device buffers and streams come from PyTorch
(``tensor.data_ptr()``, ``torch.cuda.current_stream().cuda_stream``).  If the
library is missing the import fails loudly: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libtcng.so")

# Mirrors of the C structs (layout checked against the header sizes).
GATE_DTYPE = np.dtype(
    [("op", "<u2"), ("nq", "u1"), ("pad", "u1"), ("q", "<i4", (5,)),
     ("param", "<i4"), ("scale", "<f8"), ("angle0", "<f8"), ("mat_off", "<i8")],
    align=True)
PAULI_DTYPE = np.dtype([("xmask", "<u8"), ("zmask", "<u8"), ("coeff", "<f8")], align=True)
assert GATE_DTYPE.itemsize == 56 and PAULI_DTYPE.itemsize == 24

C64, C128 = 0, 1
(OPT_FUSE_WIDTH, OPT_TILE_BITS, OPT_CHUNK_BITS, OPT_USE_GRAPHS, OPT_UNFUSED, OPT_TENSOR_CORES,
 OPT_STATE_ADJOINT_N, OPT_TC_FP16, OPT_STATE_ADJOINT_SMALL) = range(9)
STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "EUNSUPPORTED", 5: "ETIMEOUT"}


class TcngError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class _Problem(C.Structure):
    _fields_ = [("n", C.c_int), ("ops", C.c_void_p), ("n_ops", C.c_size_t),
                ("mat_pool", C.c_void_p), ("n_mat", C.c_size_t), ("P", C.c_int),
                ("H", C.c_void_p), ("n_terms", C.c_size_t)]


_lib = None


def lib():
    """Load libtcng.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with "
                              "`python -m paper_2602_14167_b300.build`")
        L = C.CDLL(LIB_PATH)
        vp, sz, i32, dp, fp = C.c_void_p, C.c_size_t, C.c_int, C.c_double, C.c_float
        sig = {
            "tcng_state_init": [C.POINTER(vp), i32, i32, vp, vp, sz, vp],
            "tcng_state_bytes": [i32, i32, vp, C.POINTER(sz)],
            "tcng_state_free": [vp],
            "tcng_state_ptr": [vp, i32, C.POINTER(vp), C.POINTER(sz)],
            "tcng_state_reset": [vp, vp],
            "tcng_apply_circuit": [vp, vp, sz, vp, sz, vp, i32, vp],
            "tcng_apply_circuit_pooled": [vp, vp, sz, vp, sz, vp, sz, vp, i32, vp],
            "tcng_expect_pauli": [vp, vp, sz, vp, vp],
            "tcng_expect_pauli_noalloc": [vp, i32, i32, vp, sz, vp, vp],
            "tcng_energy": [vp, vp, sz, vp, vp, vp],
            "tcng_expect_energy": [vp, vp, sz, vp, vp, vp, vp],
            "tcng_hamiltonian_apply": [vp, vp, sz, vp, vp, vp],
            "tcng_energy_grad": [vp, vp, sz, vp, sz, vp, i32, vp, sz, vp, vp, vp, vp],
            "tcng_energy_grad_ragged": [vp, i32, vp, i32, vp, vp, vp, vp, vp],
            "tcng_apply_shared_unitary": [vp, vp, i32, vp, vp],
            "tcng_marginal_probs": [vp, vp, i32, vp, vp],
            "tcng_measure": [vp, vp, vp, vp, vp, vp],
            "tcng_adam_step": [vp, vp, vp, vp, sz, dp, dp, dp, dp, vp, vp],
            "tcng_adam_step_f32": [vp, vp, vp, vp, sz, fp, fp, fp, fp, vp, vp],
            "tcng_mlp_forward": [vp, i32, i32, i32, i32, vp, vp, vp, vp, vp, vp, vp, vp, vp],
            "tcng_mlp_backward": [vp, i32, i32, i32, i32, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp],
            "tcng_set_option": [i32, i32],
            "tcng_get_option": [i32, C.POINTER(i32)],
            "tcng_autotune": [i32, i32, i32, C.c_char_p],
            "tcng_autotune_circuit": [vp, vp, sz, vp, sz, vp, i32, C.c_char_p, C.POINTER(dp)],
            "tcng_autotune_report": [C.c_char_p, sz],
            "tcng_fma_peak": [i32, C.POINTER(dp)],
            "tcng_plan_lock_layouts": [vp, i32, vp, C.POINTER(i32)],
            "tcng_sync_status": [],
            "tcng_profile_enable": [i32],
            "tcng_profile_read": [C.c_char_p, sz, i32],
        }
        for name, args in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = C.c_int
        L.tcng_describe_plan.argtypes = [i32, vp, sz, vp, sz, i32, i32]
        L.tcng_describe_plan.restype = C.c_char_p
        L.tcng_describe_state_adjoint.argtypes = [i32, vp, sz, vp, sz, i32, vp, sz, i32]
        L.tcng_describe_state_adjoint.restype = C.c_char_p
        L.tcng_last_error.restype = C.c_char_p
        L.tcng_version.restype = C.c_char_p
        L.tcng_launch_count.restype = C.c_uint64
        _lib = L
    return _lib


def _check(status):
    if status != 0:
        raise TcngError(status, lib().tcng_last_error().decode())


def _ptr(x):
    """Device/host address of a torch tensor, numpy array, int or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    raise TypeError(f"cannot take the address of {type(x)}")


def _stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _gates(gates):
    g = np.ascontiguousarray(gates)
    if g.dtype.itemsize != 56 or g.dtype.names is None or "mat_off" not in g.dtype.names:
        raise TypeError("gates must be a structured array with the tcng_gate layout")
    return g


def _pool(pool):
    p = np.ascontiguousarray(pool if pool is not None else np.zeros(0), dtype=np.float64)
    return p, p.size // 2


def _terms(terms):
    t = np.ascontiguousarray(terms)
    if t.dtype.itemsize != 24 or t.dtype.names is None or "zmask" not in t.dtype.names:
        raise TypeError("terms must be a structured array with the tcng_pauli layout")
    return t


# ------------------------------------------------------------- entry points --
def tcng_state_init(dtype, n_qubits, dev_buf=None, buf_bytes=0, stream=None):
    nq = np.ascontiguousarray(np.atleast_1d(n_qubits), dtype=np.int32)
    h = C.c_void_p()
    _check(lib().tcng_state_init(C.byref(h), int(dtype), int(nq.size), nq.ctypes.data,
                                 _ptr(dev_buf), int(buf_bytes), _stream(stream)))
    return h.value


def tcng_state_bytes(dtype, n_qubits):
    nq = np.ascontiguousarray(np.atleast_1d(n_qubits), dtype=np.int32)
    b = C.c_size_t()
    _check(lib().tcng_state_bytes(int(dtype), int(nq.size), nq.ctypes.data, C.byref(b)))
    return b.value


def tcng_state_free(handle):
    _check(lib().tcng_state_free(handle))


def tcng_state_ptr(handle, item=0):
    p, b = C.c_void_p(), C.c_size_t()
    _check(lib().tcng_state_ptr(handle, int(item), C.byref(p), C.byref(b)))
    return p.value, b.value


def tcng_state_reset(handle, stream=None):
    _check(lib().tcng_state_reset(handle, _stream(stream)))


def tcng_apply_circuit(handle, gates, pool, params_dev, P, stream=None):
    g = _gates(gates)
    p, n_mat = _pool(pool)
    _check(lib().tcng_apply_circuit(handle, g.ctypes.data, len(g), p.ctypes.data if n_mat else None,
                                    n_mat, _ptr(params_dev), int(P), _stream(stream)))


def tcng_expect_pauli(handle, terms, out_dev, stream=None):
    t = _terms(terms)
    _check(lib().tcng_expect_pauli(handle, t.ctypes.data, len(t), _ptr(out_dev), _stream(stream)))


def tcng_expect_pauli_noalloc(psi_dev, n, dtype, terms, out_dev, stream=None):
    """Expectations of one state without any device allocation (static scratch)."""
    t = _terms(terms)
    _check(lib().tcng_expect_pauli_noalloc(_ptr(psi_dev), int(n), int(dtype), t.ctypes.data, len(t),
                                           _ptr(out_dev), _stream(stream)))


def tcng_energy(handle, terms, coeffs_dev, energy_dev, stream=None):
    t = _terms(terms)
    _check(lib().tcng_energy(handle, t.ctypes.data, len(t), _ptr(coeffs_dev), _ptr(energy_dev),
                             _stream(stream)))


def tcng_expect_energy(handle, terms, coeffs_dev, out_dev, energy_dev, stream=None):
    t = _terms(terms)
    _check(lib().tcng_expect_energy(handle, t.ctypes.data, len(t), _ptr(coeffs_dev), _ptr(out_dev),
                                    _ptr(energy_dev), _stream(stream)))


def tcng_hamiltonian_apply(handle, terms, coeffs_dev, out_handle, stream=None):
    t = _terms(terms)
    _check(lib().tcng_hamiltonian_apply(handle, t.ctypes.data, len(t), _ptr(coeffs_dev), out_handle,
                                        _stream(stream)))


def tcng_energy_grad(handle, gates, pool, params_dev, P, terms, coeffs_dev, energy_dev, grad_dev,
                     stream=None):
    g = _gates(gates)
    p, n_mat = _pool(pool)
    t = _terms(terms)
    _check(lib().tcng_energy_grad(handle, g.ctypes.data, len(g), p.ctypes.data if n_mat else None,
                                  n_mat, _ptr(params_dev), int(P), t.ctypes.data, len(t),
                                  _ptr(coeffs_dev), _ptr(energy_dev), _ptr(grad_dev),
                                  _stream(stream)))


def tcng_energy_grad_ragged(problems, item_problem, params_dev, coeffs_dev, energy_dev, grad_dev,
                            stream=None):
    """problems: list of dicts(n, gates, pool, P, terms)."""
    keep = []
    arr = (_Problem * len(problems))()
    for i, pr in enumerate(problems):
        g = _gates(pr["gates"])
        p, n_mat = _pool(pr.get("pool"))
        t = _terms(pr["terms"])
        keep += [g, p, t]
        arr[i] = _Problem(int(pr["n"]), g.ctypes.data, len(g), p.ctypes.data if n_mat else None,
                          n_mat, int(pr["P"]), t.ctypes.data, len(t))
    ip = np.ascontiguousarray(item_problem, dtype=np.int32)
    _check(lib().tcng_energy_grad_ragged(C.cast(arr, C.c_void_p), len(problems), ip.ctypes.data,
                                         int(ip.size), _ptr(params_dev), _ptr(coeffs_dev),
                                         _ptr(energy_dev), _ptr(grad_dev), _stream(stream)))
    del keep


def tcng_apply_shared_unitary(handle, qubits, U, stream=None):
    q = np.ascontiguousarray(qubits, dtype=np.int32)
    u = np.ascontiguousarray(np.asarray(U, dtype=np.complex128)).view(np.float64)
    _check(lib().tcng_apply_shared_unitary(handle, q.ctypes.data, int(q.size), u.ctypes.data,
                                           _stream(stream)))


def tcng_marginal_probs(handle, qubits, out_dev, stream=None):
    q = np.ascontiguousarray(qubits, dtype=np.int32)
    _check(lib().tcng_marginal_probs(handle, q.ctypes.data, int(q.size), _ptr(out_dev), _stream(stream)))


def tcng_measure(handle, mask_dev, u_dev, outcome_dev, logp_dev=None, stream=None):
    _check(lib().tcng_measure(handle, _ptr(mask_dev), _ptr(u_dev), _ptr(outcome_dev), _ptr(logp_dev),
                              _stream(stream)))


def tcng_apply_circuit_pooled(handle, gates, pool, item_pool_dev, pool_stride, params_dev=None, P=0,
                              stream=None):
    """Per-item explicit matrices: item b reads its gate matrices from
    item_pool_dev[b * pool_stride ...] (device complex128); ``pool`` is a host
    pool of the same layout used for planning."""
    g = _gates(gates)
    p, n_mat = _pool(pool)
    _check(lib().tcng_apply_circuit_pooled(handle, g.ctypes.data, len(g), p.ctypes.data if n_mat else None,
                                           n_mat, _ptr(item_pool_dev), int(pool_stride), _ptr(params_dev),
                                           int(P), _stream(stream)))


def tcng_adam_step(theta, m, v, grad, n, lr, b1, b2, eps, step_dev, stream=None):
    _check(lib().tcng_adam_step(_ptr(theta), _ptr(m), _ptr(v), _ptr(grad), int(n), float(lr),
                                float(b1), float(b2), float(eps), _ptr(step_dev), _stream(stream)))


def tcng_adam_step_f32(theta, m, v, grad, n, lr, b1, b2, eps, step_dev, stream=None):
    _check(lib().tcng_adam_step_f32(_ptr(theta), _ptr(m), _ptr(v), _ptr(grad), int(n), float(lr),
                                    float(b1), float(b2), float(eps), _ptr(step_dev), _stream(stream)))


def tcng_mlp_forward(x, N, F, H, O, w1, b1, w2, b2, w3, b3, act, y, stream=None):
    _check(lib().tcng_mlp_forward(_ptr(x), N, F, H, O, _ptr(w1), _ptr(b1), _ptr(w2), _ptr(b2),
                                  _ptr(w3), _ptr(b3), _ptr(act), _ptr(y), _stream(stream)))


def tcng_mlp_backward(x, N, F, H, O, w1, w2, w3, act, y, target, mask, grads, loss_dev, stream=None):
    _check(lib().tcng_mlp_backward(_ptr(x), N, F, H, O, _ptr(w1), _ptr(w2), _ptr(w3), _ptr(act),
                                   _ptr(y), _ptr(target), _ptr(mask), _ptr(grads), _ptr(loss_dev),
                                   _stream(stream)))


def tcng_set_option(opt, value):
    _check(lib().tcng_set_option(int(opt), int(value)))


def tcng_get_option(opt):
    v = C.c_int()
    _check(lib().tcng_get_option(int(opt), C.byref(v)))
    return v.value


def tcng_fma_peak(fp64=False):
    """Measured FMA throughput in TFLOP/s (FP32, or FP64 with fp64=True)."""
    out = C.c_double(0.0)
    _check(lib().tcng_fma_peak(int(bool(fp64)), C.byref(out)))
    return out.value


def tcng_autotune(n, dtype, batch, cache_path=None):
    _check(lib().tcng_autotune(int(n), int(dtype), int(batch),
                               cache_path.encode() if cache_path else None))


def tcng_autotune_circuit(handle, gates, pool, params_dev, P, cache_path=None):
    """Time every option candidate on this circuit and state; returns the best ms
    per call (None when the choice came from the cache)."""
    g = _gates(gates)
    p, n_mat = _pool(pool)
    best = C.c_double(-1.0)
    _check(lib().tcng_autotune_circuit(handle, g.ctypes.data, len(g), p.ctypes.data if n_mat else None,
                                       n_mat, _ptr(params_dev), int(P),
                                       cache_path.encode() if cache_path else None, C.byref(best)))
    return None if best.value < 0 else best.value


def tcng_autotune_report():
    """[(fuse_width, tile_bits, chunk_bits, tensor_cores, ms)] of the last autotune
    run, or [("cached", line)] when its choice was loaded from the cache."""
    buf = C.create_string_buffer(1 << 16)
    _check(lib().tcng_autotune_report(buf, len(buf)))
    out = []
    for line in buf.value.decode().splitlines():
        if line.startswith("cached"):
            out.append(("cached", line[7:]))
        elif line.strip():
            f = line.split()
            out.append((int(f[0]), int(f[1]), int(f[2]), int(f[3]), float(f[4])))
    return out


def tcng_sync_status():
    _check(lib().tcng_sync_status())


def tcng_profile_enable(on=True):
    _check(lib().tcng_profile_enable(int(bool(on))))


def tcng_profile_read(reset=True):
    """{kernel: (launches, total_ms)} of the event-timed launches since the last reset."""
    buf = C.create_string_buffer(1 << 16)
    _check(lib().tcng_profile_read(buf, len(buf), int(reset)))
    out = {}
    for line in buf.value.decode().splitlines():
        name, cnt, ms = line.split()
        out[name] = (int(cnt), float(ms))
    return out


def tcng_describe_plan(n, gates, pool, P, adjoint=False):
    g = _gates(gates)
    p, n_mat = _pool(pool)
    return lib().tcng_describe_plan(int(n), g.ctypes.data, len(g), p.ctypes.data if n_mat else None,
                                    n_mat, int(P), int(adjoint)).decode()


def tcng_describe_state_adjoint(n, gates, pool, P, terms, dtype=C64):
    """Host-only summary of the state-pass adjoint's plan (segments, H passes)."""
    g = _gates(gates)
    p, n_mat = _pool(pool)
    t = _terms(terms)
    return lib().tcng_describe_state_adjoint(int(n), g.ctypes.data, len(g), p.ctypes.data if n_mat else None,
                                             n_mat, int(P), t.ctypes.data if len(t) else None, len(t),
                                             int(dtype)).decode()


def tcng_plan_lock_layouts(rbit):
    """Shared-memory layouts of a lock-step FP16 pass: rbit is an (nst, 4) array of
    register tile bits; returns (layouts (nst, 8) uint8, relocated)."""
    import numpy as np
    rb = np.ascontiguousarray(np.asarray(rbit, dtype=np.uint8).reshape(-1, 4))
    out = np.zeros((rb.shape[0], 8), dtype=np.uint8)
    rel = C.c_int(0)
    _check(lib().tcng_plan_lock_layouts(rb.ctypes.data, int(rb.shape[0]), out.ctypes.data, C.byref(rel)))
    return out, bool(rel.value)


def tcng_launch_count():
    return int(lib().tcng_launch_count())


def tcng_last_error():
    return lib().tcng_last_error().decode()


def tcng_version():
    return lib().tcng_version().decode()


EXPORTED = [
    "tcng_state_init", "tcng_state_bytes", "tcng_state_free", "tcng_state_ptr", "tcng_state_reset",
    "tcng_apply_circuit", "tcng_apply_circuit_pooled", "tcng_expect_pauli", "tcng_expect_pauli_noalloc", "tcng_energy", "tcng_expect_energy",
    "tcng_hamiltonian_apply",
    "tcng_energy_grad", "tcng_energy_grad_ragged", "tcng_apply_shared_unitary", "tcng_marginal_probs", "tcng_measure",
    "tcng_adam_step",
    "tcng_adam_step_f32", "tcng_mlp_forward", "tcng_mlp_backward", "tcng_set_option", "tcng_fma_peak",
    "tcng_get_option", "tcng_autotune", "tcng_autotune_circuit", "tcng_autotune_report", "tcng_sync_status", "tcng_describe_plan", "tcng_describe_state_adjoint",
    "tcng_plan_lock_layouts",
    "tcng_profile_enable", "tcng_profile_read",
    "tcng_launch_count", "tcng_last_error", "tcng_version",
]
