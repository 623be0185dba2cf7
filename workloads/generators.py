"""Seeded synthetic inputs (circuits, observables, batches) for both sides.

Holds no simulation arithmetic: every function here only draws random numbers
and lays them out in the flat input format of ``workloads.ir``.  Random draws
use ``numpy.random.default_rng(seed)`` in the order documented per function so
the same seed gives bit-identical inputs to the oracle and to the CUDA path.

Workload shapes follow the paper's circuits: the TFIM VQE ansatz of Sec. I.B,
the SU(4) brickwork of the QML and MIPT demonstrations (Sec. VII.B, VII.C),
and the parameter layouts they quote.
"""
from __future__ import annotations

import math

import numpy as np

from .ir import Circuit, PAULI_DTYPE

TWO_PI = 2.0 * math.pi


# ---------------------------------------------------------------------------
# random unitaries
# ---------------------------------------------------------------------------
def haar_su4(rng: np.random.Generator) -> np.ndarray:
    """Haar-random SU(4) matrix (MIPT/QML brickwork gates, Sec. VII.C).

    Z = (A + iB)/sqrt(2) with A, B = rng.standard_normal((2, 4, 4)) (A first);
    Q, R = qr(Z); Q <- Q diag(R_ii/|R_ii|) (Mezzadri's phase fix);
    U = Q / det(Q)^(1/4) with the principal fourth root.
    """
    a, b = rng.standard_normal((2, 4, 4))
    z = (a + 1j * b) / math.sqrt(2.0)
    q, r = np.linalg.qr(z)
    d = np.diag(r)
    q = q * (d / np.abs(d))[None, :]
    det = np.linalg.det(q)
    return q / np.power(det, 0.25)


def haar_unitary(rng: np.random.Generator, dim: int) -> np.ndarray:
    """Haar-random U(dim) by the same QR recipe (no determinant fix)."""
    a, b = rng.standard_normal((2, dim, dim))
    z = (a + 1j * b) / math.sqrt(2.0)
    q, r = np.linalg.qr(z)
    d = np.diag(r)
    return q * (d / np.abs(d))[None, :]


# ---------------------------------------------------------------------------
# circuits
# ---------------------------------------------------------------------------
def ry_cx_ladder(n: int = 10, layers: int = 4, seed: int = 0):
    """Layers of [RY(theta[l, q]) on every qubit, CX(0,1), CX(1,2), ... CX(n-2, n-1)].

    theta = rng.uniform(-pi, pi, (layers, n)); param index = l*n + q.
    Returns (Circuit, theta flat float64[layers*n]).
    """
    rng = np.random.default_rng(seed)
    theta = rng.uniform(-math.pi, math.pi, size=(layers, n))
    c = Circuit(n)
    for l in range(layers):
        for q in range(n):
            c.ry(q, param=l * n + q)
        for q in range(n - 1):
            c.cx(q, q + 1)
    return c, theta.reshape(-1).copy()


def brickwork_bonds(n: int, t: int):
    """Bonds (i, i+1) of brickwork layer t on an open chain: i = t mod 2, step 2."""
    return [(i, i + 1) for i in range(t % 2, n - 1, 2)]


def su4_brickwork(n: int, depth: int, rot: str = "RX", seed: int = 0):
    """Haar SU(4) brickwork interleaved with a rotation layer.

    Layer t: one Haar SU(4) on every bond of ``brickwork_bonds(n, t)``, then
    ``rot``(theta[t, q]) on every qubit q.  Draw order: all SU(4) matrices in
    gate order, then theta = rng.uniform(-pi, pi, (depth, n)).
    Param index = t*n + q.  Returns (Circuit, theta flat).
    """
    rng = np.random.default_rng(seed)
    mats = [[haar_su4(rng) for _ in brickwork_bonds(n, t)] for t in range(depth)]
    theta = rng.uniform(-math.pi, math.pi, size=(depth, n))
    c = Circuit(n)
    for t in range(depth):
        for (a, b), u in zip(brickwork_bonds(n, t), mats[t]):
            c.unitary((a, b), u)
        for q in range(n):
            c.add(rot, (q,), param=t * n + q)
    return c, theta.reshape(-1).copy()


def cut_brickwork(n: int, depth: int, block: int, rot: str = "RZ", seed: int = 0):
    """``su4_brickwork(n, depth, rot, seed)`` without the SU(4) gates on the bonds
    that cross a multiple of ``block`` ((block-1, block), (2 block-1, 2 block), ...).

    Every other gate, matrix and angle is the one ``su4_brickwork`` draws for the
    same seed, so the circuit keeps the full workload's layer structure while its
    state stays the tensor product of n/block independent block circuits (see
    ``block_circuit``).  Returns (Circuit, theta flat).
    """
    c, theta = su4_brickwork(n, depth, rot, seed)
    out = Circuit(n)
    for (name, qubits, param, scale, angle0, mat) in c.ops:
        if len(qubits) == 2 and min(qubits) // block != max(qubits) // block:
            continue
        out.add(name, qubits, param=param, scale=scale, angle0=angle0, matrix=mat)
    out.n_params = c.n_params
    return out, theta


def block_circuit(c: Circuit, lo: int, nq: int) -> Circuit:
    """The ops of ``c`` acting only inside qubits lo..lo+nq-1, moved to qubits 0..nq-1
    (params keep their indices)."""
    out = Circuit(nq)
    for (name, qubits, param, scale, angle0, mat) in c.ops:
        if all(lo <= q < lo + nq for q in qubits):
            out.add(name, tuple(q - lo for q in qubits), param=param, scale=scale,
                    angle0=angle0, matrix=mat)
    out.n_params = c.n_params
    return out


def inverse_circuit(c: Circuit) -> Circuit:
    """The circuit U^dagger: ops in reverse order, rotation angles negated, explicit
    matrices conjugate-transposed, S and T replaced by their inverses."""
    inv = Circuit(c.n)
    for (name, qubits, param, scale, angle0, mat) in reversed(c.ops):
        if name in ("RX", "RY", "RZ", "RZZ", "CP", "RP"):
            inv.add(name, qubits, param=param, scale=-scale, angle0=-angle0, matrix=mat)
        elif name in ("U1", "U2", "UK"):
            inv.unitary(qubits, mat.conj().T)
        elif name == "S":
            inv.unitary(qubits, np.diag([1, -1j]))
        elif name == "T":
            inv.unitary(qubits, np.diag([1, np.exp(-1j * math.pi / 4)]))
        else:
            inv.add(name, qubits)
    inv.n_params = c.n_params
    return inv


def slice_circuit(c: Circuit, nq: int) -> Circuit:
    """Drop every op whose support is not inside {0..nq-1}; params keep indices."""
    out = Circuit(nq)
    for (name, qubits, param, scale, angle0, mat) in c.ops:
        if all(q < nq for q in qubits):
            out.add(name, qubits, param=param, scale=scale, angle0=angle0, matrix=mat)
    out.n_params = c.n_params
    return out


def qml_brickwall(n: int, layers: int, seed: int = 0):
    """The QML ansatz of Sec. VII.B: per layer one SU(4) on every even pair
    (0,1), (2,3), ... then on every odd pair (1,2), (3,4), ...; each gate a Haar
    SU(4) matrix (``haar_su4``) drawn in gate order (the trained weights are
    replaced by random gates; the gate count is 15 parameters per gate in the
    paper: layers * (n - 1) * 15).  No parameters: one circuit for the whole batch.
    """
    rng = np.random.default_rng(seed)
    c = Circuit(n)
    for _ in range(layers):
        for i in list(range(0, n - 1, 2)) + list(range(1, n - 1, 2)):
            c.unitary((i, i + 1), haar_su4(rng))
    return c


SU4_WORDS = [a + b for a in "IXYZ" for b in "IXYZ" if a + b != "II"]


def su4_ladder(n: int, layers: int):
    """The SU(4)-ladder ansatz of the paper's distributed VQE benchmark (Sec. VI.B):
    per layer su4(i, i+1) for i = 0..n-2 in order, 15 parameters per gate
    (15 L (n-1) in all).  su4(i, j; t_1..t_15) is written as the ordered product of
    the 15 two-qubit Pauli rotations exp(-i t_a P_a / 2), P_a over SU4_WORDS
    (lexicographic in I, X, Y, Z; first letter on qubit i), applied a = 1 first.
    Param index = (layer (n-1) + i) 15 + a.  Returns the Circuit."""
    c = Circuit(n)
    for l in range(layers):
        for i in range(n - 1):
            base = (l * (n - 1) + i) * 15
            for a, w in enumerate(SU4_WORDS):
                c.rp((i, i + 1), w, param=base + a)
    c.n_params = 15 * layers * (n - 1)
    return c


def cut_su4_ladder(n: int, layers: int, block: int):
    """``su4_ladder`` without the su4 gates on the bonds between blocks of ``block``
    qubits (their 15 parameters are read by no gate): the state stays a product of
    n / block independent ladders."""
    c = su4_ladder(n, layers)
    out = Circuit(n)
    for (name, qubits, param, scale, angle0, mat) in c.ops:
        if min(qubits) // block != max(qubits) // block:
            continue
        out.add(name, qubits, param=param, scale=scale, angle0=angle0, matrix=mat)
    out.n_params = c.n_params
    return out


def hea_ring(n: int, layers: int = 12):
    """Hardware-efficient ring ansatz (TFIM VQE ansatz of Sec. I.B, widened).

    Layer l: RX(theta[l,0,q]) for all q, RY(theta[l,1,q]) for all q, then
    RZZ(theta[l,2,i]) on (i, (i+1) mod n) for i = 0..n-1.
    Param index = l*3n + k*n + q; P = 3*n*layers.
    """
    c = Circuit(n)
    for l in range(layers):
        base = l * 3 * n
        for q in range(n):
            c.rx(q, param=base + q)
        for q in range(n):
            c.ry(q, param=base + n + q)
        for i in range(n):
            c.rzz(i, (i + 1) % n, param=base + 2 * n + i)
    c.n_params = 3 * n * layers
    return c


def random_circuit(n: int, n_ops: int, seed: int = 0, kinds=None):
    """Random mix of every op kind on random qubits (test input)."""
    rng = np.random.default_rng(seed)
    kinds = kinds or ["X", "Y", "Z", "H", "S", "T", "RX", "RY", "RZ", "CX", "CZ",
                      "CP", "SWAP", "RZZ", "U1", "U2", "U3", "U4", "U5"]
    c = Circuit(n)
    p = 0
    for _ in range(n_ops):
        k = kinds[int(rng.integers(len(kinds)))]
        if k in ("U3", "U4", "U5") and n < int(k[1]):
            k = "U2"
        if k in ("CX", "CZ", "CP", "SWAP", "RZZ", "U2", "RP") and n < 2:
            k = "RX"
        if k in ("X", "Y", "Z", "H", "S", "T"):
            c.add(k, (int(rng.integers(n)),))
        elif k in ("RX", "RY", "RZ"):
            c.add(k, (int(rng.integers(n)),), param=p,
                  scale=float(rng.choice([1.0, -0.5, 2.0])),
                  angle0=float(rng.uniform(-1, 1)))
            p += 1
        elif k in ("CX", "CZ", "SWAP"):
            a, b = rng.choice(n, 2, replace=False)
            c.add(k, (int(a), int(b)))
        elif k == "RP":
            kq = 1 + int(rng.integers(2))
            qs = rng.choice(n, kq, replace=False)
            word = "".join("XYZ"[int(v)] for v in rng.integers(0, 3, kq))
            c.rp(tuple(int(q) for q in qs), word, param=p, scale=float(rng.choice([1.0, -0.5])),
                 angle=float(rng.uniform(-1, 1)))
            p += 1
        elif k in ("CP", "RZZ"):
            a, b = rng.choice(n, 2, replace=False)
            c.add(k, (int(a), int(b)), param=p, scale=1.0,
                  angle0=float(rng.uniform(-1, 1)))
            p += 1
        elif k == "U1":
            c.unitary((int(rng.integers(n)),), haar_unitary(rng, 2))
        elif k == "U2":
            a, b = rng.choice(n, 2, replace=False)
            c.unitary((int(a), int(b)), haar_unitary(rng, 4))
        else:
            kq = int(k[1])
            qs = rng.choice(n, kq, replace=False)
            c.unitary(tuple(int(q) for q in qs), haar_unitary(rng, 1 << kq))
    c.n_params = p
    theta = rng.uniform(-math.pi, math.pi, size=p)
    return c, theta


# ---------------------------------------------------------------------------
# observables
# ---------------------------------------------------------------------------
def tfim_terms(n: int, J=1.0, g=1.0) -> np.ndarray:
    """Open-chain TFIM H = -sum_i J_i Z_i Z_{i+1} - g sum_i X_i (Sec. I.B).

    Term order: the n-1 ZZ bonds, then the n X fields.
    """
    J = np.broadcast_to(np.asarray(J, dtype=np.float64), (max(n - 1, 0),))
    out = np.zeros(max(n - 1, 0) + n, dtype=PAULI_DTYPE)
    for i in range(n - 1):
        out[i] = (0, (1 << i) | (1 << (i + 1)), -float(J[i]))
    for i in range(n):
        out[n - 1 + i] = (1 << i, 0, -float(g))
    return out


def xxz_terms(n: int, J, delta: float, g: float) -> np.ndarray:
    """Open-chain XXZ: sum_i J_i (X X + Y Y + delta Z Z)_{i,i+1} - g sum_i X_i.

    Term order: per bond XX, YY, ZZ; then the n X fields.
    """
    J = np.broadcast_to(np.asarray(J, dtype=np.float64), (max(n - 1, 0),))
    out = np.zeros(3 * (n - 1) + n, dtype=PAULI_DTYPE)
    k = 0
    for i in range(n - 1):
        m = (1 << i) | (1 << (i + 1))
        out[k] = (m, 0, float(J[i])); k += 1
        out[k] = (m, m, float(J[i])); k += 1
        out[k] = (0, m, float(J[i]) * float(delta)); k += 1
    for i in range(n):
        out[k] = (1 << i, 0, -float(g)); k += 1
    return out


def random_pauli_strings(n: int, count: int, weight: int = 4, seed: int = 0) -> np.ndarray:
    """Random weight-w Pauli strings, coefficient 1.

    Per string: qubits = rng.choice(n, w, replace=False), then
    kinds = rng.integers(0, 3, w) with 0 -> X, 1 -> Y, 2 -> Z.
    """
    rng = np.random.default_rng(seed)
    out = np.zeros(count, dtype=PAULI_DTYPE)
    for s in range(count):
        qs = rng.choice(n, weight, replace=False)
        ks = rng.integers(0, 3, weight)
        xm = zm = 0
        for q, k in zip(qs, ks):
            if k in (0, 1):
                xm |= 1 << int(q)
            if k in (1, 2):
                zm |= 1 << int(q)
        out[s] = (xm, zm, 1.0)
    return out


# ---------------------------------------------------------------------------
# batched VQE inputs
# ---------------------------------------------------------------------------
def tfim_batch(n: int, batch: int, layers: int = 12, seed: int = 0):
    """B TFIM chains on the ring ansatz.

    Draw order: J = rng.uniform(0.5, 1.5, (B, n-1)); g = rng.uniform(0.2, 2.0, B);
    theta = rng.uniform(-pi, pi, (B, 3*n*layers)).
    Returns dict(circuit, terms (structure, coeff -1), coeffs [B][T], theta, J, g).
    """
    rng = np.random.default_rng(seed)
    J = rng.uniform(0.5, 1.5, size=(batch, n - 1))
    g = rng.uniform(0.2, 2.0, size=batch)
    P = 3 * n * layers
    theta = rng.uniform(-math.pi, math.pi, size=(batch, P))
    terms = tfim_terms(n, 1.0, 1.0)
    coeffs = np.concatenate([-J, -np.repeat(g[:, None], n, axis=1)], axis=1)
    return dict(n=n, circuit=hea_ring(n, layers), terms=terms, coeffs=coeffs,
                theta=theta, J=J, g=g)


def ragged_sizes(batch: int, choices=(12, 14, 16, 18, 20), seed: int = 0) -> np.ndarray:
    """n_b drawn uniformly from ``choices`` (rng.integers index draw)."""
    rng = np.random.default_rng(seed)
    return np.asarray(choices)[rng.integers(0, len(choices), batch)]


def ragged_vqe_batch(batch: int, layers: int = 12, choices=(12, 14, 16, 18, 20),
                     seed_sizes: int = 0, seed_values: int = 1):
    """Ragged batched-VQE input: item b is a TFIM chain of n_b qubits on the ring
    ansatz with ``layers`` layers.

    n_b = ``ragged_sizes(batch, choices, seed_sizes)``.  One structure per distinct n
    (ascending n): dict(n, gates, pool, P, terms) with the open-chain TFIM terms.
    Then with ``default_rng(seed_values)``: per item in order theta_b =
    uniform(-pi, pi, P_b); then per item coefficients (-J_1..-J_{n-1}, -g x n) with
    J_i, g drawn together as uniform(0.5, 1.5, 2n-1) (one value per term).
    Returns (problems, item_problem, theta flat, coeffs flat, sizes).
    """
    ns = ragged_sizes(batch, choices, seed=seed_sizes)
    problems, index = [], {}
    for n in sorted(set(int(x) for x in ns)):
        c = hea_ring(n, layers)
        g, p = c.to_ir()
        index[n] = len(problems)
        problems.append(dict(n=n, gates=g, pool=p, P=c.n_params, terms=tfim_terms(n, 1.0, 1.0)))
    item_problem = [index[int(x)] for x in ns]
    rng = np.random.default_rng(seed_values)
    theta = np.concatenate([rng.uniform(-math.pi, math.pi, problems[s]["P"]) for s in item_problem])
    coeffs = np.concatenate([-rng.uniform(0.5, 1.5, 2 * problems[s]["n"] - 1) for s in item_problem])
    return problems, item_problem, theta, coeffs, ns


def haar_su4_stack(rng: np.random.Generator, shape) -> np.ndarray:
    """Haar SU(4) matrices of ``shape`` in C order, by the ``haar_su4`` recipe in
    one vectorised draw: standard_normal(shape + (2, 4, 4)) gives the same A, B
    per matrix as consecutive ``haar_su4`` calls."""
    g = rng.standard_normal(tuple(shape) + (2, 4, 4))
    z = (g[..., 0, :, :] + 1j * g[..., 1, :, :]) / math.sqrt(2.0)
    q, r = np.linalg.qr(z)
    d = np.diagonal(r, axis1=-2, axis2=-1)
    q = q * (d / np.abs(d))[..., None, :]
    det = np.linalg.det(q)
    return q / np.power(det, 0.25)[..., None, None]


def mipt_batch(n: int, depth: int, batch: int, p: float, seed: int = 0):
    """Measurement-induced phase transition trajectories (Sec. VII.C).

    Time step t of trajectory b: an independent Haar SU(4) on every even bond
    (0,1), (2,3), ..., then on every odd bond (1,2), (3,4), ...; then each qubit
    is measured in the Z basis with probability p.  Draw order:
    Haar matrices for all (b, t, gate) (``haar_su4_stack``), then
    meas = rng.random((batch, depth, n)) < p, then u = rng.random((batch, depth, n))
    (the Born-rule uniform of each (b, t, q)).
    Returns dict(circuit: the gates of one time step with mat_off 16 g,
    pools complex128 [depth][batch][16 G] (gate g of step t of item b at
    pools[t, b, 16 g:16 g + 16], row-major 4x4), masks uint64 [depth][batch],
    u float64 [depth][batch][n]).
    """
    rng = np.random.default_rng(seed)
    bonds = list(range(0, n - 1, 2)) + list(range(1, n - 1, 2))
    G = len(bonds)
    mats = haar_su4_stack(rng, (batch, depth, G))
    meas = rng.random((batch, depth, n)) < p
    u = rng.random((batch, depth, n))
    c = Circuit(n)
    for i in bonds:
        c.unitary((i, i + 1), np.eye(4, dtype=np.complex128))
    pools = np.ascontiguousarray(mats.transpose(1, 0, 2, 3, 4).reshape(depth, batch, 16 * G))
    masks = (meas.astype(np.uint64) << np.arange(n, dtype=np.uint64)).sum(axis=2, dtype=np.uint64)
    return dict(n=n, depth=depth, batch=batch, p=p, circuit=c, pools=pools,
                masks=np.ascontiguousarray(masks.T), u=np.ascontiguousarray(u.transpose(1, 0, 2)))


def shadow_bases(snapshots: int, n: int, seed: int = 0):
    """Random Pauli measurement bases and Born uniforms of classical-shadow
    snapshots (Sec. VII.A): bases = rng.integers(1, 4, (snapshots, n)) with
    1 = X, 2 = Y, 3 = Z (the paper's pauli_strings), then
    u = rng.random((snapshots, n))."""
    rng = np.random.default_rng(seed)
    bases = rng.integers(1, 4, size=(snapshots, n))
    u = rng.random((snapshots, n))
    return bases, u


def warmstart_chains(count: int, n_min: int = 14, n_max: int = 20, seed: int = 0):
    """TFIM/XXZ chains for the learned warm start.

    Per chain, in order: kind = rng.integers(0, 2) (0 TFIM, 1 XXZ);
    n = rng.integers(n_min, n_max + 1); J = rng.uniform(0.5, 1.5, n-1);
    delta = rng.uniform(0, 1.5) (kept for TFIM, unused there);
    g = rng.uniform(0.2, 2.0).
    """
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        kind = int(rng.integers(0, 2))
        n = int(rng.integers(n_min, n_max + 1))
        J = rng.uniform(0.5, 1.5, n - 1)
        delta = float(rng.uniform(0.0, 1.5))
        g = float(rng.uniform(0.2, 2.0))
        out.append(dict(kind=kind, n=n, J=J, delta=delta, g=g))
    return out


def chain_terms(chain) -> np.ndarray:
    """Observable of one warm-start chain."""
    if chain["kind"] == 0:
        return tfim_terms(chain["n"], chain["J"], chain["g"])
    return xxz_terms(chain["n"], chain["J"], chain["delta"], chain["g"])


def random_thetas(shape, seed: int = 0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.uniform(-math.pi, math.pi, size=shape)


def amplitude_encoded_batch(batch: int, n: int, seed: int = 0) -> np.ndarray:
    """Normalised non-negative real vectors of length 2^n (pixel-like amplitude
    encoding of Sec. VII.B); draw rng.random((B, 2^n)). complex128."""
    rng = np.random.default_rng(seed)
    x = rng.random((batch, 1 << n))
    x /= np.linalg.norm(x, axis=1, keepdims=True)
    return x.astype(np.complex128)


def random_state(n: int, seed: int = 0) -> np.ndarray:
    """Normalised complex Gaussian state (test input)."""
    rng = np.random.default_rng(seed)
    a, b = rng.standard_normal((2, 1 << n))
    v = a + 1j * b
    return v / np.linalg.norm(v)
