"""Pins for the oracle: closed forms, invariants, an independent dense route.

Every check here ties ``oracle/`` to something other than itself: textbook
states (Bell, GHZ, QFT of basis states), norm and echo invariants, the dense
Kronecker/expm construction of ``oracle/dense.py``, exact diagonalisation,
the free-fermion closed form of the open TFIM, and finite differences.
"""
import math

import numpy as np
import pytest

from oracle import dense, sv
from oracle.adam import adam_step
from workloads import Circuit, PAULI_DTYPE, pauli_terms
from workloads import generators as gen

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


def ir(c):
    return c.to_ir()


# ---------------------------------------------------------------- conventions
def test_little_endian_qubit_order():
    for q in range(5):
        c = Circuit(5).x(q)
        g, p = ir(c)
        psi = sv.apply(5, g, p, None)
        assert psi[1 << q] == 1 and np.count_nonzero(psi) == 1


def test_gate_matrices_match_generator_route():
    """Closed-form entries of every gate == expm/projector construction."""
    rng = np.random.default_rng(5)
    names1 = ["I", "X", "Y", "Z", "H", "S", "T", "RX", "RY", "RZ"]
    names2 = ["CX", "CZ", "CP", "SWAP", "RZZ"]
    for name in names1 + names2:
        for _ in range(3):
            th = rng.uniform(-4, 4)
            c = Circuit(2)
            qs = (0,) if name in names1 else (1, 0)
            if name in ("RX", "RY", "RZ", "CP", "RZZ"):
                c.add(name, qs, param=0, scale=0.7, angle0=0.1)
            else:
                c.add(name, qs)
            g, p = ir(c)
            params = np.array([th])
            M = sv.gate_matrix(g[0], p, params)
            n = len(qs)
            g1 = g.copy()
            if n == 2:
                g1["q"][0][:2] = (1, 0)
            D = dense.gate_operator(n, g1[0], p, params)
            np.testing.assert_allclose(M, D, atol=1e-14)


# ------------------------------------------------------------- textbook states
def test_bell_and_ghz():
    c = Circuit(2).h(0).cx(0, 1)
    psi = sv.apply(2, *ir(c), None)
    np.testing.assert_allclose(psi, [2 ** -0.5, 0, 0, 2 ** -0.5], atol=1e-15)
    n = 7
    c = Circuit(n).h(0)
    for q in range(n - 1):
        c.cx(q, q + 1)
    psi = sv.apply(n, *ir(c), None)
    ref = np.zeros(1 << n, complex)
    ref[0] = ref[-1] = 2 ** -0.5
    np.testing.assert_allclose(psi, ref, atol=1e-14)


def qft_circuit(n):
    c = Circuit(n)
    for a in range(n - 1, -1, -1):
        c.h(a)
        for b in range(a - 1, -1, -1):
            c.cp(b, a, angle=math.pi / (1 << (a - b)))
    for i in range(n // 2):
        c.swap(i, n - 1 - i)
    return c


@pytest.mark.parametrize("n", [3, 5, 6])
def test_qft_of_basis_states(n):
    """QFT|j> = N^-1/2 sum_k e^{2 pi i j k / N} |k>: uniform magnitudes, known phases."""
    N = 1 << n
    g, p = ir(qft_circuit(n))
    for j in [0, 1, 3, N - 1, N // 2 + 1]:
        psi0 = np.zeros(N, complex)
        psi0[j] = 1
        psi = sv.apply(n, g, p, None, psi=psi0)
        k = np.arange(N)
        ref = np.exp(2j * math.pi * j * k / N) / math.sqrt(N)
        np.testing.assert_allclose(psi, ref, atol=1e-13)


# ----------------------------------------------------------------- invariants
inverse_circuit = gen.inverse_circuit


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_norm_and_echo(seed):
    n = 8
    c, th = gen.random_circuit(n, 150, seed=seed)
    psi0 = gen.random_state(n, seed + 10)
    psi = sv.apply(n, *ir(c), th, psi=psi0)
    assert abs(np.linalg.norm(psi) - 1) < 1e-13
    back = sv.apply(n, *ir(inverse_circuit(c)), th, psi=psi)
    np.testing.assert_allclose(back, psi0, atol=1e-12)


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_against_dense_kron_route(seed):
    n = 6
    c, th = gen.random_circuit(n, 60, seed=seed)
    g, p = ir(c)
    psi = sv.apply(n, g, p, th)
    ref = dense.run(n, g, p, th)
    np.testing.assert_allclose(psi, ref, atol=1e-12)


# ------------------------------------------------------------------ config 1
def test_ry_cx_ladder_is_real_and_theta0_values():
    c, th = gen.ry_cx_ladder(10, 4, seed=0)
    g, p = ir(c)
    psi = sv.apply(10, g, p, th)
    assert np.all(psi.imag == 0.0)
    psi0 = sv.apply(10, g, p, np.zeros_like(th))
    terms = gen.tfim_terms(10, 1.0, 1.0)
    zz = pauli_terms([{0: "Z", 1: "Z"}])
    assert abs(sv.expect(10, psi0, zz)[0] - 1) < 1e-14
    assert abs(sv.energy(10, g, p, np.zeros_like(th), terms) + 9) < 1e-13


def test_product_state_closed_form_energy_and_gradient():
    """No CX: <Z_i> = cos t_i, <X_i> = sin t_i with t_i = sum_l theta[l, i]."""
    n, L, gfield = 6, 3, 0.8
    rng = np.random.default_rng(3)
    th = rng.uniform(-math.pi, math.pi, (L, n))
    c = Circuit(n)
    for l in range(L):
        for q in range(n):
            c.ry(q, param=l * n + q)
    g, p = ir(c)
    terms = gen.tfim_terms(n, 1.0, gfield)
    t = th.sum(0)
    E = -np.sum(np.cos(t[:-1]) * np.cos(t[1:])) - gfield * np.sum(np.sin(t))
    assert abs(sv.energy(n, g, p, th.ravel(), terms) - E) < 1e-13
    dE = np.zeros(n)
    for i in range(n):
        if i > 0:
            dE[i] += np.sin(t[i]) * np.cos(t[i - 1])
        if i < n - 1:
            dE[i] += np.sin(t[i]) * np.cos(t[i + 1])
        dE[i] -= gfield * np.cos(t[i])
    ps = sv.grad_param_shift(n, g, p, th.ravel(), terms)
    np.testing.assert_allclose(ps, np.tile(dE, L), atol=1e-12)


# ------------------------------------------------------------------ observables
def test_pauli_y_phase_and_z_basis_signs():
    c = Circuit(1).h(0).s(0)            # (|0> + i|1>)/sqrt2
    psi = sv.apply(1, *ir(c), None)
    assert abs(sv.expect(1, psi, pauli_terms([{0: "Y"}]))[0] - 1) < 1e-15
    n = 5
    for x in [0, 5, 31, 18]:
        psi = np.zeros(1 << n, complex)
        psi[x] = 1
        z = pauli_terms([{0: "Z", 2: "Z", 4: "Z"}])
        sign = (-1) ** bin(x & 0b10101).count("1")
        assert sv.expect(n, psi, z)[0] == sign


@pytest.mark.parametrize("seed", [0, 1])
def test_expectations_and_h_apply_against_dense(seed):
    n = 6
    psi = gen.random_state(n, seed)
    strings = gen.random_pauli_strings(n, 20, weight=3, seed=seed)
    vals = sv.expect(n, psi, strings)
    for s, v in zip(strings, vals):
        P = dense.pauli_operator(n, s["xmask"], s["zmask"])
        assert abs(np.vdot(psi, P @ psi) - v) < 1e-13
        assert abs(v.imag) < 1e-13
    terms = gen.xxz_terms(n, np.linspace(0.5, 1.5, n - 1), 0.7, 0.4)
    Hd = dense.hamiltonian_matrix(n, terms)
    np.testing.assert_allclose(sv.hamiltonian_apply(n, psi, terms), Hd @ psi, atol=1e-13)


# ------------------------------------------------------------- exact energies
def test_free_fermion_special_cases():
    assert abs(dense.tfim_ground_energy_free_fermion([], [0.7]) + 0.7) < 1e-15
    J = np.array([0.6, 1.2, 0.9])
    g = np.array([0.3, 0.5, 1.1, 0.2])
    assert abs(dense.tfim_ground_energy_free_fermion(np.zeros(3), g) + g.sum()) < 1e-14
    assert abs(dense.tfim_ground_energy_free_fermion(J, np.zeros(4)) + J.sum()) < 1e-14


def test_critical_open_chain_closed_form():
    """J = g = 1 open chain: E0(N) = 1 - csc(pi / (4N + 2))."""
    for N in [1, 2, 3, 10, 40, 400]:
        ref = 1 - 1 / math.sin(math.pi / (4 * N + 2))
        assert abs(dense.tfim_ground_energy_free_fermion(np.ones(N - 1), np.ones(N)) - ref) < 1e-9 * N


@pytest.mark.parametrize("n", [2, 3, 5, 8, 10])
def test_ed_equals_free_fermion(n):
    rng = np.random.default_rng(n)
    J = rng.uniform(0.5, 1.5, n - 1)
    g = rng.uniform(0.2, 2.0)
    terms = gen.tfim_terms(n, J, g)
    e_ed = dense.ground_energy_ed(n, terms)
    e_ff = dense.tfim_ground_energy_free_fermion(J, np.full(n, g))
    assert abs(e_ed - e_ff) < 1e-10


def test_variational_energy_above_ground():
    n = 8
    b = gen.tfim_batch(n, 4, layers=2, seed=1)
    g, p = ir(b["circuit"])
    for i in range(4):
        e = sv.energy(n, g, p, b["theta"][i], b["terms"], b["coeffs"][i])
        e0 = dense.tfim_ground_energy_free_fermion(b["J"][i], np.full(n, b["g"][i]))
        assert e >= e0 - 1e-12


def test_energy_equals_dense_quadratic_form():
    n = 7
    c, th = gen.ry_cx_ladder(n, 3, seed=4)
    g, p = ir(c)
    terms = gen.tfim_terms(n, 1.0, 1.0)
    psi = dense.run(n, g, p, th)
    Hd = dense.hamiltonian_matrix(n, terms)
    assert abs(sv.energy(n, g, p, th, terms) - np.vdot(psi, Hd @ psi).real) < 1e-12


# ------------------------------------------------------------------ gradients
@pytest.mark.parametrize("seed", [0, 1])
def test_param_shift_equals_finite_difference(seed):
    n = 5
    c, th = gen.random_circuit(n, 40, seed=seed)
    g, p = ir(c)
    terms = gen.xxz_terms(n, 1.0, 0.5, 0.3)
    ps = sv.grad_param_shift(n, g, p, th, terms)
    fd = sv.grad_fd(n, g, p, th, terms, h=1e-5)
    np.testing.assert_allclose(ps, fd, atol=2e-9)


def test_shared_parameter_gradient_sums_over_gates():
    n = 3
    c = Circuit(n)
    c.rx(0, param=0).ry(1, param=0, scale=-2.0).rzz(0, 1, param=0, scale=0.5).cx(1, 2)
    g, p = ir(c)
    terms = gen.tfim_terms(n, 1.0, 0.7)
    th = np.array([0.37])
    ps = sv.grad_param_shift(n, g, p, th, terms)
    fd = sv.grad_fd(n, g, p, th, terms, h=1e-5)
    assert abs(ps[0] - fd[0]) < 1e-9


# ---------------------------------------------------------------- optimiser
def test_adam_first_step_closed_form():
    th0 = np.array([0.3, -1.0, 2.0])
    grad = np.array([0.5, -2e-3, 0.0])
    th1, m, v = adam_step(th0, np.zeros(3), np.zeros(3), grad, 1, lr=0.02, eps=1e-8)
    np.testing.assert_allclose(th1, th0 - 0.02 * grad / (np.abs(grad) + 1e-8), rtol=1e-14)


def test_adam_quadratic_converges():
    th = np.array([3.0, -2.0])
    m = v = np.zeros(2)
    for t in range(1, 2001):
        th, m, v = adam_step(th, m, v, 2 * th, t, lr=0.05)
    assert np.all(np.abs(th) < 1e-2)


# ------------------------------------------------------------------- inputs
def test_haar_su4_is_special_unitary():
    rng = np.random.default_rng(0)
    for _ in range(20):
        u = gen.haar_su4(rng)
        assert np.linalg.norm(u.conj().T @ u - np.eye(4)) < 1e-14
        assert abs(np.linalg.det(u) - 1) < 1e-13


def test_rejects_bad_gates():
    c = Circuit(3).cx(0, 0)
    with pytest.raises(ValueError):
        sv.apply(3, *ir(c), None)
    c = Circuit(3).x(3)
    with pytest.raises(ValueError):
        sv.apply(3, *ir(c), None)
    with pytest.raises(ValueError):
        sv.expect(3, sv.zero_state(3), np.array([(8, 0, 1.0)], dtype=PAULI_DTYPE))


# ------------------------------------------------- Born probabilities, measurement
def test_marginal_probs_bit_order_and_basis_states():
    psi = np.zeros(8, complex)
    psi[1] = 1.0                      # qubit 0 set
    np.testing.assert_array_equal(sv.marginal_probs(3, psi, [0, 1]), [0, 0, 1, 0])   # q[0] most significant
    np.testing.assert_array_equal(sv.marginal_probs(3, psi, [1, 0]), [0, 1, 0, 0])
    np.testing.assert_array_equal(sv.marginal_probs(3, psi, [2]), [1, 0])


def test_marginal_probs_product_state_closed_form():
    """RY(t_q) on every qubit: P(bits) = prod_q (cos^2(t_q/2) or sin^2(t_q/2))."""
    n = 7
    th = np.linspace(-2.5, 2.9, n)
    c = Circuit(n)
    for q in range(n):
        c.ry(q, param=q)
    psi = sv.apply(n, *ir(c), th)
    qs = [5, 0, 3]
    p = sv.marginal_probs(n, psi, qs)
    for j in range(8):
        ref = 1.0
        for i, q in enumerate(qs):
            bit = (j >> (len(qs) - 1 - i)) & 1
            ref *= math.sin(th[q] / 2) ** 2 if bit else math.cos(th[q] / 2) ** 2
        assert abs(p[j] - ref) < 1e-14
    assert abs(p.sum() - 1) < 1e-14


def test_marginal_probs_ghz():
    n = 6
    c = Circuit(n).h(0)
    for q in range(n - 1):
        c.cx(q, q + 1)
    psi = sv.apply(n, *ir(c), None)
    p = sv.marginal_probs(n, psi, [1, 3, 4])
    np.testing.assert_allclose(p, [0.5, 0, 0, 0, 0, 0, 0, 0.5], atol=1e-15)


def test_measure_bell_state_collapses():
    c = Circuit(2).h(0).cx(0, 1)
    for u, want in ((0.3, 0), (0.7, 1)):
        psi = sv.apply(2, *ir(c), None)
        out, prob, p0 = sv.measure_qubit(2, psi, 0, u)
        assert out == want and abs(prob - 0.5) < 1e-15 and abs(p0 - 0.5) < 1e-15
        ref = np.zeros(4, complex)
        ref[3 * want] = 1.0
        np.testing.assert_allclose(psi, ref, atol=1e-15)
        out1, prob1, _ = sv.measure_qubit(2, psi, 1, 0.999)   # now certain
        assert out1 == want and abs(prob1 - 1) < 1e-15


def test_sequential_measurement_matches_joint_distribution():
    """P(o_a) P(o_b | o_a) from two single-qubit measurements equals the joint
    Born probability of (o_a, o_b); the post-measurement state has unit norm and
    lives on the measured outcome."""
    n = 6
    psi0 = gen.random_state(n, seed=3)
    joint = sv.marginal_probs(n, psi0, [4, 1])
    for oa in (0, 1):
        for ob in (0, 1):
            psi = psi0.copy()
            _, pa, _ = sv.measure_qubit(n, psi, 4, 0.0, forced=oa)
            _, pb, _ = sv.measure_qubit(n, psi, 1, 0.0, forced=ob)
            assert abs(pa * pb - joint[2 * oa + ob]) < 1e-14
            assert abs(np.linalg.norm(psi) - 1) < 1e-14
            m = sv.marginal_probs(n, psi, [4, 1])
            assert abs(m[2 * oa + ob] - 1) < 1e-14


# --------------------------------------------- MIPT trajectories, shadow snapshots
def _pool_of(mats):
    return np.ascontiguousarray(np.concatenate([m.reshape(-1) for m in mats]))


def test_mipt_trajectory_without_measurement_is_the_circuit():
    from oracle import trajectories as tr
    b = gen.mipt_batch(6, 4, 2, 0.0, seed=2)
    g, _ = b["circuit"].to_ir()
    out = tr.mipt_trajectory(6, g, b["pools"][:, 1], b["masks"][:, 1], b["u"][:, 1])
    assert np.all(out["outcomes"] == -1) and out["logp"] == 0.0
    psi = sv.zero_state(6)
    for t in range(4):
        pool = np.empty(2 * b["pools"][t, 1].size)
        pool[0::2], pool[1::2] = b["pools"][t, 1].real, b["pools"][t, 1].imag
        psi = dense.run(6, g, pool, None, psi0=psi)
    np.testing.assert_allclose(out["psi"], psi, atol=1e-12)


def test_mipt_trajectory_closed_form_hadamard_steps():
    """Even bonds H (x) I, odd bonds I: after each step qubits 0 and 2 of four are in
    |+> (or re-measured basis states turned into |+>/|->), qubits 1 and 3 stay |0>;
    measuring all four gives P = 1/2 for qubits 0, 2 (outcome u < 1/2 -> 0) and
    certainty for 1, 3: log P = 2 log(1/2) per step."""
    from oracle import trajectories as tr
    n, D = 4, 3
    Hm = np.array([[1, 1], [1, -1]]) / math.sqrt(2)
    HI = np.kron(Hm, np.eye(2)).astype(np.complex128)
    c = Circuit(n)
    for i in (0, 2, 1):
        c.unitary((i, i + 1), np.eye(4, dtype=np.complex128))
    g, _ = ir(c)
    pools = [_pool_of([HI, HI, np.eye(4, dtype=np.complex128)]) for _ in range(D)]
    u = np.array([[0.2, 0.9, 0.7, 0.1], [0.6, 0.3, 0.4, 0.8], [0.49, 0.5, 0.51, 0.0]])
    out = tr.mipt_trajectory(n, g, pools, [0b1111] * D, u)
    for t in range(D):
        assert out["outcomes"][t, 0] == (0 if u[t, 0] < 0.5 else 1)
        assert out["outcomes"][t, 2] == (0 if u[t, 2] < 0.5 else 1)
        assert out["outcomes"][t, 1] == 0 and out["outcomes"][t, 3] == 0
        np.testing.assert_allclose(out["p0"][t], [0.5, 1.0, 0.5, 1.0], atol=1e-15)
    assert abs(out["logp"] - 2 * D * math.log(0.5)) < 1e-12
    ref = np.zeros(16, complex)
    ref[out["outcomes"][-1, 0] | (out["outcomes"][-1, 2] << 2)] = 1.0
    np.testing.assert_allclose(out["psi"], ref, atol=1e-15)


def test_shadow_basis_change_measures_the_right_basis():
    """X basis on |+>/|->, Y basis on |+i>/|-i>, Z basis on |0>/|1> give certain
    outcomes 0/1."""
    from oracle import trajectories as tr
    n = 6
    prep = Circuit(n)
    prep.h(0).x(1).h(1)                      # |+>, |->
    prep.rx(2, angle=-math.pi / 2)           # |+i>
    prep.x(3).rx(3, angle=-math.pi / 2)      # |-i> (up to phase)
    prep.x(5)                                # qubit 4 |0>, qubit 5 |1>
    psi = sv.apply(n, *ir(prep), None)
    out, p0, _ = tr.shadow_snapshot(n, psi, [1, 1, 2, 2, 3, 3], np.full(n, 0.5))
    np.testing.assert_array_equal(out, [0, 1, 0, 1, 0, 1])
    np.testing.assert_allclose(p0, [1, 0, 1, 0, 1, 0], atol=1e-14)


def test_shadow_outcome_statistics_match_pauli_expectations():
    """For each basis the outcome probabilities are (1 +- <P_q>)/2 with P_q the
    basis Pauli: P(0) - P(1) on qubit q equals <X_q>, <Y_q> or <Z_q>."""
    from oracle import trajectories as tr
    n = 5
    psi0 = gen.random_state(n, seed=8)
    for b, name in ((1, "X"), (2, "Y"), (3, "Z")):
        g, p = tr.basis_change(n, [b] * n)
        phi = sv.apply(n, g, p, None, psi=psi0)
        for q in range(n):
            pz = sv.marginal_probs(n, phi, [q])
            ev = sv.expect(n, psi0, pauli_terms([{q: name}]))[0].real
            assert abs((pz[0] - pz[1]) - ev) < 1e-13


def test_mipt_generator_draws_like_sequential_haar():
    rng = np.random.default_rng(11)
    seq = np.array([[gen.haar_su4(rng) for _ in range(3)] for _ in range(2)])
    stack = gen.haar_su4_stack(np.random.default_rng(11), (2, 3))
    np.testing.assert_array_equal(seq, stack)
    for U in stack.reshape(-1, 4, 4):
        np.testing.assert_allclose(U.conj().T @ U, np.eye(4), atol=1e-14)
        assert abs(np.linalg.det(U) - 1) < 1e-13


# ------------------------------------------------ Pauli-word rotations, su4 ladder
def test_pauli_rotation_special_cases():
    """RP on one qubit equals RX/RY/RZ; RP(ZZ) equals RZZ; RP(XY) equals the
    dense route's expm(-i t X(x)Y / 2)."""
    n = 3
    for word, name in (("X", "RX"), ("Y", "RY"), ("Z", "RZ")):
        a = Circuit(n).rp((1,), word, angle=0.83)
        b = Circuit(n).add(name, (1,), angle0=0.83)
        psi0 = gen.random_state(n, seed=1)
        np.testing.assert_allclose(sv.apply(n, *ir(a), None, psi=psi0), sv.apply(n, *ir(b), None, psi=psi0),
                                   atol=1e-15)
    a = Circuit(n).rp((0, 2), "ZZ", angle=-1.3)
    b = Circuit(n).rzz(0, 2, angle=-1.3)
    psi0 = gen.random_state(n, seed=2)
    np.testing.assert_allclose(sv.apply(n, *ir(a), None, psi=psi0), sv.apply(n, *ir(b), None, psi=psi0), atol=1e-15)
    c = Circuit(n).rp((2, 0), "XY", angle=0.4).rp((1, 2, 0), "YZX", angle=1.7)
    g, p = ir(c)
    np.testing.assert_allclose(sv.apply(n, g, p, None, psi=psi0), dense.run(n, g, p, None, psi0=psi0), atol=1e-14)


def test_su4_gate_is_special_unitary_and_counts():
    """The 15-rotation su4 gate is in SU(4); the ladder has 15 L (n - 1)
    parameters (the paper's 7440 for n = 32, L = 16)."""
    c = gen.su4_ladder(2, 1)
    th = gen.random_thetas(15, seed=3)
    g, p = ir(c)
    U = dense.circuit_unitary(2, g, p, th)
    np.testing.assert_allclose(U.conj().T @ U, np.eye(4), atol=1e-14)
    assert abs(np.linalg.det(U) - 1) < 1e-13
    assert gen.su4_ladder(32, 16).n_params == 7440
    assert len(gen.SU4_WORDS) == 15 and len(set(gen.SU4_WORDS)) == 15


def test_su4_ladder_parameter_shift_equals_finite_differences():
    n = 4
    c = gen.su4_ladder(n, 1)
    g, p = ir(c)
    th = gen.random_thetas(c.n_params, seed=5)
    terms = gen.tfim_terms(n, 1.0, 0.7)
    ps = sv.grad_param_shift(n, g, p, th, terms)
    fd = sv.grad_fd(n, g, p, th, terms, h=1e-5)
    assert np.max(np.abs(ps - fd)) < 1e-8
    assert np.linalg.norm(ps) > 1e-2
