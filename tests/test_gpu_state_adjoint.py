"""State-pass adjoint (tcng_energy_grad for large states and for RP parameters):
the su4 parameterisation (15 Pauli rotations per gate) of the paper's SU(4)-ladder
VQE (Sec. VI.B), checked against the oracle's exact parameter-shift gradient and
finite differences; the same path forced onto circuits the per-item kernel also
handles gives the same energies and gradients."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import sv  # noqa: E402
from workloads import generators as gen  # noqa: E402

TOL = {"c64": 1e-5, "c128": 1e-12}


@pytest.fixture(scope="module")
def T():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2602_14167_b300 import build
    build.build()
    from paper_2602_14167_b300 import tcng
    return tcng


@pytest.fixture(autouse=True)
def options(T):
    saved = {o: T.tcng_get_option(o) for o in range(9)}
    yield
    for o, v in saved.items():
        T.tcng_set_option(o, v)
    torch.cuda.synchronize()
    torch.cuda.empty_cache()


def energy_grad(T, n, gates, pool, theta, terms, coeffs=None, dtype="c128"):
    from paper_2602_14167_b300 import StateBatch
    theta = np.atleast_2d(theta)
    B, P = theta.shape
    st = StateBatch(n, batch=B, dtype=dtype)
    prm = torch.tensor(theta, dtype=torch.float64, device="cuda")
    cf = None if coeffs is None else torch.tensor(np.atleast_2d(coeffs), dtype=torch.float64, device="cuda")
    e = torch.empty(B, dtype=torch.float64, device="cuda")
    g = torch.empty((B, P), dtype=torch.float64, device="cuda")
    T.tcng_energy_grad(st.handle, gates, pool, prm, P, terms, cf, e, g)
    T.tcng_sync_status()
    return e.cpu().numpy(), g.cpu().numpy(), st


def check(e, g, e_ref, g_ref, csum, dtype):
    assert abs(e - e_ref) / csum < TOL[dtype], (e, e_ref)
    den = max(np.linalg.norm(g_ref), 1e-3 * csum)
    assert np.linalg.norm(g - g_ref) / den < TOL[dtype], np.linalg.norm(g - g_ref) / den


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("n,L", [(4, 2), (7, 1), (9, 2), (14, 2), (16, 1)])
def test_su4_ladder_against_parameter_shift(T, n, L, dtype):
    c = gen.su4_ladder(n, L)
    g, p = c.to_ir()
    th = gen.random_thetas(c.n_params, seed=n)
    terms = gen.tfim_terms(n, 1.0, 1.0)
    e, gr, st = energy_grad(T, n, g, p, th, terms, dtype=dtype)
    e_ref = sv.energy(n, g, p, th, terms)
    g_ref = sv.grad_param_shift(n, g, p, th, terms)
    check(e[0], gr[0], e_ref, g_ref, np.abs(terms["coeff"]).sum(), dtype)
    if dtype == "c128" and n <= 7:
        fd = sv.grad_fd(n, g, p, th, terms, h=1e-5)
        assert np.max(np.abs(gr[0] - fd)) < 1e-8


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_forced_state_path_matches_per_item_kernel(T, dtype):
    """Ring ansatz (RX, RY, RZZ), per-item couplings, a batch of three: the
    state-pass adjoint (forced) against the per-item kernel and the oracle."""
    n, B = 10, 3
    b = gen.tfim_batch(n, B, layers=2, seed=6)
    g, p = b["circuit"].to_ir()
    e1, g1, _ = energy_grad(T, n, g, p, b["theta"], b["terms"], b["coeffs"], dtype)
    T.tcng_set_option(T.OPT_STATE_ADJOINT_N, 1)
    e2, g2, _ = energy_grad(T, n, g, p, b["theta"], b["terms"], b["coeffs"], dtype)
    for i in range(B):
        csum = np.abs(b["coeffs"][i]).sum()
        e_ref = sv.energy(n, g, p, b["theta"][i], b["terms"], b["coeffs"][i])
        g_ref = sv.grad_param_shift(n, g, p, b["theta"][i], b["terms"], b["coeffs"][i])
        check(e2[i], g2[i], e_ref, g_ref, csum, dtype)
        check(e2[i], g2[i], e1[i], g1[i], csum, dtype)


@pytest.mark.parametrize("n,seed", [(7, 0), (7, 1), (14, 2)])
def test_state_path_every_gate_kind(T, n, seed):
    """Random circuits of every kind up to 3-qubit explicit matrices, with RP
    parameters (1- and 2-qubit words), CP, RZZ, shared parameters: oracle PS and FD.
    At 14 qubits the fused runs of blocks span several tiles and alternate with the
    3-qubit blocks' own passes."""
    c, th = gen.random_circuit(n, 60, seed=seed,
                               kinds=["X", "Y", "Z", "H", "S", "T", "RX", "RY", "RZ", "CX", "CZ", "CP",
                                      "SWAP", "RZZ", "U1", "U2", "U3", "RP"])
    g, p = c.to_ir()
    assert np.any(g["op"] == 18)
    terms = np.concatenate([gen.xxz_terms(n, 0.9, 0.6, 0.4), gen.random_pauli_strings(n, 6, 3, seed)])
    e, gr, _ = energy_grad(T, n, g, p, th, terms)
    check(e[0], gr[0], sv.energy(n, g, p, th, terms), sv.grad_param_shift(n, g, p, th, terms),
          np.abs(terms["coeff"]).sum(), "c128")
    fd = sv.grad_fd(n, g, p, th, terms, h=1e-5)
    assert np.max(np.abs(gr[0] - fd)) < 1e-8


def factorized_energy_grad(n, block, c, th, terms):
    """Oracle energy and gradient of a circuit whose state is a product of
    independent blocks: <P_t> is the product of block values, and the gradient
    in block k is that of the block-k Pauli sum whose coefficients carry the
    other blocks' values (exact parameter shift on each block)."""
    nb = n // block
    m = np.uint64((1 << block) - 1)
    circ = [gen.block_circuit(c, k * block, block).to_ir() for k in range(nb)]
    vals = np.ones((len(terms), nb))
    subs = []
    for k in range(nb):
        t = terms.copy()
        t["xmask"] = (terms["xmask"] >> np.uint64(k * block)) & m
        t["zmask"] = (terms["zmask"] >> np.uint64(k * block)) & m
        t["coeff"] = 1.0
        subs.append(t)
        vals[:, k] = sv.expect(block, sv.apply(block, *circ[k], th), t).real
    E = float(np.dot(terms["coeff"], np.prod(vals, axis=1)))
    grad = np.zeros(th.size)
    for k in range(nb):
        others = np.prod(np.delete(vals, k, axis=1), axis=1)
        grad += sv.grad_param_shift(block, *circ[k], th, subs[k], terms["coeff"] * others)
    return E, grad


def test_su4_ladder_n32_cut_against_oracle_blocks(T):
    """n = 32, L = 16 SU(4) ladder (7440 parameters) without the gates on bonds
    (7,8), (15,16), (23,24): energy and full gradient of the open TFIM (J = g = 1)
    against the oracle's block-factorised values (complex64 tolerances)."""
    n, L, block = 32, 16, 8
    c = gen.cut_su4_ladder(n, L, block)
    g, p = c.to_ir()
    th = gen.random_thetas(c.n_params, seed=7) * 0.3
    terms = gen.tfim_terms(n, 1.0, 1.0)
    e, gr, st = energy_grad(T, n, g, p, th, terms, dtype="c64")
    st.free()
    del st
    torch.cuda.empty_cache()
    e_ref, g_ref = factorized_energy_grad(n, block, c, th, terms)
    check(e[0], gr[0], e_ref, g_ref, np.abs(terms["coeff"]).sum(), "c64")
    cut = np.array([(i % block) == block - 1 for l in range(L) for i in range(n - 1)])
    cut_params = np.repeat(cut, 15)
    assert np.all(gr[0][cut_params] == 0.0)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_wide_x_term_and_multi_pass_lambda(T, dtype):
    """lambda = H psi with terms in several tile passes plus one X string on 12
    qubits (wider than a tile with the lowest qubits: the whole Pauli sum then
    takes the per-amplitude gather kernel), 14 qubits: energy and gradient against
    the oracle's parameter shift, both sums."""
    n = 14
    c = gen.su4_ladder(n, 1)
    g, p = c.to_ir()
    th = gen.random_thetas(c.n_params, seed=3)
    base = np.concatenate([gen.tfim_terms(n, 1.0, 0.7), gen.random_pauli_strings(n, 8, 3, seed=4)])
    wide = base[:1].copy()
    wide["xmask"] = np.uint64(((1 << 12) - 1) << 2)
    wide["zmask"] = np.uint64(1 << 5)
    wide["coeff"] = 0.3
    plan = T.tcng_describe_state_adjoint(n, g, p, c.n_params, base).splitlines()[0]
    assert "hampasses=-1" not in plan and int(plan.split("hampasses=")[1]) >= 2
    assert "hampasses=-1" in T.tcng_describe_state_adjoint(n, g, p, c.n_params, np.concatenate([base, wide]))
    for terms in (base, np.concatenate([base, wide])):
        e, gr, _ = energy_grad(T, n, g, p, th, terms, dtype=dtype)
        check(e[0], gr[0], sv.energy(n, g, p, th, terms), sv.grad_param_shift(n, g, p, th, terms),
              np.abs(terms["coeff"]).sum(), dtype)


@pytest.mark.parametrize("n,B,state,dtype", [(16, 2, True, "c64"), (16, 12, False, "c64"), (18, 8, True, "c64"),
                                              (12, 1, False, "c64"), (15, 6, True, "c128"), (14, 6, False, "c128")])
def test_small_batches_take_the_state_pass(T, n, B, state, dtype):
    """Below the qubit threshold, batches too small for the per-item kernel take
    the state-pass adjoint (TCNG_OPT_STATE_ADJOINT_SMALL, on by default): the path
    taken (seen in the kernels launched) follows the cost model, and both paths
    give the oracle's energies and gradients."""
    b = gen.tfim_batch(n, B, layers=2, seed=n + B)
    g, p = b["circuit"].to_ir()
    out = {}
    for small in (1, 0):
        T.tcng_set_option(T.OPT_STATE_ADJOINT_SMALL, small)
        T.tcng_profile_read(reset=True)
        T.tcng_profile_enable(True)
        e, gr, st = energy_grad(T, n, g, p, b["theta"], b["terms"], b["coeffs"], dtype)
        T.tcng_profile_enable(False)
        used = "sa_seg_kernel" in T.tcng_profile_read(reset=True)
        assert used == (state and small == 1)
        out[small] = (e, gr)
        st.free()
    for i in range(min(B, 2)):
        csum = np.abs(b["coeffs"][i]).sum()
        e_ref = sv.energy(n, g, p, b["theta"][i], b["terms"], b["coeffs"][i])
        g_ref = sv.grad_param_shift(n, g, p, b["theta"][i], b["terms"], b["coeffs"][i])
        for small in (1, 0):
            check(out[small][0][i], out[small][1][i], e_ref, g_ref, csum, dtype)
