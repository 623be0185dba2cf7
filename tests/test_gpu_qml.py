"""QML-shaped batches (Sec. VII.B): one brickwall of Haar SU(4) gates applied to
a batch of amplitude-encoded inputs by one tcng_apply_circuit call (several
small items per tensor-core tile), and the readout probabilities of the first
qubits (tcng_marginal_probs), each checked against the oracle item by item.
Shapes: 12 qubits x 30 layers x 5000 inputs and 10 qubits x 40 layers x 15000."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import sv  # noqa: E402
from workloads import generators as gen  # noqa: E402


@pytest.fixture(scope="module")
def T():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2602_14167_b300 import build
    build.build()
    from paper_2602_14167_b300 import tcng
    return tcng


@pytest.fixture(autouse=True)
def release_memory():
    yield
    torch.cuda.synchronize()
    torch.cuda.empty_cache()


@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("n,qubits", [(6, [0, 1, 2]), (12, [0, 1, 2, 3, 4, 5, 6]), (12, [11]),
                                      (16, [15, 3, 9, 0]), (16, list(range(6, 16))), (20, [19, 0])])
def test_marginal_probs_against_oracle(T, n, qubits, dtype):
    from paper_2602_14167_b300 import StateBatch
    B = 3
    st = StateBatch(n, batch=B, dtype=dtype)
    psis = [gen.random_state(n, seed=10 * n + i) for i in range(B)]
    for i in range(B):
        st.amplitudes(i).copy_(torch.tensor(psis[i], dtype=st.cdtype, device="cuda"))
    p = st.probs(qubits).cpu().numpy()
    for i in range(B):
        ref = sv.marginal_probs(n, st.amplitudes(i).cpu().numpy().astype(np.complex128), qubits)
        assert np.max(np.abs(p[i] - ref)) < (1e-6 if dtype == "c64" else 1e-13)
    p2 = st.probs(qubits).cpu().numpy()
    assert np.array_equal(p, p2)        # fixed summation order


def test_marginal_probs_rejects_bad_qubits(T):
    from paper_2602_14167_b300 import StateBatch
    st = StateBatch(8, dtype="c64")
    for bad in ([8], [1, 1], list(range(11))):
        with pytest.raises(T.TcngError):
            st.probs(bad)


def qml_run(T, n, layers, B, seed=0, dtype="c64"):
    from paper_2602_14167_b300 import StateBatch
    c = gen.qml_brickwall(n, layers, seed=seed)
    g, p = c.to_ir()
    x = gen.amplitude_encoded_batch(B, n, seed=seed + 1)
    st = StateBatch(n, batch=B, dtype=dtype)
    st.batch_view().copy_(torch.tensor(x, dtype=st.cdtype, device="cuda"))
    T.tcng_profile_enable(True)
    T.tcng_profile_read(reset=True)
    try:
        st.apply(g, p)
        probs = st.probs(list(range(7)))
        torch.cuda.synchronize()
        prof = T.tcng_profile_read(reset=True)
    finally:
        T.tcng_profile_enable(False)
    return st, g, p, x, probs.cpu().numpy(), prof


@pytest.mark.parametrize("n,layers,B", [(12, 30, 5000), (10, 40, 15000), (12, 30, 5001), (9, 6, 37)])
def test_qml_batch_against_oracle(T, n, layers, B):
    st, g, p, x, probs, prof = qml_run(T, n, layers, B)
    if (B << n) >= (1 << 13) * 148:
        tc = sum(prof.get(k, (0, 0.0))[0] for k in ("pass_tcs_kernel_c64", "pass_tch_kernel_c64"))
        assert tc >= 1      # packed tiles on the tensor cores
    rng = np.random.default_rng(3)
    picks = sorted({0, B - 1, B // 2} | set(int(i) for i in rng.integers(0, B, 4)))
    for i in picks:
        ref = sv.apply(n, g, p, None, psi=x[i])
        got = st.amplitudes(i).cpu().numpy()
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert err < 1e-5, (i, err)
        pref = sv.marginal_probs(n, ref, list(range(7)))
        assert np.max(np.abs(probs[i] - pref)) < 1e-6, i
    assert np.allclose(probs.sum(axis=1), 1.0, atol=1e-5)


def test_qml_packed_complex128(T):
    """complex128: 2^12-amplitude tiles hold 4 items of 10 qubits."""
    n, layers, B = 10, 8, 64
    st, g, p, x, probs, _ = qml_run(T, n, layers, B, dtype="c128")
    for i in (0, 17, 63):
        ref = sv.apply(n, g, p, None, psi=x[i])
        got = st.amplitudes(i).cpu().numpy()
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-12
        assert np.max(np.abs(probs[i] - sv.marginal_probs(n, ref, list(range(7))))) < 1e-13
