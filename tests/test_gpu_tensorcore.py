"""GPU: shared-unitary batched apply on tcgen05 tensor cores vs the oracle.

Every item of a complex64 batch gets the same k-qubit unitary; the result must
match the oracle's complex128 UK gate within 1e-5 relative L2 error per item.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import sv  # noqa: E402
from workloads import Circuit  # noqa: E402
from workloads import generators as gen  # noqa: E402


@pytest.fixture(scope="module")
def T():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2602_14167_b300 import build
    build.build()
    from paper_2602_14167_b300 import tcng
    return tcng


@pytest.mark.parametrize("n,B,qubits", [
    (6, 3, (0,)), (8, 5, (3, 1)), (8, 7, (0, 1, 2)), (9, 4, (7, 2, 5, 0)),
    (10, 6, (4, 0, 9, 2, 6)), (12, 33, (1, 0, 3, 2, 4)), (7, 1, (6, 5))])
def test_matches_oracle(T, n, B, qubits):
    from paper_2602_14167_b300 import StateBatch
    k = len(qubits)
    rng = np.random.default_rng(n * 10 + k)
    U = gen.haar_unitary(rng, 1 << k)
    psi0 = [gen.random_state(n, seed=100 * n + b) for b in range(B)]
    st = StateBatch(n, batch=B, dtype="c64")
    for b in range(B):
        st.amplitudes(b).copy_(torch.tensor(psi0[b], dtype=torch.complex64, device="cuda"))
    T.tcng_apply_shared_unitary(st.handle, list(qubits), U)
    T.tcng_sync_status()
    c = Circuit(n).unitary(qubits, U)
    g, p = c.to_ir()
    for b in range(B):
        ref = sv.apply(n, g, p, None, psi=psi0[b].astype(np.complex64).astype(np.complex128))
        got = st.amplitudes(b).cpu().numpy()
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-5


def test_qml_brickwork_layer_stack(T):
    """A 10-qubit SU(4) brickwork (QML shape) applied layer by layer to a batch of
    amplitude-encoded inputs, two bonds fused per 4-qubit unitary, vs the oracle."""
    from paper_2602_14167_b300 import StateBatch
    n, B, depth = 10, 64, 4
    x = gen.amplitude_encoded_batch(B, n, seed=0)
    rng = np.random.default_rng(1)
    st = StateBatch(n, batch=B, dtype="c64")
    for b in range(B):
        st.amplitudes(b).copy_(torch.tensor(x[b], dtype=torch.complex64, device="cuda"))
    c = Circuit(n)
    for t in range(depth):
        for (a, bb) in gen.brickwork_bonds(n, t):
            u = gen.haar_su4(rng)
            T.tcng_apply_shared_unitary(st.handle, [a, bb], u)
            c.unitary((a, bb), u)
    T.tcng_sync_status()
    g, p = c.to_ir()
    for b in [0, 17, B - 1]:
        ref = sv.apply(n, g, p, None, psi=x[b].astype(np.complex64).astype(np.complex128))
        got = st.amplitudes(b).cpu().numpy()
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-5


def test_rejects_complex128(T):
    from paper_2602_14167_b300 import StateBatch
    st = StateBatch(6, dtype="c128")
    with pytest.raises(T.TcngError):
        T.tcng_apply_shared_unitary(st.handle, [0, 1], np.eye(4))
