"""CUDA graph per circuit structure (TCNG_OPT_USE_GRAPHS): replayed calls give the
same bits as eager calls through the C ABI, for new parameter values too, and
the launches of a replay are counted."""
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
def graphs_option(T):
    saved = T.tcng_get_option(T.OPT_USE_GRAPHS)
    yield
    T.tcng_set_option(T.OPT_USE_GRAPHS, saved)


def apply_runs(T, use_graphs, n, g, p, thetas, dtype):
    """Apply the circuit to fresh |0..0> for each parameter set; returns states."""
    from paper_2602_14167_b300 import StateBatch
    T.tcng_set_option(T.OPT_USE_GRAPHS, use_graphs)
    st = StateBatch(n, dtype=dtype)
    prm = torch.empty((1, thetas.shape[1]), dtype=torch.float64, device="cuda")
    out = []
    for th in thetas:
        prm.copy_(torch.tensor(th).reshape(1, -1))
        T.tcng_state_reset(st.handle)
        T.tcng_apply_circuit(st.handle, g, p, prm, prm.shape[1])
        out.append(st.amplitudes(0).clone())
    torch.cuda.synchronize()
    return out


@pytest.mark.parametrize("n,dtype", [(10, "c128"), (16, "c64"), (20, "c64")])
def test_apply_replay_matches_eager_bitwise(T, n, dtype):
    c, th0 = gen.su4_brickwork(n, 6, "RZ", seed=n)
    g, p = c.to_ir()
    thetas = np.stack([th0, th0 + 0.3, th0 - 1.1, th0 * 0.5])
    eager = apply_runs(T, 0, n, g, p, thetas, dtype)
    l0 = T.tcng_launch_count()
    graph = apply_runs(T, 1, n, g, p, thetas, dtype)
    assert T.tcng_launch_count() > l0
    for a, b in zip(eager, graph):
        assert torch.equal(a, b)
    ref = sv.apply(n, g, p, thetas[3])
    got = graph[3].cpu().numpy()
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < (1e-12 if dtype == "c128" else 1e-5)


def energy_grad_runs(T, use_graphs, n, B, layers):
    from paper_2602_14167_b300 import StateBatch
    T.tcng_set_option(T.OPT_USE_GRAPHS, use_graphs)
    b = gen.tfim_batch(n, B, layers=layers, seed=7)
    g, p = b["circuit"].to_ir()
    st = StateBatch(n, batch=B, dtype="c64")
    P = b["theta"].shape[1]
    prm = torch.empty((B, P), dtype=torch.float64, device="cuda")
    cf = torch.tensor(b["coeffs"], dtype=torch.float64, device="cuda")
    e = torch.empty(B, dtype=torch.float64, device="cuda")
    gr = torch.empty((B, P), dtype=torch.float64, device="cuda")
    res = []
    for k in range(4):
        prm.copy_(torch.tensor(b["theta"] + 0.25 * k))
        T.tcng_energy_grad(st.handle, g, p, prm, P, b["terms"], cf, e, gr)
        res.append((e.clone(), gr.clone()))
    T.tcng_sync_status()
    return res, b


def test_energy_grad_replay_matches_eager_bitwise(T):
    eager, b = energy_grad_runs(T, 0, 12, 8, 3)
    graph, _ = energy_grad_runs(T, 1, 12, 8, 3)
    for (e0, g0), (e1, g1) in zip(eager, graph):
        assert torch.equal(e0, e1) and torch.equal(g0, g1)
    g, p = b["circuit"].to_ir()
    th = b["theta"][2] + 0.75
    e_ref = sv.energy(12, g, p, th, b["terms"], b["coeffs"][2])
    assert abs(float(graph[3][0][2]) - e_ref) / np.abs(b["coeffs"][2]).sum() < 1e-5


def test_ragged_replay_matches_eager_bitwise(T):
    probs, item_problem, theta, coeffs, _ = gen.ragged_vqe_batch(40, layers=2, choices=(6, 9, 12))
    outs = []
    for use in (0, 1):
        T.tcng_set_option(T.OPT_USE_GRAPHS, use)
        prm = torch.tensor(theta, dtype=torch.float64, device="cuda")
        cf = torch.tensor(coeffs, dtype=torch.float64, device="cuda")
        e = torch.empty(40, dtype=torch.float64, device="cuda")
        gr = torch.empty_like(prm)
        res = []
        for k in range(3):
            prm.copy_(torch.tensor(theta + 0.1 * k))
            T.tcng_energy_grad_ragged(probs, item_problem, prm, cf, e, gr)
            res.append((e.clone(), gr.clone()))
        T.tcng_sync_status()
        outs.append(res)
    for (e0, g0), (e1, g1) in zip(*outs):
        assert torch.equal(e0, e1) and torch.equal(g0, g1)


def test_replay_inside_caller_capture_runs_eagerly(T):
    """A call on a stream the caller is capturing is recorded into the caller's
    graph (no nested recording); replaying the caller's graph gives the eager bits."""
    from paper_2602_14167_b300 import StateBatch
    n = 14
    c, th = gen.su4_brickwork(n, 4, "RZ", seed=2)
    g, p = c.to_ir()
    T.tcng_set_option(T.OPT_USE_GRAPHS, 1)
    st = StateBatch(n, dtype="c64")
    prm = torch.tensor(th.reshape(1, -1), dtype=torch.float64, device="cuda")
    T.tcng_apply_circuit(st.handle, g, p, prm, prm.shape[1])     # warm: plans, scratch
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(graph, stream=s):
            T.tcng_state_reset(st.handle)
            T.tcng_apply_circuit(st.handle, g, p, prm, prm.shape[1])
    graph.replay()
    torch.cuda.synchronize()
    got = st.amplitudes(0).clone()
    T.tcng_set_option(T.OPT_USE_GRAPHS, 0)
    T.tcng_state_reset(st.handle)
    T.tcng_apply_circuit(st.handle, g, p, prm, prm.shape[1])
    torch.cuda.synchronize()
    assert torch.equal(got, st.amplitudes(0))
