"""MIPT trajectories (Sec. VII.C) and classical-shadow snapshots (Sec. VII.A) on
the GPU against the oracle, trajectory by trajectory.

Outcomes are integers decided by floating point (u < p0): the oracle takes each
decision from its own complex128 state, the GPU from its complex64 (or
complex128) state.  Outcomes must agree; a first disagreement is accepted only
where u lies within the precision's tolerance of the oracle's p0 (both outcomes
are then correct), after which that trajectory is not compared further.
Where outcomes agree, the log-probability (|d logp| <= tol per measurement) and
the final state (fidelity >= 1 - tol) are compared."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import sv  # noqa: E402
from oracle import trajectories as tr  # noqa: E402
from workloads import generators as gen  # noqa: E402

TOL = {"c64": 1e-5, "c128": 1e-11}


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


def compare_decisions(got, ref, p0, u, tol):
    """got/ref [steps][n] outcomes (-1 = not measured).  True if identical; False
    if they first differ where |u - p0| <= tol (asserts that otherwise)."""
    assert np.array_equal(got < 0, ref < 0)          # the same qubits were measured
    diff = np.argwhere(got != ref)
    if diff.size == 0:
        return True
    t, q = diff[0]
    assert abs(u[t, q] - p0[t, q]) <= tol, (t, q, u[t, q], p0[t, q])
    return False


def run_mipt(T, n, D, B, p, seed, dtype):
    from paper_2602_14167_b300.trajectories import MIPTBatch
    b = gen.mipt_batch(n, D, B, p, seed=seed)
    g, _ = b["circuit"].to_ir()
    rep = np.empty(2 * b["pools"][0, 0].size)
    rep[0::2], rep[1::2] = b["pools"][0, 0].real, b["pools"][0, 0].imag
    pools = torch.tensor(b["pools"], dtype=torch.complex128, device="cuda")
    masks = torch.tensor(b["masks"].astype(np.int64), device="cuda")
    u = torch.tensor(b["u"], dtype=torch.float64, device="cuda")
    mb = MIPTBatch(n, B, dtype=dtype)
    out, logp = mb.run(g, rep, pools, masks, u)
    torch.cuda.synchronize()
    return b, g, mb, out.cpu().numpy(), logp.cpu().numpy()


def check_trajectories(b, g, mb, out, logp, items, dtype):
    n = b["n"]
    compared = 0
    for i in items:
        ref = tr.mipt_trajectory(n, g, b["pools"][:, i], b["masks"][:, i], b["u"][:, i])
        same = compare_decisions(out[:, i], ref["outcomes"], ref["p0"], b["u"][:, i], TOL[dtype])
        if not same:
            continue
        compared += 1
        n_meas = int((ref["outcomes"] >= 0).sum())
        assert abs(logp[i] - ref["logp"]) <= TOL[dtype] * max(1, n_meas), (i, logp[i], ref["logp"])
        psi = mb.state.amplitudes(i).cpu().numpy().astype(np.complex128)
        fid = abs(np.vdot(ref["psi"], psi)) ** 2 / np.vdot(psi, psi).real
        assert fid >= 1 - TOL[dtype], (i, fid)
        assert abs(np.linalg.norm(psi) - 1) < TOL[dtype] * 10
    return compared


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_mipt_small_batch_every_trajectory(T, dtype):
    n, D, B, p = 10, 8, 48, 0.3
    b, g, mb, out, logp = run_mipt(T, n, D, B, p, seed=4, dtype=dtype)
    assert check_trajectories(b, g, mb, out, logp, range(B), dtype) >= B - 2


def test_mipt_edge_probabilities(T):
    """p = 0: no outcome, log-probability 0, the plain circuit; p = 1: every qubit
    measured every step, every trajectory a basis state at the end."""
    n, D, B = 9, 3, 16
    b, g, mb, out, logp = run_mipt(T, n, D, B, 0.0, seed=5, dtype="c64")
    assert np.all(out == -1) and np.all(logp == 0.0)
    assert check_trajectories(b, g, mb, out, logp, range(4), "c64") == 4
    b, g, mb, out, logp = run_mipt(T, n, D, B, 1.0, seed=6, dtype="c64")
    assert np.all(out >= 0)
    for i in range(B):
        psi = mb.state.amplitudes(i).cpu().numpy()
        x = int(sum(int(out[-1, i, q]) << q for q in range(n)))
        assert abs(abs(psi[x]) - 1) < 1e-5
    assert check_trajectories(b, g, mb, out, logp, range(6), "c64") >= 5


def test_mipt_full_shape_sampled(T):
    """N = 20, D = 40, batch 1000, p = 0.2 (the benchmark's shape): two sampled
    trajectories against the oracle; every trajectory's outcome pattern follows
    its masks and its log-probability is finite and <= 0."""
    n, D, B, p = 20, 40, 1000, 0.2
    b, g, mb, out, logp = run_mipt(T, n, D, B, p, seed=0, dtype="c64")
    meas = ((b["masks"][:, :, None] >> np.arange(n, dtype=np.uint64)[None, None, :]) & np.uint64(1)).astype(bool)
    assert np.array_equal(out >= 0, meas)
    assert np.all(np.isfinite(logp)) and np.all(logp <= 1e-9)
    assert check_trajectories(b, g, mb, out, logp, [0, 777], "c64") >= 1


@pytest.mark.parametrize("n,S,picks", [(12, 64, None), (20, 256, [0, 100, 255])])
def test_shadow_snapshots_against_oracle(T, n, S, picks):
    from paper_2602_14167_b300 import StateBatch
    from paper_2602_14167_b300.trajectories import shadow_snapshots
    c, th = gen.su4_brickwork(n, 6, "RZ", seed=n)
    g, p = c.to_ir()
    st = StateBatch(n, dtype="c64")
    st.apply(g, p, torch.tensor(th.reshape(1, -1), device="cuda"))
    psi = st.amplitudes(0)
    bases, u = gen.shadow_bases(S, n, seed=3)
    out = shadow_snapshots(psi, bases, torch.tensor(u, device="cuda")).cpu().numpy()
    assert out.shape == (S, n) and np.all((out == 0) | (out == 1))
    psi_ref = sv.apply(n, g, p, th)
    agree = 0
    for s in (range(S) if picks is None else picks):
        ref, p0, _ = tr.shadow_snapshot(n, psi_ref, bases[s], u[s])
        if compare_decisions(out[s][None], ref[None], p0[None], u[s][None], TOL["c64"]):
            agree += 1
    assert agree >= (S - 2 if picks is None else len(picks) - 1)


def test_measure_leaves_unselected_items_alone(T):
    from paper_2602_14167_b300 import StateBatch
    n, B = 11, 4
    st = StateBatch(n, batch=B, dtype="c128")
    psis = [gen.random_state(n, seed=30 + i) for i in range(B)]
    for i in range(B):
        st.amplitudes(i).copy_(torch.tensor(psis[i], device="cuda"))
    masks = torch.tensor([0, 0b101, 0, (1 << n) - 1], dtype=torch.int64, device="cuda")
    u = torch.full((B, n), 0.5, dtype=torch.float64, device="cuda")
    out = torch.full((B, n), -1, dtype=torch.int8, device="cuda")
    logp = torch.zeros(B, dtype=torch.float64, device="cuda")
    T.tcng_measure(st.handle, masks, u, out, logp)
    torch.cuda.synchronize()
    o = out.cpu().numpy()
    for i in (0, 2):
        assert np.all(o[i] == -1) and float(logp[i]) == 0.0
        assert np.array_equal(st.amplitudes(i).cpu().numpy(), psis[i])
    for i, m in ((1, 0b101), (3, (1 << n) - 1)):
        psi = psis[i].copy()
        lp = 0.0
        for q in range(n):
            if (m >> q) & 1:
                oc, pr, _ = sv.measure_qubit(n, psi, q, 0.5)
                assert o[i, q] == oc
                lp += np.log(pr)
            else:
                assert o[i, q] == -1
        assert abs(float(logp[i]) - lp) < 1e-11
        assert np.linalg.norm(st.amplitudes(i).cpu().numpy() - psi) < 1e-11
