"""GPU: device Adam, the autograd Function, and a short batched VQE run."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import dense, sv  # noqa: E402
from oracle.adam import adam_step  # noqa: E402
from workloads import generators as gen  # noqa: E402


@pytest.fixture(scope="module")
def T():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2602_14167_b300 import build
    build.build()
    from paper_2602_14167_b300 import tcng
    return tcng


def test_device_adam_matches_oracle(T):
    rng = np.random.default_rng(0)
    n = 1000
    th = rng.standard_normal(n)
    m = np.zeros(n)
    v = np.zeros(n)
    d = {k: torch.tensor(a, device="cuda") for k, a in dict(th=th, m=m, v=v).items()}
    step = torch.zeros(1, dtype=torch.int32, device="cuda")
    for t in range(1, 6):
        g = rng.standard_normal(n)
        gd = torch.tensor(g, device="cuda")
        T.tcng_adam_step(d["th"], d["m"], d["v"], gd, n, 0.02, 0.9, 0.999, 1e-8, step)
        th, m, v = adam_step(th, m, v, g, t, lr=0.02)
    torch.cuda.synchronize()
    assert int(step.item()) == 5
    np.testing.assert_allclose(d["th"].cpu().numpy(), th, rtol=0, atol=1e-14)
    # float32 variant
    th32 = torch.tensor(rng.standard_normal(n), dtype=torch.float32, device="cuda")
    ref = th32.double().cpu().numpy()
    m32, v32 = torch.zeros_like(th32), torch.zeros_like(th32)
    s32 = torch.zeros(1, dtype=torch.int32, device="cuda")
    g = rng.standard_normal(n).astype(np.float32)
    T.tcng_adam_step_f32(th32, m32, v32, torch.tensor(g, device="cuda"), n, 0.01, 0.9, 0.999, 1e-8, s32)
    r, _, _ = adam_step(ref, np.zeros(n), np.zeros(n), g.astype(np.float64), 1, lr=0.01)
    np.testing.assert_allclose(th32.cpu().numpy(), r, atol=1e-6)


def test_autograd_function_backward(T):
    from paper_2602_14167_b300.vqe import VQEBatch, energy
    n, B = 8, 3
    b = gen.tfim_batch(n, B, layers=2, seed=2)
    g, p = b["circuit"].to_ir()
    vb = VQEBatch(n, g, p, b["terms"], B, coeffs=b["coeffs"], dtype="c128")
    th = torch.tensor(b["theta"], device="cuda", requires_grad=True)
    w = torch.tensor([1.0, -2.0, 0.5], dtype=torch.float64, device="cuda")
    loss = (energy(th, vb) * w).sum()
    loss.backward()
    for i in range(B):
        gref = sv.grad_param_shift(n, g, p, b["theta"][i], b["terms"], b["coeffs"][i])
        np.testing.assert_allclose(th.grad[i].cpu().numpy(), w[i].item() * gref, atol=1e-11)


@pytest.mark.parametrize("use_graph", [False, True])
def test_batched_vqe_descends_and_respects_ground_bound(T, use_graph):
    from paper_2602_14167_b300.vqe import VQEBatch
    n, B = 10, 16
    b = gen.tfim_batch(n, B, layers=3, seed=5)
    g, p = b["circuit"].to_ir()
    vb = VQEBatch(n, g, p, b["terms"], B, coeffs=b["coeffs"], dtype="c64")
    theta, hist = vb.optimize(b["theta"], steps=60, lr=0.05, use_graph=use_graph, record_every=10)
    torch.cuda.synchronize()
    e0 = hist[0].cpu().numpy()
    e1 = hist[-1].cpu().numpy()
    assert np.all(e1 < e0 - 1e-3)
    for i in range(B):
        ef = dense.tfim_ground_energy_free_fermion(b["J"][i], np.full(n, b["g"][i]))
        assert e1[i] >= ef - 1e-5
        # the final theta's energy is what the oracle says
        e_or = sv.energy(n, g, p, theta[i].cpu().numpy(), b["terms"], b["coeffs"][i])
        vb.energy_and_grad(theta)
        assert abs(vb.energy[i].item() - e_or) < 1e-5 * np.abs(b["coeffs"][i]).sum()


def test_graph_and_eager_runs_agree(T):
    from paper_2602_14167_b300.vqe import VQEBatch
    n, B = 9, 4
    b = gen.tfim_batch(n, B, layers=2, seed=8)
    g, p = b["circuit"].to_ir()
    vb = VQEBatch(n, g, p, b["terms"], B, coeffs=b["coeffs"], dtype="c128")
    t1, _ = vb.optimize(b["theta"], steps=20, lr=0.03, use_graph=False)
    t2, _ = vb.optimize(b["theta"], steps=20, lr=0.03, use_graph=True)
    torch.cuda.synchronize()
    assert torch.equal(t1, t2)


def test_autotune_sets_options_and_caches(T, tmp_path):
    """The synthetic-brickwork search: every candidate (k = 1..5, tensor cores
    off/on, two tile and two chunk sizes) is timed, the fastest becomes the
    option set and the cache line; a second call loads the line."""
    cache = str(tmp_path / "tune.txt")
    saved = {o: T.tcng_get_option(o) for o in range(6)}
    try:
        T.tcng_autotune(18, T.C64, 1, cache)
        rep = T.tcng_autotune_report()
        assert len(rep) == 5 * 2 * 2 * 2
        assert {r[0] for r in rep} == {1, 2, 3, 4, 5} and {r[3] for r in rep} == {0, 1}
        timed = [r for r in rep if r[4] >= 0]
        best = min(timed, key=lambda r: r[4])
        opts = tuple(T.tcng_get_option(o) for o in (T.OPT_FUSE_WIDTH, T.OPT_TILE_BITS, T.OPT_CHUNK_BITS,
                                                     T.OPT_TENSOR_CORES))
        assert opts == best[:4]
        line = open(cache).read().split()
        assert [int(v) for v in line[:7]] == [18, 0, 1, *best[:4]]
        for o, v in saved.items():
            T.tcng_set_option(o, v)
        T.tcng_autotune(18, T.C64, 1, cache)
        assert T.tcng_autotune_report()[0][0] == "cached"
        assert tuple(T.tcng_get_option(o) for o in (T.OPT_FUSE_WIDTH, T.OPT_TILE_BITS, T.OPT_CHUNK_BITS,
                                                     T.OPT_TENSOR_CORES)) == best[:4]
        assert len(open(cache).read().splitlines()) == 1
    finally:
        for o, v in saved.items():
            T.tcng_set_option(o, v)


def test_autotune_circuit_choice_is_fastest_and_correct(T, tmp_path):
    """Tuning on the caller's circuit: the chosen candidate is the fastest timed,
    and the circuit run with it still matches the oracle."""
    from oracle import sv
    from paper_2602_14167_b300 import StateBatch
    cache = str(tmp_path / "tune2.txt")
    saved = {o: T.tcng_get_option(o) for o in range(6)}
    n = 17
    c, th = gen.su4_brickwork(n, 6, "RZ", seed=4)
    g, p = c.to_ir()
    try:
        st = StateBatch(n, dtype="c64")
        prm = torch.tensor(th.reshape(1, -1), dtype=torch.float64, device="cuda")
        best_ms = T.tcng_autotune_circuit(st.handle, g, p, prm, prm.shape[1], cache)
        rep = T.tcng_autotune_report()
        timed = [r for r in rep if r[4] >= 0]
        best = min(timed, key=lambda r: r[4])
        assert abs(best[4] - best_ms) <= 1e-9 * max(1.0, best_ms)
        assert tuple(T.tcng_get_option(o) for o in (T.OPT_FUSE_WIDTH, T.OPT_TILE_BITS, T.OPT_CHUNK_BITS,
                                                     T.OPT_TENSOR_CORES)) == best[:4]
        st.reset()
        st.apply(g, p, prm)
        psi = st.amplitudes(0).cpu().numpy()
        ref = sv.apply(n, g, p, th)
        assert np.linalg.norm(psi - ref) / np.linalg.norm(ref) < 1e-5
        assert T.tcng_autotune_circuit(st.handle, g, p, prm, prm.shape[1], cache) is None   # cached
    finally:
        for o, v in saved.items():
            T.tcng_set_option(o, v)
