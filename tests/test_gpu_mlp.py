"""GPU: warm-start MLP kernels vs the float64 oracle, and what the warm start gains.

MLP parity: relative L2 error <= 1e-2 of outputs and of every gradient against
oracle/mlp.py with BF16 rounding at the kernels' rounding points (the oracle's
own gradients are pinned by finite differences in test_oracle_mlp.py).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import mlp as omlp  # noqa: E402
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


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)


@pytest.mark.parametrize("N", [1, 37, 96])
def test_mlp_forward_backward_parity(T, N):
    from paper_2602_14167_b300.warmstart import MLP
    F, H, O = 24, 512, 720
    net = MLP(F, H, O, seed=3)
    rng = np.random.default_rng(N)
    # non-zero biases so every term of the backward pass is exercised
    for i in (1, 3, 5):
        net.p(i).copy_(torch.tensor(rng.standard_normal(net.p(i).numel()) * 0.1, dtype=torch.float32))
    x = rng.standard_normal((N, F)).astype(np.float32)
    t = rng.uniform(-3, 3, (N, O)).astype(np.float32)
    mask = (rng.random((N, O)) < 0.7).astype(np.float32)
    xd, td, md = (torch.tensor(a, device="cuda") for a in (x, t, mask))
    y = net.forward(xd)
    loss = net.backward(xd, y, td, md)
    torch.cuda.synchronize()
    w = [net.p(i).cpu().numpy().astype(np.float64) for i in range(6)]
    z1, z2, yref = omlp.forward(x.astype(np.float64), w[0].reshape(F, H), w[1], w[2].reshape(H, H), w[3],
                                w[4].reshape(H, O), w[5])
    assert rel(y.cpu().numpy(), yref) < 1e-2
    lref, dy = omlp.loss_and_dy(yref, t.astype(np.float64), mask.astype(np.float64))
    assert abs(float(loss.item()) - lref) <= 1e-2 * abs(lref)
    gref = omlp.backward(x.astype(np.float64), w[0].reshape(F, H), w[2].reshape(H, H), w[4].reshape(H, O),
                         z1, z2, dy)
    flat = net.grads.cpu().numpy()
    off = 0
    for g in gref:
        got = flat[off:off + g.size].reshape(g.shape)
        off += g.size
        assert rel(got, g) < 1e-2


def test_ragged_vqe_energies_match_oracle(T):
    from paper_2602_14167_b300.warmstart import RaggedVQE, ring_ansatz
    chains = gen.warmstart_chains(5, n_min=5, n_max=8, seed=4)
    rv = RaggedVQE(chains, gen.chain_terms, layers=2)
    rng = np.random.default_rng(0)
    th = [rng.uniform(-np.pi, np.pi, 3 * c["n"] * 2) for c in chains]
    e, _ = rv.energy_and_grad(rv.pack(th))
    e = e.cpu().numpy()
    for i, c in enumerate(chains):
        g = ring_ansatz(c["n"], 2)
        ref = sv.energy(c["n"], g, None, th[i], gen.chain_terms(c))
        assert abs(e[i] - ref) < 1e-5 * np.abs(gen.chain_terms(c)["coeff"]).sum()


def test_warm_start_beats_random_initialisation(T):
    """Train on converged angles of 192 chains, evaluate on 16 held-out chains."""
    from paper_2602_14167_b300.warmstart import MLP, RaggedVQE, features, predict_init, targets_for
    n_max, layers, steps = 8, 2, 150
    train = gen.warmstart_chains(192, n_min=6, n_max=n_max, seed=11)
    held = gen.warmstart_chains(16, n_min=6, n_max=n_max, seed=12)
    rv = RaggedVQE(train, gen.chain_terms, layers=layers)
    common = np.random.default_rng(5).uniform(-0.3, 0.3, 3 * n_max * layers)
    th0 = [common[:3 * c["n"] * layers] for c in train]
    th_star, _ = rv.optimize(rv.pack(th0), steps=steps, lr=0.05)
    tgt, mask = targets_for(train, rv.unpack(th_star), layers, n_max)
    x = torch.tensor(np.stack([features(c, n_max) for c in train]), device="cuda")
    net = MLP(x.shape[1], 128, 3 * layers * n_max, seed=0)
    hist = net.train(x, torch.tensor(tgt, device="cuda"), torch.tensor(mask, device="cuda"),
                     steps=400, lr=2e-3)
    assert hist[-1] < 0.5 * hist[0]
    # held-out: warm start vs 4 random starts, energy after k Adam steps
    rh = RaggedVQE(held, gen.chain_terms, layers=layers)
    warm = predict_init(net, held, layers, n_max)
    _, hw = rh.optimize(rh.pack(warm), steps=20, lr=0.05)
    rng = np.random.default_rng(7)
    rand_e = []
    for r in range(4):
        th = [rng.uniform(-np.pi, np.pi, 3 * c["n"] * layers) for c in held]
        _, hr = rh.optimize(rh.pack(th), steps=20, lr=0.05)
        rand_e.append(hr[-1].cpu().numpy())
    warm_e = hw[-1].cpu().numpy()
    rand_e = np.mean(rand_e, axis=0)
    # lower (better) energy after 20 steps on most held-out chains
    assert np.mean(warm_e < rand_e) >= 0.75, (warm_e, rand_e)
