"""Pins for the MLP oracle: bf16 rounding and finite-difference gradients."""
import numpy as np

from oracle import mlp


def test_bf16_rounding_known_values():
    # 1 + 2^-8 is halfway between bf16 neighbours 1 and 1 + 2^-7: ties go to even (1).
    vals = np.array([1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8, -2.5, 1e-3])
    r = mlp.bf16(vals)
    assert r[0] == 1.0 and r[1] == 1.0 and r[2] == 1 + 2 ** -6 and r[3] == -2.5
    assert abs(r[4] - 1e-3) / 1e-3 < 2 ** -8


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(0)
    N, F, H, O = 7, 5, 6, 4
    p = {k: v.astype(np.float64) for k, v in mlp.init(F, H, O, seed=1).items()}
    p["b1"] = rng.standard_normal(H) * 0.1
    p["b2"] = rng.standard_normal(H) * 0.1
    x = rng.standard_normal((N, F))
    t = rng.uniform(-3, 3, (N, O))
    mask = (rng.random((N, O)) < 0.8).astype(np.float64)

    def L(q):
        _, _, y = mlp.forward(x, q["w1"], q["b1"], q["w2"], q["b2"], q["w3"], q["b3"], bf=False)
        return mlp.loss_and_dy(y, t, mask)[0]

    z1, z2, y = mlp.forward(x, p["w1"], p["b1"], p["w2"], p["b2"], p["w3"], p["b3"], bf=False)
    _, dy = mlp.loss_and_dy(y, t, mask)
    grads = mlp.backward(x, p["w1"], p["w2"], p["w3"], z1, z2, dy, bf=False)
    names = ["w1", "b1", "w2", "b2", "w3", "b3"]
    h = 1e-6
    for name, g in zip(names, grads):
        fd = np.zeros_like(p[name])
        it = np.nditer(p[name], flags=["multi_index"])
        for _ in it:
            i = it.multi_index
            q = {k: v.copy() for k, v in p.items()}
            q[name][i] += h
            lp = L(q)
            q[name][i] -= 2 * h
            lm = L(q)
            fd[i] = (lp - lm) / (2 * h)
        np.testing.assert_allclose(g, fd, atol=1e-7)
