"""Learned warm start, end to end (no counterpart in the paper).

Protocol (run on one GPU, all steps on the library's kernels):
  1. training chains (TFIM / XXZ, n in [n_min, n_max], couplings as in
     ``workloads.generators.warmstart_chains``) are optimised from one common
     initial vector by the batched adjoint simulator + device Adam;
  2. the BF16 MLP maps chain features to those converged angles;
  3. on held-out chains, one run starts from the network's prediction and 16
     runs from uniform random angles; the threshold of a chain is the best
     final energy of its 16 random runs + 1e-3, and each run reports the first
     Adam step whose energy is at or below the threshold (steps + 1 if never).

Usage: python -m paper_2602_14167_b300.warmstart_experiment [--train 1024 ...]
Prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np
import torch

from . import tcng as T  # noqa: F401  (loads the library: fails loudly without it)
from .warmstart import MLP, RaggedVQE, features, predict_init, targets_for


def run(train=1024, held=32, restarts=16, n_min=14, n_max=20, layers=12, steps=200, lr=0.05,
        mlp_width=512, mlp_steps=2000, mlp_lr=1e-3, chunk=1024, seed=0):
    from workloads import generators as gen

    t0 = time.perf_counter()
    tr = gen.warmstart_chains(train, n_min=n_min, n_max=n_max, seed=seed + 11)
    ho = gen.warmstart_chains(held, n_min=n_min, n_max=n_max, seed=seed + 12)
    common = np.random.default_rng(seed + 5).uniform(-0.3, 0.3, 3 * n_max * layers)

    # 1. targets: converged angles from the common start, in chunks of `chunk` chains
    thetas = []
    for c0 in range(0, train, chunk):
        part = tr[c0:c0 + chunk]
        rv = RaggedVQE(part, gen.chain_terms, layers=layers)
        th0 = [common[:3 * c["n"] * layers] for c in part]
        th, _ = rv.optimize(rv.pack(th0), steps=steps, lr=lr)
        thetas += rv.unpack(th)
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t0

    # 2. the network
    t1 = time.perf_counter()
    tgt, mask = targets_for(tr, thetas, layers, n_max)
    x = torch.tensor(np.stack([features(c, n_max) for c in tr]), device="cuda")
    net = MLP(x.shape[1], mlp_width, 3 * layers * n_max, seed=seed)
    loss = net.train(x, torch.tensor(tgt, device="cuda"), torch.tensor(mask, device="cuda"),
                     steps=mlp_steps, lr=mlp_lr)
    torch.cuda.synchronize()
    t_mlp = time.perf_counter() - t1

    # 3. held-out: 1 warm + `restarts` random runs per chain, one ragged batch
    t2 = time.perf_counter()
    warm = predict_init(net, ho, layers, n_max)
    rng = np.random.default_rng(seed + 7)
    items, th0 = [], []
    for i, c in enumerate(ho):
        items.append(c)
        th0.append(warm[i])
        for _ in range(restarts):
            items.append(c)
            th0.append(rng.uniform(-np.pi, np.pi, 3 * c["n"] * layers))
    rh = RaggedVQE(items, gen.chain_terms, layers=layers)
    _, hist = rh.optimize(rh.pack(th0), steps=steps, lr=lr)
    h = hist.cpu().numpy().reshape(steps + 1, held, restarts + 1)
    torch.cuda.synchronize()
    t_eval = time.perf_counter() - t2

    best_rand = h[-1, :, 1:].min(axis=1)

    def reach_steps(tol):   # first step within tol of the best random final energy
        thr = best_rand + tol
        out = np.full((held, restarts + 1), steps + 1, dtype=np.int64)
        for i in range(held):
            for r in range(restarts + 1):
                idx = np.nonzero(h[:, i, r] <= thr[i])[0]
                if idx.size:
                    out[i, r] = idx[0]
        return out

    reach = reach_steps(1e-3)
    warm_steps = reach[:, 0]
    rand_steps = reach[:, 1:]
    looser = {}
    for tol in (1e-1, 1e-2):
        r = reach_steps(tol)
        looser[f"{tol:g}"] = {"warm_median": float(np.median(r[:, 0])),
                              "random_median": float(np.median(r[:, 1:])),
                              "warm_reached": float(np.mean(r[:, 0] <= steps)),
                              "random_reached": float(np.mean(r[:, 1:] <= steps))}
    thr = best_rand + 1e-3
    return {
        "protocol": {"train_chains": train, "held_out": held, "restarts": restarts, "n": [n_min, n_max],
                     "layers": layers, "adam_steps": steps, "adam_lr": lr, "mlp_width": mlp_width,
                     "mlp_steps": mlp_steps},
        "steps_to_threshold": {
            "warm_median": float(np.median(warm_steps)),
            "random_median": float(np.median(rand_steps)),
            "warm_mean": float(warm_steps.mean()),
            "random_mean": float(rand_steps.mean()),
            "warm_reached": float(np.mean(warm_steps <= steps)),
            "random_reached": float(np.mean(rand_steps <= steps)),
        },
        "looser_thresholds": looser,
        "energy_after_20_steps": {
            "warm_mean": float(h[min(20, steps), :, 0].mean()),
            "random_mean": float(h[min(20, steps), :, 1:].mean()),
        },
        "warm_initial_gap_to_threshold_mean": float((h[0, :, 0] - thr).mean()),
        "mlp_loss_first_last": [float(loss[0]), float(loss[-1])],
        "seconds": {"data": t_data, "mlp": t_mlp, "held_out": t_eval},
        "adjoint_evals": int(train * (steps + 1) + held * (restarts + 1) * (steps + 1)),
    }


def main():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--train", type=int, default=1024)
    ap.add_argument("--held", type=int, default=32)
    ap.add_argument("--restarts", type=int, default=16)
    ap.add_argument("--n-min", type=int, default=14)
    ap.add_argument("--n-max", type=int, default=20)
    ap.add_argument("--layers", type=int, default=12)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--lr", type=float, default=0.05)
    ap.add_argument("--mlp-steps", type=int, default=2000)
    ap.add_argument("--seed", type=int, default=0)
    a = ap.parse_args()
    out = run(train=a.train, held=a.held, restarts=a.restarts, n_min=a.n_min, n_max=a.n_max,
              layers=a.layers, steps=a.steps, lr=a.lr, mlp_steps=a.mlp_steps, seed=a.seed)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
