"""Host-side logic without a GPU: planner invariants, IR validation, multi-rank timing."""
import os
import re
import socket

import numpy as np
import pytest

from workloads import Circuit
from workloads import generators as gen


@pytest.fixture(scope="module")
def T():
    from paper_2602_14167_b300 import build
    build.build()
    from paper_2602_14167_b300 import tcng
    return tcng


def plan_summary(T, n, c, P=None, adjoint=False):
    g, p = c.to_ir()
    s = T.tcng_describe_plan(n, g, p, c.n_params if P is None else P, adjoint)
    assert not s.startswith("error"), s
    head = dict(re.findall(r"(\w+)=(\d+)", s.splitlines()[0]))
    passes = [dict(m=int(a), chunk=int(b), gather=[int(x) for x in cgt.split(",") if x])
              for a, b, cgt in re.findall(r"m=(\d+) chunk=(\d+) gather=\[([\d,]*)\]", s)]
    return {k: int(v) for k, v in head.items()}, passes


def test_brickwork_plan_structure(T):
    c, _ = gen.su4_brickwork(32, 14, "RZ", seed=0)
    head, passes = plan_summary(T, 32, c)
    assert head["ops"] == len(c) and head["blocks"] == 217   # one 2-qubit block per SU(4) (+RZ absorbed)
    assert head["passes"] == len(passes) >= 14
    for p in passes:
        assert p["m"] == 13 and p["chunk"] + len(p["gather"]) == 13
        assert p["gather"] == sorted(p["gather"]) and all(q >= p["chunk"] for q in p["gather"])


def test_small_state_is_one_pass(T):
    c, _ = gen.random_circuit(9, 80, seed=1)
    head, passes = plan_summary(T, 9, c)
    assert all(p["m"] == 9 and not p["gather"] for p in passes)


def test_adjoint_plan_keeps_parameterised_gates_single(T):
    c = gen.hea_ring(12, 3)
    head, _ = plan_summary(T, 12, c, adjoint=True)
    assert head["grads"] == c.n_params == head["blocks"]


def test_fusion_width_reduces_blocks(T):
    c, _ = gen.su4_brickwork(20, 8, "RZ", seed=2)
    counts = []
    for w in (1, 2, 3, 4):
        T.tcng_set_option(T.OPT_FUSE_WIDTH, w)
        counts.append(plan_summary(T, 20, c)[0]["blocks"])
    T.tcng_set_option(T.OPT_FUSE_WIDTH, 2)
    assert counts[0] > counts[1] >= counts[2] >= counts[3]


@pytest.mark.parametrize("bad", [
    lambda: Circuit(4).cx(1, 1),          # repeated qubit
    lambda: Circuit(5).x(4),              # qubit outside a 4-qubit register
    lambda: Circuit(4).add("H", (0,), param=0),   # a parameter on a fixed gate
])
def test_ir_validation(T, bad):
    c = bad()
    g, p = c.to_ir()
    s = T.tcng_describe_plan(4, g, p, max(c.n_params, 1))
    assert s.startswith("error")


def test_options_are_validated(T):
    with pytest.raises(T.TcngError):
        T.tcng_set_option(T.OPT_FUSE_WIDTH, 9)
    with pytest.raises(T.TcngError):
        T.tcng_set_option(T.OPT_TILE_BITS, 20)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t = bench.max_over_ranks(10.0 + 5.0 * rank, dist)
    q.put((rank, t))
    dist.barrier()
    dist.destroy_process_group()


def test_bench_timing_is_max_over_ranks_gloo():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
    assert out == {0: 15.0, 1: 15.0}
