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


def stage_widths(T, n, c):
    g, p = c.to_ir()
    out = []
    for line in T.tcng_describe_plan(n, g, p, c.n_params, False).splitlines()[1:]:
        if "regs=" in line:
            out.append([tok[tok.index("{") + 1:tok.index("}")].count(",") + 1
                        for tok in line.split("regs=")[1].split()])
    return out


def test_fp16_plans_cap_stages_and_use_wide_stages(T):
    """Plans for the FP16 tensor-core passes (the default options) keep at most 22
    stages per pass (every W resident) and take 5-qubit stages where two of them
    replace three 4-qubit ones; with the FP16 split off the plan has only 4-qubit
    stages and the long passes of a deep circuit on one tile stay whole."""
    T.tcng_set_option(T.OPT_TC_FP16, 1)
    long = stage_widths(T, 13, gen.qml_brickwall(12, 30, seed=0))
    assert max(len(s) for s in long) <= 22 and sum(len(s) for s in long) >= 100
    c, _ = gen.su4_brickwork(32, 14, "RZ", seed=0)
    wide = stage_widths(T, 32, c)
    assert sum(1 for s in wide if s and all(w == 5 for w in s)) >= 10
    try:
        T.tcng_set_option(T.OPT_TC_FP16, 0)
        narrow = stage_widths(T, 32, c)
        assert all(w == 4 for s in narrow for w in s)
        assert max(len(s) for s in stage_widths(T, 13, gen.qml_brickwall(12, 30, seed=0))) > 22
    finally:
        T.tcng_set_option(T.OPT_TC_FP16, 1)


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
