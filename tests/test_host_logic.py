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


# ---- shared-memory layouts of the lock-step FP16 passes (host planner) ----
def _insert_zeros(row, positions):
    g = row
    for b in sorted(positions):
        low = (1 << b) - 1
        g = (g & low) | ((g & ~low) << 1)
    return g


def _swizzle(o):   # 128-byte swizzle on 8-byte elements: 16-byte chunk ^= 128-byte row & 7
    return o ^ ((o >> 3) & 0xE)


def _move_tile(stages, lay):
    """Move a tile (values = tile indices) through the stages' read/write layouts as
    the lock-step kernel does: row r of stage s reads positions with zeros inserted
    at the read positions plus register offsets, writes the same values at the write
    positions.  Returns the final memory and asserts each row is one register group."""
    mem = list(range(8192))
    for s, regs in enumerate(stages):
        rp, wp = [int(x) for x in lay[s][:4]], [int(x) for x in lay[s][4:]]
        new = [-1] * 8192
        for row in range(512):
            gr, gw = _insert_zeros(row, rp), _insert_zeros(row, wp)
            t0 = None
            for v in range(16):
                a, b, lin = gr, gw, 0
                for i in range(4):
                    if (v >> i) & 1:
                        a |= 1 << rp[i]
                        b |= 1 << wp[i]
                        lin |= 1 << regs[i]
                t = mem[a]
                t0 = t if v == 0 else t0
                assert t ^ t0 == lin and new[b] == -1
                new[b] = t
        mem = new
    return mem


def _wavefronts(positions):
    """Shared-memory wavefronts of one stage phase (read or write) over a tile: 16
    warps x 32 lanes (lane = row bits 0..4), 8-byte accesses served per half warp,
    16-byte pair accesses (tile position 0 a register bit) per quarter warp."""
    pos = [int(x) for x in positions]
    pairs = 0 in pos
    total = 0
    for w in range(16):
        for v in range(0, 16, 2 if pairs else 1):
            words = []
            for lane in range(32):
                g = _insert_zeros((w // 4) * 128 + (w % 4) * 32 + lane, pos)
                for i in range(4):
                    if (v >> i) & 1:
                        g |= 1 << pos[i]
                ws = []
                for k in range(2 if pairs else 1):
                    o = _swizzle(g | k)
                    ws += [2 * o, 2 * o + 1]
                words.append(ws)
            phase = 8 if pairs else 16
            for p0 in range(0, 32, phase):
                ph = [x for ws in words[p0:p0 + phase] for x in ws]
                banks = {}
                for x in ph:
                    banks.setdefault(x % 32, set()).add(x)
                total += max(max(len(b) for b in banks.values()), len(set(ph)) // 32)
    return total


def test_lock_layouts_move_the_tile_consistently_and_spread_banks(T):
    """The planned layouts of a 13-qubit brickwork pass (stages on {2,3,4,5} and
    {1,2,5,6} conflict on the tile map's layout): every row is one register group,
    the last stage writes the tile map's layout, and each stage's reads and writes
    take the minimum wavefronts (512 per tile) where the tile map's layout takes more."""
    stages = [(0, 1, 2, 3), (4, 5, 6, 7), (8, 9, 10, 11), (3, 4, 7, 8), (2, 3, 4, 5), (6, 7, 8, 9),
              (1, 2, 5, 6), (0, 1, 2, 3), (4, 5, 6, 7), (2, 3, 4, 5), (0, 1, 2, 3)]
    lay, relocated = T.tcng_plan_lock_layouts(stages)
    assert relocated
    assert [tuple(lay[0][:4])] == [stages[0]] and tuple(lay[-1][4:]) == stages[-1]
    assert _move_tile(stages, lay) == list(range(8192))
    before = sum(2 * _wavefronts(s) for s in stages)
    after = sum(_wavefronts(l[:4]) + _wavefronts(l[4:]) for l in lay)
    assert after == 2 * len(stages) * 512 < before


def test_lock_layouts_random_passes_and_rejects(T):
    rng = np.random.default_rng(7)
    for _ in range(6):
        nst = int(rng.integers(2, 12))
        stages = [tuple(sorted(rng.choice(13, 4, replace=False).tolist())) for _ in range(nst)]
        lay, relocated = T.tcng_plan_lock_layouts(stages)
        assert _move_tile(stages, lay) == list(range(8192))
        if not relocated:
            assert all(tuple(l[:4]) == s and tuple(l[4:]) == s for l, s in zip(lay, stages))
    for bad in ([(0, 1, 2, 13)], [(3, 2, 1, 0)], []):
        with pytest.raises(T.TcngError):
            T.tcng_plan_lock_layouts(bad if bad else np.zeros((0, 4)))


# ---- state-pass adjoint plan (host planner: fused segments, H passes) ----
def _state_plan(T, n, c, terms, dtype=0):
    g, p = c.to_ir()
    s = T.tcng_describe_state_adjoint(n, g, p, max(c.n_params, 1), terms, dtype)
    assert not s.startswith("error"), s
    lines = s.splitlines()
    head = {k: int(v) for k, v in re.findall(r"(\w+)=(-?\d+)", lines[0])}
    steps, ham = [], []
    for ln in lines[1:]:
        kind, tm, rest = re.match(r"(\w+) tmask=([0-9a-f]+) (?:blocks|terms)=(.*)", ln).groups()
        if kind == "ham":
            ham.append((int(tm, 16), [int(t) for t in rest.split(",") if t]))
        else:
            blk = [tuple(int(x, 16) if i else int(x) for i, x in enumerate(b.split(":"))) for b in rest.split(",")]
            steps.append((kind, int(tm, 16), blk))
    return head, steps, ham


def _popc(x):
    return bin(x).count("1")


@pytest.mark.parametrize("dtype,tbits,cmask", [(0, 12, 0b11), (1, 11, 0b1)])
def test_state_adjoint_segments_of_the_su4_ladder(T, dtype, tbits, cmask):
    """32-qubit, 16-layer SU(4) ladder: every block once, last first; each segment's
    tile holds its blocks' qubits and the lowest qubits in exactly tbits qubits, at
    most 16 blocks; a segment ends only where the next block does not fit."""
    n = 32
    c = gen.su4_ladder(n, 16)
    head, steps, ham = _state_plan(T, n, c, gen.tfim_terms(n, 1.0, 1.0), dtype)
    assert head["blocks"] == 496 and head["lone"] == 0 and head["tbits"] == tbits
    order = [b for _, _, blk in steps for b, _ in blk]
    assert order == list(range(495, -1, -1))
    for i, (kind, tm, blk) in enumerate(steps):
        assert kind == "seg" and _popc(tm) == tbits and tm & cmask == cmask and len(blk) <= 16
        used = 0
        for _, qm in blk:
            assert _popc(qm) == 2 and qm & tm == qm
            used |= qm
        if i + 1 < len(steps) and len(blk) < 16:
            assert _popc(cmask | used | steps[i + 1][2][0][1]) > tbits
    if dtype == 0:
        assert head["segments"] == 54


def test_state_adjoint_plan_keeps_wide_blocks_alone(T):
    """A circuit with explicit 3-qubit gates: the 3-qubit blocks are lone steps, the
    segments around them keep the block order."""
    n = 14
    c, _ = gen.random_circuit(n, 80, seed=4, kinds=["RX", "RY", "RZ", "CX", "RZZ", "U2", "U3", "RP"])
    head, steps, _ = _state_plan(T, n, c, gen.tfim_terms(n, 1.0, 1.0))
    order = [b for _, _, blk in steps for b, _ in blk]
    assert order == list(range(head["blocks"] - 1, -1, -1))
    lone = [blk for kind, _, blk in steps if kind == "lone"]
    assert head["lone"] == len(lone) >= 1
    assert all(len(b) == 1 and _popc(b[0][1]) >= 3 for b in lone)
    assert all(_popc(qm) <= 2 for kind, _, blk in steps if kind == "seg" for _, qm in blk)


@pytest.mark.parametrize("n,seed", [(32, 0), (20, 1)])
def test_hamiltonian_passes_cover_every_term_once(T, n, seed):
    """lambda = H psi passes: every term in exactly one pass, its X mask inside the
    pass's tile (12 qubits with qubits 0 and 1), the diagonal terms in the first."""
    terms = np.concatenate([gen.tfim_terms(n, 1.0, 1.0), gen.random_pauli_strings(n, 40, 4, seed)])
    head, _, ham = _state_plan(T, n, gen.su4_ladder(n, 1), terms)
    assert head["hampasses"] == len(ham) >= 2
    seen = sorted(t for _, ts in ham for t in ts)
    assert seen == list(range(len(terms)))
    for i, (tm, ts) in enumerate(ham):
        assert _popc(tm) == 12 and tm & 3 == 3 and len(ts) <= 64
        for t in ts:
            xm = int(terms["xmask"][t])
            assert xm & tm == xm
            if xm == 0 and i > 0:
                assert all(int(terms["xmask"][u]) == 0 for u in ts)   # overflow bins hold diagonals only
    wide = terms[:1].copy()
    wide["xmask"] = (1 << 11) - 1 << 5
    wide["zmask"] = 0
    assert _state_plan(T, n, gen.su4_ladder(n, 1), wide)[0]["hampasses"] == -1
