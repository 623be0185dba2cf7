"""GPU parity: tcng_apply_circuit / tcng_expect_pauli / tcng_energy vs the oracle.

Tolerances (relative L2 error of amplitudes; absolute for <P> with |<P>| <= 1;
|dE| / sum|c| for energies): complex128 1e-12, complex64 1e-5 and fidelity
>= 1 - 1e-5.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import sv  # noqa: E402
from workloads import generators as gen  # noqa: E402

TOL = {"c64": 1e-5, "c128": 1e-12}


@pytest.fixture(scope="module")
def T():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2602_14167_b300 import build
    build.build()
    from paper_2602_14167_b300 import tcng
    return tcng


@pytest.fixture(autouse=True)
def default_options(T):
    saved = {o: T.tcng_get_option(o) for o in range(8)}
    yield
    for o, v in saved.items():
        T.tcng_set_option(o, v)


def run(n, gates, pool, theta, dtype, batch=1):
    from paper_2602_14167_b300 import StateBatch
    st = StateBatch(n, batch=batch, dtype=dtype)
    prm = None
    if theta is not None and np.size(theta):
        prm = torch.tensor(np.atleast_2d(theta), dtype=torch.float64, device="cuda")
        if prm.shape[0] != batch:
            prm = prm.expand(batch, -1).contiguous()
    st.apply(gates, pool, prm)
    torch.cuda.synchronize()
    return st


def relerr(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def check_state(psi, ref, dtype):
    assert relerr(psi, ref) < TOL[dtype], relerr(psi, ref)
    if dtype == "c64":
        fid = abs(np.vdot(ref, psi)) ** 2 / (np.vdot(psi, psi).real * np.vdot(ref, ref).real)
        assert fid >= 1 - 1e-5


@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("n", [5, 7, 10, 13, 15, 17])
def test_random_circuit_all_ops(T, n, dtype):
    c, th = gen.random_circuit(n, 120, seed=n)
    g, p = c.to_ir()
    st = run(n, g, p, th, dtype)
    check_state(st.amplitudes(0).cpu().numpy(), sv.apply(n, g, p, th), dtype)


@pytest.mark.parametrize("width", [1, 2, 3, 4, 5])
def test_fusion_widths(T, width):
    T.tcng_set_option(T.OPT_FUSE_WIDTH, width)
    n = 14
    c, th = gen.random_circuit(n, 150, seed=100 + width)
    g, p = c.to_ir()
    st = run(n, g, p, th, "c128")
    check_state(st.amplitudes(0).cpu().numpy(), sv.apply(n, g, p, th), "c128")


@pytest.mark.parametrize("tile,chunk", [(6, 2), (8, 3), (9, 1), (13, 7), (12, 12)])
def test_small_tiles_many_passes(T, tile, chunk):
    """Small tiles force many gather passes at a size the oracle does instantly."""
    T.tcng_set_option(T.OPT_TILE_BITS, tile)
    T.tcng_set_option(T.OPT_CHUNK_BITS, chunk)
    n = 12
    c, th = gen.su4_brickwork(n, 6, "RZ", seed=7)
    g, p = c.to_ir()
    for dtype in ("c64", "c128"):
        st = run(n, g, p, th, dtype)
        check_state(st.amplitudes(0).cpu().numpy(), sv.apply(n, g, p, th), dtype)


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_unfused_pair_quartet_kernels(T, dtype):
    T.tcng_set_option(T.OPT_UNFUSED, 1)
    n = 11
    c, th = gen.random_circuit(n, 100, seed=3)
    g, p = c.to_ir()
    st = run(n, g, p, th, dtype)
    check_state(st.amplitudes(0).cpu().numpy(), sv.apply(n, g, p, th), dtype)


def test_batch_with_per_item_params(T):
    n, B = 9, 5
    c = gen.hea_ring(n, 3)
    g, p = c.to_ir()
    th = gen.random_thetas((B, c.n_params), seed=1)
    st = run(n, g, p, th, "c128", batch=B)
    for b in range(B):
        check_state(st.amplitudes(b).cpu().numpy(), sv.apply(n, g, p, th[b]), "c128")


def test_config1_ry_cx_ladder(T):
    """n=10 complex128: full state, <Z0 Z1> and the TFIM energy (g=1)."""
    c, th = gen.ry_cx_ladder(10, 4, seed=0)
    g, p = c.to_ir()
    st = run(10, g, p, th, "c128")
    ref = sv.apply(10, g, p, th)
    check_state(st.amplitudes(0).cpu().numpy(), ref, "c128")
    from workloads import pauli_terms
    zz = pauli_terms([{0: "Z", 1: "Z"}])
    assert abs(float(st.expect(zz)[0, 0]) - sv.expect(10, ref, zz)[0].real) < 1e-12
    terms = gen.tfim_terms(10, 1.0, 1.0)
    e = float(st.energy(terms)[0])
    e_ref = sv.energy(10, g, p, th, terms)
    assert abs(e - e_ref) / np.abs(terms["coeff"]).sum() < 1e-12


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_config2_n24_brickwork(T, dtype):
    """n=24, depth-20 SU(4) brickwork with RX layers; energy and 32 weight-4 strings."""
    n = 24
    c, th = gen.su4_brickwork(n, 20, "RX", seed=0)
    g, p = c.to_ir()
    st = run(n, g, p, th, dtype)
    ref = sv.apply(n, g, p, th)
    check_state(st.amplitudes(0).cpu().numpy(), ref, dtype)
    strings = gen.random_pauli_strings(n, 32, 4, seed=1)
    vals = st.expect(strings)[0].cpu().numpy()
    vref = sv.expect(n, ref, strings).real
    assert np.max(np.abs(vals - vref)) < TOL[dtype]
    terms = gen.tfim_terms(n, 1.0, 1.0)
    e = float(st.energy(terms)[0])
    e_ref = float(np.dot(terms["coeff"], sv.expect(n, ref, terms).real))
    assert abs(e - e_ref) / np.abs(terms["coeff"]).sum() < TOL[dtype]


@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("n", [6, 11, 16])
def test_expectations_random_strings(T, n, dtype):
    psi0 = gen.random_state(n, seed=n)
    from paper_2602_14167_b300 import StateBatch
    st = StateBatch(n, dtype=dtype)
    st.amplitudes(0).copy_(torch.tensor(psi0, dtype=st.cdtype, device="cuda"))
    strings = np.concatenate([gen.random_pauli_strings(n, 40, min(4, n), seed=2),
                              gen.random_pauli_strings(n, 10, 1, seed=3),
                              gen.tfim_terms(n, 0.7, 0.3)])
    vals = st.expect(strings)[0].cpu().numpy()
    ref_psi = st.amplitudes(0).cpu().numpy().astype(np.complex128)
    vref = sv.expect(n, ref_psi, strings).real
    assert np.max(np.abs(vals - vref)) < (1e-6 if dtype == "c64" else 1e-12)


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_expectation_forms(T, dtype):
    """Every specialised form of the complex64 expectation pass (2^13 tiles over
    qubits 0..12): X on register qubits 10..12 (all 8 patterns; the half-pair forms
    for the non-zero ones), with and without X on qubit 0 (swapped pairs), an even
    or odd number of Y factors, the partner on a lane bit (qubit 3), a warp bit
    (qubit 7; the alternating warp-half form), both, or the thread itself, the top
    X bit on qubit 4 or 5 (lane bits 3, 4), alone or with lower X bits; random Z
    factors on the tile and on qubits 13..15 (the tile's global sign)."""
    n = 16
    psi0 = gen.random_state(n, seed=31)
    from paper_2602_14167_b300 import StateBatch
    from workloads import pauli_terms
    rng = np.random.default_rng(5)
    specs = []
    for xr in range(8):
        for sw in (0, 1):
            for part in ((), (3,), (7,), (3, 7), (4,), (5,), (1, 5), (2, 3, 4)):
                for im in (0, 1):
                    xq = [10 + k for k in range(3) if (xr >> k) & 1] + ([0] if sw else []) + list(part)
                    if not xq:
                        continue
                    d = {q: "X" for q in xq}
                    if im:
                        d[xq[0]] = "Y"
                    for q in rng.choice([q for q in range(n) if q not in d], size=3, replace=False):
                        d[int(q)] = "Z"
                    specs.append(d)
    strings = pauli_terms(specs)
    st = StateBatch(n, dtype=dtype)
    st.amplitudes(0).copy_(torch.tensor(psi0, dtype=st.cdtype, device="cuda"))
    vals = st.expect(strings)[0].cpu().numpy()
    ref_psi = st.amplitudes(0).cpu().numpy().astype(np.complex128)
    vref = sv.expect(n, ref_psi, strings).real
    assert np.max(np.abs(vals - vref)) < (1e-6 if dtype == "c64" else 1e-12)


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_expectations_batch_scattered(T, dtype):
    """A batch of three different states, terms whose X bits scatter over the high
    qubits (tiles copied piecewise, each item from its own offset), checked item by
    item against the oracle."""
    n = 17
    from paper_2602_14167_b300 import StateBatch
    from workloads import pauli_terms
    st = StateBatch(n, batch=3, dtype=dtype)
    for i in range(3):
        st.amplitudes(i).copy_(torch.tensor(gen.random_state(n, seed=40 + i), dtype=st.cdtype, device="cuda"))
    strings = np.concatenate([
        pauli_terms([{4: "X", 9: "Y", 13: "X", 16: "Z"}, {5: "Y", 11: "X", 15: "X"},
                     {0: "X", 8: "X", 12: "Y", 16: "X"}, {3: "Z", 10: "X", 14: "Y"}]),
        gen.random_pauli_strings(n, 12, 4, seed=9)])
    vals = st.expect(strings).cpu().numpy()
    for i in range(3):
        ref_psi = st.amplitudes(i).cpu().numpy().astype(np.complex128)
        vref = sv.expect(n, ref_psi, strings).real
        assert np.max(np.abs(vals[i] - vref)) < (1e-6 if dtype == "c64" else 1e-12), i


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_expectations_scattered_gathers(T, dtype):
    """Terms whose X bits scatter over the high qubits: tiles that need more than five
    tensor-map dimensions (gather4 rows for 2^7 chunks, bulk copies for wider chunks)."""
    n = 20
    psi0 = gen.random_state(n, seed=21)
    from paper_2602_14167_b300 import StateBatch
    from workloads import pauli_terms
    st = StateBatch(n, dtype=dtype)
    st.amplitudes(0).copy_(torch.tensor(psi0, dtype=st.cdtype, device="cuda"))
    strings = pauli_terms([{8: "X", 10: "X", 12: "Y", 14: "X", 16: "X", 18: "Y"},   # 2^7 chunk rows
                           {8: "X", 11: "Y", 14: "X", 17: "Z", 19: "X"},
                           {8: "Y", 11: "X", 14: "Y", 17: "X", 19: "Y", 2: "Z"},
                           {9: "X", 12: "X", 15: "Y", 18: "X", 0: "Y"},
                           {10: "X", 16: "Y", 19: "Z", 3: "X"}])
    vals = st.expect(strings)[0].cpu().numpy()
    ref_psi = st.amplitudes(0).cpu().numpy().astype(np.complex128)
    vref = sv.expect(n, ref_psi, strings).real
    assert np.max(np.abs(vals - vref)) < (1e-6 if dtype == "c64" else 1e-12)


@pytest.mark.parametrize("dtype,n", [("c128", 16), ("c64", 17), ("c64", 22)])
def test_expectation_terms_wider_than_a_tile(T, dtype, n):
    """Strings with more X/Y factors than a tile gathers (the parity X...X, Y-heavy
    and random high-weight strings) run from global memory; together with
    ordinary terms in one call, every value against the oracle."""
    from paper_2602_14167_b300 import StateBatch
    from workloads import pauli_terms
    rng = np.random.default_rng(n)
    wide = [{q: "X" for q in range(n)}, {q: "Y" for q in range(1, n)},
            {q: "XYZ"[int(rng.integers(3))] for q in range(n)},
            {q: "XY"[q % 2] for q in range(2, n, 1)}]
    terms = np.concatenate([pauli_terms(wide), gen.random_pauli_strings(n, 12, 4, seed=n),
                            gen.tfim_terms(n, 1.0, 0.7)])
    st = StateBatch(n, dtype=dtype)
    psi = gen.random_state(n, seed=2 * n)
    st.amplitudes(0).copy_(torch.tensor(psi, dtype=st.cdtype, device="cuda"))
    got = st.expect(terms)[0].cpu().numpy()
    ref = sv.expect(n, psi, terms).real
    assert np.max(np.abs(got - ref)) < (1e-12 if dtype == "c128" else 1e-5)
    e = st.energy(terms)[0].item()
    assert abs(e - float(np.dot(terms["coeff"], ref))) < (1e-11 if dtype == "c128" else 1e-4)
    st.free()


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_expectations_of_a_ragged_batch(T, dtype):
    """A batch of states of 9, 14 and 17 qubits: one expectation call per size class
    inside the library, values and energies in the items' own rows."""
    from paper_2602_14167_b300 import StateBatch
    ns = [14, 9, 17, 14, 9]
    st = StateBatch(ns, dtype=dtype)
    terms = np.concatenate([gen.random_pauli_strings(9, 10, 3, seed=4), gen.tfim_terms(9, 1.0, 0.5)])
    psis = [gen.random_state(n, seed=30 + i) for i, n in enumerate(ns)]
    for i, psi in enumerate(psis):
        st.amplitudes(i).copy_(torch.tensor(psi, dtype=st.cdtype, device="cuda"))
    coeffs = torch.tensor(np.random.default_rng(1).normal(size=(len(ns), len(terms))), device="cuda")
    vals = torch.empty((len(ns), len(terms)), dtype=torch.float64, device="cuda")
    energy = torch.empty(len(ns), dtype=torch.float64, device="cuda")
    T.tcng_expect_energy(st.handle, terms, coeffs, vals, energy)
    vals, energy, cf = vals.cpu().numpy(), energy.cpu().numpy(), coeffs.cpu().numpy()
    tol = 1e-12 if dtype == "c128" else 1e-5
    for i, (n, psi) in enumerate(zip(ns, psis)):
        ref = sv.expect(n, psi, terms).real
        assert np.max(np.abs(vals[i] - ref)) < tol
        assert abs(energy[i] - float(np.dot(cf[i], ref))) < 50 * tol
    st.free()


def test_energy_per_item_coefficients(T):
    n, B = 12, 4
    b = gen.tfim_batch(n, B, layers=2, seed=3)
    g, p = b["circuit"].to_ir()
    st = run(n, g, p, b["theta"], "c128", batch=B)
    coeffs = torch.tensor(b["coeffs"], dtype=torch.float64, device="cuda")
    e = st.energy(b["terms"], coeffs).cpu().numpy()
    for i in range(B):
        e_ref = sv.energy(n, g, p, b["theta"][i], b["terms"], b["coeffs"][i])
        assert abs(e[i] - e_ref) < 1e-11


def test_expect_energy_matches_separate_calls(T):
    """One plan for strings + Hamiltonian: same values and energy as two calls."""
    n = 18
    c, th = gen.su4_brickwork(n, 4, "RZ", seed=9)
    g, p = c.to_ir()
    st = run(n, g, p, th, "c64")
    strings = gen.random_pauli_strings(n, 24, 4, seed=10)
    ham = gen.tfim_terms(n, 1.0, 0.8)
    terms = np.concatenate([strings, ham])
    terms["coeff"][:len(strings)] = 0.0
    vals = torch.empty((1, len(terms)), dtype=torch.float64, device="cuda")
    e = torch.empty(1, dtype=torch.float64, device="cuda")
    T.tcng_expect_energy(st.handle, terms, None, vals, e)
    v_sep = st.expect(strings)[0].cpu().numpy()
    e_sep = float(st.energy(ham)[0])
    v = vals[0].cpu().numpy()
    assert np.max(np.abs(v[:len(strings)] - v_sep)) < 1e-6
    assert abs(float(e[0]) - e_sep) < 1e-6 * np.abs(ham["coeff"]).sum()
    ref = sv.apply(n, g, p, th)
    assert abs(float(e[0]) - float(np.dot(ham["coeff"], sv.expect(n, ref, ham).real))) < 1e-5 * np.abs(ham["coeff"]).sum()


def test_hamiltonian_apply(T):
    n = 10
    from paper_2602_14167_b300 import StateBatch
    st = StateBatch(n, dtype="c128")
    out = StateBatch(n, dtype="c128")
    psi0 = gen.random_state(n, seed=4)
    st.amplitudes(0).copy_(torch.tensor(psi0, device="cuda"))
    terms = gen.xxz_terms(n, np.linspace(0.5, 1.5, n - 1), 0.6, 0.4)
    T.tcng_hamiltonian_apply(st.handle, terms, None, out.handle)
    torch.cuda.synchronize()
    ref = sv.hamiltonian_apply(n, psi0, terms)
    assert relerr(out.amplitudes(0).cpu().numpy(), ref) < 1e-12


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_hamiltonian_apply_ragged_batch(T, dtype):
    """lambda_b = H_b psi_b over a batch of 8-, 11- and 13-qubit states with
    per-item coefficients: one size class at a time, each item against the oracle."""
    from paper_2602_14167_b300 import StateBatch
    ns = [11, 8, 13, 8]
    st, out = StateBatch(ns, dtype=dtype), StateBatch(ns, dtype=dtype)
    terms = gen.xxz_terms(8, np.linspace(0.5, 1.5, 7), 0.6, 0.4)
    cf = np.random.default_rng(3).normal(size=(len(ns), len(terms)))
    psis = [gen.random_state(n, seed=40 + i) for i, n in enumerate(ns)]
    for i, psi in enumerate(psis):
        st.amplitudes(i).copy_(torch.tensor(psi, dtype=st.cdtype, device="cuda"))
    T.tcng_hamiltonian_apply(st.handle, terms, torch.tensor(cf, device="cuda"), out.handle)
    torch.cuda.synchronize()
    tol = 1e-12 if dtype == "c128" else 1e-5
    for i, (n, psi) in enumerate(zip(ns, psis)):
        ref = sv.hamiltonian_apply(n, psi, terms, cf[i])
        assert relerr(out.amplitudes(i).cpu().numpy().astype(np.complex128), ref) < tol
    st.free()
    out.free()


def test_expectation_is_deterministic(T):
    n = 18
    c, th = gen.su4_brickwork(n, 4, "RZ", seed=5)
    g, p = c.to_ir()
    st = run(n, g, p, th, "c64")
    s = gen.random_pauli_strings(n, 20, 4, seed=6)
    a = st.expect(s).cpu().numpy()
    b = st.expect(s).cpu().numpy()
    assert np.array_equal(a, b)


def test_invalid_arguments_are_rejected(T):
    from paper_2602_14167_b300 import StateBatch
    st = StateBatch(6, dtype="c64")
    from workloads import Circuit
    bad = Circuit(7).x(6)
    g, p = bad.to_ir()
    with pytest.raises(T.TcngError):
        st.apply(g, p)
    with pytest.raises(T.TcngError):
        st.expect(np.array([(1 << 6, 0, 1.0)], dtype=T.PAULI_DTYPE))
    T.tcng_sync_status()


TC_KERNELS = ("pass_tcs_kernel_c64", "pass_tch_kernel_c64")   # TF32-, FP16-split stages


def tc_run(T, n, g, p, th, batch=1, fp16=1, per_kernel=False):
    """complex64 run with register stages on the tensor cores; returns (state, tc
    launches) or, with per_kernel, (state, {kernel: launches})."""
    T.tcng_set_option(T.OPT_TENSOR_CORES, 1)
    T.tcng_set_option(T.OPT_TC_FP16, fp16)
    T.tcng_profile_enable(True)
    T.tcng_profile_read(reset=True)
    try:
        st = run(n, g, p, th, "c64", batch=batch)
        prof = T.tcng_profile_read(reset=True)
    finally:
        T.tcng_profile_enable(False)
    counts = {k: prof.get(k, (0, 0.0))[0] for k in TC_KERNELS}
    return st, (counts if per_kernel else sum(counts.values()))


@pytest.mark.parametrize("fp16", [1, 0])
@pytest.mark.parametrize("n,depth,width", [(13, 6, 4), (16, 8, 4), (19, 6, 3), (21, 5, 2), (22, 6, 2)])
def test_tensor_core_stages(T, n, depth, width, fp16):
    """complex64 register stages on the tensor cores (FP16 and TF32 splits) vs the
    oracle and vs the SIMT stages."""
    c, th = gen.su4_brickwork(n, depth, "RZ", seed=n)
    g, p = c.to_ir()
    ref = sv.apply(n, g, p, th)
    T.tcng_set_option(T.OPT_FUSE_WIDTH, width)
    st, counts = tc_run(T, n, g, p, th, fp16=fp16, per_kernel=True)
    assert counts["pass_tch_kernel_c64" if fp16 else "pass_tcs_kernel_c64"] > 0
    if not fp16:
        assert counts["pass_tch_kernel_c64"] == 0
    check_state(st.amplitudes(0).cpu().numpy(), ref, "c64")
    T.tcng_set_option(T.OPT_TENSOR_CORES, 0)
    st2 = run(n, g, p, th, "c64")
    check_state(st2.amplitudes(0).cpu().numpy(), ref, "c64")


@pytest.mark.parametrize("n,depth,fw", [(15, 6, 2), (18, 10, 2), (20, 8, 2), (16, 12, 4)])
def test_fp16_passes_every_kernel_form(T, n, depth, fw):
    """Unitary single-item plans: every tensor-core pass takes the FP16 kernels
    (independent slices, lock-step with three tile buffers and with two); the state
    matches the oracle and the TF32 form."""
    c, th = gen.su4_brickwork(n, depth, "RZ", seed=100 + n)
    g, p = c.to_ir()
    ref = sv.apply(n, g, p, th)
    T.tcng_set_option(T.OPT_FUSE_WIDTH, fw)
    st, counts = tc_run(T, n, g, p, th, fp16=1, per_kernel=True)
    assert counts["pass_tch_kernel_c64"] > 0
    psi = st.amplitudes(0).cpu().numpy()
    check_state(psi, ref, "c64")
    st.free()
    st2, counts2 = tc_run(T, n, g, p, th, fp16=0, per_kernel=True)
    assert counts2["pass_tch_kernel_c64"] == 0
    psi2 = st2.amplitudes(0).cpu().numpy()
    assert relerr(psi, psi2) < 2 * TOL["c64"]


def stage_widths(T, n, g, p, P):
    """Register bits of every stage of the plan tcng_apply_circuit runs."""
    out = []
    for line in T.tcng_describe_plan(n, g, p, P, False).split("\n"):
        if "regs=" in line:
            for tok in line.split("regs=")[1].split():
                out.append(tok[tok.index("{") + 1:tok.index("}")].count(",") + 1)
    return out


@pytest.mark.parametrize("n,depth", [(18, 10), (22, 14)])
def test_fp16_five_bit_stages(T, n, depth):
    """Gathered passes whose gates fit two 5-qubit register stages instead of three
    4-qubit ones run 32x32 complex (64x64 real) FP16 GEMMs: the plan has such stages,
    they run on the FP16 kernels, and the state matches the oracle."""
    c, th = gen.su4_brickwork(n, depth, "RZ", seed=100 + n)
    g, p = c.to_ir()
    T.tcng_set_option(T.OPT_TENSOR_CORES, 1)
    T.tcng_set_option(T.OPT_TC_FP16, 1)
    assert 5 in stage_widths(T, n, g, p, len(th))
    st, counts = tc_run(T, n, g, p, th, fp16=1, per_kernel=True)
    assert counts["pass_tch_kernel_c64"] > 0 and counts["pass_tcs_kernel_c64"] == 0
    check_state(st.amplitudes(0).cpu().numpy(), sv.apply(n, g, p, th), "c64")
    T.tcng_set_option(T.OPT_TC_FP16, 0)   # the TF32 path plans 4-qubit stages only
    assert set(stage_widths(T, n, g, p, len(th))) == {4}


@pytest.mark.parametrize("scale_log2", [-70, -20, 0, 30, 60])
def test_fp16_passes_scaled_states(T, scale_log2):
    """The FP16 split scales each tile by a power of two: states of any magnitude
    (here 2^k times a random unit state, far outside FP16's range at both ends) and
    with a wide spread (an RY product state) come back as the oracle's."""
    from paper_2602_14167_b300 import StateBatch
    n = 16
    c, th = gen.su4_brickwork(n, 6, "RZ", seed=7)
    g, p = c.to_ir()
    f = 2.0 ** scale_log2
    t = np.random.default_rng(9).uniform(-np.pi, np.pi, n)
    prod = np.ones(1, dtype=np.complex128)
    for q in range(n):   # qubit q is index bit q
        prod = np.kron(np.array([np.cos(t[q] / 2), np.sin(t[q] / 2)]), prod)
    for psi0 in (gen.random_state(n, seed=8) * f, prod * f):
        T.tcng_set_option(T.OPT_TENSOR_CORES, 1)
        T.tcng_set_option(T.OPT_TC_FP16, 1)
        st = StateBatch(n, dtype="c64")
        st.amplitudes(0).copy_(torch.tensor(psi0, dtype=st.cdtype, device="cuda"))
        prm = torch.tensor(th, dtype=torch.float64, device="cuda").reshape(1, -1)
        st.apply(g, p, prm)
        torch.cuda.synchronize()
        psi = st.amplitudes(0).cpu().numpy().astype(np.complex128)
        ref = sv.apply(n, g, p, th, psi=psi0)
        assert np.all(np.isfinite(psi))
        assert relerr(psi, ref) < TOL["c64"], relerr(psi, ref)
        st.free()


def test_tensor_core_stages_with_diagonal_and_random_ops(T):
    n = 15
    c, th = gen.random_circuit(n, 200, seed=77,
                               kinds=["H", "RX", "RY", "RZ", "CX", "CZ", "CP", "RZZ", "U1", "U2", "U3", "U4", "T", "S"])
    g, p = c.to_ir()
    st, launches = tc_run(T, n, g, p, th)
    assert launches > 0
    check_state(st.amplitudes(0).cpu().numpy(), sv.apply(n, g, p, th), "c64")


def test_tensor_core_stages_config2(T):
    """n=24 depth-20 SU(4) brickwork + RX: the longest circuit of the parity set."""
    n = 24
    c, th = gen.su4_brickwork(n, 20, "RX", seed=0)
    g, p = c.to_ir()
    st, launches = tc_run(T, n, g, p, th)
    assert launches > 0
    check_state(st.amplitudes(0).cpu().numpy(), sv.apply(n, g, p, th), "c64")


def test_tensor_core_stages_batch_per_item_params(T):
    n, B = 14, 3
    c = gen.hea_ring(n, 2)
    g, p = c.to_ir()
    th = gen.random_thetas((B, c.n_params), seed=5)
    st, launches = tc_run(T, n, g, p, th, batch=B)
    assert launches > 0
    for b in range(B):
        check_state(st.amplitudes(b).cpu().numpy(), sv.apply(n, g, p, th[b]), "c64")


def test_tensor_core_stages_shared_params_batch(T):
    """Several items, one parameter set: every item runs the same W operands."""
    n, B = 15, 4
    c, th = gen.su4_brickwork(n, 5, "RZ", seed=3)
    g, p = c.to_ir()
    from paper_2602_14167_b300 import StateBatch
    T.tcng_set_option(T.OPT_TENSOR_CORES, 1)
    st = StateBatch(n, batch=B, dtype="c64")
    prm = torch.tensor(th, dtype=torch.float64, device="cuda").reshape(1, -1).expand(B, -1).contiguous()
    st.apply(g, p, prm)
    ref = sv.apply(n, g, p, th)
    for b in range(B):
        check_state(st.amplitudes(b).cpu().numpy(), ref, "c64")


def test_tensor_core_stages_parameter_free_batch(T):
    """A circuit without parameters (angles fixed in the gates) on three different
    states: one W set serves every tile of every item, and the lock-step pass over
    the 13 lowest qubits (10 register stages) keeps it resident; each item against
    the oracle."""
    n, B = 15, 3
    c, th = gen.su4_brickwork(n, 6, "RZ", seed=11)
    g, p = c.to_ir()
    g = g.copy()
    sel = g["param"] >= 0
    g["angle0"][sel] = g["angle0"][sel] + g["scale"][sel] * np.asarray(th, dtype=np.float64)[g["param"][sel]]
    g["scale"][sel] = 0.0
    g["param"][sel] = -1
    from paper_2602_14167_b300 import StateBatch
    psi0 = [gen.random_state(n, seed=60 + i) for i in range(B)]
    T.tcng_set_option(T.OPT_TENSOR_CORES, 1)
    T.tcng_profile_enable(True)
    T.tcng_profile_read(reset=True)
    try:
        st = StateBatch(n, batch=B, dtype="c64")
        for i in range(B):
            st.amplitudes(i).copy_(torch.tensor(psi0[i], dtype=st.cdtype, device="cuda"))
        st.apply(g, p)
        torch.cuda.synchronize()
        prof = T.tcng_profile_read(reset=True)
        launches = sum(prof.get(k, (0, 0.0))[0] for k in TC_KERNELS)
    finally:
        T.tcng_profile_enable(False)
    assert launches > 0
    for i in range(B):
        check_state(st.amplitudes(i).cpu().numpy(), sv.apply(n, g, p, None, psi=psi0[i]), "c64")


def test_tensor_core_option_values(T):
    for v in (0, 1, 2):
        T.tcng_set_option(T.OPT_TENSOR_CORES, v)
        assert T.tcng_get_option(T.OPT_TENSOR_CORES) == v
    with pytest.raises(T.TcngError):
        T.tcng_set_option(T.OPT_TENSOR_CORES, 3)


def test_tensor_core_stages_non_unitary_matrix(T):
    """An explicit non-unitary block (a projector times a scale) must not be renormalised."""
    from workloads import Circuit
    n = 14
    c = Circuit(n)
    for q in range(n):
        c.h(q)
    c.unitary((3, 4), np.diag([1.0, 0.0, 0.0, 0.5]).astype(np.complex128))
    c.unitary((9, 11), np.array([[1, 1, 0, 0], [0, 1, 0, 0], [0, 0, 1, 0.5j], [0, 0, 0, 0.5]],
                                dtype=np.complex128))
    for q in range(0, n - 1, 2):
        c.cx(q, q + 1)
    g, p = c.to_ir()
    st, launches = tc_run(T, n, g, p, None)
    ref = sv.apply(n, g, p, None)
    psi = st.amplitudes(0).cpu().numpy()
    assert relerr(psi, ref) < TOL["c64"], relerr(psi, ref)
