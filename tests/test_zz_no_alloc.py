"""tcng_expect_pauli_noalloc against tcng_expect_pauli (GPU).

The allocation-free entry point exists for callers that must not let the
library call cudaMalloc (their allocator owns the free memory, or their hot
path bans allocation).  It keeps its
partial sums in a static device array instead.  Here it must reproduce the
ordinary entry point's values and the oracle's within the complex64/complex128
tolerances of the other expectation tests, on two calls in a row (the second call reuses the
array the first one left behind), and reject requests larger than its array.
This file is collected last so a failure here comes after every other test.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import sv  # noqa: E402
from workloads import generators as gen  # noqa: E402

TOL = {"c64": 1e-6, "c128": 1e-12}


@pytest.fixture(scope="module")
def T():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2602_14167_b300 import build
    build.build()
    from paper_2602_14167_b300 import tcng
    return tcng


@pytest.mark.parametrize("dtype,n", [("c64", 17), ("c64", 9), ("c128", 14)])
def test_matches_allocating_entry_point_twice(T, dtype, n):
    from paper_2602_14167_b300 import StateBatch
    st = StateBatch(n, dtype=dtype)
    dt = T.C64 if dtype == "c64" else T.C128
    for call in range(2):
        psi = gen.random_state(n, seed=10 * n + call)
        st.amplitudes(0).copy_(torch.tensor(psi, dtype=st.cdtype, device="cuda"))
        strings = np.concatenate([gen.random_pauli_strings(n, 48, min(4, n), seed=call),
                                  gen.tfim_terms(n, 1.0, 1.0)])
        ref = torch.empty((1, len(strings)), dtype=torch.float64, device="cuda")
        T.tcng_expect_pauli(st.handle, strings, ref)
        out = torch.full((len(strings),), float("nan"), dtype=torch.float64, device="cuda")
        ptr, _ = T.tcng_state_ptr(st.handle, 0)
        status = T.lib().tcng_expect_pauli_noalloc(ptr, n, dt, strings.ctypes.data, len(strings),
                                                   out.data_ptr(), T._stream(None))
        assert status == 0, T.tcng_last_error()
        torch.cuda.synchronize()
        got, want = out.cpu().numpy(), ref[0].cpu().numpy()
        assert np.all(np.isfinite(got))
        assert np.max(np.abs(got - want)) < TOL[dtype]
        # and against the oracle directly (the state as stored on the device)
        stored = st.amplitudes(0).cpu().numpy().astype(np.complex128)
        assert np.max(np.abs(got - sv.expect(n, stored, strings).real)) < TOL[dtype]
    st.free()


def test_rejects_requests_beyond_the_static_scratch(T):
    from paper_2602_14167_b300 import StateBatch
    n = 24          # 2^11 tiles: one CTA per SM, so 4096 terms need far more than 65536 slots
    st = StateBatch(n, dtype="c64")
    strings = gen.random_pauli_strings(n, 4096, 2, seed=3)
    out = torch.empty(len(strings), dtype=torch.float64, device="cuda")
    ptr, _ = T.tcng_state_ptr(st.handle, 0)
    with pytest.raises(T.TcngError) as ei:
        T.tcng_expect_pauli_noalloc(ptr, n, T.C64, strings, out)
    assert "static scratch" in str(ei.value)
    st.free()


@pytest.mark.parametrize("dtype,n", [("c64", 17), ("c128", 12)])
def test_call_recorded_in_a_cuda_graph(T, dtype, n):
    """The entry point allocates nothing and copies nothing, so after one ordinary
    call it can be recorded into a CUDA graph: the replay reads the state as it
    is at replay time (changed after the capture) and matches tcng_expect_pauli."""
    from paper_2602_14167_b300 import StateBatch
    st = StateBatch(n, dtype=dtype)
    dt = T.C64 if dtype == "c64" else T.C128
    strings = np.concatenate([gen.random_pauli_strings(n, 24, min(4, n), seed=5), gen.tfim_terms(n, 1.0, 1.0)])
    ptr, _ = T.tcng_state_ptr(st.handle, 0)
    out = torch.full((len(strings),), float("nan"), dtype=torch.float64, device="cuda")
    st.amplitudes(0).copy_(torch.tensor(gen.random_state(n, seed=1), dtype=st.cdtype, device="cuda"))
    T.tcng_expect_pauli_noalloc(ptr, n, dt, strings, out)   # first call outside any capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        T.tcng_expect_pauli_noalloc(ptr, n, dt, strings, out)
    for seed in (2, 3):
        st.amplitudes(0).copy_(torch.tensor(gen.random_state(n, seed=seed), dtype=st.cdtype, device="cuda"))
        out.fill_(float("nan"))
        g.replay()
        ref = torch.empty((1, len(strings)), dtype=torch.float64, device="cuda")
        T.tcng_expect_pauli(st.handle, strings, ref)
        torch.cuda.synchronize()
        got, want = out.cpu().numpy(), ref[0].cpu().numpy()
        assert np.all(np.isfinite(got))
        assert np.max(np.abs(got - want)) < TOL[dtype]
    del g
    st.free()
