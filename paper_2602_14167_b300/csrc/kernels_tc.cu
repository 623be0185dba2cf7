// Shared-unitary batched apply (tcng_apply_shared_unitary).
//
// B states that all see the same k-qubit unitary U (the batched layer of the
// paper's QML demonstration, Sec. VII.B) are one complex GEMM [2^k x 2^k] x
// [2^k x B 2^(n-k)].  The call is a one-gate circuit without parameters: the
// tile passes then hold one W set for every tile of every item and run it on
// the tensor cores (FP16 hi/lo operands, kernels_pass_tch.cu), with items of
// fewer than 13 qubits packed several to a tile.
#include <cuda_runtime.h>

#include "capi_internal.hpp"

using namespace tcng;

extern "C" tcng_status tcng_apply_shared_unitary(tcng_state* st, const int* qubits, int k,
                                                 const double* U, void* stream) {
    if (!st || !qubits || !U) return fail(TCNG_EINVAL, "null argument");
    if (k < 1 || k > 5) return fail(TCNG_EINVAL, "k must be 1..5");
    if (st->dt != TCNG_C64) return fail(TCNG_EUNSUPPORTED, "shared-unitary apply needs complex64 states");
    for (int j = 0; j < k; ++j)
        for (int i = 0; i < j; ++i)
            if (qubits[i] == qubits[j]) return fail(TCNG_EINVAL, "repeated qubit");
    tcng_gate g{};
    g.op = (uint16_t)(k == 1 ? TCNG_U1 : (k == 2 ? TCNG_U2 : TCNG_UK));
    g.nq = (uint8_t)k;
    for (int j = 0; j < 5; ++j) g.q[j] = j < k ? qubits[j] : -1;
    g.param = -1;
    g.scale = 0.0;
    g.angle0 = 0.0;
    g.mat_off = 0;
    // qubit range checks (per size class) happen in the circuit call
    return tcng_apply_circuit(st, &g, 1, U, (size_t)1 << (2 * k), nullptr, 0, stream);
}
