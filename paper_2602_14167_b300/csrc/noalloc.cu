// Pauli expectations with no device allocation (tcng_expect_pauli_noalloc).
//
// Some callers cannot let a library allocate device memory: a host framework
// whose own allocator has already reserved the GPU's free memory, or a serving
// loop that forbids allocation (and the device synchronisation cudaFree brings)
// on its hot path.  This entry point runs the same expectation passes
// as tcng_expect_pauli but keeps the per-CTA partial sums in a fixed-size array
// in this file's device memory, so it calls no cudaMalloc or cudaFree and never
// touches the library's other caches.  Every GPU that loads the library holds
// that array (512 KiB) until the process exits.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <stdexcept>
#include <string>
#include <vector>

#include "capi_internal.hpp"

namespace {

constexpr size_t kNoAllocPartials = 1u << 16;   // doubles of per-CTA partial sums (512 KiB)
constexpr int kNoAllocMaxDevices = 64;

// Partial sums of the expectation passes.  Every call writes each slot it later
// reads (one per term per CTA), so stale contents from an earlier call are
// never used and nothing needs clearing.
static __device__ __align__(256) double g_noalloc_partials[kNoAllocPartials];
// Element offset of the single state vector (always 0; never written).
static __device__ __align__(256) long long g_noalloc_item_off[1];

struct NoAllocPtrs {
    double* partials = nullptr;
    long long* item_off = nullptr;
};
NoAllocPtrs g_ptrs[kNoAllocMaxDevices];
std::mutex g_ptr_mu;

// Device addresses of the static arrays for the current device (set up once
// per device, on its first call).
tcng_status noalloc_setup(NoAllocPtrs* out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return tcng::cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kNoAllocMaxDevices) return tcng::fail(TCNG_EUNSUPPORTED, "device index too large");
    std::lock_guard<std::mutex> lk(g_ptr_mu);
    NoAllocPtrs& p = g_ptrs[dev];
    if (!p.partials) {
        void* a = nullptr;
        void* b = nullptr;
        e = cudaGetSymbolAddress(&a, g_noalloc_partials);
        if (e != cudaSuccess) return tcng::cuda_fail(e, "cudaGetSymbolAddress(partials)");
        e = cudaGetSymbolAddress(&b, g_noalloc_item_off);
        if (e != cudaSuccess) return tcng::cuda_fail(e, "cudaGetSymbolAddress(item offset)");
        p.item_off = static_cast<long long*>(b);
        p.partials = static_cast<double*>(a);
    }
    *out = p;
    return TCNG_OK;
}

}  // namespace

using namespace tcng;

extern "C" tcng_status tcng_expect_pauli_noalloc(const void* psi_dev, int n, tcng_dtype dt,
                                                 const tcng_pauli* terms, size_t n_terms,
                                                 double* out_dev, void* stream) {
    if (!psi_dev || !out_dev || (!terms && n_terms)) return fail(TCNG_EINVAL, "null argument");
    if (dt != TCNG_C64 && dt != TCNG_C128) return fail(TCNG_EINVAL, "bad dtype");
    if (n < 1 || n > TCNG_MAX_QUBITS) return fail(TCNG_EINVAL, "qubit count out of range");
    if (reinterpret_cast<uintptr_t>(psi_dev) & 255)
        return fail(TCNG_EINVAL, "psi_dev must be 256-byte aligned");
    if (n_terms == 0) return TCNG_OK;
    if (n_terms > 4096) return fail(TCNG_EINVAL, "at most 4096 terms per call");
    // the options and the launchers' per-device attribute caches are shared with
    // every other entry point: read and use them under the library lock
    std::lock_guard<std::mutex> lk(g_mu);
    try {
        const PlanOptions o = plan_options(dt, false);
        std::vector<DevPass> passes;
        std::vector<ExpPass> eps;
        plan_expectation(n, o.tile_bits, o.chunk_bits, terms, n_terms, passes, eps);
        const long long tpi = 1ll << (n - passes[0].m);
        const int nblk = (int)std::max<long long>(1, std::min<long long>(tpi, num_sms()));
        const size_t need = n_terms * (size_t)nblk;
        if (need > kNoAllocPartials)
            return fail(TCNG_EINVAL, "tcng_expect_pauli_noalloc: " + std::to_string(n_terms) +
                                         " terms need " + std::to_string(need) +
                                         " partial sums; the static scratch holds " +
                                         std::to_string(kNoAllocPartials));
        NoAllocPtrs ptrs;
        tcng_status st = noalloc_setup(&ptrs);
        if (st) return st;
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        for (size_t i = 0; i < passes.size(); ++i) {
            cudaError_t e;
            if (dt == TCNG_C64)
                e = launch_expect_pass<float2>(static_cast<const float2*>(psi_dev), ptrs.item_off, 1, n,
                                               passes[i], eps[i], ptrs.partials, (int)n_terms, nblk,
                                               nullptr, s);
            else
                e = launch_expect_pass<double2>(static_cast<const double2*>(psi_dev), ptrs.item_off, 1, n,
                                                passes[i], eps[i], ptrs.partials, (int)n_terms, nblk,
                                                nullptr, s);
            if (e != cudaSuccess) return cuda_fail(e, "expectation pass");
        }
        cudaError_t e = launch_expect_finalize(ptrs.partials, nblk, (int)n_terms, out_dev, nullptr,
                                               nullptr, nullptr, 1, s);
        if (e != cudaSuccess) return cuda_fail(e, "expectation finalize");
        return TCNG_OK;
    } catch (const std::invalid_argument& ex) {
        return fail(TCNG_EINVAL, ex.what());
    } catch (const std::exception& ex) {
        return fail(TCNG_EINVAL, ex.what());
    }
}
