// Shared-unitary batched apply on the tensor cores (tcgen05, TMEM accumulators).
//
// Paper: Sec. VII.B (QML on CIFAR-100/MNIST) -- every input state of a batch is
// evolved by the same parameterised circuit, so one layer's fused k-qubit
// unitary U multiplies every length-2^k slice of every state: a complex GEMM
// [batch * 2^(n-k) rows] x [2^k] times U^T.  Written as a real GEMM on
// interleaved (re, im) pairs: row (.., re_l, im_l, ..) times W with
//   W[2l][2j] = Re U_jl,  W[2l+1][2j] = -Im U_jl,  W[2l][2j+1] = Im U_jl,  W[2l+1][2j+1] = Re U_jl.
// fp32 accuracy from TF32 operands by the 3-term split a = a_hi + a_lo,
// w = w_hi + w_lo: D = a_hi w_hi + a_hi w_lo + a_lo w_hi (a_lo w_lo dropped).
//
// Per CTA (128 threads, persistent over 128-row tiles): warps gather the rows of
// a tile from the state, split them into TF32 hi/lo and store them K-major with
// the 128-byte swizzle; one thread issues 24 tcgen05.mma (M=128, N=64, K=8) into a
// 64-column TMEM accumulator and commits to an mbarrier; the four warps read their
// 32 TMEM lanes (tcgen05.ld 32x32b) and scatter the new amplitudes back.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "capi_internal.hpp"
#include "device.cuh"
#include "tc.cuh"

namespace tcng {

struct TcArgs {
    float2* state;              // complex64 amplitudes
    const long long* item_off;  // element offset of each item
    int items;
    int n;                      // qubits per item
    int k;                      // qubits of U
    uint32_t qmask;             // ascending qubits of U
    const float* w;             // [2][TC_N][TC_K]: W^T hi then lo (row = output column)
    unsigned* err;
};

__global__ void __launch_bounds__(128) shared_unitary_tc_kernel(TcArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // 1024-byte aligned operand region: A_hi, A_lo, B_hi, B_lo
    const uint32_t base_s = smem_u32(smem_raw);
    const uint32_t pad = (1024u - (base_s & 1023u)) & 1023u;
    unsigned char* ops = smem_raw + pad;
    unsigned char* a_hi = ops;
    unsigned char* a_lo = ops + TC_A_BYTES;
    unsigned char* b_hi = ops + 2 * TC_A_BYTES;
    unsigned char* b_lo = b_hi + TC_B_BYTES;
    __shared__ uint64_t bar;
    __shared__ uint32_t tmem_base;
    __shared__ int s_abort;
    // warp index and TMEM base broadcast from lane 0: warp-uniform for the compiler
    const int tid = threadIdx.x, warp = __shfl_sync(0xffffffffu, tid >> 5, 0), lane = tid & 31;
    const int kq = a.k, D = 1 << kq;
    int qs[TCNG_MAX_FUSE];
    {
        int j = 0;
        for (int b = 0; b < a.n && j < kq; ++b)
            if ((a.qmask >> b) & 1) qs[j++] = b;
    }
    // B operand (same for every tile), zero-padded to 64 x 64
    for (int e = tid; e < TC_N * TC_K; e += blockDim.x) {
        const int nn = e / TC_K, kk = e % TC_K;
        const uint32_t off = sw128_offset(nn, kk, TC_N);
        *reinterpret_cast<float*>(b_hi + off) = a.w[e];
        *reinterpret_cast<float*>(b_lo + off) = a.w[TC_N * TC_K + e];
    }
    // zero the A padding columns once (columns >= 2*D are never overwritten)
    for (int e = tid; e < TC_M * TC_K; e += blockDim.x) {
        const int row = e / TC_K, kk = e % TC_K;
        if (kk >= 2 * D) {
            const uint32_t off = sw128_offset(row, kk, TC_M);
            *reinterpret_cast<float*>(a_hi + off) = 0.f;
            *reinterpret_cast<float*>(a_lo + off) = 0.f;
        }
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_base)),
                     "r"(TC_N)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
        s_abort = 0;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = __shfl_sync(0xffffffffu, tmem_base, 0);
    const long long rows_per_item = 1ll << (a.n - kq);
    const long long total_rows = rows_per_item * a.items;
    const long long ntiles = (total_rows + TC_M - 1) / TC_M;
    uint32_t phase = 0;
    const uint32_t idesc = tf32_idesc(TC_M, TC_N);
    for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const long long r0 = t * TC_M;
        // ---- gather rows, split to TF32 hi/lo, store swizzled ----
        for (int e = tid; e < TC_M * D; e += blockDim.x) {
            const int l = e / TC_M, row = e % TC_M;
            const long long r = r0 + row;
            float2 v = make_float2(0.f, 0.f);
            if (r < total_rows) {
                const long long item = r >> (a.n - kq);
                long long x = r & (rows_per_item - 1);
                for (int j = 0; j < kq; ++j) x = ((x >> qs[j]) << (qs[j] + 1)) | (x & ((1ll << qs[j]) - 1));
                for (int j = 0; j < kq; ++j)
                    if ((l >> j) & 1) x |= 1ll << qs[j];
                v = a.state[a.item_off[item] + x];
            }
            const float hr = tf32_round(v.x), hi_ = tf32_round(v.y);
            const uint32_t o0 = sw128_offset(row, 2 * l, TC_M), o1 = sw128_offset(row, 2 * l + 1, TC_M);
            *reinterpret_cast<float*>(a_hi + o0) = hr;
            *reinterpret_cast<float*>(a_hi + o1) = hi_;
            *reinterpret_cast<float*>(a_lo + o0) = tf32_round(v.x - hr);
            *reinterpret_cast<float*>(a_lo + o1) = tf32_round(v.y - hi_);
        }
        fence_proxy_async_smem();   // generic smem writes -> tensor-core (async proxy) reads
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        // ---- 3-term TF32 product on the tensor cores ----
        if (warp == 0 && elect_one()) {
            // small cross terms first, the large hi*hi products last: the tensor-core
            // accumulator rounds toward zero, so each full-magnitude accumulation costs
            // up to an ulp; this order has 4 of them per output instead of 12
            int first = 1;
            for (int kb = 0; kb < TC_KBLK; ++kb)
                for (int kk = 0; kk < 4; ++kk) {
                    const uint32_t ka = (uint32_t)kb * TC_M * TC_ROWB + kk * 32u;
                    const uint32_t kbb = (uint32_t)kb * TC_N * TC_ROWB + kk * 32u;
                    tc_mma(tmem, sw128_desc(smem_u32(a_hi) + ka), sw128_desc(smem_u32(b_lo) + kbb), idesc,
                           first ? 0 : 1);
                    tc_mma(tmem, sw128_desc(smem_u32(a_lo) + ka), sw128_desc(smem_u32(b_hi) + kbb), idesc, 1);
                    first = 0;
                }
            for (int kb = 0; kb < TC_KBLK; ++kb)
                for (int kk = 0; kk < 4; ++kk) {
                    const uint32_t ka = (uint32_t)kb * TC_M * TC_ROWB + kk * 32u;
                    const uint32_t kbb = (uint32_t)kb * TC_N * TC_ROWB + kk * 32u;
                    tc_mma(tmem, sw128_desc(smem_u32(a_hi) + ka), sw128_desc(smem_u32(b_hi) + kbb), idesc, 1);
                }
            tc_commit(&bar);
        }
        if (!mbar_wait_bounded(&bar, phase, a.err)) s_abort = 1;
        phase ^= 1u;
        tc_fence_after();
        __syncthreads();
        if (s_abort) break;
        // ---- epilogue: TMEM lanes -> amplitudes ----
        {
            const int row = warp * 32 + lane;
            const long long r = r0 + row;
            float v[2][32];
            tc_ld32(tmem + ((uint32_t)(warp * 32) << 16) + 0u, v[0]);
            tc_ld32(tmem + ((uint32_t)(warp * 32) << 16) + 32u, v[1]);
            if (r < total_rows) {
                const long long item = r >> (a.n - kq);
                long long x = r & (rows_per_item - 1);
                for (int j = 0; j < kq; ++j) x = ((x >> qs[j]) << (qs[j] + 1)) | (x & ((1ll << qs[j]) - 1));
                float2* psi = a.state + a.item_off[item];
#pragma unroll
                for (int jj = 0; jj < 32; ++jj) {
                    if (jj < D) {
                        long long y = x;
                        for (int j = 0; j < kq; ++j)
                            if ((jj >> j) & 1) y |= 1ll << qs[j];
                        const int c = 2 * jj;
                        psi[y] = make_float2(v[c >> 5][c & 31], v[(c + 1) >> 5][(c + 1) & 31]);
                    }
                }
            }
        }
        tc_fence_before();
        __syncthreads();
    }
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_N)
                     : "memory");
}

}  // namespace tcng

using namespace tcng;

extern "C" tcng_status tcng_apply_shared_unitary(tcng_state* st, const int* qubits, int k,
                                                 const double* U, void* stream) {
    if (!st || !qubits || !U) return fail(TCNG_EINVAL, "null argument");
    if (k < 1 || k > 5) return fail(TCNG_EINVAL, "k must be 1..5");
    if (st->dt != TCNG_C64) return fail(TCNG_EUNSUPPORTED, "shared-unitary apply needs complex64 states");
    std::lock_guard<std::mutex> lk(g_mu);
    for (auto& kv : st->groups) {
        const int n = kv.first;
        for (int j = 0; j < k; ++j) {
            if (qubits[j] < 0 || qubits[j] >= n) return fail(TCNG_EINVAL, "qubit out of range");
            for (int i = 0; i < j; ++i)
                if (qubits[i] == qubits[j]) return fail(TCNG_EINVAL, "repeated qubit");
        }
    }
    // U in the ascending local order of the kernel: bit j <-> j-th smallest qubit
    int sorted[5];
    for (int j = 0; j < k; ++j) sorted[j] = qubits[j];
    std::sort(sorted, sorted + k);
    int pos_of[5];   // position of gate qubit j (q[0] most significant) in ascending order
    for (int j = 0; j < k; ++j)
        for (int i = 0; i < k; ++i)
            if (sorted[i] == qubits[j]) pos_of[j] = i;
    const int D = 1 << k;
    auto asc = [&](int r) {   // gate-local index -> ascending-local index
        int o = 0;
        for (int j = 0; j < k; ++j)
            if ((r >> (k - 1 - j)) & 1) o |= 1 << pos_of[j];
        return o;
    };
    std::vector<double> Ur(D * D), Ui(D * D);
    for (int r = 0; r < D; ++r)
        for (int c = 0; c < D; ++c) {
            Ur[asc(r) * D + asc(c)] = U[2 * (r * D + c)];
            Ui[asc(r) * D + asc(c)] = U[2 * (r * D + c) + 1];
        }
    // W^T (row = output column nn = 2j+b, col = kk = 2l+a), split into TF32 hi/lo
    std::vector<float> w(2 * TC_N * TC_K, 0.f);
    auto tf32 = [](float x) {
        uint32_t u;
        std::memcpy(&u, &x, 4);
        u += 0xfffu + ((u >> 13) & 1u);
        u &= 0xffffe000u;
        float y;
        std::memcpy(&y, &u, 4);
        return y;
    };
    for (int j = 0; j < D; ++j)
        for (int l = 0; l < D; ++l) {
            const double re = Ur[j * D + l], im = Ui[j * D + l];
            const double W[2][2] = {{re, im}, {-im, re}};   // W[a][b] = W(2l+a, 2j+b)
            for (int a2 = 0; a2 < 2; ++a2)
                for (int b2 = 0; b2 < 2; ++b2) {
                    const int nn = 2 * j + b2, kk = 2 * l + a2;
                    const float f = (float)W[a2][b2];
                    const float h = tf32(f);
                    w[nn * TC_K + kk] = h;
                    w[TC_N * TC_K + nn * TC_K + kk] = tf32((float)(W[a2][b2] - (double)h));
                }
        }
    DeviceCtx& c = ctx();
    float* dw = static_cast<float*>(c.scratch("tc_w", sizeof(float) * w.size()));
    if (!dw) return fail(TCNG_ENOMEM, "unitary scratch");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemcpyAsync(dw, w.data(), sizeof(float) * w.size(), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e, "upload");
    e = cudaStreamSynchronize(s);   // w is a host temporary
    if (e != cudaSuccess) return cuda_fail(e, "upload");
    const size_t smem = 2 * TC_A_BYTES + 2 * TC_B_BYTES + 1024;
    static bool attr[kMaxDeviceSlots] = {};   // the attribute is per device
    const int d = device_slot();
    if (!attr[d]) {
        e = cudaFuncSetAttribute(shared_unitary_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return cuda_fail(e, "smem attribute");
        attr[d] = true;
    }
    for (auto& kv : st->groups) {
        TcArgs a{};
        a.state = static_cast<float2*>(st->buf);
        a.item_off = kv.second.d_off;
        a.items = (int)kv.second.items.size();
        a.n = kv.first;
        a.k = k;
        a.qmask = 0;
        for (int j = 0; j < k; ++j) a.qmask |= 1u << qubits[j];
        a.w = dw;
        a.err = c.err;
        const long long rows = (1ll << (a.n - k)) * a.items;
        const long long tiles = (rows + TC_M - 1) / TC_M;
        const int grid = (int)std::max<long long>(1, std::min<long long>(tiles, 2ll * num_sms()));
        ProfScope ps("shared_unitary_tc", s);
        shared_unitary_tc_kernel<<<grid, 128, smem, s>>>(a);
        count_launch();
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "tensor-core kernel");
    }
    return TCNG_OK;
}
