// Warm-start MLP: forward, loss and backward with BF16 operands, FP32 accumulation.
//
// No counterpart in the paper: a small network maps Hamiltonian couplings to
// initial ansatz angles.  y = W3 relu(W2 relu(W1 x + b1) + b2) + b3; the loss
// is periodic in the angle, L = sum mask * 2 (1 - cos(y - target)) / sum mask.
//
// Every GEMM goes through one tiled kernel: operand tiles are read from FP32
// (with arbitrary strides, so transposes are free), optionally passed through
// relu, rounded to BF16 (round to nearest even) into 128-byte-swizzled shared
// memory, multiplied by tcgen05 kind::f16 MMAs into an FP32 TMEM accumulator,
// and written back through an epilogue (bias add, or multiply by the relu mask
// of a saved pre-activation).  Column sums (bias gradients) run in a fixed order.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "capi_internal.hpp"
#include "device.cuh"
#include "tc.cuh"

namespace tcng {

struct GemmArgs {
    int M, N, K;
    const float* A;               // A(i,k) = A[i*a_i + k*a_k]
    long long a_i, a_k;
    const float* B;               // B(k,j) = B[k*b_k + j*b_j]
    long long b_k, b_j;
    float* C;                     // C(i,j) = C[i*ldc + j]
    long long ldc;
    int relu_a;                   // 1: A <- max(A, 0) before rounding
    const float* bias;            // epilogue: C += bias[j]
    const float* gate;            // epilogue: C *= (gate[i*ldc + j] > 0)
    int kslice;                   // split K: CTA z takes K range [z kslice, (z+1) kslice) ...
    float* part;                  // ... and writes raw sums to part[z][i][j] (no epilogue)
};

constexpr int GT_M = 128, GT_N = 64, GT_K = 64;   // CTA tile; K chunk = one 128-byte swizzle row
constexpr uint32_t GT_A_BYTES = GT_M * GT_K * 2, GT_B_BYTES = GT_N * GT_K * 2;

// Instruction descriptor, kind::f16 with BF16 A and B, FP32 D, both K-major.
__host__ __device__ constexpr uint32_t bf16_idesc(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
// D (TMEM) += A (shared-memory descriptor) * B (shared-memory descriptor)
__device__ __forceinline__ void mma_bf16_ss(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, int accum) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accum)
        : "memory");
}

// C tile [128 x 64] of one CTA: 128 threads convert their share of each K chunk
// of A (128 rows) and B (64 columns) from FP32 to BF16 into 128-byte-swizzled
// K-major shared memory; one thread issues four kind::f16 MMAs (M=128, N=64,
// K=16) into a 64-column TMEM accumulator; each warp reads its 32 TMEM lanes
// back for the epilogue.
__global__ void __launch_bounds__(128) gemm_bf16_kernel(GemmArgs g) {
    __shared__ __align__(1024) unsigned char sa[GT_A_BYTES];
    __shared__ __align__(1024) unsigned char sb[GT_B_BYTES];
    __shared__ uint64_t mma_bar;
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int i0 = blockIdx.y * GT_M, j0 = blockIdx.x * GT_N;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_base)),
                     "r"(64)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        mbar_init(&mma_bar, 1);
        fence_mbar_init();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;
    constexpr uint32_t idesc = bf16_idesc(GT_M, GT_N);
    uint32_t chunk = 0;
    bool ok = true;
    const int kb = g.part ? (int)blockIdx.z * g.kslice : 0;
    const int ke = g.part ? min(g.K, kb + g.kslice) : g.K;
    for (int k0 = kb; k0 < ke; k0 += GT_K, ++chunk) {
        // the previous chunk's MMAs have read the tiles
        if (chunk > 0 && !mbar_wait_bounded(&mma_bar, (chunk - 1) & 1u, nullptr)) ok = false;
        for (int e = tid; e < GT_M * GT_K; e += blockDim.x) {
            const int r = e / GT_K, c = e % GT_K;
            const int i = i0 + r, k = k0 + c;
            float v = 0.f;
            if (i < g.M && k < ke) {
                v = g.A[i * g.a_i + k * g.a_k];
                if (g.relu_a) v = fmaxf(v, 0.f);
            }
            *reinterpret_cast<__nv_bfloat16*>(sa + sw128_offset_h(r, c)) = __float2bfloat16_rn(v);
        }
        for (int e = tid; e < GT_N * GT_K; e += blockDim.x) {
            const int r = e / GT_K, c = e % GT_K;   // row r = output column j0 + r, K-major
            const int k = k0 + c, j = j0 + r;
            float v = 0.f;
            if (k < ke && j < g.N) v = g.B[k * g.b_k + j * g.b_j];
            *reinterpret_cast<__nv_bfloat16*>(sb + sw128_offset_h(r, c)) = __float2bfloat16_rn(v);
        }
        fence_proxy_async_smem();   // generic-proxy writes before the tensor core reads them
        tc_fence_before();
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
            const uint64_t da = sw128_desc(smem_u32(sa)), db = sw128_desc(smem_u32(sb));
#pragma unroll
            for (int kk = 0; kk < GT_K / 16; ++kk)   // +32 bytes per K step: +2 in the start field
                mma_bf16_ss(tmem, da + 2u * kk, db + 2u * kk, idesc, (k0 > kb || kk > 0) ? 1 : 0);
            tc_commit(&mma_bar);
        }
    }
    if (chunk > 0 && !mbar_wait_bounded(&mma_bar, (chunk - 1) & 1u, nullptr)) ok = false;
    tc_fence_after();
    const int i = i0 + 32 * warp + lane;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        float y[32];
        tc_ld32(tmem + ((uint32_t)(32 * warp) << 16) + 32u * h, y);
        if (i < g.M && ok) {
#pragma unroll
            for (int c = 0; c < 32; ++c) {
                const int j = j0 + 32 * h + c;
                if (j >= g.N) break;
                float v = chunk > 0 ? y[c] : 0.f;
                if (g.part) {   // raw partial sum of this K slice
                    g.part[((long long)blockIdx.z * g.M + i) * g.N + j] = v;
                    continue;
                }
                if (g.bias) v += g.bias[j];
                if (g.gate && !(g.gate[i * g.ldc + j] > 0.f)) v = 0.f;
                g.C[i * g.ldc + j] = v;
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(64) : "memory");
}

// C = sum over the K slices in order (+ the epilogue of the unsplit GEMM).
__global__ void splitk_reduce_kernel(GemmArgs g, int splits) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)g.M * g.N) return;
    const int i = (int)(e / g.N), j = (int)(e % g.N);
    float v = 0.f;
    for (int z = 0; z < splits; ++z) v += g.part[(long long)z * g.M * g.N + e];
    if (g.bias) v += g.bias[j];
    if (g.gate && !(g.gate[i * g.ldc + j] > 0.f)) v = 0.f;
    g.C[i * g.ldc + j] = v;
}

// dy = mask * 2 sin(y - t) / sum(mask); loss = sum mask * 2 (1 - cos(y - t)) / sum(mask).
// Three steps, each in a fixed order (deterministic): per-CTA FP64 sums of the
// mask and the loss terms, their sum over CTAs (and 1/sum(mask)), then dy.
constexpr int kLossBlocks = 296;
__global__ void __launch_bounds__(256) loss_partial_kernel(const float* __restrict__ y, const float* __restrict__ t,
                                                           const float* __restrict__ mask, long long n,
                                                           double* __restrict__ part) {
    __shared__ double s_m[256], s_l[256];
    double msum = 0, lsum = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double m = mask[i];
        msum += m;
        lsum += m * 2.0 * (1.0 - cos((double)y[i] - (double)t[i]));
    }
    s_m[threadIdx.x] = msum;
    s_l[threadIdx.x] = lsum;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            s_m[threadIdx.x] += s_m[threadIdx.x + o];
            s_l[threadIdx.x] += s_l[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = s_m[0];
        part[2 * blockIdx.x + 1] = s_l[0];
    }
}
__global__ void loss_final_kernel(const double* __restrict__ part, int nb, double* __restrict__ inv,
                                  double* __restrict__ loss) {
    double m = 0, l = 0;
    for (int b = 0; b < nb; ++b) {
        m += part[2 * b];
        l += part[2 * b + 1];
    }
    const double iv = m > 0 ? 1.0 / m : 0.0;
    *inv = iv;
    *loss = l * iv;
}
__global__ void dy_kernel(const float* __restrict__ y, const float* __restrict__ t, const float* __restrict__ mask,
                          long long n, const double* __restrict__ inv, float* __restrict__ dy) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    dy[i] = (float)(mask[i] * 2.0 * sin((double)y[i] - (double)t[i]) * *inv);
}

// out[j] = sum_i X[i*cols + j]: row blocks of kColRows rows summed per column,
// then the blocks in order.
constexpr int kColRows = 128;
__global__ void colsum_partial_kernel(const float* __restrict__ X, int rows, int cols, float* __restrict__ part) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= cols) return;
    const int r0 = blockIdx.y * kColRows, r1 = min(rows, r0 + kColRows);
    float s = 0.f;
    for (int i = r0; i < r1; ++i) s += X[(long long)i * cols + j];
    part[(long long)blockIdx.y * cols + j] = s;
}
__global__ void colsum_final_kernel(const float* __restrict__ part, int nrb, int cols, float* __restrict__ out) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= cols) return;
    float s = 0.f;
    for (int b = 0; b < nrb; ++b) s += part[(long long)b * cols + j];
    out[j] = s;
}

// One GEMM.  Few output tiles over a long K (the weight gradients, K = batch)
// split K over more CTAs into a scratch of partial sums (part: room for
// part_floats floats), then add the slices in a fixed order (deterministic).
static cudaError_t gemm(GemmArgs g, cudaStream_t s, float* part = nullptr, size_t part_floats = 0) {
    dim3 grid((g.N + GT_N - 1) / GT_N, (g.M + GT_M - 1) / GT_M);
    const int tiles = (int)(grid.x * grid.y);
    int splits = 1;
    if (part && g.K >= 4 * GT_K && tiles < num_sms()) {
        splits = std::min((g.K + GT_K - 1) / GT_K, std::max(1, 2 * num_sms() / tiles));
        while (splits > 1 && (size_t)splits * g.M * g.N > part_floats) --splits;
    }
    if (splits > 1) {
        g.kslice = ((g.K + splits - 1) / splits + GT_K - 1) / GT_K * GT_K;
        splits = (g.K + g.kslice - 1) / g.kslice;
        g.part = part;
        grid.z = (unsigned)splits;
        gemm_bf16_kernel<<<grid, 128, 0, s>>>(g);
        count_launch();
        const long long n = (long long)g.M * g.N;
        splitk_reduce_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(g, splits);
        count_launch();
        return cudaGetLastError();
    }
    g.part = nullptr;
    gemm_bf16_kernel<<<grid, 128, 0, s>>>(g);
    count_launch();
    return cudaGetLastError();
}

static GemmArgs mk(int M, int N, int K, const float* A, long long ai, long long ak, const float* B,
                   long long bk, long long bj, float* C, long long ldc) {
    GemmArgs g{};
    g.M = M; g.N = N; g.K = K;
    g.A = A; g.a_i = ai; g.a_k = ak;
    g.B = B; g.b_k = bk; g.b_j = bj;
    g.C = C; g.ldc = ldc;
    return g;
}

}  // namespace tcng

using namespace tcng;

extern "C" {

tcng_status tcng_mlp_forward(const float* x, int N, int F, int H, int O, const float* w1,
                             const float* b1, const float* w2, const float* b2, const float* w3,
                             const float* b3, float* act, float* y, void* stream) {
    if (!x || !w1 || !b1 || !w2 || !b2 || !w3 || !b3 || !act || !y) return fail(TCNG_EINVAL, "null argument");
    if (N < 1 || F < 1 || H < 1 || O < 1) return fail(TCNG_EINVAL, "sizes must be positive");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    float* z1 = act;
    float* z2 = act + (long long)N * H;
    ProfScope ps("mlp_forward", s);
    GemmArgs g = mk(N, H, F, x, F, 1, w1, H, 1, z1, H);
    g.bias = b1;
    cudaError_t e = gemm(g, s);
    if (e == cudaSuccess) {
        g = mk(N, H, H, z1, H, 1, w2, H, 1, z2, H);
        g.relu_a = 1;
        g.bias = b2;
        e = gemm(g, s);
    }
    if (e == cudaSuccess) {
        g = mk(N, O, H, z2, H, 1, w3, O, 1, y, O);
        g.relu_a = 1;
        g.bias = b3;
        e = gemm(g, s);
    }
    if (e != cudaSuccess) return cuda_fail(e, "mlp forward");
    return TCNG_OK;
}

tcng_status tcng_mlp_backward(const float* x, int N, int F, int H, int O, const float* w1,
                              const float* w2, const float* w3, const float* act, const float* y,
                              const float* target, const float* mask, float* grads, double* loss_dev,
                              void* stream) {
    if (!x || !w1 || !w2 || !w3 || !act || !y || !target || !mask || !grads || !loss_dev)
        return fail(TCNG_EINVAL, "null argument");
    if (N < 1 || F < 1 || H < 1 || O < 1) return fail(TCNG_EINVAL, "sizes must be positive");
    std::lock_guard<std::mutex> lk(g_mu);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    DeviceCtx& c = ctx();
    // dy, dz2, dz1; split-K partial sums; column-sum partials; loss partials
    const size_t part_floats = (size_t)1 << 22;
    const int nrb = (N + kColRows - 1) / kColRows;
    const size_t col_floats = (size_t)nrb * std::max(H, O);
    const size_t floats = (size_t)N * O + 2 * (size_t)N * H + part_floats + col_floats + 4 * (kLossBlocks + 2);
    float* tmp = static_cast<float*>(c.scratch("mlp_tmp", sizeof(float) * floats));
    if (!tmp) return fail(TCNG_ENOMEM, "mlp scratch");
    float* dy = tmp;
    float* dz2 = dy + (size_t)N * O;
    float* dz1 = dz2 + (size_t)N * H;
    float* part = dz1 + (size_t)N * H;
    float* colp = part + part_floats;
    double* lossp = reinterpret_cast<double*>(colp + col_floats + ((reinterpret_cast<uintptr_t>(colp + col_floats) & 7) ? 1 : 0));
    const float* z1 = act;
    const float* z2 = act + (long long)N * H;
    float* gw1 = grads;
    float* gb1 = gw1 + (size_t)F * H;
    float* gw2 = gb1 + H;
    float* gb2 = gw2 + (size_t)H * H;
    float* gw3 = gb2 + H;
    float* gb3 = gw3 + (size_t)H * O;
    ProfScope ps("mlp_backward", s);
    const long long ny = (long long)N * O;
    loss_partial_kernel<<<kLossBlocks, 256, 0, s>>>(y, target, mask, ny, lossp);
    loss_final_kernel<<<1, 1, 0, s>>>(lossp, kLossBlocks, lossp + 2 * kLossBlocks, loss_dev);
    dy_kernel<<<(unsigned)((ny + 255) / 256), 256, 0, s>>>(y, target, mask, ny, lossp + 2 * kLossBlocks, dy);
    count_launch();
    count_launch();
    count_launch();
    cudaError_t e = cudaGetLastError();
    auto cs = [&](const float* X, int rows, int cols, float* out) {
        colsum_partial_kernel<<<dim3((cols + 255) / 256, nrb), 256, 0, s>>>(X, rows, cols, colp);
        colsum_final_kernel<<<(cols + 255) / 256, 256, 0, s>>>(colp, nrb, cols, out);
        count_launch();
        count_launch();
    };
    if (e == cudaSuccess) {   // dW3 = relu(z2)^T dy ; db3 = colsum(dy)
        GemmArgs g = mk(H, O, N, z2, 1, H, dy, O, 1, gw3, O);
        g.relu_a = 1;
        e = gemm(g, s, part, part_floats);
        cs(dy, N, O, gb3);
    }
    if (e == cudaSuccess) {   // dz2 = (dy W3^T) * (z2 > 0)
        GemmArgs g = mk(N, H, O, dy, O, 1, w3, 1, O, dz2, H);
        g.gate = z2;
        e = gemm(g, s);
    }
    if (e == cudaSuccess) {   // dW2 = relu(z1)^T dz2 ; db2
        GemmArgs g = mk(H, H, N, z1, 1, H, dz2, H, 1, gw2, H);
        g.relu_a = 1;
        e = gemm(g, s, part, part_floats);
        cs(dz2, N, H, gb2);
    }
    if (e == cudaSuccess) {   // dz1 = (dz2 W2^T) * (z1 > 0)
        GemmArgs g = mk(N, H, H, dz2, H, 1, w2, 1, H, dz1, H);
        g.gate = z1;
        e = gemm(g, s);
    }
    if (e == cudaSuccess) {   // dW1 = x^T dz1 ; db1
        GemmArgs g = mk(F, H, N, x, 1, F, dz1, H, 1, gw1, H);
        e = gemm(g, s, part, part_floats);
        cs(dz1, N, H, gb1);
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "mlp backward");
    return TCNG_OK;
}

}  // extern "C"
