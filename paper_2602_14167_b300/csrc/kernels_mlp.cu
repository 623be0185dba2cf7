// Warm-start MLP: forward, loss and backward with BF16 operands, FP32 accumulation.
//
// No counterpart in the paper: a small network maps Hamiltonian couplings to
// initial ansatz angles.  y = W3 relu(W2 relu(W1 x + b1) + b2) + b3; the loss
// is periodic in the angle, L = sum mask * 2 (1 - cos(y - target)) / sum mask.
//
// Every GEMM goes through one tiled kernel: operand tiles are read from FP32
// (with arbitrary strides, so transposes are free), optionally passed through
// relu, rounded to BF16 (round to nearest even) into shared memory, multiplied
// on the tensor cores with FP32 accumulators (16x16x16 warp tiles), and written
// back through an epilogue (bias add, or multiply by the relu mask of a saved
// pre-activation).  Column sums (bias gradients) run in a fixed order.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <mma.h>

#include <algorithm>

#include "capi_internal.hpp"

namespace tcng {

using namespace nvcuda;

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
};

constexpr int GT_M = 64, GT_N = 64, GT_K = 32;

__global__ void __launch_bounds__(128) gemm_bf16_kernel(GemmArgs g) {
    __shared__ __align__(32) __nv_bfloat16 As[GT_M][GT_K + 8];
    __shared__ __align__(32) __nv_bfloat16 Bs[GT_K][GT_N + 8];
    __shared__ __align__(32) float Cs[GT_M][GT_N + 4];
    const int tid = threadIdx.x, warp = tid >> 5;
    const int i0 = blockIdx.y * GT_M, j0 = blockIdx.x * GT_N;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;   // 2x2 warps, 32x32 each
    wmma::fragment<wmma::accumulator, 16, 16, 16, float> acc[2][2];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) wmma::fill_fragment(acc[a][b], 0.0f);
    for (int k0 = 0; k0 < g.K; k0 += GT_K) {
        for (int e = tid; e < GT_M * GT_K; e += blockDim.x) {
            const int r = e / GT_K, c = e % GT_K;
            const int i = i0 + r, k = k0 + c;
            float v = 0.f;
            if (i < g.M && k < g.K) {
                v = g.A[i * g.a_i + k * g.a_k];
                if (g.relu_a) v = fmaxf(v, 0.f);
            }
            As[r][c] = __float2bfloat16_rn(v);
        }
        for (int e = tid; e < GT_K * GT_N; e += blockDim.x) {
            const int r = e / GT_N, c = e % GT_N;
            const int k = k0 + r, j = j0 + c;
            float v = 0.f;
            if (k < g.K && j < g.N) v = g.B[k * g.b_k + j * g.b_j];
            Bs[r][c] = __float2bfloat16_rn(v);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GT_K; kk += 16) {
            wmma::fragment<wmma::matrix_a, 16, 16, 16, __nv_bfloat16, wmma::row_major> fa[2];
            wmma::fragment<wmma::matrix_b, 16, 16, 16, __nv_bfloat16, wmma::row_major> fb[2];
#pragma unroll
            for (int a = 0; a < 2; ++a) wmma::load_matrix_sync(fa[a], &As[wm + 16 * a][kk], GT_K + 8);
#pragma unroll
            for (int b = 0; b < 2; ++b) wmma::load_matrix_sync(fb[b], &Bs[kk][wn + 16 * b], GT_N + 8);
#pragma unroll
            for (int a = 0; a < 2; ++a)
#pragma unroll
                for (int b = 0; b < 2; ++b) wmma::mma_sync(acc[a][b], fa[a], fb[b], acc[a][b]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b)
            wmma::store_matrix_sync(&Cs[wm + 16 * a][wn + 16 * b], acc[a][b], GT_N + 4, wmma::mem_row_major);
    __syncthreads();
    for (int e = tid; e < GT_M * GT_N; e += blockDim.x) {
        const int r = e / GT_N, c = e % GT_N;
        const int i = i0 + r, j = j0 + c;
        if (i >= g.M || j >= g.N) continue;
        float v = Cs[r][c];
        if (g.bias) v += g.bias[j];
        if (g.gate && !(g.gate[i * g.ldc + j] > 0.f)) v = 0.f;
        g.C[i * g.ldc + j] = v;
    }
}

// dy = mask * 2 sin(y - t) / sum(mask); loss = sum mask * 2 (1 - cos(y - t)) / sum(mask).
// One CTA, fixed-order reduction (deterministic).
__global__ void periodic_loss_kernel(const float* __restrict__ y, const float* __restrict__ t,
                                     const float* __restrict__ mask, long long n, float* __restrict__ dy,
                                     double* __restrict__ loss) {
    __shared__ double s_m[1024], s_l[1024];
    double msum = 0, lsum = 0;
    for (long long i = threadIdx.x; i < n; i += blockDim.x) {
        const double m = mask[i];
        msum += m;
        lsum += m * 2.0 * (1.0 - cos((double)y[i] - (double)t[i]));
    }
    s_m[threadIdx.x] = msum;
    s_l[threadIdx.x] = lsum;
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0, b = 0;
        for (int k = 0; k < (int)blockDim.x; ++k) {
            a += s_m[k];
            b += s_l[k];
        }
        s_m[0] = a;
        s_l[0] = b;
    }
    __syncthreads();
    const double inv = s_m[0] > 0 ? 1.0 / s_m[0] : 0.0;
    if (threadIdx.x == 0) *loss = s_l[0] * inv;
    for (long long i = threadIdx.x; i < n; i += blockDim.x)
        dy[i] = (float)(mask[i] * 2.0 * sin((double)y[i] - (double)t[i]) * inv);
}

// out[j] = sum_i X[i*ld + j] over i in order.
__global__ void colsum_kernel(const float* __restrict__ X, int rows, int cols, float* __restrict__ out) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= cols) return;
    float s = 0.f;
    for (int i = 0; i < rows; ++i) s += X[(long long)i * cols + j];
    out[j] = s;
}

static cudaError_t gemm(const GemmArgs& g, cudaStream_t s) {
    dim3 grid((g.N + GT_N - 1) / GT_N, (g.M + GT_M - 1) / GT_M);
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
    float* tmp = static_cast<float*>(c.scratch("mlp_tmp", sizeof(float) * ((size_t)N * O + 2 * (size_t)N * H)));
    if (!tmp) return fail(TCNG_ENOMEM, "mlp scratch");
    float* dy = tmp;
    float* dz2 = dy + (size_t)N * O;
    float* dz1 = dz2 + (size_t)N * H;
    const float* z1 = act;
    const float* z2 = act + (long long)N * H;
    float* gw1 = grads;
    float* gb1 = gw1 + (size_t)F * H;
    float* gw2 = gb1 + H;
    float* gb2 = gw2 + (size_t)H * H;
    float* gw3 = gb2 + H;
    float* gb3 = gw3 + (size_t)H * O;
    ProfScope ps("mlp_backward", s);
    periodic_loss_kernel<<<1, 1024, 0, s>>>(y, target, mask, (long long)N * O, dy, loss_dev);
    count_launch();
    cudaError_t e = cudaGetLastError();
    auto cs = [&](const float* X, int rows, int cols, float* out) {
        colsum_kernel<<<(cols + 255) / 256, 256, 0, s>>>(X, rows, cols, out);
        count_launch();
    };
    if (e == cudaSuccess) {   // dW3 = relu(z2)^T dy ; db3 = colsum(dy)
        GemmArgs g = mk(H, O, N, z2, 1, H, dy, O, 1, gw3, O);
        g.relu_a = 1;
        e = gemm(g, s);
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
        e = gemm(g, s);
        cs(dz2, N, H, gb2);
    }
    if (e == cudaSuccess) {   // dz1 = (dz2 W2^T) * (z1 > 0)
        GemmArgs g = mk(N, H, H, dz2, H, 1, w2, 1, H, dz1, H);
        g.gate = z1;
        e = gemm(g, s);
    }
    if (e == cudaSuccess) {   // dW1 = x^T dz1 ; db1
        GemmArgs g = mk(F, H, N, x, 1, F, dz1, H, 1, gw1, H);
        e = gemm(g, s);
        cs(dz1, N, H, gb1);
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "mlp backward");
    return TCNG_OK;
}

}  // extern "C"
