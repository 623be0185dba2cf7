// Pauli strings with more X/Y factors than a tile can gather (Sec. I.B,
// expectation_ps takes any string), e.g. the parity <X X ... X>.
//
// <P> = sum_x Re( i^{#Y} conj(psi[x ^ m]) (-1)^{popc(x & z)} psi[x] ).  The terms
// of x and x ^ m are complex conjugates (P is Hermitian), so the sum runs over
// the pairs with bit h of x clear (h = the highest bit of m) and doubles the
// real part: one read of the state per string, straight from global memory
// (x and x ^ m lie in the same aligned 32-element blocks up to a permutation, so
// a warp's two loads are coalesced).  Each thread takes four consecutive pair
// indices per step (eight loads in flight); FP32 (complex64) products fold into
// FP64 every 64 steps; CTAs reduce in a fixed order and write one partial sum
// each, in the layout of the tile passes' partial sums.
#include <cuda_runtime.h>

#include "capi_internal.hpp"
#include "device.cuh"

namespace tcng {
namespace {

constexpr int kWideThreads = 1024;
constexpr int kWideUnroll = 4;

template <typename C>
__global__ void __launch_bounds__(kWideThreads) expect_wide_kernel(const C* __restrict__ state,
                                                                  const long long* __restrict__ item_off, int n,
                                                                  unsigned long long xm, unsigned long long zm,
                                                                  int ny, int out, double* __restrict__ partial,
                                                                  int n_out) {
    using R = typename Real<C>::T;
    __shared__ double red[kWideThreads];
    const int item = blockIdx.y;
    const C* __restrict__ psi = state + item_off[item];
    const int h = 63 - __clzll((long long)xm);
    const unsigned long long lowmask = (1ull << h) - 1;
    const unsigned long long pairs = 1ull << (n - 1);
    const unsigned long long step = (unsigned long long)gridDim.x * kWideThreads * kWideUnroll;
    double acc = 0.0;
    R part = 0;
    int cnt = 0;
    for (unsigned long long j0 = ((unsigned long long)blockIdx.x * kWideThreads + threadIdx.x) * kWideUnroll;
         j0 < pairs; j0 += step) {
        C a[kWideUnroll], b[kWideUnroll];
        unsigned long long xs[kWideUnroll];
#pragma unroll
        for (int u = 0; u < kWideUnroll; ++u) {
            const unsigned long long j = j0 + u;   // pairs is a multiple of kWideUnroll for n >= 3
            const unsigned long long x = ((j & ~lowmask) << 1) | (j & lowmask);
            xs[u] = x;
            if (j < pairs) {
                a[u] = psi[x];
                b[u] = psi[x ^ xm];
            } else {
                a[u] = C{0, 0};
                b[u] = C{0, 0};
            }
        }
#pragma unroll
        for (int u = 0; u < kWideUnroll; ++u) {
            // w = conj(b) a; Re(i^ny w)
            const R wr = b[u].x * a[u].x + b[u].y * a[u].y;
            const R wi = b[u].x * a[u].y - b[u].y * a[u].x;
            R v = ny == 0 ? wr : (ny == 1 ? -wi : (ny == 2 ? -wr : wi));
            if (__popcll(xs[u] & zm) & 1) v = -v;
            part += v;
        }
        if (++cnt == 64) {
            acc += (double)part;
            part = 0;
            cnt = 0;
        }
    }
    acc += (double)part;
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = kWideThreads / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[((long long)item * n_out + out) * gridDim.x + blockIdx.x] = 2.0 * red[0];
}

}  // namespace

template <typename C>
cudaError_t launch_expect_wide(const C* state, const long long* item_off, int items, int n, const tcng_pauli& t,
                               int out, double* partial, int n_out, int nblk, cudaStream_t s) {
    const int ny = __builtin_popcountll(t.xmask & t.zmask) & 3;
    dim3 grid((unsigned)nblk, (unsigned)items);
    expect_wide_kernel<C><<<grid, kWideThreads, 0, s>>>(state, item_off, n, t.xmask, t.zmask, ny, out, partial,
                                                        n_out);
    count_launch();
    return cudaGetLastError();
}

template cudaError_t launch_expect_wide<float2>(const float2*, const long long*, int, int, const tcng_pauli&, int,
                                                double*, int, int, cudaStream_t);
template cudaError_t launch_expect_wide<double2>(const double2*, const long long*, int, int, const tcng_pauli&,
                                                 int, double*, int, int, cudaStream_t);

}  // namespace tcng
