// Computational-basis probabilities of a subset of qubits (tcng_marginal_probs).
//
// p_b(k) = sum over x whose bits at qubits q_0..q_{K-1} spell k of |psi_b(x)|^2,
// k = sum_j bit(x, q_j) << (K-1-j): the diagonal of the reduced density matrix
// of those qubits, which the paper's QML pipeline reads out as class
// probabilities (Sec. VII.B, reduced_density_matrix over the first 7 qubits),
// and the Born probabilities of measuring those qubits.
//
// Layout: a block of 256 threads = NBt bin lanes x JL index lanes (NBt = min(2^K,
// 256)); thread (bin lane r, index lane l) sums |psi|^2 over the amplitudes of
// bins r, r + NBt, ... whose free-bit index j = l, l + JL, ... lies in the
// block's split of the free index range.  The free-bit index is advanced with
// the masked increment x' = ((x | ~free) + pdep(JL)) & free, so no bit
// deposit runs per element.  Bin-lane-fastest threads read consecutive
// addresses when the kept qubits are the low ones (the QML readout); with high
// kept qubits a warp reads NBt contiguous runs.  Per-thread FP32 partial sums
// (complex64) fold into FP64 every 256 elements; lanes of one bin then add in a
// fixed order, and splits add in a fixed order in a second kernel, so results
// are bitwise reproducible.
#include <cuda_runtime.h>

#include "capi_internal.hpp"
#include "device.cuh"

namespace tcng {

namespace {

constexpr int kMpThreads = 256;

struct MarginalArgs {
    const void* state;
    const long long* item_off;   // element offset of each item
    int items;
    int n;
    int k;                       // kept qubits
    int q[10];                   // kept qubits, q[0] -> most significant bit of the bin
    unsigned long long free_mask;   // index bits not kept
    int splits;
    double* out;                 // splits == 1: [items][2^k]; else partial [items][2^k][splits]
    int out_stride;              // bins per item in out
};

__device__ __forceinline__ unsigned long long pdep64(unsigned long long v, unsigned long long mask) {
    unsigned long long r = 0;
    for (unsigned long long bb = 1; mask; bb <<= 1) {
        const unsigned long long low = mask & (~mask + 1);
        if (v & bb) r |= low;
        mask ^= low;
    }
    return r;
}

template <typename C>
__global__ void __launch_bounds__(kMpThreads) marginal_kernel(MarginalArgs a) {
    using R = typename Real<C>::T;
    const int item = blockIdx.y;
    const int split = blockIdx.x;
    const int tid = threadIdx.x;
    const int nb = 1 << a.k;
    const int nbt = nb < kMpThreads ? nb : kMpThreads;
    const int jl = kMpThreads / nbt;
    const int r = tid % nbt;
    const int l = tid / nbt;
    const C* psi = static_cast<const C*>(a.state) + a.item_off[item];
    const long long J = 1ll << (a.n - a.k);          // free index range
    const long long per = (J + a.splits - 1) / a.splits;
    const long long j0 = (long long)split * per;
    const long long j1 = j0 + per < J ? j0 + per : J;
    __shared__ double red[kMpThreads];
    for (int bb = 0; bb < nb; bb += nbt) {
        const int bin = bb + r;
        unsigned long long xb = 0;   // kept bits of the bin
        for (int i = 0; i < a.k; ++i)
            if ((bin >> (a.k - 1 - i)) & 1) xb |= 1ull << a.q[i];
        double acc = 0.0;
        if (j0 + l < j1) {
            unsigned long long xf = pdep64((unsigned long long)(j0 + l), a.free_mask);
            const unsigned long long step = pdep64((unsigned long long)jl, a.free_mask);
            R part = 0;
            int cnt = 0;
            for (long long j = j0 + l; j < j1; j += jl) {
                const C v = psi[xf | xb];
                part = fma(v.x, v.x, fma(v.y, v.y, part));
                if (++cnt == 256) {
                    acc += (double)part;
                    part = 0;
                    cnt = 0;
                }
                xf = ((xf | ~a.free_mask) + step) & a.free_mask;
            }
            acc += (double)part;
        }
        red[tid] = acc;
        __syncthreads();
        if (l == 0) {   // lanes of this bin in order
            double s = 0.0;
            for (int i = 0; i < jl; ++i) s += red[i * nbt + r];
            if (a.splits == 1)
                a.out[(long long)item * a.out_stride + bin] = s;
            else
                a.out[((long long)item * a.out_stride + bin) * a.splits + split] = s;
        }
        __syncthreads();
    }
}

__global__ void marginal_finalize_kernel(const double* __restrict__ partial, int splits, int bins,
                                         int items, double* __restrict__ out) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)items * bins) return;
    double s = 0.0;
    for (int k = 0; k < splits; ++k) s += partial[i * splits + k];
    out[i] = s;
}

}  // namespace

template <typename C>
cudaError_t launch_marginal(const C* state, const long long* item_off, int items, int n, const int* q, int k,
                            double* out, double* partial, int splits, cudaStream_t s) {
    MarginalArgs a{};
    a.state = state;
    a.item_off = item_off;
    a.items = items;
    a.n = n;
    a.k = k;
    unsigned long long kept = 0;
    for (int i = 0; i < k; ++i) {
        a.q[i] = q[i];
        kept |= 1ull << q[i];
    }
    const unsigned long long all = n >= 64 ? ~0ull : ((1ull << n) - 1);
    a.free_mask = all & ~kept;
    a.splits = splits;
    a.out = splits == 1 ? out : partial;
    a.out_stride = 1 << k;
    dim3 grid((unsigned)splits, (unsigned)items);
    marginal_kernel<C><<<grid, kMpThreads, 0, s>>>(a);
    count_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || splits == 1) return e;
    const long long tot = (long long)items << k;
    marginal_finalize_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(partial, splits, 1 << k, items, out);
    count_launch();
    return cudaGetLastError();
}

// Splits of the free index range per item so that the grid fills the GPU
// (at least ~4 blocks per SM) while each thread still sums >= 32 elements.
int marginal_splits(int items, int n, int k) {
    const long long J = 1ll << (n - k);
    const int nbt = (1 << k) < kMpThreads ? (1 << k) : kMpThreads;
    const long long jl = kMpThreads / nbt;
    const long long want = (4ll * num_sms() + items - 1) / items;
    const long long cap = std::max<long long>(1, J / (jl * 32));
    return (int)std::max<long long>(1, std::min<long long>(want, std::min<long long>(cap, 4096)));
}

// ---------------------------------------------------------------- measure --
// Projective measurement of per-item qubit sets (tcng_measure), in rounds of up
// to 10 qubits: the histogram of the round's qubits (bin bit i = the item's
// i-th measured qubit of the round, counted from the lowest), sequential Born
// sampling of the round's outcomes from it (one thread per item), then the
// projection and renormalisation of the state.  The conditional probabilities
// P(o_i | o_0..o_{i-1}) read from the joint histogram equal those of measuring
// the qubits one at a time in increasing order.

namespace {

constexpr int kMeasRoundBits = 10;

// Bits of mask whose rank among the set bits lies in [lo, lo + cnt).
__device__ __forceinline__ unsigned long long rank_bits(unsigned long long mask, int lo, int cnt) {
    unsigned long long out = 0;
    int r = 0;
    while (mask) {
        const unsigned long long b = mask & (~mask + 1);
        if (r >= lo && r < lo + cnt) out |= b;
        mask ^= b;
        ++r;
    }
    return out;
}

struct MeasHistArgs {
    const void* state;
    const long long* item_off;
    const unsigned long long* mask;   // [items]
    int n;
    int round;
    int splits;
    double* hist;                      // [items][1024][splits]
};

template <typename C>
__global__ void __launch_bounds__(kMpThreads) measure_hist_kernel(MeasHistArgs a) {
    using R = typename Real<C>::T;
    const int item = blockIdx.y;
    const int split = blockIdx.x;
    const int tid = threadIdx.x;
    const unsigned long long km = rank_bits(a.mask[item], a.round * kMeasRoundBits, kMeasRoundBits);
    if (!km) return;
    const int m = __popcll(km);
    const int nb = 1 << m;
    const int nbt = nb < kMpThreads ? nb : kMpThreads;
    const int jl = kMpThreads / nbt;
    const int r = tid % nbt;
    const int l = tid / nbt;
    const C* psi = static_cast<const C*>(a.state) + a.item_off[item];
    const unsigned long long all = a.n >= 64 ? ~0ull : ((1ull << a.n) - 1);
    const unsigned long long free_mask = all & ~km;
    const long long J = 1ll << (a.n - m);
    const long long per = (J + a.splits - 1) / a.splits;
    const long long j0 = (long long)split * per;
    const long long j1 = j0 + per < J ? j0 + per : J;
    __shared__ double red[kMpThreads];
    for (int bb = 0; bb < nb; bb += nbt) {
        const int bin = bb + r;
        const unsigned long long xb = pdep64((unsigned long long)bin, km);
        double acc = 0.0;
        if (j0 + l < j1) {
            unsigned long long xf = pdep64((unsigned long long)(j0 + l), free_mask);
            const unsigned long long step = pdep64((unsigned long long)jl, free_mask);
            R part = 0;
            int cnt = 0;
            for (long long j = j0 + l; j < j1; j += jl) {
                const C v = psi[xf | xb];
                part = fma(v.x, v.x, fma(v.y, v.y, part));
                if (++cnt == 256) {
                    acc += (double)part;
                    part = 0;
                    cnt = 0;
                }
                xf = ((xf | ~free_mask) + step) & free_mask;
            }
            acc += (double)part;
        }
        red[tid] = acc;
        __syncthreads();
        if (l == 0) {
            double s = 0.0;
            for (int i = 0; i < jl; ++i) s += red[i * nbt + r];
            a.hist[((long long)item * 1024 + bin) * a.splits + split] = s;
        }
        __syncthreads();
    }
}

struct MeasProj {
    unsigned long long km;   // qubits projected in this round
    unsigned long long ob;   // their outcomes, deposited on km
    double scale;            // 1 / sqrt(probability mass kept)
    int pad[2];
};

// One thread per item: sum the splits, sample the round's outcomes in increasing
// qubit order, record them and the projection.
__global__ void measure_sample_kernel(const double* __restrict__ hist, int splits,
                                      const unsigned long long* __restrict__ mask, int round, int n,
                                      const double* __restrict__ u, signed char* __restrict__ outcome,
                                      double* __restrict__ logp, MeasProj* __restrict__ proj, int items) {
    const int item = blockIdx.x * blockDim.x + threadIdx.x;
    if (item >= items) return;
    const unsigned long long km = rank_bits(mask[item], round * kMeasRoundBits, kMeasRoundBits);
    MeasProj pr{};
    pr.km = km;
    pr.scale = 1.0;
    if (!km) {
        proj[item] = pr;
        return;
    }
    const int m = __popcll(km);
    const int nb = 1 << m;
    const double* h = hist + (long long)item * 1024 * splits;
    auto H = [&](int bin) {
        double s = 0.0;
        for (int k = 0; k < splits; ++k) s += h[(long long)bin * splits + k];
        return s;
    };
    double total = 0.0;
    for (int b = 0; b < nb; ++b) total += H(b);
    int prefix = 0;   // outcomes of the round's first i qubits (bit i = qubit i)
    unsigned long long rest = km;
    for (int i = 0; i < m; ++i) {
        const unsigned long long qb = rest & (~rest + 1);
        rest ^= qb;
        const int q = __ffsll((long long)qb) - 1;
        double s0 = 0.0, s1 = 0.0;
        const int low = (1 << i) - 1;
        for (int b = 0; b < nb; ++b) {
            if ((b & low) != prefix) continue;
            if ((b >> i) & 1) s1 += H(b); else s0 += H(b);
        }
        const double p0 = (s0 + s1) > 0.0 ? s0 / (s0 + s1) : 1.0;
        const int o = u[(long long)item * n + q] < p0 ? 0 : 1;
        prefix |= o << i;
        outcome[(long long)item * n + q] = (signed char)o;
    }
    const double kept = H(prefix);
    if (logp) logp[item] += log(kept / total);
    pr.ob = pdep64((unsigned long long)prefix, km);
    pr.scale = kept > 0.0 ? 1.0 / sqrt(kept) : 0.0;
    proj[item] = pr;
}

template <typename C>
__global__ void measure_project_kernel(C* state, const long long* __restrict__ item_off,
                                       const MeasProj* __restrict__ proj, long long N) {
    const int item = blockIdx.y;
    const MeasProj pr = proj[item];
    if (!pr.km) return;
    C* psi = state + item_off[item];
    using R = typename Real<C>::T;
    const R sc = (R)pr.scale;
    for (long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x; x < N; x += (long long)gridDim.x * blockDim.x) {
        C v = psi[x];
        if (((unsigned long long)x & pr.km) == pr.ob) {
            v.x *= sc;
            v.y *= sc;
        } else {
            v.x = 0;
            v.y = 0;
        }
        psi[x] = v;
    }
}

}  // namespace

template <typename C>
cudaError_t launch_measure(C* state, const long long* item_off, int items, int n,
                           const unsigned long long* mask, const double* u, signed char* outcome, double* logp,
                           double* hist, int splits, void* proj, cudaStream_t s) {
    const int rounds = (n + kMeasRoundBits - 1) / kMeasRoundBits;
    const long long N = 1ll << n;
    for (int r = 0; r < rounds; ++r) {
        MeasHistArgs a{};
        a.state = state;
        a.item_off = item_off;
        a.mask = mask;
        a.n = n;
        a.round = r;
        a.splits = splits;
        a.hist = hist;
        measure_hist_kernel<C><<<dim3((unsigned)splits, (unsigned)items), kMpThreads, 0, s>>>(a);
        count_launch();
        measure_sample_kernel<<<(items + 127) / 128, 128, 0, s>>>(hist, splits, mask, r, n, u, outcome, logp,
                                                                   static_cast<MeasProj*>(proj), items);
        count_launch();
        const long long per_blk = 256ll * 8;
        const unsigned gx = (unsigned)std::max<long long>(1, std::min<long long>((N + per_blk - 1) / per_blk, 4096));
        measure_project_kernel<C><<<dim3(gx, (unsigned)items), 256, 0, s>>>(state, item_off,
                                                                            static_cast<const MeasProj*>(proj), N);
        count_launch();
    }
    return cudaGetLastError();
}

size_t measure_proj_bytes(int items) { return sizeof(MeasProj) * (size_t)items; }
int measure_splits(int items, int n) { return marginal_splits(items, n, std::min(n, kMeasRoundBits)); }

template cudaError_t launch_measure<float2>(float2*, const long long*, int, int, const unsigned long long*,
                                            const double*, signed char*, double*, double*, int, void*, cudaStream_t);
template cudaError_t launch_measure<double2>(double2*, const long long*, int, int, const unsigned long long*,
                                             const double*, signed char*, double*, double*, int, void*,
                                             cudaStream_t);

template cudaError_t launch_marginal<float2>(const float2*, const long long*, int, int, const int*, int, double*,
                                             double*, int, cudaStream_t);
template cudaError_t launch_marginal<double2>(const double2*, const long long*, int, int, const int*, int,
                                              double*, double*, int, cudaStream_t);

}  // namespace tcng
