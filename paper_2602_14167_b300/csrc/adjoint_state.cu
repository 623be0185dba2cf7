// State-pass adjoint: energy and gradient of single large states (the 32-qubit
// SU(4)-ladder TFIM VQE of the paper's distributed VQE benchmark, Sec. VI.B),
// and of any circuit whose parameterised gates include Pauli-word rotations
// (RP: the 15 generators of the su4 parameterisation).
//
// The gradient follows the adjoint method that replaces reverse-mode AD
// (Sec. I.B "Paradigms: AD"): with psi = U|0> and lambda = H psi, walk the
// circuit backwards block by block, keeping two states.  Gates are fused into
// blocks of at most two qubits whatever their parameters (all 15 rotations of
// an su4 gate form one block).  For a block B (matrix U_B = M_m ... M_1 over its
// ops, in the block's ascending-qubit local order), over both states:
//     psi_in = U_B^dagger psi_out,
//     N_B[a][b] = sum over the other qubits of psi_in(a) conj(lambda_out(b)),
//     lambda_in = U_B^dagger lambda_out,
// and afterwards, for each parameterised op j of B,
//     dE/dtheta_j = 2 scale_j Re Tr(D_j N_B),
//     D_j = M_m ... M_{j+1} (dM_j/dangle) M_{j-1} ... M_1,
// with dM/dangle exact from two evaluations of the gate at shifted angles:
// (M(a + pi) - M(a - pi)) / 4 for exp(-i a G / 2) with G^2 = I (RX, RY, RZ,
// RZZ, RP), (M(a + pi/2) - M(a - pi/2)) / 2 for CP.  So the 15 gradients of an
// su4 block cost one pass over the two states (one 4 x 4 cross-density matrix)
// instead of fifteen.
//
// Blocks of at most two qubits run in fused segments: consecutive blocks (last
// first) whose qubits, with the lowest qubits (32-byte pieces in memory), fit in
// a tile of 2^12 (complex64) or 2^11 (complex128) amplitudes.  Each CTA holds a
// tile of psi and of lambda in shared memory, applies the segment's blocks one
// after the other (a CTA barrier between blocks) and writes the tile back, so a
// segment costs one read and one write of the two states (the SU(4) ladder: about
// ten blocks per segment instead of one pass per block).  The kernels sum the
// block's outputs, M[c][b] = sum psi_out(c) conj(lambda_out(b)), and the gradient
// kernel forms N_B = U_B^dagger M in FP64 (the same 192 FMAs per class of four
// amplitudes, fewer live registers).  M partials: per thread in FP32 over its
// classes of the tile, summed over the warp by a transposing shuffle tree (lane
// i ends with element i), added to the warp's FP32 row in shared memory and
// folded into FP64 every 16 tiles; CTA partials, then a fixed-order reduction
// (bitwise reproducible).  Blocks of 3..5 qubits (no parameter) end a segment
// and run on their own.  The forward runs on the ordinary tile passes; lambda =
// H psi on tile passes of its own (below).
#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <cstdio>
#include <stdexcept>
#include <string>
#include <vector>

#include "capi_internal.hpp"
#include "device.cuh"
#include "gates.cuh"

namespace tcng {

namespace {

constexpr int kSaThreads = 256;

__device__ __forceinline__ unsigned long long sa_pdep(unsigned long long v, unsigned long long mask) {
    unsigned long long r = 0;
    for (unsigned long long bb = 1; mask; bb <<= 1) {
        const unsigned long long low = mask & (~mask + 1);
        if (v & bb) r |= low;
        mask ^= low;
    }
    return r;
}

// ---- fused segments: runs of consecutive blocks (reverse order) on one tile ----
//
// A segment is a run of blocks of at most two qubits whose qubits, together with
// the lowest qubits (contiguous 32-byte pieces in memory), fit in TB tile bits.
// Each CTA loads a tile of psi and of lambda (the segment's qubits free, all other
// qubits fixed) into shared memory once, applies every block of the run to both
// (with its M partials), and writes the tile back: one pass over the two states
// per segment instead of one per block.
constexpr int kSegMax = 16;      // blocks per segment
constexpr int kSegThreads = 256; // complex64: two CTAs per SM (shared memory and registers)
constexpr int kSegFold = 16;     // tiles between folds of the FP32 warp sums into FP64

struct SaSegBlk {
    int tb0, tb1;   // tile bits of the block's qubits (ascending; tb1 = -1 for one qubit)
    int k, diag;
    int grad;       // gradient-block index, -1 none
    int out_off;    // matrix offset in the block table
};
struct SaSeg {
    unsigned long long tmask;   // qubits of the tile
    int tbits, nblk;
    SaSegBlk b[kSegMax];
};

template <typename C, int TB>
constexpr size_t sa_seg_smem() {
    using R = typename Real<C>::T;
    return 2 * sizeof(C) * (size_t(1) << TB) + sizeof(C) * kSegMax * 16 + 128 * sizeof(unsigned long long) +
           sizeof(R) * (kSegThreads / 32) * kSegMax * 32 + sizeof(double) * kSegMax * 32;
}

__device__ __forceinline__ float sa_fma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double sa_fma(double a, double b, double c) { return fma(a, b, c); }

__device__ __forceinline__ int sa_ins0(int j, int b) { return ((j >> b) << (b + 1)) | (j & ((1 << b) - 1)); }

// Shared-memory place of tile position p (complex64 tiles): tile bit 4 flips
// bits 1 and 2, bit 5 flips bits 2 and 3.  Linear (place(p ^ o) = place(p) ^
// place(o)), a bijection, and bit 0 is kept (a 16-byte piece stays whole); with
// 16 eight-byte words per 128-byte row it spreads the half-warps of blocks on
// tile bits (1,2), (2,3), (3,4) over all banks (and halves the conflict of (0,1)).
template <typename C>
__device__ __forceinline__ int sa_place(int p) {
    if (sizeof(C) != 8) return p;
    return p ^ ((0xAC60 >> (((p >> 4) & 3) * 4)) & 15);
}

// v[0..V) per lane; afterwards, for V = 32, lane l holds the warp total of
// element l in v[0]; for V = 8 the four lanes 4e..4e+3 hold that of element e.
template <typename R, int V>
__device__ __forceinline__ void sa_warp_transpose_sum(R (&v)[32], int lane) {
#pragma unroll
    for (int h = V / 2, o = 16; h >= 1; h >>= 1, o >>= 1) {
        const bool up = lane & o;
#pragma unroll
        for (int i = 0; i < h; ++i) {
            const R keep = up ? v[i + h] : v[i];
            const R send = up ? v[i] : v[i + h];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
    if (V == 8) {
#pragma unroll
        for (int o = 2; o >= 1; o >>= 1) v[0] += __shfl_xor_sync(0xffffffffu, v[0], o);
    }
}

// One block of K qubits over the tile: psi, lambda <- U^dagger (psi, lambda)
// and, for a gradient block, the warp's partials of M[l][m] = sum psi_out(l)
// conj(lambda_out(m)) (the block's outputs, before U^dagger) added to wr (this
// warp's row).  Every product is one fused multiply-add on a running sum.
template <typename C, int K, bool DIAG>
__device__ __forceinline__ void sa_seg_block(C* __restrict__ sp, C* __restrict__ sl, const C* __restrict__ su,
                                             const SaSegBlk& bk, int E, typename Real<C>::T* __restrict__ wr) {
    using R = typename Real<C>::T;
    constexpr int D = 1 << K;
    const int lane = threadIdx.x & 31;
    const bool grad = bk.grad >= 0;
    C u[DIAG ? D : D * D];
#pragma unroll
    for (int i = 0; i < (DIAG ? D : D * D); ++i) u[i] = su[i];
    int off[D];   // places of the class's amplitudes relative to the class's first
#pragma unroll
    for (int l = 0; l < D; ++l)
        off[l] = sa_place<C>(((l & 1) ? (1 << bk.tb0) : 0) | ((K == 2 && (l & 2)) ? (1 << bk.tb1) : 0));
    R macc[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) macc[i] = 0;
    const int classes = E >> K;
    for (int j = threadIdx.x; j < classes; j += kSegThreads) {
        int p = sa_ins0(j, bk.tb0);
        if (K == 2) p = sa_ins0(p, bk.tb1);
        p = sa_place<C>(p);
        C a[D], b[D];
#pragma unroll
        for (int l = 0; l < D; ++l) {
            a[l] = sp[p ^ off[l]];
            b[l] = sl[p ^ off[l]];
        }
        if (grad) {   // M[l][m] += a_l conj(b_m)
#pragma unroll
            for (int l = 0; l < D; ++l)
#pragma unroll
                for (int m = 0; m < D; ++m) {
                    R& mr = macc[2 * (l * D + m)];
                    R& mi = macc[2 * (l * D + m) + 1];
                    mr = sa_fma(a[l].y, b[m].y, sa_fma(a[l].x, b[m].x, mr));
                    mi = sa_fma(-a[l].x, b[m].y, sa_fma(a[l].y, b[m].x, mi));
                }
        }
#pragma unroll
        for (int l = 0; l < D; ++l) {   // y_l = sum_m conj(U[m][l]) a_m (diagonal: conj(u_l) a_l)
            R yr = 0, yi = 0, zr = 0, zi = 0;
#pragma unroll
            for (int m = 0; m < D; ++m) {
                if (DIAG && m != l) continue;
                const C w = DIAG ? u[l] : u[m * D + l];
                yr = sa_fma(w.y, a[m].y, sa_fma(w.x, a[m].x, yr));
                yi = sa_fma(-w.y, a[m].x, sa_fma(w.x, a[m].y, yi));
                zr = sa_fma(w.y, b[m].y, sa_fma(w.x, b[m].x, zr));
                zi = sa_fma(-w.y, b[m].x, sa_fma(w.x, b[m].y, zi));
            }
            sp[p ^ off[l]] = cmk<C>(yr, yi);
            sl[p ^ off[l]] = cmk<C>(zr, zi);
        }
    }
    if (grad) {   // block-uniform branch: every lane of every warp takes it
        sa_warp_transpose_sum<R, 2 * D * D>(macc, lane);
        if (K == 2)
            wr[lane] += macc[0];
        else if ((lane & 3) == 0)
            wr[lane >> 2] += macc[0];
    }
}

template <typename C, int TB>
__global__ void __launch_bounds__(kSegThreads, sizeof(C) == 8 ? 2 : 1)
    sa_seg_kernel(C* __restrict__ psi, C* __restrict__ lam, const C* __restrict__ table,
                  const __grid_constant__ SaSeg seg, int n, double* __restrict__ npart) {
    using R = typename Real<C>::T;
    constexpr int W = kSegThreads / 32;
    extern __shared__ __align__(16) unsigned char sa_smem[];
    C* sp = reinterpret_cast<C*>(sa_smem);
    C* sl = sp + (1 << TB);
    C* su = sl + (1 << TB);
    unsigned long long* dep = reinterpret_cast<unsigned long long*>(su + kSegMax * 16);   // [2][64]
    R* wr = reinterpret_cast<R*>(dep + 128);                                               // [W][kSegMax][32]
    double* w64 = reinterpret_cast<double*>(wr + W * kSegMax * 32);                        // [kSegMax][32]
    const int tid = threadIdx.x, warp = tid >> 5;
    const int nb = seg.nblk;
    for (int i = tid; i < nb * 16; i += kSegThreads) {
        const SaSegBlk& bk = seg.b[i >> 4];
        const int e = i & 15, d = 1 << bk.k;
        if (e < (bk.diag ? d : d * d)) su[i] = table[bk.out_off + e];
    }
    if (tid < 128) {   // tile position bits 0..5 (dep[0..63]) and 6..11 (dep[64..127]) -> qubit bits
        const int lo = (tid >> 6) * 6, v = tid & 63;
        unsigned long long g = 0;
        for (int b = 0, c = 0; b < 64; ++b) {
            if (!((seg.tmask >> b) & 1)) continue;
            if (c >= lo && c < lo + 6 && ((v >> (c - lo)) & 1)) g |= 1ull << b;
            ++c;
        }
        dep[tid] = g;
    }
    for (int i = tid; i < W * kSegMax * 32; i += kSegThreads) wr[i] = 0;
    for (int i = tid; i < kSegMax * 32; i += kSegThreads) w64[i] = 0.0;
    __syncthreads();
    auto fold = [&]() {
        for (int i = tid; i < nb * 32; i += kSegThreads) {
            R s = 0;
#pragma unroll
            for (int w = 0; w < W; ++w) {
                s += wr[w * kSegMax * 32 + i];
                wr[w * kSegMax * 32 + i] = 0;
            }
            w64[i] += (double)s;
        }
    };
    const unsigned long long all = (n >= 64) ? ~0ull : ((1ull << n) - 1);
    const unsigned long long fm = all & ~seg.tmask;
    const long long ntiles = 1ll << (n - seg.tbits);
    const int E = 1 << seg.tbits;
    constexpr int PW = 16 / sizeof(C);   // amplitudes per 16-byte piece (tile bit 0 is qubit 0)
    unsigned long long base = sa_pdep((unsigned long long)blockIdx.x, fm);
    const unsigned long long step = sa_pdep((unsigned long long)gridDim.x, fm);
    int since = 0;
    for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
        for (int q = tid; q < E / PW; q += kSegThreads) {
            const int pos = q * PW;
            const unsigned long long g = base | dep[pos & 63] | dep[64 + (pos >> 6)];
            const int sq = sa_place<C>(pos);
            *reinterpret_cast<float4*>(sp + sq) = __ldcs(reinterpret_cast<const float4*>(psi + g));
            *reinterpret_cast<float4*>(sl + sq) = __ldcs(reinterpret_cast<const float4*>(lam + g));
        }
        __syncthreads();
        for (int bi = 0; bi < nb; ++bi) {
            const SaSegBlk& bk = seg.b[bi];
            R* w = wr + (warp * kSegMax + bi) * 32;
            if (bk.k == 2) {
                if (bk.diag)
                    sa_seg_block<C, 2, true>(sp, sl, su + bi * 16, bk, E, w);
                else
                    sa_seg_block<C, 2, false>(sp, sl, su + bi * 16, bk, E, w);
            } else {
                if (bk.diag)
                    sa_seg_block<C, 1, true>(sp, sl, su + bi * 16, bk, E, w);
                else
                    sa_seg_block<C, 1, false>(sp, sl, su + bi * 16, bk, E, w);
            }
            __syncthreads();
        }
        for (int q = tid; q < E / PW; q += kSegThreads) {
            const int pos = q * PW;
            const unsigned long long g = base | dep[pos & 63] | dep[64 + (pos >> 6)];
            const int sq = sa_place<C>(pos);
            __stcs(reinterpret_cast<float4*>(psi + g), *reinterpret_cast<const float4*>(sp + sq));
            __stcs(reinterpret_cast<float4*>(lam + g), *reinterpret_cast<const float4*>(sl + sq));
        }
        if (++since == kSegFold) {   // CTA-uniform
            fold();
            since = 0;
        }
        base = ((base | ~fm) + step) & fm;
        __syncthreads();
    }
    fold();
    __syncthreads();
    for (int i = tid; i < nb * 32; i += kSegThreads) {
        const int g = seg.b[i >> 5].grad;
        if (g >= 0) npart[((long long)g * gridDim.x + blockIdx.x) * 32 + (i & 31)] = w64[i];
    }
}

// ---- lambda = H psi in tile passes ----
//
// (H psi)(y) = sum_t c_t i^{ny_t} (-1)^{popc((y ^ x_t) & z_t)} psi(y ^ x_t).  The
// terms are grouped into passes whose X masks, with the lowest qubits, fit in
// a tile of 2^12 (complex64) / 2^11 (complex128) amplitudes; a pass loads each
// psi tile into shared memory once, takes every partner psi(y ^ x_t) from it and
// writes (first pass) or adds to lambda.  The Z sign splits into the tile part,
// popc(pos & z_t (tile bits)), and the tile's fixed part; diagonal terms (x_t =
// 0) sum into one real factor per amplitude.
constexpr int kHamMax = 64;      // terms per pass
constexpr int kHamThreads = 256;
struct SaHamPass {
    unsigned long long tmask;
    int tbits, nt, ndiag, first;   // terms [0, ndiag) are diagonal
    int idx[kHamMax];              // term index
    int xt[kHamMax], zt[kHamMax];  // X and Z masks in tile bits
};

template <typename C, int TB>
constexpr size_t sa_ham_smem() {
    using R = typename Real<C>::T;
    return sizeof(C) * (size_t(1) << TB) + 128 * sizeof(unsigned long long) + kHamMax * sizeof(unsigned long long) +
           2 * kHamMax * sizeof(R) + 3 * kHamMax * sizeof(int);
}

template <typename C, int TB>
__global__ void __launch_bounds__(kHamThreads)
    sa_ham_tile_kernel(const C* __restrict__ psi, C* __restrict__ lam, const HTerm* __restrict__ terms,
                       const double* __restrict__ coeffs, const double* __restrict__ term_coeff,
                       const __grid_constant__ SaHamPass hp, int n) {
    using R = typename Real<C>::T;
    constexpr int EPT = (1 << TB) / kHamThreads;   // amplitudes per thread
    extern __shared__ __align__(16) unsigned char sh_smem[];
    C* sp = reinterpret_cast<C*>(sh_smem);
    unsigned long long* dep = reinterpret_cast<unsigned long long*>(sp + (1 << TB));   // [128]
    unsigned long long* zout = dep + 128;   // Z mask outside the tile
    R* cre = reinterpret_cast<R*>(zout + kHamMax);
    R* cim = cre + kHamMax;
    int* xt = reinterpret_cast<int*>(cim + kHamMax);
    int* zt = xt + kHamMax;
    int* pb = zt + kHamMax;   // per tile: popc(base & z_t) & 1
    const int tid = threadIdx.x, nt = hp.nt;
    if (tid < nt) {   // c_t i^{ny} (-1)^{popc(x_t & z_t)} as (re, im)
        const HTerm h = terms[hp.idx[tid]];
        const double c0 = coeffs ? coeffs[hp.idx[tid]] : term_coeff[hp.idx[tid]];
        const double c = (__popcll(h.xm & h.zm) & 1) ? -c0 : c0;
        const int ny = h.ny & 3;
        cre[tid] = (R)(ny == 0 ? c : (ny == 2 ? -c : 0.0));
        cim[tid] = (R)(ny == 1 ? c : (ny == 3 ? -c : 0.0));
        xt[tid] = hp.xt[tid];
        zt[tid] = hp.zt[tid];
        zout[tid] = h.zm & ~hp.tmask;
    }
    if (tid < 128) {   // tile position bits 0..5 (dep[0..63]) and 6..11 (dep[64..127]) -> qubit bits
        const int lo = (tid >> 6) * 6, v = tid & 63;
        unsigned long long g = 0;
        for (int b = 0, c = 0; b < 64; ++b) {
            if (!((hp.tmask >> b) & 1)) continue;
            if (c >= lo && c < lo + 6 && ((v >> (c - lo)) & 1)) g |= 1ull << b;
            ++c;
        }
        dep[tid] = g;
    }
    __syncthreads();
    const unsigned long long all = (n >= 64) ? ~0ull : ((1ull << n) - 1);
    const unsigned long long fm = all & ~hp.tmask;
    const long long ntiles = 1ll << (n - hp.tbits);
    const int E = 1 << hp.tbits;
    constexpr int PW = 16 / sizeof(C);
    unsigned long long base = sa_pdep((unsigned long long)blockIdx.x, fm);
    const unsigned long long step = sa_pdep((unsigned long long)gridDim.x, fm);
    for (long long t = blockIdx.x; t < ntiles; t += gridDim.x) {
        for (int q = tid; q < E / PW; q += kHamThreads) {
            const int pos = q * PW;
            const unsigned long long g = base | dep[pos & 63] | dep[64 + (pos >> 6)];
            *reinterpret_cast<float4*>(sp + pos) = __ldcs(reinterpret_cast<const float4*>(psi + g));
        }
        if (tid < nt) pb[tid] = __popcll(base & zout[tid]) & 1;
        __syncthreads();
        R ar[EPT], ai[EPT], d[EPT];
#pragma unroll
        for (int k = 0; k < EPT; ++k) ar[k] = ai[k] = d[k] = 0;
        for (int i = 0; i < hp.ndiag; ++i) {   // real diagonal factor
            const int z = zt[i];
            const R c = pb[i] ? -cre[i] : cre[i];
#pragma unroll
            for (int k = 0; k < EPT; ++k) {
                const int pos = tid + k * kHamThreads;
                d[k] += (__popc(pos & z) & 1) ? -c : c;
            }
        }
        for (int i = hp.ndiag; i < nt; ++i) {
            const int x = xt[i], z = zt[i];
            const R sr = pb[i] ? -cre[i] : cre[i], si = pb[i] ? -cim[i] : cim[i];
#pragma unroll
            for (int k = 0; k < EPT; ++k) {
                const int pos = tid + k * kHamThreads;
                if (pos >= E) break;
                const C v = sp[pos ^ x];
                const bool neg = __popc(pos & z) & 1;
                const R cr = neg ? -sr : sr, ci = neg ? -si : si;
                ar[k] = sa_fma(cr, v.x, sa_fma(-ci, v.y, ar[k]));
                ai[k] = sa_fma(cr, v.y, sa_fma(ci, v.x, ai[k]));
            }
        }
#pragma unroll
        for (int k = 0; k < EPT; ++k) {
            const int pos = tid + k * kHamThreads;
            if (pos >= E) break;
            const unsigned long long g = base | dep[pos & 63] | dep[64 + (pos >> 6)];
            const C v = sp[pos];
            R yr = sa_fma(d[k], v.x, ar[k]), yi = sa_fma(d[k], v.y, ai[k]);
            if (!hp.first) {
                const C o = lam[g];
                yr += o.x;
                yi += o.y;
            }
            lam[g] = cmk<C>(yr, yi);
        }
        base = ((base | ~fm) + step) & fm;
        __syncthreads();
    }
}

// Blocks of 3..5 qubits carry no parameter: psi <- U^dagger psi on one state
// (called for psi and for lambda).
template <typename C, int K>
__global__ void __launch_bounds__(kSaThreads) sa_uncompute_kernel(C* __restrict__ st, const C* __restrict__ U,
                                                                  int diag, unsigned long long qmask, int n) {
    using R = typename Real<C>::T;
    constexpr int D = 1 << K;
    __shared__ C su[D * D];
    for (int i = threadIdx.x; i < (diag ? D : D * D); i += blockDim.x) su[i] = U[i];
    __syncthreads();
    const unsigned long long all = (n >= 64) ? ~0ull : ((1ull << n) - 1);
    const unsigned long long fm = all & ~qmask;
    const long long classes = 1ll << (n - K);
    const long long stride = (long long)gridDim.x * blockDim.x;
    long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long x0 = sa_pdep((unsigned long long)j, fm);
    const unsigned long long step = sa_pdep((unsigned long long)stride, fm);
    for (; j < classes; j += stride) {
        C a[D];
#pragma unroll
        for (int l = 0; l < D; ++l) a[l] = st[x0 | sa_pdep((unsigned long long)l, qmask)];
#pragma unroll
        for (int l = 0; l < D; ++l) {
            R yr = 0, yi = 0;
            if (diag) {
                const C u = su[l];
                yr = u.x * a[l].x + u.y * a[l].y;
                yi = u.x * a[l].y - u.y * a[l].x;
            } else {
#pragma unroll
                for (int m = 0; m < D; ++m) {
                    const C u = su[m * D + l];
                    yr += u.x * a[m].x + u.y * a[m].y;
                    yi += u.x * a[m].y - u.y * a[m].x;
                }
            }
            st[x0 | sa_pdep((unsigned long long)l, qmask)] = cmk<C>(yr, yi);
        }
        x0 = ((x0 | ~fm) + step) & fm;
    }
}

// M of every gradient block: the CTA partials summed in order.
__global__ void sa_nfinal_kernel(const double* __restrict__ npart, int ncta, int nblocks, double* __restrict__ N) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nblocks * 32) return;
    const int g = i >> 5, e = i & 31;
    const double* p = npart + (long long)g * ncta * 32 + e;
    double s = 0.0;
    for (int c = 0; c < ncta; ++c) s += p[(long long)c * 32];
    N[i] = s;
}

struct SaEntry {     // one parameterised op: its block, its place in the block
    int gblock;      // gradient-block index (row of N)
    int op_begin;    // the block's first BuildOp
    int op_count;
    int j;           // the op within the block
    int k;           // block qubits (1 or 2)
    int pad;
};

// Apply a k-qubit op matrix (its own local order, q[0] most significant) to
// every column of the D x D block-space matrix L (ascending-qubit local order).
__device__ void sa_apply_op(double2* L, int D, const BuildOp& op, const double2* M) {
    const int ko = op.k, dk = 1 << ko;
    int qm = 0;
    for (int i = 0; i < ko; ++i) qm |= 1 << op.pos[i];
    for (int c = 0; c < D; ++c)
        for (int x = 0; x < D; ++x) {
            if (x & qm) continue;
            double2 v[4], w[4];
            int idx[4];
            for (int r = 0; r < dk; ++r) {
                int y = x;
                for (int i = 0; i < ko; ++i)
                    if ((r >> (ko - 1 - i)) & 1) y |= 1 << op.pos[i];
                idx[r] = y;
                v[r] = L[y * D + c];
            }
            for (int r = 0; r < dk; ++r) {
                double re = 0, im = 0;
                for (int s = 0; s < dk; ++s) {
                    const double2 m = M[r * dk + s];
                    re += m.x * v[s].x - m.y * v[s].y;
                    im += m.x * v[s].y + m.y * v[s].x;
                }
                w[r] = make_double2(re, im);
            }
            for (int r = 0; r < dk; ++r) L[idx[r] * D + c] = w[r];
        }
}

// contrib[e] = 2 scale Re Tr(D_j N) for parameterised op e, with the segment
// kernels' M (outputs of the block: M[c][b] = sum psi_out(c) conj(lambda_out(b)))
// and N = U_B^dagger M:  Tr(D_j N) = sum_{b,c} (D_j U_B^dagger)[b][c] M[c][b].
__global__ void sa_grad_kernel(const SaEntry* __restrict__ ents, int n_ent, const BuildOp* __restrict__ bops,
                               const double2* __restrict__ pool, const double* __restrict__ params,
                               const double* __restrict__ Mblk, double* __restrict__ contrib) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_ent) return;
    const SaEntry en = ents[e];
    const int D = 1 << en.k;
    double2 L[16], U[16], M[16], Mp[16];
    for (int i = 0; i < D * D; ++i) L[i] = U[i] = make_double2((i / D) == (i % D) ? 1.0 : 0.0, 0.0);
    const double pi = 3.14159265358979323846;
    double scale = 1.0;
    for (int o = 0; o < en.op_count; ++o) {
        const BuildOp op = bops[en.op_begin + o];
        const int dk = 1 << op.k;
        double ang = op.angle0;
        if (op.param >= 0) ang += op.scale * params[op.param];
        gate_matrix_d(op, ang, M, dk, pool);
        sa_apply_op(U, D, op, M);
        if (o == en.j) {   // dM/dangle from two shifted evaluations
            scale = op.scale;
            const bool cp = op.code == TCNG_CP;
            const double h = cp ? 0.5 * pi : pi, f = cp ? 0.5 : 0.25;
            gate_matrix_d(op, ang + h, M, dk, pool);
            gate_matrix_d(op, ang - h, Mp, dk, pool);
            for (int i = 0; i < dk * dk; ++i) M[i] = make_double2(f * (M[i].x - Mp[i].x), f * (M[i].y - Mp[i].y));
        }
        sa_apply_op(L, D, op, M);
    }
    const double* Mb = Mblk + (long long)en.gblock * 32;
    double re = 0.0;
    for (int b = 0; b < D; ++b)
        for (int c = 0; c < D; ++c) {
            double pr = 0.0, pim = 0.0;   // (D U^dagger)[b][c] = sum_a D[b][a] conj(U[c][a])
            for (int a = 0; a < D; ++a) {
                const double2 d = L[b * D + a], u = U[c * D + a];
                pr += d.x * u.x + d.y * u.y;
                pim += d.y * u.x - d.x * u.y;
            }
            re += pr * Mb[2 * (c * D + b)] - pim * Mb[2 * (c * D + b) + 1];
        }
    contrib[e] = 2.0 * scale * re;
}

// grad[p] = sum of its contributions in op order (CSR over entries).
__global__ void sa_param_sum_kernel(const int* __restrict__ start, const int* __restrict__ list,
                                    const double* __restrict__ contrib, int P, double* __restrict__ grad) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    double s = 0.0;
    for (int i = start[p]; i < start[p + 1]; ++i) s += contrib[list[i]];
    grad[p] = s;
}

// Re <a|b> over one state: CTA partials, then a fixed-order sum.
template <typename C>
__global__ void __launch_bounds__(kSaThreads) sa_dot_kernel(const C* __restrict__ a, const C* __restrict__ b,
                                                            long long N, double* __restrict__ part) {
    double acc = 0.0;
    float f = 0.f;
    int cnt = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        const C x = a[i], y = b[i];
        if (sizeof(x.x) == 8) {
            acc += (double)x.x * (double)y.x + (double)x.y * (double)y.y;
        } else {
            f = fmaf((float)x.x, (float)y.x, fmaf((float)x.y, (float)y.y, f));
            if (++cnt == 64) {
                acc += (double)f;
                f = 0.f;
                cnt = 0;
            }
        }
    }
    acc += (double)f;
    __shared__ double red[kSaThreads / 32];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < kSaThreads / 32; ++w) s += red[w];
        part[blockIdx.x] = s;
    }
}

__global__ void sa_sum_kernel(const double* __restrict__ part, int m, double* __restrict__ out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < m; ++i) s += part[i];
        *out = s;
    }
}

}  // namespace

// ------------------------------------------------------------- host side --
namespace {

struct SaPlan {           // per adjoint block plan: blocks in order, gradient entries
    struct Blk {
        unsigned long long qmask;
        int k, diag, out_off, grad;   // grad: gradient-block index, -1 none
    };
    std::vector<Blk> blocks;
    int n_grad_blocks = 0;
    SaEntry* d_ents = nullptr;
    int n_ents = 0;
    int* d_start = nullptr;
    int* d_list = nullptr;
    ~SaPlan() {
        cudaFree(d_ents);
        cudaFree(d_start);
        cudaFree(d_list);
    }
};
std::map<const DevPlan*, std::unique_ptr<SaPlan>> g_saplans;

SaPlan* get_saplan(DevPlan* dp) {
    auto it = g_saplans.find(dp);
    if (it != g_saplans.end()) return it->second.get();
    const Plan& pl = dp->plan;
    std::unique_ptr<SaPlan> sp(new SaPlan());
    std::vector<SaEntry> ents;
    std::vector<std::vector<int>> per_param(std::max(pl.P, 1));
    for (size_t bi = 0; bi < pl.blocks.size(); ++bi) {
        const Block& b = pl.blocks[bi];
        const BuildBlock& bb = pl.bblocks[bi];
        SaPlan::Blk k{};
        k.qmask = b.qmask;
        k.k = b.k;
        k.diag = b.diag ? 1 : 0;
        k.out_off = b.out_off;
        k.grad = -1;
        bool has = false;
        for (int oi : b.ops) has = has || pl.ops[oi].param >= 0;
        if (has) {
            if (b.k > 2) throw std::invalid_argument("state-pass adjoint: a parameterised gate on more than 2 qubits");
            k.grad = sp->n_grad_blocks++;
            for (int o = 0; o < (int)b.ops.size(); ++o) {
                const HostOp& op = pl.ops[b.ops[o]];
                if (op.param < 0) continue;
                SaEntry e{};
                e.gblock = k.grad;
                e.op_begin = bb.op_begin;
                e.op_count = bb.op_count;
                e.j = o;
                e.k = b.k;
                per_param[op.param].push_back((int)ents.size());
                ents.push_back(e);
            }
        }

        sp->blocks.push_back(k);
    }
    std::vector<int> start(1, 0), list;
    for (int p = 0; p < pl.P; ++p) {
        for (int e : per_param[p]) list.push_back(e);
        start.push_back((int)list.size());
    }
    if (list.empty()) list.push_back(0);
    sp->n_ents = (int)ents.size();
    if (!ents.empty()) sp->d_ents = dev_copy(ents);
    sp->d_start = dev_copy(start);
    sp->d_list = dev_copy(list);
    SaPlan* raw = sp.get();
    g_saplans[dp] = std::move(sp);
    return raw;
}

template <typename C, int TB>
cudaError_t launch_seg(C* psi, C* lam, const C* table, const SaSeg& sg, int n, double* npart, int grid,
                       cudaStream_t s) {
    static bool attr[kMaxDeviceSlots] = {};   // the attribute is per device
    const int d = device_slot();
    if (!attr[d]) {
        const cudaError_t e = cudaFuncSetAttribute(sa_seg_kernel<C, TB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)sa_seg_smem<C, TB>());
        if (e != cudaSuccess) return e;
        attr[d] = true;
    }
    ProfScope ps("sa_seg_kernel", s);
    sa_seg_kernel<C, TB><<<grid, kSegThreads, sa_seg_smem<C, TB>(), s>>>(psi, lam, table, sg, n, npart);
    count_launch();
    return cudaGetLastError();
}

// Tile geometry of the state-pass kernels: tile bits and the lowest qubits that
// every tile holds (32-byte pieces in memory).
template <typename C>
void sa_tile_geometry(int n, int* tbits, unsigned long long* cmask) {
    constexpr int TB = sizeof(C) == 8 ? 12 : 11;
    *tbits = std::min(TB, n);
    *cmask = (unsigned long long)std::min(32 / (int)sizeof(C), 1 << *tbits) - 1;
}

// Pad a tile mask with the lowest qubits it lacks, up to tbits qubits.
unsigned long long sa_pad_mask(unsigned long long tm, int n, int tbits) {
    for (int q = 0; q < n && __builtin_popcountll(tm) < tbits; ++q) tm |= 1ull << q;
    return tm;
}

// The reverse sweep's steps, last block first: segments (runs of blocks of <= 2
// qubits whose qubits and cmask fit in tbits, at most kSegMax) and lone blocks
// of 3..5 qubits (tmask 0).
struct SaStep {
    std::vector<int> blk;
    unsigned long long tmask = 0;
};
std::vector<SaStep> plan_reverse_steps(const std::vector<unsigned long long>& qmask, const std::vector<int>& k,
                                       int n, int tbits, unsigned long long cmask) {
    std::vector<SaStep> out;
    SaStep cur;
    unsigned long long used = 0;
    auto close = [&]() {
        if (cur.blk.empty()) return;
        cur.tmask = sa_pad_mask(cmask | used, n, tbits);
        out.push_back(cur);
        cur = SaStep{};
        used = 0;
    };
    for (int bi = (int)qmask.size() - 1; bi >= 0; --bi) {
        if (k[bi] <= 2) {
            if ((int)cur.blk.size() == kSegMax || __builtin_popcountll(cmask | used | qmask[bi]) > tbits) close();
            cur.blk.push_back(bi);
            used |= qmask[bi];
            continue;
        }
        close();
        SaStep big;
        big.blk.push_back(bi);
        out.push_back(big);
    }
    close();
    return out;
}

// The passes of lambda = H psi: diagonal terms (no X) in the first pass, each
// other term in the first pass whose tile mask, widened by its X mask, stays
// within tbits qubits (at most kHamMax terms a pass).  False when a term's X
// mask does not fit in a tile with cmask.
struct HamBin {
    unsigned long long mask;   // before padding
    std::vector<int> diag, off;
};
bool plan_ham_passes(const tcng_pauli* H, size_t n_terms, int tbits, unsigned long long cmask,
                     std::vector<HamBin>& bins) {
    bins.clear();
    for (size_t t = 0; t < n_terms; ++t) {
        const unsigned long long x = H[t].xmask;
        if (__builtin_popcountll(cmask | x) > tbits) return false;
        if (x == 0) {
            if (bins.empty()) bins.push_back(HamBin{cmask, {}, {}});
            bins[0].diag.push_back((int)t);
            continue;
        }
        bool placed = false;
        for (HamBin& b : bins) {
            if (b.diag.size() + b.off.size() < (size_t)kHamMax && __builtin_popcountll(b.mask | x) <= tbits) {
                b.mask |= x;
                b.off.push_back((int)t);
                placed = true;
                break;
            }
        }
        if (!placed) bins.push_back(HamBin{cmask | x, {}, {(int)t}});
    }
    if (!bins.empty())   // diagonal terms beyond the first bin's room go to bins of their own
        while (bins[0].diag.size() + bins[0].off.size() > (size_t)kHamMax) {
            HamBin extra{cmask, {}, {}};
            while (extra.diag.size() < (size_t)kHamMax && bins[0].diag.size() + bins[0].off.size() > (size_t)kHamMax) {
                extra.diag.push_back(bins[0].diag.back());
                bins[0].diag.pop_back();
            }
            bins.push_back(extra);
        }
    return true;
}

// lambda = H psi by tile passes; returns false (nothing launched) when a term's
// X mask does not fit in a tile with the lowest qubits.
template <typename C>
bool ham_apply_tiled(const C* psi, C* lam, const tcng_pauli* H, size_t n_terms, const TermSet* ts,
                     const double* coeffs, int n, cudaStream_t s, cudaError_t* err) {
    constexpr int TB = sizeof(C) == 8 ? 12 : 11;
    int tbits;
    unsigned long long cmask;
    sa_tile_geometry<C>(n, &tbits, &cmask);
    std::vector<HamBin> bins;
    if (!plan_ham_passes(H, n_terms, tbits, cmask, bins)) return false;
    static bool attr[kMaxDeviceSlots] = {};
    const int d = device_slot();
    if (!attr[d]) {
        *err = cudaFuncSetAttribute(sa_ham_tile_kernel<C, TB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)sa_ham_smem<C, TB>());
        if (*err != cudaSuccess) return true;
        attr[d] = true;
    }
    const int grid = std::max(1, num_sms() * 4);
    bool first = true;
    for (const HamBin& b : bins) {
        SaHamPass hp{};
        const unsigned long long tm = sa_pad_mask(b.mask, n, tbits);
        hp.tmask = tm;
        hp.tbits = tbits;
        hp.first = first ? 1 : 0;
        auto tile_bits = [&](unsigned long long m) {   // m's bits inside the tile, in tile positions
            int r = 0;
            for (int q = 0, c = 0; q < n; ++q)
                if ((tm >> q) & 1) {
                    if ((m >> q) & 1) r |= 1 << c;
                    ++c;
                }
            return r;
        };
        for (int t : b.diag) {
            hp.idx[hp.nt] = t;
            hp.xt[hp.nt] = 0;
            hp.zt[hp.nt++] = tile_bits(H[t].zmask);
        }
        hp.ndiag = hp.nt;
        for (int t : b.off) {
            hp.idx[hp.nt] = t;
            hp.xt[hp.nt] = tile_bits(H[t].xmask);
            hp.zt[hp.nt++] = tile_bits(H[t].zmask);
        }
        sa_ham_tile_kernel<C, TB><<<grid, kHamThreads, sa_ham_smem<C, TB>(), s>>>(psi, lam, ts->d_h, coeffs,
                                                                                  ts->d_c, hp, n);
        count_launch();
        first = false;
    }
    if (bins.empty()) {   // no terms: lambda = 0
        *err = cudaMemsetAsync(lam, 0, sizeof(C) << n, s);
        return true;
    }
    *err = cudaGetLastError();
    return true;
}

}  // namespace

// Energy and gradient of item `item` of st (a single size class) by the
// state-pass adjoint.  params/coeffs/energy/grad point at the item's rows.
template <typename C>
tcng_status run_state_adjoint(tcng_state* st, int item, const tcng_gate* ops, size_t n_ops, const double* pool,
                              size_t n_mat, const double* params, int P, const tcng_pauli* H, size_t n_terms,
                              const double* coeffs, double* energy, double* grad, cudaStream_t s) {
    const int n = st->n[item];
    DeviceCtx& c = ctx();
    const long long N = 1ll << n;
    C* psi = static_cast<C*>(st->buf) + st->off[item];
    cudaError_t e;
    // forward on the tile passes
    {
        const PlanOptions o = plan_options(st->dt, false);
        DevPlan* dp = get_plan(n, ops, n_ops, pool, n_mat, P, o);
        e = cudaMemsetAsync(psi, 0, sizeof(C) * (size_t)N, s);
        if (e == cudaSuccess) e = launch_set_basis<C>(static_cast<C*>(st->buf), st->d_off + item, 1, s);
        if (e != cudaSuccess) return cuda_fail(e, "state reset");
        const tcng_status r = run_plan<C>(dp, static_cast<C*>(st->buf), st->d_off + item, 1, params, s, psi, 0);
        if (r) return r;
    }
    // lambda = H psi, E = Re <psi|lambda>
    C* lam = static_cast<C*>(c.scratch("sa_lambda", sizeof(C) * (size_t)N));
    long long* zero = static_cast<long long*>(c.scratch("sa_zero", sizeof(long long)));
    const int grid = std::max(1, num_sms() * 4);
    double* dpart = static_cast<double*>(c.scratch("sa_dot", sizeof(double) * grid));
    if (!lam || !zero || !dpart) return fail(TCNG_ENOMEM, "state-pass adjoint scratch");
    e = cudaMemsetAsync(zero, 0, sizeof(long long), s);
    if (e != cudaSuccess) return cuda_fail(e, "memset");
    TermSet* ts = get_terms(H, n_terms, n);
    {
    ProfScope ps("ham_apply_kernel", s);
    if (!ham_apply_tiled<C>(psi, lam, H, n_terms, ts, coeffs, n, s, &e))
        e = launch_ham_apply<C>(static_cast<const C*>(st->buf), st->d_off + item, lam, zero, 1, n, ts->d_h,
                            (int)n_terms, coeffs, ts->d_c, s);
    }
    if (e != cudaSuccess) return cuda_fail(e, "H apply");
    {
    ProfScope ps("sa_dot_kernel", s);
    sa_dot_kernel<C><<<grid, kSaThreads, 0, s>>>(psi, lam, N, dpart);
    sa_sum_kernel<<<1, 32, 0, s>>>(dpart, grid, energy);
    }
    count_launch();
    count_launch();
    if (!grad || P == 0) {
        e = cudaGetLastError();
        return e == cudaSuccess ? TCNG_OK : cuda_fail(e, "energy");
    }
    // reverse sweep over blocks of <= 2 qubits (parameterised gates fused too)
    PlanOptions ob = plan_options(st->dt, false);
    ob.fuse_width = 2;
    ob.unfused = 0;
    DevPlan* dq = get_plan(n, ops, n_ops, pool, n_mat, P, ob);
    SaPlan* sp = get_saplan(dq);
    C* table = static_cast<C*>(plan_table(dq, sizeof(C), 1));
    if (!table) return fail(TCNG_ENOMEM, "matrix table");
    const Plan& pl = dq->plan;
    e = launch_build_matrices<C>(dq->d_bblocks, (int)pl.bblocks.size(), dq->d_bops, dq->d_pool, params, P, table,
                                 pl.table_size, 1, s);
    if (e != cudaSuccess) return cuda_fail(e, "block matrices");
    const int ng = std::max(1, sp->n_grad_blocks);
    double* npart = static_cast<double*>(c.scratch("sa_npart", sizeof(double) * 32 * (size_t)grid * ng));
    double* Nfin = static_cast<double*>(c.scratch("sa_n", sizeof(double) * 32 * (size_t)ng));
    double* contrib = static_cast<double*>(c.scratch("sa_contrib", sizeof(double) * std::max(1, sp->n_ents)));
    if (!npart || !Nfin || !contrib) return fail(TCNG_ENOMEM, "state-pass adjoint scratch");
    // scratch may have moved: re-read lambda
    lam = static_cast<C*>(c.scratch("sa_lambda", sizeof(C) * (size_t)N));
    // blocks of <= 2 qubits run in fused segments (one pass over both states per
    // segment): consecutive blocks, last first, while their qubits and the lowest
    // qubits fit in the tile
    constexpr int TB = sizeof(C) == 8 ? 12 : 11;
    int tbits;
    unsigned long long cmask;
    sa_tile_geometry<C>(n, &tbits, &cmask);
    std::vector<unsigned long long> qms;
    std::vector<int> ks;
    for (const SaPlan::Blk& b : sp->blocks) {
        qms.push_back(b.qmask);
        ks.push_back(b.k);
    }
    for (const SaStep& st_ : plan_reverse_steps(qms, ks, n, tbits, cmask)) {
        if (st_.tmask) {
            SaSeg sg{};
            sg.tmask = st_.tmask;
            sg.tbits = tbits;
            sg.nblk = (int)st_.blk.size();
            for (int i = 0; i < sg.nblk; ++i) {
                const SaPlan::Blk& b = sp->blocks[st_.blk[i]];
                SaSegBlk& sb = sg.b[i];
                sb.k = b.k;
                sb.diag = b.diag;
                sb.grad = b.grad;
                sb.out_off = b.out_off;
                const int q0 = __builtin_ctzll(b.qmask);
                const unsigned long long rest = b.qmask & (b.qmask - 1);
                sb.tb0 = __builtin_popcountll(st_.tmask & ((1ull << q0) - 1));
                sb.tb1 = rest ? __builtin_popcountll(st_.tmask & ((1ull << __builtin_ctzll(rest)) - 1)) : -1;
            }
            e = launch_seg<C, TB>(psi, lam, table, sg, n, npart, grid, s);
            if (e != cudaSuccess) return cuda_fail(e, "adjoint segment kernel");
            continue;
        }
        const SaPlan::Blk& b = sp->blocks[st_.blk[0]];   // 3..5 qubits, no parameter: each state on its own
        const C* U = table + b.out_off;
        for (C* x : {psi, lam}) {
            if (b.k == 3)
                sa_uncompute_kernel<C, 3><<<grid, kSaThreads, 0, s>>>(x, U, b.diag, b.qmask, n);
            else if (b.k == 4)
                sa_uncompute_kernel<C, 4><<<grid, kSaThreads, 0, s>>>(x, U, b.diag, b.qmask, n);
            else
                sa_uncompute_kernel<C, 5><<<grid, kSaThreads, 0, s>>>(x, U, b.diag, b.qmask, n);
            count_launch();
        }
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "adjoint block kernel");
    }
    ProfScope ps("sa_grad_kernels", s);
    if (sp->n_ents > 0) {
        sa_nfinal_kernel<<<(sp->n_grad_blocks * 32 + 255) / 256, 256, 0, s>>>(npart, grid, sp->n_grad_blocks, Nfin);
        sa_grad_kernel<<<(sp->n_ents + 63) / 64, 64, 0, s>>>(sp->d_ents, sp->n_ents, dq->d_bops, dq->d_pool, params,
                                                             Nfin, contrib);
        count_launch();
        count_launch();
    }
    sa_param_sum_kernel<<<(P + 255) / 256, 256, 0, s>>>(sp->d_start, sp->d_list, contrib, P, grad);
    count_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "gradient assembly");
    return TCNG_OK;
}

template tcng_status run_state_adjoint<float2>(tcng_state*, int, const tcng_gate*, size_t, const double*, size_t,
                                               const double*, int, const tcng_pauli*, size_t, const double*,
                                               double*, double*, cudaStream_t);
template tcng_status run_state_adjoint<double2>(tcng_state*, int, const tcng_gate*, size_t, const double*, size_t,
                                                const double*, int, const tcng_pauli*, size_t, const double*,
                                                double*, double*, cudaStream_t);

}  // namespace tcng

// Host-only summary of the state-pass adjoint's plan: the reverse sweep's steps
// and the passes of lambda = H psi (no device call).
extern "C" const char* tcng_describe_state_adjoint(int n, const tcng_gate* ops, size_t n_ops,
                                                   const double* mat_pool, size_t n_mat, int P,
                                                   const tcng_pauli* H, size_t n_terms, tcng_dtype dt) {
    using namespace tcng;
    static thread_local std::string out;
    try {
        if (dt != TCNG_C64 && dt != TCNG_C128) throw std::invalid_argument("bad dtype");
        if (n_terms && !H) throw std::invalid_argument("null terms");
        Plan pl;
        pl.n = n;
        pl.P = P;
        pl.opt = plan_options(dt, false);
        pl.opt.fuse_width = 2;   // as the state-pass adjoint plans its blocks
        pl.opt.unfused = 0;
        pl.ops = import_ops(n, ops, n_ops, n_mat, P, mat_pool);
        build_plan(pl);
        int tbits;
        unsigned long long cmask;
        if (dt == TCNG_C64)
            sa_tile_geometry<float2>(n, &tbits, &cmask);
        else
            sa_tile_geometry<double2>(n, &tbits, &cmask);
        std::vector<unsigned long long> qms;
        std::vector<int> ks;
        for (const Block& b : pl.blocks) {
            qms.push_back(b.qmask);
            ks.push_back(b.k);
        }
        const std::vector<SaStep> steps = plan_reverse_steps(qms, ks, n, tbits, cmask);
        std::vector<HamBin> bins;
        const bool tiled = plan_ham_passes(H, n_terms, tbits, cmask, bins);
        int nseg = 0;
        for (const SaStep& st : steps) nseg += st.tmask != 0;
        char buf[160];
        snprintf(buf, sizeof buf, "blocks=%zu segments=%d lone=%d tbits=%d hampasses=%d\n", pl.blocks.size(),
                 nseg, (int)steps.size() - nseg, tbits, tiled ? (int)bins.size() : -1);
        out = buf;
        for (const SaStep& st : steps) {
            snprintf(buf, sizeof buf, "%s tmask=%llx blocks=", st.tmask ? "seg" : "lone", st.tmask);
            out += buf;
            for (size_t i = 0; i < st.blk.size(); ++i) {
                snprintf(buf, sizeof buf, "%s%d:%llx", i ? "," : "", st.blk[i], (unsigned long long)qms[st.blk[i]]);
                out += buf;
            }
            out += "\n";
        }
        if (tiled)
            for (const HamBin& b : bins) {
                snprintf(buf, sizeof buf, "ham tmask=%llx terms=", sa_pad_mask(b.mask, n, tbits));
                out += buf;
                bool first = true;
                for (const std::vector<int>* v : {&b.diag, &b.off})
                    for (int t : *v) {
                        snprintf(buf, sizeof buf, "%s%d", first ? "" : ",", t);
                        out += buf;
                        first = false;
                    }
                out += "\n";
            }
    } catch (const std::exception& ex) {
        out = std::string("error: ") + ex.what();
    }
    return out.c_str();
}
