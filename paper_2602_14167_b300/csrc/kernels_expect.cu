// Pauli-string expectations of complex64 states, 2^13-amplitude tiles (the fast
// form of the expectation pass; Sec. I.B, expectation_ps).
//
// One pass over the state evaluates every term whose X bits lie in the tile:
// <P> = sum_x Re( i^{#Y} conj(psi[x ^ m]) (-1)^{popc(x & z)} psi[x] ).
//
// Thread t of 512 holds tile offsets e + 2t + 1024 i (e = 0, 1; i = 0..7) in
// registers r = e + 2i, read as eight 16-byte pairs.  For a term with X mask m:
//   * m's bits 1..9 (xt) name the partner thread, m's bits 10..12 (XR) permute
//     the pairs, m's bit 0 swaps the two amplitudes of a pair;
//   * the Z parity splits into the thread's part (tile bits 1..9, a bit per term
//     prepared once per pass), the tile's part (global bits, one ballot per tile
//     for all terms) and the register part (tile bits 0, 10, 11, 12: a butterfly
//     with +-1 factors).
// The host sorts the pass's terms into runs of one form (XR, swap, Re/Im, and
// the warp-skip bit below); the kernel dispatches once per run to code
// specialised on the form, so the partner pairs are read at fixed offsets from
// one base, and takes two terms of a run per step in one basic block.  The term
// constants are a kernel parameter (constant bank).  A Pauli string is
// Hermitian, so the terms of x and x ^ m are complex conjugates: one member of
// each pair, doubled, gives the same sum.  With XR != 0 only the register pairs
// with XR's top bit clear are evaluated (four partner loads instead of eight);
// otherwise, with X bits on tile bits 6..9 (warp bits), the warps on one side of
// the lowest such bit (alternating per tile) skip the term.  The butterflies run
// on packed FP32 pairs.  Per term and tile each thread adds its value, times the
// term's scale and sign, to its own FP32 sum in shared memory; every 64 tiles the
// warps fold those sums into FP64 in a fixed order.  Each tile's base index is
// one warp OR-reduction.
// Tiles whose bit runs fit a tensor map arrive by one TMA copy (warp 0 refills a
// buffer once every warp has released it).  Others (gathered qubits scattered
// over more than five dimensions) are copied by all 512 threads with 16-byte
// cp.async pieces, which stream these scattered rows at the contiguous rate
// where per-row TMA copies do not; each warp loads its share of tile i + 2 at
// the end of tile i, once every warp has left tile i - 1.
#include <cuda_runtime.h>

#include <algorithm>

#include "device.cuh"
#include "launch.hpp"
#include "tile_io.cuh"

namespace tcng {

namespace {

__device__ __forceinline__ void cp_async16(void* dst_smem, const void* src_gmem) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst_smem)), "l"(src_gmem) : "memory");
}
// The mbarrier counts one arrival when all of this thread's earlier cp.async copies land.
__device__ __forceinline__ void cp_async_arrive(uint64_t* bar) {
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Global element offset (from the tile base) of tile element x: the low chunk
// bits stay, the row bits land on the gathered qubits.  Linear in x (an OR of
// per-bit parts), so disjoint parts of x can be mapped separately.
__device__ __forceinline__ long long ef_tile_offset(const DevPass& p, int x) {
    return (long long)(x & ((1 << p.chunk) - 1)) | chunk_offset(p, x >> p.chunk);
}

constexpr int kEfTileBits = 13;
constexpr int kEfNbuf = 3;

struct EfTerm {          // a term of the pass, prepared once per CTA (32 bytes)
    float2 s1, s2, s3;   // (-1)^{z bit} of pair-index bits 0, 1, 2 (tile bits 10, 11, 12), duplicated
    float sx;            // (-1)^{z bit} of tile bit 0
    int32_t code;        // bits 0..8: xt (partner thread t ^ xt); 9..14: form (0: Z only, else
                         // 1 + 4 XR + 2 swap + im); 15..17: wskip + 1 (warps with bit wskip of the
                         // warp index xor tile parity set skip the term; 0: none)
};
struct EfPass {          // the pass's term constants: a kernel parameter, read from the
                         // constant bank at the (warp-uniform) term index
    EfTerm e[kExpTermsPerPass];
    float sf[kExpTermsPerPass];   // Re(i^ny w) sign x (2: half forms and the warp-half form)
    // terms sorted by (form, wskip): run r holds terms run_end[r - 1] .. run_end[r] - 1,
    // all with form and wskip + 1 packed in run_code[r] (form | (wskip + 1) << 6)
    int nrun;
    int run_code[kExpTermsPerPass];
    int run_end[kExpTermsPerPass];
};

// Global index of a tile's offset 0 (tile_global_base) by one warp OR-reduction:
// lane i holds 1 << rest[i] split into 32-bit halves (zero for i >= nrest).
__device__ __forceinline__ long long ef_tile_base(uint32_t tile, uint32_t bit_lo, uint32_t bit_hi, int lane) {
    const bool on = (tile >> lane) & 1u;
    const uint32_t lo = __reduce_or_sync(0xffffffffu, on ? bit_lo : 0u);
    const uint32_t hi = __reduce_or_sync(0xffffffffu, on ? bit_hi : 0u);
    return (long long)(((unsigned long long)hi << 32) | lo);
}

// sum_r (-1)^{popc(r & zr)} w_r over the 16 registers, w packed by register pair
// (W_i = (w_2i, w_2i+1)): three packed levels over the pair index, then the pair bit.
__device__ __forceinline__ float ef_butterfly(const float2 (&w)[kExpSlots / 2], const EfTerm& T) {
    float2 u[4], v[2];
#pragma unroll
    for (int k = 0; k < 4; ++k) u[k] = __ffma2_rn(T.s1, w[2 * k + 1], w[2 * k]);
#pragma unroll
    for (int k = 0; k < 2; ++k) v[k] = __ffma2_rn(T.s2, u[2 * k + 1], u[2 * k]);
    const float2 z = __ffma2_rn(T.s3, v[1], v[0]);
    return fmaf(T.sx, z.y, z.x);
}

// The same over the four register pairs whose index has bit K clear (pair jj: the
// index with a 0 inserted at bit K).
template <int K>
__device__ __forceinline__ float ef_butterfly_half(const float2 (&w)[kExpSlots / 4], const EfTerm& T) {
    const float2 sa = K == 0 ? T.s2 : T.s1, sb = K == 2 ? T.s2 : T.s3;
    const float2 u0 = __ffma2_rn(sa, w[1], w[0]), u1 = __ffma2_rn(sa, w[3], w[2]);
    const float2 z = __ffma2_rn(sb, u1, u0);
    return fmaf(T.sx, z.y, z.x);
}

template <bool SWAP, bool IM>
__device__ __forceinline__ float2 ef_pair(const float4 q, const float2 a0, const float2 a1) {
    float2 b0 = make_float2(q.x, q.y), b1 = make_float2(q.z, q.w);
    if (SWAP) {
        const float2 tmp = b0;
        b0 = b1;
        b1 = tmp;
    }
    if (!IM) return make_float2(fmaf(b0.x, a0.x, b0.y * a0.y), fmaf(b1.x, a1.x, b1.y * a1.y));
    return make_float2(fmaf(b0.x, a0.y, -b0.y * a0.x), fmaf(b1.x, a1.y, -b1.y * a1.x));
}

// Term with X bits: w_r = Re (IM: Im) of conj(partner) * a_r.  The partner of
// register pair i is pair i ^ XR of thread t ^ xt: pb[512 (i ^ XR)] with pb the
// partner thread's first pair.  XR != 0: the half form (pairs with bit K of i
// clear, K = XR's top bit; the 2 is in the term's scale).  (Taking the partner
// from the thread's own registers when xt = 0 is left out: those forms raise the
// register count of the whole term loop past the limit.)
template <int XR, bool SWAP, bool IM>
__device__ __forceinline__ float ef_xterm(const float2 (&a)[kExpSlots], const float4* __restrict__ pb,
                                          const EfTerm& T) {
    if constexpr (XR != 0) {
        constexpr int K = XR >= 4 ? 2 : (XR >= 2 ? 1 : 0);
        float2 w[kExpSlots / 4];
#pragma unroll
        for (int jj = 0; jj < kExpSlots / 4; ++jj) {
            const int i = ((jj >> K) << (K + 1)) | (jj & ((1 << K) - 1));   // jj with a 0 inserted at bit K
            w[jj] = ef_pair<SWAP, IM>(pb[kExpThreads * (i ^ XR)], a[2 * i], a[2 * i + 1]);
        }
        return ef_butterfly_half<K>(w, T);
    } else {
        float2 w[kExpSlots / 2];
#pragma unroll
        for (int i = 0; i < kExpSlots / 2; ++i) w[i] = ef_pair<SWAP, IM>(pb[kExpThreads * i], a[2 * i], a[2 * i + 1]);
        return ef_butterfly(w, T);
    }
}

// The terms j .. end - 1 of one run (one form): two terms per step in one basic
// block, so that the second term's partner reads overlap the first one's products.
template <int XR, bool SWAP, bool IM>
__device__ __forceinline__ void ef_run(const float2 (&a)[kExpSlots], const float4* __restrict__ buf4, int tid,
                                       const EfPass& ef, int j, int end, uint32_t fm, float* __restrict__ acc) {
    auto scale = [&](int k) { return __uint_as_float(__float_as_uint(ef.sf[k]) ^ (((fm >> k) & 1u) << 31)); };
    for (; j + 1 < end; j += 2) {
        float* ap0 = acc + j * kExpThreads + tid;
        float* ap1 = ap0 + kExpThreads;
        const float acc0 = *ap0, acc1 = *ap1;
        const float v0 = ef_xterm<XR, SWAP, IM>(a, buf4 + (tid ^ (ef.e[j].code & 511)), ef.e[j]);
        const float v1 = ef_xterm<XR, SWAP, IM>(a, buf4 + (tid ^ (ef.e[j + 1].code & 511)), ef.e[j + 1]);
        *ap0 = fmaf(scale(j), v0, acc0);
        *ap1 = fmaf(scale(j + 1), v1, acc1);
    }
    if (j < end) {
        float* ap = acc + j * kExpThreads + tid;
        const float accv = *ap;
        const float v = ef_xterm<XR, SWAP, IM>(a, buf4 + (tid ^ (ef.e[j].code & 511)), ef.e[j]);
        *ap = fmaf(scale(j), v, accv);
    }
}
// ... of the Z-only terms, two per step.
__device__ __forceinline__ void ef_run_z(const float2 (&pz)[kExpSlots / 2], int tid, const EfPass& ef, int j,
                                         int end, uint32_t fm, float* __restrict__ acc) {
    auto scale = [&](int k) { return __uint_as_float(__float_as_uint(ef.sf[k]) ^ (((fm >> k) & 1u) << 31)); };
    for (; j + 1 < end; j += 2) {
        float* ap0 = acc + j * kExpThreads + tid;
        float* ap1 = ap0 + kExpThreads;
        const float acc0 = *ap0, acc1 = *ap1;
        const float v0 = ef_butterfly(pz, ef.e[j]), v1 = ef_butterfly(pz, ef.e[j + 1]);
        *ap0 = fmaf(scale(j), v0, acc0);
        *ap1 = fmaf(scale(j + 1), v1, acc1);
    }
    if (j < end) {
        float* ap = acc + j * kExpThreads + tid;
        const float accv = *ap;
        *ap = fmaf(scale(j), ef_butterfly(pz, ef.e[j]), accv);
    }
}

__global__ void __launch_bounds__(kExpThreads, 1)
    expect_fast_kernel(const float2* __restrict__ state, const long long* __restrict__ item_off,
                       const __grid_constant__ DevPass p, const __grid_constant__ ExpPass ep, TileCtx tc,
                       double* __restrict__ partial, int n_out, unsigned* __restrict__ err,
                       const __grid_constant__ TmaTile tma, const __grid_constant__ EfPass ef) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int tile_elems = 1 << kEfTileBits;
    float2* bufs = reinterpret_cast<float2*>(smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u));
    uint64_t* bars = reinterpret_cast<uint64_t*>(bufs + (size_t)kEfNbuf * tile_elems);
    uint64_t* ebars = bars + kEfNbuf;                             // buffer released by every warp
    float* acc = reinterpret_cast<float*>(ebars + kEfNbuf);      // [term][thread]
    __shared__ double red[kExpThreads / 32][kExpTermsPerPass];
    __shared__ unsigned long long szg[kExpTermsPerPass];         // Z mask on global bits
    __shared__ int s_abort, s_hasz;
    __shared__ long long s_koff[3];   // cp.async form: offsets of tile elements 1024, 2048, 4096
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int item = blockIdx.y;
    const int nt = ep.nterms;
    for (int i = tid; i < (kExpThreads / 32) * kExpTermsPerPass; i += kExpThreads) (&red[0][0])[i] = 0.0;
    for (int i = tid; i < kExpTermsPerPass * kExpThreads; i += kExpThreads) acc[i] = 0.f;
    if (tid == 0) s_hasz = 0;
    __syncthreads();
    if (tid < nt) {
        const ExpTerm T = ep.t[tid];
        szg[tid] = T.zm_glob;
        if (T.xm_tile == 0) s_hasz = 1;
    }
    // per thread and term: Z parity over tile bits 1..9
    uint32_t fm0 = 0;
    for (int j = 0; j < nt; ++j)
        fm0 |= (uint32_t)(__popc(((unsigned)tid << 1) & ep.t[j].zm_tile & 0x3feu) & 1) << j;
    // this lane's part of every tile base (ef_tile_base); the loop form past 32 global bits
    const bool wbase = p.nrest <= 32;
    const int rb = lane < p.nrest ? p.rest[lane] : -1;
    const uint32_t bit_lo = (rb >= 0 && rb < 32) ? 1u << rb : 0u, bit_hi = rb >= 32 ? 1u << (rb - 32) : 0u;
    auto tbase = [&](long long t) {
        const long long tt = t & (tc.tiles_per_item - 1);
        return wbase ? ef_tile_base((uint32_t)tt, bit_lo, bit_hi, lane) : tile_global_base(p, tt);
    };
    const bool simt = tma.rank == 0;   // no tile map: cp.async pieces by every thread
    if (tid == 0) {
        for (int i = 0; i < kEfNbuf; ++i) {
            mbar_init(&bars[i], simt ? (uint32_t)kExpThreads : 1u);
            mbar_init(&ebars[i], (uint32_t)(kExpThreads / 32));
        }
        for (int k = 0; k < 3; ++k) s_koff[k] = ef_tile_offset(p, 1024 << k);
        fence_mbar_init();
        s_abort = 0;
    }
    __syncthreads();
    const bool hasz = s_hasz != 0;
    const long long t0 = (long long)item * tc.tiles_per_item;
    const long long t1 = t0 + tc.tiles_per_item;
    const long long first = t0 + blockIdx.x;
    const long long stride = gridDim.x;
    // cp.async form: this thread copies pieces tid + 512 k (elements 2 tid + 1024 k, k = 0..7)
    const long long my_off = ef_tile_offset(p, 2 * tid);
    const float2* item_state = state + item_off[item];
    auto simt_load = [&](long long t, int bb) {
        const long long gb = tbase(t);
        float2* dst = bufs + (size_t)bb * tile_elems + 2 * tid;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const long long ko = ((k & 1) ? s_koff[0] : 0) | ((k & 2) ? s_koff[1] : 0) | ((k & 4) ? s_koff[2] : 0);
            cp_async16(dst + 1024 * k, item_state + (gb + (my_off | ko)));
        }
        cp_async_arrive(&bars[bb]);
    };
    if (simt) {
        for (int i = 0; i < 2; ++i) {
            const long long t = first + i * stride;
            if (t < t1) simt_load(t, i);
        }
    } else if (warp == 0) {
        for (int i = 0; i < kEfNbuf; ++i) {
            const long long t = first + i * stride;
            if (t < t1) issue_tile_load(state, item_off, p, tc, t, bufs + (size_t)i * tile_elems, &bars[i], lane, tma);
        }
    }
    const unsigned long long lane_zg = lane < nt ? szg[lane] : 0ull;
    auto flush = [&]() {   // per-thread FP32 sums -> warp sum (fixed order) -> FP64
        for (int j = 0; j < nt; ++j) {
            float v = acc[j * kExpThreads + tid];
            acc[j * kExpThreads + tid] = 0.f;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) red[warp][j] += (double)v;
        }
    };
    int it = 0;
    for (long long t = first; t < t1; t += stride, ++it) {
        const int b = it % kEfNbuf;
        const float2* buf = bufs + (size_t)b * tile_elems;
        if (!mbar_wait_bounded(&bars[b], (uint32_t)((it / kEfNbuf) & 1), err)) s_abort = 1;
        const long long gbase = tbase(t);
        // the tile's part of every term's Z parity: one term per lane, one ballot
        const uint32_t fm =
            fm0 ^ __ballot_sync(0xffffffffu, (__popcll((unsigned long long)gbase & lane_zg) & 1) != 0);
        const float4* buf4 = reinterpret_cast<const float4*>(buf);
        float2 a[kExpSlots];
#pragma unroll
        for (int i = 0; i < kExpSlots / 2; ++i) {
            const float4 q = buf4[tid + kExpThreads * i];
            a[2 * i] = make_float2(q.x, q.y);
            a[2 * i + 1] = make_float2(q.z, q.w);
        }
        float2 pz[kExpSlots / 2];   // |a_r|^2 for the Z-only terms, by register pair
        if (hasz) {
#pragma unroll
            for (int i = 0; i < kExpSlots / 2; ++i)
                pz[i] = make_float2(fmaf(a[2 * i].x, a[2 * i].x, a[2 * i].y * a[2 * i].y),
                                    fmaf(a[2 * i + 1].x, a[2 * i + 1].x, a[2 * i + 1].y * a[2 * i + 1].y));
        }
        for (int r = 0, j = 0; r < ef.nrun; j = ef.run_end[r], ++r) {
            const int code = ef.run_code[r], end = ef.run_end[r];
            const int wskip = (code >> 6) - 1;
            // one half of the warps carries a warp-form term (doubled); the halves take
            // turns tile by tile, so no warp runs ahead of the others
            if (wskip >= 0 && (((warp >> wskip) ^ it) & 1)) continue;
            switch (code & 63) {
            case 0: ef_run_z(pz, tid, ef, j, end, fm, acc); break;
#define TCNG_EF1(XR, SW, IM) \
    case 1 + 4 * (XR) + 2 * (SW) + (IM): ef_run<XR, SW, IM>(a, buf4, tid, ef, j, end, fm, acc); break;
#define TCNG_EF4(XR) TCNG_EF1(XR, 0, 0) TCNG_EF1(XR, 0, 1) TCNG_EF1(XR, 1, 0) TCNG_EF1(XR, 1, 1)
                TCNG_EF4(0) TCNG_EF4(1) TCNG_EF4(2) TCNG_EF4(3)
                TCNG_EF4(4) TCNG_EF4(5) TCNG_EF4(6) TCNG_EF4(7)
#undef TCNG_EF4
#undef TCNG_EF1
            default: break;
            }
        }
        if ((it & 63) == 63 || t + stride >= t1) flush();
        __syncwarp();
        if (lane == 0) mbar_arrive(&ebars[b]);   // this warp is done with buf
        if (simt) {   // this warp's share of tile it + 2, into the buffer of tile it - 1
            const long long tn = t + 2 * stride;
            if (tn < t1) {
                if (it >= 1 && !mbar_wait_bounded(&ebars[(it + 2) % kEfNbuf], (uint32_t)(((it - 1) / kEfNbuf) & 1), err))
                    s_abort = 1;
                simt_load(tn, (it + 2) % kEfNbuf);
            }
        } else if (warp == 0) {
            const long long tn = t + (long long)kEfNbuf * stride;
            if (tn < t1) {
                if (!mbar_wait_bounded(&ebars[b], (uint32_t)((it / kEfNbuf) & 1), err)) s_abort = 1;
                __syncwarp();
                issue_tile_load(state, item_off, p, tc, tn, bufs + (size_t)b * tile_elems, &bars[b], lane, tma);
            }
        }
        if (s_abort) break;
    }
    asm volatile("cp.async.wait_all;" ::: "memory");   // this thread's copies (cp.async form)
    if (s_abort && tid == 0 && !simt) {   // drain loads still in flight before the shared memory goes away
        for (int i = 0; i < kEfNbuf; ++i) {
            const long long ti = first + (long long)(it + 1 + i) * stride;
            if (ti < t1) mbar_wait_bounded(&bars[(it + 1 + i) % kEfNbuf], (uint32_t)(((it + 1 + i) / kEfNbuf) & 1), err);
        }
    }
    __syncthreads();
    if (tid < nt) {   // warps in order
        double s = 0;
        for (int w = 0; w < kExpThreads / 32; ++w) s += red[w][tid];
        // a timed-out wait leaves the sum short: report NaN rather than a wrong value
        partial[((long long)item * n_out + ep.t[tid].out) * gridDim.x + blockIdx.x] = s_abort ? __longlong_as_double(0x7ff8000000000000ll) : s;
    }
}

}  // namespace

size_t expect_fast_smem_bytes() {
    return 128 + (size_t)kEfNbuf * (sizeof(float2) << kEfTileBits) + 16 * kEfNbuf +
           sizeof(float) * kExpTermsPerPass * kExpThreads;
}

cudaError_t launch_expect_fast(const float2* state, const long long* item_off, int items, const DevPass& p,
                               const ExpPass& ep, const TileCtx& tc, double* partial, int n_out, int nblk,
                               unsigned* err, cudaStream_t s, const TmaTile& tma) {
    if (p.m != kEfTileBits || tc.nbuf != kEfNbuf) return cudaErrorInvalidValue;
    // terms sorted by (form, wskip) into runs (stable: equal keys keep their order)
    auto key = [](const ExpTerm& T) {
        const uint32_t xr = (T.xm_tile >> 10) & 7u, xw = (T.xm_tile >> 6) & 15u;
        const int var = T.xm_tile == 0 ? 0 : 1 + 4 * (int)xr + 2 * (int)(T.xm_tile & 1u) + (T.ny & 1);
        const int wskip = (xr == 0 && xw) ? __builtin_ctz(xw) : -1;
        return var | ((wskip + 1) << 6);
    };
    ExpPass eps = ep;
    const int nt = ep.nterms < kExpTermsPerPass ? ep.nterms : kExpTermsPerPass;
    std::stable_sort(eps.t, eps.t + nt, [&](const ExpTerm& x, const ExpTerm& y) { return key(x) < key(y); });
    EfPass ef{};
    for (int j = 0; j < nt; ++j) {
        const int k = key(eps.t[j]);
        if (ef.nrun == 0 || ef.run_code[ef.nrun - 1] != k) ef.run_code[ef.nrun++] = k;
        ef.run_end[ef.nrun - 1] = j + 1;
    }
    for (int j = 0; j < nt; ++j) {
        const ExpTerm& T = eps.t[j];
        EfTerm& x = ef.e[j];
        auto sgn = [&](int b) { return ((T.zm_tile >> b) & 1u) ? -1.f : 1.f; };
        x.s1 = make_float2(sgn(10), sgn(10));
        x.s2 = make_float2(sgn(11), sgn(11));
        x.s3 = make_float2(sgn(12), sgn(12));
        x.sx = sgn(0);
        const uint32_t xr = (T.xm_tile >> 10) & 7u;
        const int var = T.xm_tile == 0 ? 0 : 1 + 4 * (int)xr + 2 * (int)(T.xm_tile & 1u) + (T.ny & 1);
        // warp form: X on tile bits 6..9 (thread bits 5..8 = warp bits 0..3), none on 10..12
        const uint32_t xw = (T.xm_tile >> 6) & 15u;
        const int wskip = (xr == 0 && xw) ? __builtin_ctz(xw) : -1;
        x.code = (int)((T.xm_tile >> 1) & 511u) | (var << 9) | ((wskip + 1) << 15);
        // Re(i^ny w) = -Re w (ny = 2), -Im w (ny = 1), Im w (ny = 3); the half forms and the
        // warp-half form count each pair (x, x ^ m) once, doubled
        const float sg = ((T.ny & 3) == 1 || (T.ny & 3) == 2) ? -1.f : 1.f;
        ef.sf[j] = (xr != 0 || wskip >= 0) ? 2.f * sg : sg;
    }
    static bool attr[kMaxDeviceSlots] = {};   // the attribute is per device
    const int d = device_slot();
    if (!attr[d]) {
        const cudaError_t e = cudaFuncSetAttribute(expect_fast_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)expect_fast_smem_bytes());
        if (e != cudaSuccess) return e;
        attr[d] = true;
    }
    dim3 grid((unsigned)nblk, (unsigned)items);
    expect_fast_kernel<<<grid, kExpThreads, expect_fast_smem_bytes(), s>>>(state, item_off, p, eps, tc, partial,
                                                                           n_out, err, tma, ef);
    count_launch();
    return cudaGetLastError();
}

}  // namespace tcng
