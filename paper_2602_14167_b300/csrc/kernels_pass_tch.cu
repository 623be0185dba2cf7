// Tile passes whose register stages run on the tensor cores with an FP16
// split (complex64 states, unitary plans, one W set for every tile).
//
// A register stage is the real GEMM of kernels_pass_tc.cu: the tile's 512 rows
// of 32 reals (re, im of one thread's 16 amplitudes) times W_s, the 32x32 real
// form of the stage's fused 16x16 unitary.  Here both operands are split into
// FP16 hi + lo (x = hi + lo to ~2^-23 relative), and one FP32 accumulator per
// output takes lo*W_hi + hi*W_lo + hi*W_hi through six kind::f16 MMAs (M=128,
// N=32, K=16); lo*W_lo (~2^-24) is dropped.
//
// Range.  FP16 spans 2^-24 .. 65504, so each tile is multiplied by a power of
// two (exact) before its first stage, chosen so that the tile's largest |re| or
// |im| lands in [2^7, 2^8).  Every stage of a unitary plan keeps the tile norm
// (the gates act inside the tile), and no element exceeds the norm, so later
// stages see values below sqrt(8192) * 2^8 < 2^15; elements far below the
// maximum keep an absolute accuracy of ~2^-25 (subnormal halves), i.e. 2^-32 of
// the maximum.  After the last stage the tile is unscaled and its norm is
// restored to the norm it had before the pass (the tensor core's accumulation
// rounds toward zero, a small systematic shrink per stage).
//
// Why: FP16 operands take half the tensor-core time of the TF32 form and half
// its TMEM traffic, and a row's TMEM share (A hi 16 + A lo 16 + D 32 columns)
// leaves room for a second tile per 128-row slice:
//   * lock-step passes (the stages touch every tile bit, so every row of a tile
//     must be written before the next stage reads any) keep two tiles in flight,
//     each run by its own group of eight warps on its own barrier: one group's
//     shared-memory phases overlap the other's tensor-core round trips;
//   * independent-slice passes (two tile bits that no stage touches, so each
//     slice's 128 rows stay closed under the pass) run one tile per slice, the
//     slice pairs half a stage apart, as in the TF32 kernel.
// A seventeenth warp moves tiles (TMA or per-chunk bulk copies, tile_io.cuh).
// In the lock-step passes on the 128-byte-swizzled tile each stage may write its
// register bits to new shared-memory positions (planned on the host by
// lock_layouts below) so that every stage's reads and writes reach all bank
// slots.  The split's residual x - hi is one mixed-precision FMA per component.
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <cstdlib>

#include <algorithm>
#include <cstring>

#include "capi_internal.hpp"
#include "device.cuh"
#include "tc.cuh"
#include "tile_io.cuh"

namespace tcng {

namespace {

constexpr int TH_THREADS = 512;                    // compute threads: 4 slices x 4 warps
constexpr int TH_CTA_THREADS = TH_THREADS + 32;    // + one producer warp
constexpr int TH_PRODUCER_WARP = TH_THREADS / 32;
constexpr int TH_TILE_BITS = 13;
constexpr int TH_TILE_ELEMS = 1 << TH_TILE_BITS;
constexpr uint32_t TH_TILE_BYTES = sizeof(float2) << TH_TILE_BITS;   // 64 KiB
constexpr uint32_t TH_TMEM_COLS = 512;             // 4 slices x 2 tiles x (A hi 16 + A lo 16 + D 32)
constexpr int TH_MAX_STAGES = kMaxWideStages;      // stages per pass (W of all resident)
constexpr int TH_MAX_STAGES_3BUF = 7;              // with three tile buffers
constexpr int TH_MAX_STAGES_5 = 2;                 // 32-amplitude stages (16 KiB W each)
constexpr int FORM_PLAIN = 0, FORM_ROT = 1, FORM_SWZ = 2;

struct StageH {             // per-stage constants, shared memory (64 bytes)
    int sr[4];              // 1 << register tile bit i
    int hm[6];              // ~((1 << b) - 1) for the bits the row index skips (ascending)
    int nj;                 // register bits on tile bits 0..3
    int sr4;                // 32-amplitude stages: 1 << register tile bit 4
    int srz[4];             // sr on the 128-byte-swizzled tile (o ^ ((o >> 3) & 0xE))
    int hmw[4], srzw[4];    // lock-step stages on the swizzled tile: hm and srz of the layout
                            // the stage writes (its register bits moved, the planner's choice)
};

struct PassTchArgs {
    int gb0, gb1;               // independent-slice passes: tile bits fixed per slice
    int renorm;                 // restore each tile's (slice's) norm after the last stage
    const TcsStage* tcs;        // this pass's stages
    const uint8_t* lay;         // per stage: read / write positions of the register bits (or null)
    const unsigned char* wops;  // FP16 W operands of the plan's tensor-core stages
    long long total_tiles;
    unsigned* err;
    float2* state;
    const long long* item_off;
    TileCtx tc;
};

__device__ __forceinline__ void sync_slice(int slice) {   // the 128 threads of one slice
    asm volatile("bar.sync %0, %1;" ::"r"(1 + slice), "r"(128) : "memory");
}

// Power-of-two scale c with m*c in [2^7, 2^8) (m >= 0; c and 1/c stay normal).
__device__ __forceinline__ void tile_scale(float m, float& c, float& ic) {
    const int e = (int)((__float_as_uint(m) >> 23) & 0xffu);
    const int f = min(253, max(1, 261 - e));
    c = __uint_as_float((uint32_t)f << 23);
    ic = __uint_as_float((uint32_t)(254 - f) << 23);
}

// x = hi + lo, both FP16 (re in the low half of each 32-bit word).  The residual
// x - hi is exact in FP32; it is formed by a mixed-precision FMA, hi * (-1) + x,
// straight from the packed halves.
__device__ __forceinline__ void split_f16(float2 x, uint32_t& hi, uint32_t& lo) {
    asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(hi) : "f"(x.y), "f"(x.x));
    float r0, r1;
    asm("{\n\t.reg .f16 h0, h1, m;\n\tmov.b32 {h0, h1}, %2;\n\tmov.b16 m, 0xBC00;\n\t"
        "fma.rn.f32.f16 %0, h0, m, %3;\n\tfma.rn.f32.f16 %1, h1, m, %4;\n\t}"
        : "=f"(r0), "=f"(r1)
        : "r"(hi), "f"(x.x), "f"(x.y));
    asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(lo) : "f"(r1), "f"(r0));
}

// a[s] holds register value s ^ tau (tau only on slots 0..nj-1): permute so
// that a[v] holds value v (the permutation is its own inverse).
__device__ __forceinline__ void unrotate_h(float2 (&a)[16], int tau, int nj) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (k < nj) {
            const bool sw = (tau >> k) & 1;
#pragma unroll
            for (int s = 0; s < 16; ++s)
                if (!(s & (1 << k))) {
                    const float2 x = a[s], y = a[s | (1 << k)];
                    a[s] = sw ? y : x;
                    a[s | (1 << k)] = sw ? x : y;
                }
        }
    }
}

// Shared-memory slots of this thread's 16 amplitudes for stage S: row g (the
// tile index with zeros at the register bits), tau the XOR rotation (ROT).
template <int FORM>
__device__ __forceinline__ void stage_slots(const StageH& S, int g, int tau, int (&L)[16]) {
    int sr[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) sr[i] = FORM == FORM_SWZ ? S.srz[i] : S.sr[i];
    if (FORM == FORM_SWZ) g ^= (g >> 3) & 0xe;   // slot offset o lies at o ^ ((o >> 3) & 0xE) (linear in o)
    int stau = 0;
    if (FORM == FORM_ROT && S.nj) {
#pragma unroll
        for (int i = 0; i < 4; ++i) stau |= ((tau >> i) & 1) ? sr[i] : 0;
    }
    L[0] = g | stau;
#pragma unroll
    for (int v = 1; v < 16; ++v)
        L[v] = L[v & (v - 1)] ^ ((v & 1) ? sr[0] : (v & 2) ? sr[1] : (v & 4) ? sr[2] : sr[3]);
}

// Row index of this thread in a lock-step stage: tid with zeros inserted at the
// four register bits.
__device__ __forceinline__ int lock_row(const StageH& S, int tid) {
    int g = tid;
#pragma unroll
    for (int i = 0; i < 4; ++i) g += g & S.hm[i];
    return g;
}
// The same row in the layout the stage writes, and its slots there (swizzled tile).
__device__ __forceinline__ int lock_row_w(const StageH& S, int tid) {
    int g = tid;
#pragma unroll
    for (int i = 0; i < 4; ++i) g += g & S.hmw[i];
    return g;
}
__device__ __forceinline__ void stage_slots_wswz(const StageH& S, int g, int (&L)[16]) {
    L[0] = g ^ ((g >> 3) & 0xe);
#pragma unroll
    for (int v = 1; v < 16; ++v)
        L[v] = L[v & (v - 1)] ^ ((v & 1) ? S.srzw[0] : (v & 2) ? S.srzw[1] : (v & 4) ? S.srzw[2] : S.srzw[3]);
}
// ... in an independent-slice stage: the slice's 128 rows, the slice index on
// the pass's two fixed tile bits.
__device__ __forceinline__ int group_row(const StageH& S, int tid, int gb0, int gb1) {
    int g = tid & 127;
#pragma unroll
    for (int i = 0; i < 6; ++i) g += g & S.hm[i];
    return g | (((tid >> 7) & 1) << gb0) | (((tid >> 8) & 1) << gb1);
}

// Stage constants: the row index skips the register bits and, in passes with
// fixed tile bits per slice (or row block), those bits (gb0 only when gb1 < 0).
__device__ __forceinline__ void load_stage(const TcsStage* tcs, int nst, int gb0, int gb1, bool grouped,
                                           StageH* sst, int tid, int nthreads, const uint8_t* lay = nullptr) {
    for (int i = tid; i < nst; i += nthreads) {
        const TcsStage S = tcs[i];
        StageH d;
        int skip[7], ns = 0;
        for (int r = 0; r < 4; ++r) {
            const int pos = lay ? lay[8 * i + r] : S.rbit[r];
            d.sr[r] = 1 << pos;
            skip[ns++] = pos;
        }
        {   // the layout this stage writes (the same one without a layout table)
            int wp[4];
            for (int r = 0; r < 4; ++r) {
                wp[r] = lay ? lay[8 * i + 4 + r] : S.rbit[r];
                const int o = 1 << wp[r];
                d.srzw[r] = o ^ ((o >> 3) & 0xe);
            }
            for (int x = 1; x < 4; ++x)
                for (int y = x; y > 0 && wp[y - 1] > wp[y]; --y) {
                    const int t = wp[y];
                    wp[y] = wp[y - 1];
                    wp[y - 1] = t;
                }
            for (int r = 0; r < 4; ++r) d.hmw[r] = ~((1 << wp[r]) - 1);
        }
        d.sr4 = 0;
        if (S.nreg == 5) {
            d.sr4 = 1 << S.rbit[4];
            skip[ns++] = S.rbit[4];
        }
        if (grouped) {
            skip[ns++] = gb0;
            if (gb1 >= 0) skip[ns++] = gb1;
        }
        for (int x = 1; x < ns; ++x)
            for (int y = x; y > 0 && skip[y - 1] > skip[y]; --y) {
                const int t = skip[y];
                skip[y] = skip[y - 1];
                skip[y - 1] = t;
            }
        for (int k = 0; k < 6; ++k) d.hm[k] = k < ns ? ~((1 << skip[k]) - 1) : 0;
        d.nj = S.nj;
        for (int k = 0; k < 4; ++k) d.srz[k] = d.sr[k] ^ ((d.sr[k] >> 3) & 0xe);
        sst[i] = d;
    }
}

// The six MMAs of one stage for one 128-row slice: D = lo*W_hi + hi*W_lo + hi*W_hi.
// A (TMEM): hi at column a, lo at a + 16, 8 columns per K step of 16 halves.
// W (shared memory, 128-byte rows [hi 32 | lo 32]): +32 bytes per K step (+2 in
// the descriptor's start field), the lo half at +64 bytes (+4).
__device__ __forceinline__ void stage_mmas(uint32_t d, uint32_t a, uint64_t dw) {
    constexpr uint32_t idesc = f16_idesc(128, 32);
    tc_mma_f16_ts(d, a + 16u, dw, idesc, 0);
    tc_mma_f16_ts(d, a + 24u, dw + 2u, idesc, 1);
    tc_mma_f16_ts(d, a, dw + 4u, idesc, 1);
    tc_mma_f16_ts(d, a + 8u, dw + 6u, idesc, 1);
    tc_mma_f16_ts(d, a, dw, idesc, 1);
    tc_mma_f16_ts(d, a + 8u, dw + 2u, idesc, 1);
}

__device__ __forceinline__ float warp_max(float m) {
#pragma unroll
    for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    return m;
}
__device__ __forceinline__ float row_max(const float2 (&x)[16]) {
    float m = 0.f;
#pragma unroll
    for (int v = 0; v < 16; ++v) m = fmaxf(m, fmaxf(fabsf(x[v].x), fabsf(x[v].y)));
    return m;
}
__device__ __forceinline__ float row_norm2(const float2 (&x)[16]) {
    float p4[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int v = 0; v < 16; ++v) p4[v & 3] = fmaf(x[v].x, x[v].x, fmaf(x[v].y, x[v].y, p4[v & 3]));
    return (p4[0] + p4[1]) + (p4[2] + p4[3]);
}
// sqrt(ti / to) * ic; tiles of zero norm keep their values (times ic)
__device__ __forceinline__ float norm_factor(int renorm, float ti, float to, float ic) {
    return (renorm && ti > 0.f && to > 0.f) ? sqrtf(ti) * rsqrtf(to) * ic : ic;
}

// Tile mover (warp TH_PRODUCER_WARP): loads run `ahead` tiles in front; a tile's
// buffer is stored once the compute side reports it done, and the load `ahead`
// tiles later goes into the same buffer once the store has read it.
template <int NBUF>
__device__ void tile_mover(const DevPass& p, const PassTchArgs& a, const TmaTile& tma, float2* bufs,
                           uint64_t* tile_bar, uint64_t* done_bar, volatile int* s_abort, long long first,
                           long long stride, long long my_tiles, int lane) {
    long long issued = 0;
    for (; issued < NBUF && issued < my_tiles; ++issued)
        issue_tile_load(a.state, a.item_off, p, a.tc, first + issued * stride, bufs + issued * TH_TILE_ELEMS,
                        &tile_bar[issued], lane, tma);
    for (long long i = 0; i < my_tiles; ++i) {
        const int b = (int)(i % NBUF);
        uint32_t done = 0;
        if (lane == 0) {
            const uint32_t par = (uint32_t)((i / NBUF) & 1);
            done = mbar_try_wait(&done_bar[b], par);
            const unsigned long long t0 = global_ns();
            for (uint32_t k = 1; !done; ++k) {
                if (*s_abort) break;
                done = mbar_try_wait(&done_bar[b], par);
                if (!done && (k & 255u) == 0 && global_ns() - t0 > kWaitLimitNs) {
                    atomicOr(a.err, ERR_TIMEOUT);
                    *s_abort = 1;
                    break;
                }
            }
        }
        if (!__shfl_sync(0xffffffffu, done, 0)) break;
        issue_tile_store(a.state, a.item_off, p, a.tc, first + i * stride, bufs + (size_t)b * TH_TILE_ELEMS,
                         lane, tma);
        if (issued < my_tiles) {
            bulk_wait_read<0>();
            __syncwarp();
            issue_tile_load(a.state, a.item_off, p, a.tc, first + issued * stride,
                            bufs + (size_t)b * TH_TILE_ELEMS, &tile_bar[b], lane, tma);
            ++issued;
        }
    }
    bulk_wait<0>();
    // after an abort the last loads may still be in flight: wait for them before
    // the shared memory goes away
    if (lane == 0)
        for (long long i = issued > NBUF ? issued - NBUF : 0; i < issued; ++i)
            mbar_wait_bounded(&tile_bar[i % NBUF], (uint32_t)((i / NBUF) & 1), a.err);
    __syncwarp();
}

// Tile mover for the lock-step kernel, whose two groups finish tiles in either
// order: buffer b holds tiles b, b + NBUF, b + 2 NBUF, ...; whichever buffer's
// tile is reported done first is stored first, and the buffer's next tile is
// loaded once the store has read it.
template <int NBUF>
__device__ void tile_mover_any(const DevPass& p, const PassTchArgs& a, const TmaTile& tma, float2* bufs,
                               uint64_t* tile_bar, uint64_t* done_bar, volatile int* s_abort,
                               volatile long long* s_issued, long long first, long long stride,
                               long long my_tiles, int lane) {
    long long cur[NBUF];   // tile in buffer b, or -1
    uint32_t ph[NBUF];     // done phases of buffer b seen so far
    int pending = 0;
#pragma unroll
    for (int b = 0; b < NBUF; ++b) {
        ph[b] = 0;
        cur[b] = b < my_tiles ? b : -1;
        if (cur[b] >= 0) {
            issue_tile_load(a.state, a.item_off, p, a.tc, first + (long long)b * stride,
                            bufs + (size_t)b * TH_TILE_ELEMS, &tile_bar[b], lane, tma);
            if (lane == 0) s_issued[b] = b;
            ++pending;
        }
    }
    unsigned long long t0 = global_ns();
    uint32_t spins = 0;
    while (pending > 0) {
        int hit = -1;
        if (lane == 0) {
#pragma unroll
            for (int b = 0; b < NBUF; ++b)
                if (hit < 0 && cur[b] >= 0 && mbar_try_wait(&done_bar[b], ph[b] & 1u)) hit = b;
        }
        hit = __shfl_sync(0xffffffffu, hit, 0);
        if (hit < 0) {
            int stop = 0;
            if (lane == 0 && (++spins & 255u) == 0) {
                if (*s_abort) {
                    stop = 1;
                } else if (global_ns() - t0 > kWaitLimitNs) {
                    atomicOr(a.err, ERR_TIMEOUT);
                    *s_abort = 1;
                    stop = 1;
                }
            }
            if (__shfl_sync(0xffffffffu, stop, 0)) break;
            continue;
        }
        t0 = global_ns();
#pragma unroll
        for (int b = 0; b < NBUF; ++b) {
            if (b != hit) continue;
            ++ph[b];
            issue_tile_store(a.state, a.item_off, p, a.tc, first + cur[b] * stride,
                             bufs + (size_t)b * TH_TILE_ELEMS, lane, tma);
            const long long nxt = cur[b] + NBUF;
            if (nxt < my_tiles) {
                bulk_wait_read<0>();
                __syncwarp();
                issue_tile_load(a.state, a.item_off, p, a.tc, first + nxt * stride,
                                bufs + (size_t)b * TH_TILE_ELEMS, &tile_bar[b], lane, tma);
                if (lane == 0) s_issued[b] = nxt;
                cur[b] = nxt;
            } else {
                cur[b] = -1;
                --pending;
            }
        }
    }
    bulk_wait<0>();
    // after an abort the loads still in flight must land before the shared memory
    // goes away: each buffer's last load is the tile in cur[b]
    if (lane == 0)
        for (int b = 0; b < NBUF; ++b)
            if (cur[b] >= 0) mbar_wait_bounded(&tile_bar[b], (uint32_t)((cur[b] / NBUF) & 1), a.err);
    __syncwarp();
}

// Wait until the tile mover has issued the load of tile `it` into its buffer.
// A buffer's tiles alternate between the two tile slots, so a slot can reach
// its next tile while the buffer's previous load (the other slot's tile) has not
// landed yet: its mbarrier is then two phases behind and a parity wait would
// pass on the older phase.  Once the load of `it` is issued, the previous one
// has been consumed, so the parity wait that follows is exact.
__device__ __forceinline__ bool wait_issued(volatile long long* s_issued, long long it, unsigned* err) {
    if (*s_issued == it) return true;
    const unsigned long long t0 = global_ns();
    for (uint32_t k = 1;; ++k) {
        __nanosleep(32);
        if (*s_issued == it) return true;
        if ((k & 255u) == 0 && global_ns() - t0 > kWaitLimitNs) {
            atomicOr(err, ERR_TIMEOUT);
            return false;
        }
    }
}

// 16 amplitudes of a row from the tile (pairs as 16-byte loads when register
// bit 0 is tile bit 0: slots v and v + 1 are then adjacent), and back.
template <int FORM>
__device__ __forceinline__ void load_row(const float2* buf, const int (&L)[16], bool pairs, float2 (&x)[16]) {
    if (FORM != FORM_ROT && pairs) {
#pragma unroll
        for (int v = 0; v < 16; v += 2) {
            const float4 q = *reinterpret_cast<const float4*>(buf + L[v]);
            x[v] = make_float2(q.x, q.y);
            x[v + 1] = make_float2(q.z, q.w);
        }
    } else {
#pragma unroll
        for (int v = 0; v < 16; ++v) x[v] = buf[L[v]];
    }
}
template <int FORM>
__device__ __forceinline__ void store_row(float2* buf, const int (&L)[16], bool pairs, const float2 (&x)[16]) {
    if (FORM != FORM_ROT && pairs) {
#pragma unroll
        for (int v = 0; v < 16; v += 2)
            *reinterpret_cast<float4*>(buf + L[v]) = make_float4(x[v].x, x[v].y, x[v + 1].x, x[v + 1].y);
    } else {
#pragma unroll
        for (int v = 0; v < 16; ++v) buf[L[v]] = x[v];
    }
}

__device__ __forceinline__ void sync_group(int grp) {   // the 256 threads of one group
    asm volatile("bar.sync %0, %1;" ::"r"(1 + grp), "r"(256) : "memory");
}
__device__ __forceinline__ bool sync_group_or(int grp, bool flag) {
    uint32_t r;
    asm volatile("{\n\t.reg .pred p, q;\n\tsetp.ne.u32 q, %1, 0;\n\t"
                 "bar.red.or.pred p, %2, 256, q;\n\tselp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(r)
                 : "r"((uint32_t)flag), "r"(1 + grp)
                 : "memory");
    return r != 0;
}

// ------------------------------------------------------- lock-step passes --
// The 16 compute warps form two groups of eight; each group runs whole tiles
// (its tiles are the CTA's tiles G, G + 2, ...) and syncs only on its own
// barrier, so one group's shared-memory phases overlap the other's tensor-core
// round trips.  A thread owns two rows of each stage (row blocks 2h and 2h + 1
// of the tile's four 128-row blocks, h = its warp's half of the group); the
// group's TMEM is 256 columns: per row block A hi 16 + A lo 16 + D 32.
template <int FORM, int NBUF>
__global__ void __launch_bounds__(TH_CTA_THREADS, 1)
    pass_tch_lock_kernel(const __grid_constant__ DevPass p, const PassTchArgs a,
                         const __grid_constant__ TmaTile tma) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char* base = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    const int nst = p.stage_count;
    unsigned char* wres = base;   // nst x 4 KiB, every stage's W
    float2* bufs = reinterpret_cast<float2*>(base + (size_t)nst * TH_W_BYTES);
    __shared__ uint64_t tile_bar[NBUF], done_bar[NBUF], mma_bar[2], w_bar;
    __shared__ long long s_issued[NBUF];
    __shared__ uint32_t tmem_base;
    __shared__ int s_abort;
    __shared__ float redm[2][8];
    __shared__ float2 redn[2][8];
    __shared__ StageH sst[TH_MAX_STAGES];
    const int tid = threadIdx.x, warp = __shfl_sync(0xffffffffu, tid >> 5, 0);
    const int lane = tid & 31;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_base)),
                     "r"(TH_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    load_stage(a.tcs, nst, 0, 0, false, sst, tid, TH_CTA_THREADS, FORM == FORM_SWZ ? a.lay : nullptr);
    if (tid == 0) {
        for (int i = 0; i < NBUF; ++i) {
            mbar_init(&tile_bar[i], 1);
            mbar_init(&done_bar[i], 1);
            s_issued[i] = -1;
        }
        mbar_init(&mma_bar[0], 1);
        mbar_init(&mma_bar[1], 1);
        mbar_init(&w_bar, 1);
        fence_mbar_init();
        s_abort = 0;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = __shfl_sync(0xffffffffu, tmem_base, 0);
    const long long first = blockIdx.x, stride = gridDim.x;
    const long long my_tiles = first < a.total_tiles ? (a.total_tiles - first + stride - 1) / stride : 0;
    if (warp == TH_PRODUCER_WARP) {
        tile_mover_any<NBUF>(p, a, tma, bufs, tile_bar, done_bar, &s_abort, s_issued, first, stride, my_tiles,
                             lane);
        tc_fence_before();
        __syncthreads();
        return;
    }
    if (tid == 0 && my_tiles > 0) {   // every stage's W: one bulk copy (consecutive operands)
        const uint32_t wb = (uint32_t)nst * TH_W_BYTES;
        mbar_arrive_expect_tx(&w_bar, wb);
        bulk_g2s(wres, a.wops + a.tcs[0].wh_off, wb, &w_bar);
    }
    if (my_tiles > 0 && !mbar_wait_bounded(&w_bar, 0u, a.err)) s_abort = 1;
    const int grp = warp >> 3, gw = warp & 7, quarter = warp & 3, half = gw >> 2;
    const uint32_t lane_base = tmem + ((uint32_t)(32 * quarter) << 16);
    const uint32_t gcol = (uint32_t)grp * 256u;
    uint32_t q = 0;
    for (long long it = grp; it < my_tiles; it += 2) {
        const int b = (int)(it % NBUF);
        float2* buf = bufs + (size_t)b * TH_TILE_ELEMS;
        const bool tile_ok = wait_issued(&s_issued[b], it, a.err) &&
                             mbar_wait_bounded(&tile_bar[b], (uint32_t)((it / NBUF) & 1), a.err);
        if (sync_group_or(grp, !tile_ok || *reinterpret_cast<volatile int*>(&s_abort) != 0)) {
            s_abort = 1;
            break;
        }
        // the tile's scale from its largest component: one extra read of row 0; row 1
        // stays in registers for the first stage
        float sc, isc;
        float2 x1[16];
        {
            const StageH& S = sst[0];
            const bool pairs = S.sr[0] == 1;
            float m = 0.f;
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                const int row = (2 * half + k) * 128 + quarter * 32 + lane;
                const int tau = (FORM == FORM_ROT && S.nj) ? (row & 15) >> (4 - S.nj) : 0;
                int L[16];
                stage_slots<FORM>(S, lock_row(S, row), tau, L);
                if (k == 0) {
                    float2 x[16];
                    load_row<FORM>(buf, L, pairs, x);
                    m = fmaxf(m, row_max(x));
                } else {
                    load_row<FORM>(buf, L, pairs, x1);
                    m = fmaxf(m, row_max(x1));
                }
            }
            m = warp_max(m);
            if (lane == 0) redm[grp][gw] = m;
            sync_group(grp);
            float mt = 0.f;
#pragma unroll
            for (int w = 0; w < 8; ++w) mt = fmaxf(mt, redm[grp][w]);
            tile_scale(mt, sc, isc);
        }
        float nin = 0.f;
        // one stage (first: stage 0, which takes row 1 from x1 and scales)
        auto stage = [&](const int s, const bool first) {
            const StageH& S = sst[s];
            const bool pairs = S.sr[0] == 1;
            // this thread's two rows (tile index with zeros at the register bits), for the
            // loads and again for the stores
            const int g0 = lock_row(S, (2 * half) * 128 + quarter * 32 + lane);
            const int g1 = lock_row(S, (2 * half + 1) * 128 + quarter * 32 + lane);
            // the same rows in the layout this stage writes (its register bits may move)
            const int gw0 = FORM == FORM_SWZ ? lock_row_w(S, (2 * half) * 128 + quarter * 32 + lane) : g0;
            const int gw1 = FORM == FORM_SWZ ? lock_row_w(S, (2 * half + 1) * 128 + quarter * 32 + lane) : g1;
#pragma unroll
            for (int kk = 0; kk < 2; ++kk) {
                const int k = first ? 1 - kk : kk;
                const int rb = 2 * half + k;
                const int row = rb * 128 + quarter * 32 + lane;
                const int tau = (FORM == FORM_ROT && S.nj) ? (row & 15) >> (4 - S.nj) : 0;
                int L[16];
                stage_slots<FORM>(S, k ? g1 : g0, tau, L);
                float2 x[16];
                if (first && kk == 0) {
#pragma unroll
                    for (int v = 0; v < 16; ++v) x[v] = x1[v];
                } else {
                    load_row<FORM>(buf, L, pairs, x);
                }
                if (FORM == FORM_ROT && S.nj) unrotate_h(x, tau, S.nj);
                if (first) {
#pragma unroll
                    for (int v = 0; v < 16; ++v) x[v] = make_float2(x[v].x * sc, x[v].y * sc);
                    nin += row_norm2(x);
                }
                uint32_t hi[16], lo[16];
#pragma unroll
                for (int v = 0; v < 16; ++v) split_f16(x[v], hi[v], lo[v]);
                const uint32_t col = gcol + (uint32_t)rb * 64u;
                tc_st16(lane_base + col, hi);
                tc_st16(lane_base + col + 16u, lo);
            }
            asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
            tc_fence_before();
            sync_group(grp);
            if (gw == 0 && elect_one()) {
                tc_fence_after();
                const uint64_t dw = sw128_desc(smem_u32(wres) + (uint32_t)s * TH_W_BYTES);
#pragma unroll
                for (int rb = 0; rb < 4; ++rb) {
                    const uint32_t col = gcol + (uint32_t)rb * 64u;
                    stage_mmas(tmem + col + 32u, tmem + col, dw);
                }
                tc_commit(&mma_bar[grp]);
            }
            if (!mbar_wait_bounded(&mma_bar[grp], q & 1u, a.err)) s_abort = 1;
            tc_fence_after();
            const bool last = s == nst - 1;
            float f = 1.f;
            if (last) {   // the output norm (D read once more below), then unscale and restore
                float nout = 0.f;
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    float y[32];
                    tc_ld32(lane_base + gcol + (uint32_t)(2 * half + k) * 64u + 32u, y);
                    float p4[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
                    for (int v = 0; v < 32; ++v) p4[v & 3] = fmaf(y[v], y[v], p4[v & 3]);
                    nout += (p4[0] + p4[1]) + (p4[2] + p4[3]);
                }
                float ni = nin;
#pragma unroll
                for (int o = 16; o; o >>= 1) {
                    ni += __shfl_xor_sync(0xffffffffu, ni, o);
                    nout += __shfl_xor_sync(0xffffffffu, nout, o);
                }
                if (lane == 0) redn[grp][gw] = make_float2(ni, nout);
                sync_group(grp);
                float ti = 0.f, to = 0.f;
#pragma unroll
                for (int w = 0; w < 8; ++w) {
                    ti += redn[grp][w].x;
                    to += redn[grp][w].y;
                }
                f = norm_factor(a.renorm, ti, to, isc);
            }
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                const int rb = 2 * half + k;
                const int row = rb * 128 + quarter * 32 + lane;
                float2 x[16];
                {
                    float y[32];
                    tc_ld32(lane_base + gcol + (uint32_t)rb * 64u + 32u, y);
                    if (last) {   // unscale and restore the norm (earlier stages keep the scale)
#pragma unroll
                        for (int v = 0; v < 32; ++v) y[v] *= f;
                    }
#pragma unroll
                    for (int v = 0; v < 16; ++v) x[v] = make_float2(y[2 * v], y[2 * v + 1]);
                }
                const int tau = (FORM == FORM_ROT && S.nj) ? (row & 15) >> (4 - S.nj) : 0;
                if (FORM == FORM_ROT && S.nj) unrotate_h(x, tau, S.nj);
                int L[16];
                if (FORM == FORM_SWZ) stage_slots_wswz(S, k ? gw1 : gw0, L);
                else stage_slots<FORM>(S, k ? g1 : g0, tau, L);
                store_row<FORM>(buf, L, pairs, x);
            }
            if (last) fence_proxy_async_smem();   // before the tile store reads them
            tc_fence_before();
            sync_group(grp);
            tc_fence_after();
            ++q;
        };
        stage(0, true);
        for (int s = 1; s < nst; ++s) stage(s, false);
        if ((tid & 255) == 0) mbar_arrive(&done_bar[b]);   // the producer stores it
    }
    if (tid == 0 && s_abort && my_tiles > 0) mbar_wait_bounded(&w_bar, 0u, a.err);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TH_TMEM_COLS)
                     : "memory");
}

// ------------------------------------------------ independent-slice passes --
template <int FORM>
__global__ void __launch_bounds__(TH_CTA_THREADS, 1)
    pass_tch_group_kernel(const __grid_constant__ DevPass p, const PassTchArgs a,
                          const __grid_constant__ TmaTile tma) {
    constexpr int NBUF = 3;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char* base = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    const int nst = p.stage_count;
    unsigned char* wres = base;
    float2* bufs = reinterpret_cast<float2*>(base + (size_t)nst * TH_W_BYTES);
    __shared__ uint64_t tile_bar[NBUF], done_bar[NBUF], mma_bar[4], w_bar, stag_bar;
    __shared__ uint32_t tmem_base;
    __shared__ int s_abort;
    __shared__ float redm[TH_THREADS / 32];
    __shared__ float2 redn[TH_THREADS / 32];
    __shared__ StageH sst[TH_MAX_STAGES_3BUF];
    const int tid = threadIdx.x, warp = __shfl_sync(0xffffffffu, tid >> 5, 0);
    const int quarter = warp & 3, slice = warp >> 2, lane = tid & 31;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_base)),
                     "r"(TH_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    load_stage(a.tcs, nst, a.gb0, a.gb1, true, sst, tid, TH_CTA_THREADS);
    if (tid == 0) {
        for (int i = 0; i < NBUF; ++i) {
            mbar_init(&tile_bar[i], 1);
            mbar_init(&done_bar[i], 4);
        }
        for (int i = 0; i < 4; ++i) mbar_init(&mma_bar[i], 1);
        mbar_init(&w_bar, 1);
        mbar_init(&stag_bar, 2);
        fence_mbar_init();
        s_abort = 0;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = __shfl_sync(0xffffffffu, tmem_base, 0);
    const long long first = blockIdx.x, stride = gridDim.x;
    const long long my_tiles = first < a.total_tiles ? (a.total_tiles - first + stride - 1) / stride : 0;
    if (warp == TH_PRODUCER_WARP) {
        tile_mover<NBUF>(p, a, tma, bufs, tile_bar, done_bar, &s_abort, first, stride, my_tiles, lane);
        tc_fence_before();
        __syncthreads();
        return;
    }
    if (tid == 0 && my_tiles > 0) {
        const uint32_t wb = (uint32_t)nst * TH_W_BYTES;
        mbar_arrive_expect_tx(&w_bar, wb);
        bulk_g2s(wres, a.wops + a.tcs[0].wh_off, wb, &w_bar);
    }
    if (my_tiles > 0 && !mbar_wait_bounded(&w_bar, 0u, a.err)) s_abort = 1;
    const uint32_t lane_base = tmem + ((uint32_t)(32 * quarter) << 16);
    const uint32_t col = (uint32_t)slice * 128u;
    uint32_t q = 0;
    long long it = 0;
    for (long long t = first; t < a.total_tiles; t += stride, ++it) {
        const int b = (int)(it % NBUF);
        float2* buf = bufs + (size_t)b * TH_TILE_ELEMS;
        const bool tile_ok = mbar_wait_bounded(&tile_bar[b], (uint32_t)((it / NBUF) & 1), a.err);
        {   // a slice-uniform abort check
            uint32_t stop;
            asm volatile("{\n\t.reg .pred p, q;\n\tsetp.ne.u32 q, %1, 0;\n\t"
                         "bar.red.or.pred p, %2, 128, q;\n\tselp.u32 %0, 1, 0, p;\n\t}"
                         : "=r"(stop)
                         : "r"((uint32_t)(!tile_ok || s_abort)), "r"(1 + slice)
                         : "memory");
            if (stop) {
                s_abort = 1;
                break;
            }
        }
        // once: slices 0 and 1 start after 2 and 3 have issued their first MMAs, so
        // the two pairs stay half a stage apart
        if (it == 0 && slice < 2) mbar_wait_bounded(&stag_bar, 0u, a.err);
        float sc = 1.f, isc = 1.f, nin = 0.f;
        for (int s = 0; s < nst; ++s, ++q) {
            const StageH& S = sst[s];
            const int tau = (FORM == FORM_ROT && S.nj) ? (tid & 15) >> (4 - S.nj) : 0;
            int L[16];
            stage_slots<FORM>(S, group_row(S, tid, a.gb0, a.gb1), tau, L);
            float2 x[16];
#pragma unroll
            for (int v = 0; v < 16; ++v) x[v] = buf[L[v]];
            if (FORM == FORM_ROT && S.nj) unrotate_h(x, tau, S.nj);
            if (s == 0) {   // the slice's scale from its largest component
                const float m = warp_max(row_max(x));
                if (lane == 0) redm[warp] = m;
                sync_slice(slice);
                float mt = 0.f;
#pragma unroll
                for (int w = 0; w < 4; ++w) mt = fmaxf(mt, redm[4 * slice + w]);
                tile_scale(mt, sc, isc);
#pragma unroll
                for (int v = 0; v < 16; ++v) x[v] = make_float2(x[v].x * sc, x[v].y * sc);
                nin = row_norm2(x);
            }
            uint32_t hi[16], lo[16];
#pragma unroll
            for (int v = 0; v < 16; ++v) split_f16(x[v], hi[v], lo[v]);
            tc_st16(lane_base + col, hi);
            tc_st16(lane_base + col + 16u, lo);
            asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
            tc_fence_before();
            sync_slice(slice);
            if (quarter == 0 && elect_one()) {
                tc_fence_after();
                stage_mmas(tmem + col + 32u, tmem + col, sw128_desc(smem_u32(wres) + (uint32_t)s * TH_W_BYTES));
                tc_commit(&mma_bar[slice]);
                if (it == 0 && s == 0 && slice >= 2) mbar_arrive(&stag_bar);
            }
            if (!mbar_wait_bounded(&mma_bar[slice], q & 1u, a.err)) s_abort = 1;
            tc_fence_after();
            {
                float y[32];
                tc_ld32(lane_base + col + 32u, y);
#pragma unroll
                for (int v = 0; v < 16; ++v) x[v] = make_float2(y[2 * v], y[2 * v + 1]);
            }
            if (s == nst - 1) {   // unscale, restore the slice norm (its rows are closed under the pass)
                float ni = nin, nout = row_norm2(x);
#pragma unroll
                for (int o = 16; o; o >>= 1) {
                    ni += __shfl_xor_sync(0xffffffffu, ni, o);
                    nout += __shfl_xor_sync(0xffffffffu, nout, o);
                }
                if (lane == 0) redn[warp] = make_float2(ni, nout);
                sync_slice(slice);
                float ti = 0.f, to = 0.f;
#pragma unroll
                for (int w = 0; w < 4; ++w) {
                    ti += redn[4 * slice + w].x;
                    to += redn[4 * slice + w].y;
                }
                const float f = norm_factor(a.renorm, ti, to, isc);
#pragma unroll
                for (int v = 0; v < 16; ++v) x[v] = make_float2(x[v].x * f, x[v].y * f);
            }
            if (FORM == FORM_ROT && S.nj) unrotate_h(x, tau, S.nj);
#pragma unroll
            for (int v = 0; v < 16; ++v) buf[L[v]] = x[v];
            tc_fence_before();
            sync_slice(slice);
            tc_fence_after();
        }
        fence_proxy_async_smem();   // this thread's tile writes before the tensor store reads them
        sync_slice(slice);
        if ((tid & 127) == 0) mbar_arrive(&done_bar[b]);
    }
    if (tid == 0 && s_abort && my_tiles > 0) mbar_wait_bounded(&w_bar, 0u, a.err);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TH_TMEM_COLS)
                     : "memory");
}

// ------------------------------------------- 32-amplitude (5-bit) stages --
// A stage of 5 register bits is the real GEMM [256 rows x 64] . [64 x 64] per
// tile.  The tile bit gb (>= 5, untouched by every stage of the pass) splits the
// rows into two 128-row blocks that stay closed under the pass.  The CTA keeps
// two tiles in flight (slots 0 and 1 run the CTA's tiles 0, 2, 4, ... and 1, 3,
// 5, ...), so its four chains of four warps each run one row block of one tile
// on their own barrier; a thread owns one row and takes its 32 amplitudes in
// two halves.  TMEM per chain: A hi 32 + A lo 32 + D 64 columns.  W (64 rows, K
// blocks of 64 halves: hi, lo) is 16 KiB per stage, every stage resident (at
// most two, with three tile buffers).
__device__ __forceinline__ void sync_chain(int c) {   // the 128 threads of one chain
    asm volatile("bar.sync %0, %1;" ::"r"(1 + c), "r"(128) : "memory");
}
__device__ __forceinline__ bool sync_chain_or(int c, bool flag) {
    uint32_t r;
    asm volatile("{\n\t.reg .pred p, q;\n\tsetp.ne.u32 q, %1, 0;\n\t"
                 "bar.red.or.pred p, %2, 128, q;\n\tselp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(r)
                 : "r"((uint32_t)flag), "r"(1 + c)
                 : "memory");
    return r != 0;
}

__global__ void __launch_bounds__(TH_CTA_THREADS, 1)
    pass_tch5_kernel(const __grid_constant__ DevPass p, const PassTchArgs a,
                     const __grid_constant__ TmaTile tma) {
    constexpr int NBUF = 3;
    constexpr uint32_t W5 = 4 * TH_W_BYTES;   // 16 KiB
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char* base = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    const int nst = p.stage_count;
    unsigned char* wres = base;
    float2* bufs = reinterpret_cast<float2*>(base + (size_t)nst * W5);
    __shared__ uint64_t tile_bar[NBUF], done_bar[NBUF], mma_bar[4], w_bar, stag_bar[2];
    __shared__ long long s_issued[NBUF];
    __shared__ uint32_t tmem_base;
    __shared__ int s_abort;
    __shared__ float redm[4][4];
    __shared__ float2 redn[4][4];
    __shared__ StageH sst[TH_MAX_STAGES_5];
    const int tid = threadIdx.x, warp = __shfl_sync(0xffffffffu, tid >> 5, 0);
    const int lane = tid & 31;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_base)),
                     "r"(TH_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    load_stage(a.tcs, nst, a.gb0, -1, true, sst, tid, TH_CTA_THREADS);
    if (tid == 0) {
        for (int i = 0; i < NBUF; ++i) {
            mbar_init(&tile_bar[i], 1);
            mbar_init(&done_bar[i], 2);
            s_issued[i] = -1;
        }
        for (int i = 0; i < 4; ++i) mbar_init(&mma_bar[i], 1);
        mbar_init(&w_bar, 1);
        mbar_init(&stag_bar[0], 1);
        mbar_init(&stag_bar[1], 1);
        fence_mbar_init();
        s_abort = 0;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = __shfl_sync(0xffffffffu, tmem_base, 0);
    const long long first = blockIdx.x, stride = gridDim.x;
    const long long my_tiles = first < a.total_tiles ? (a.total_tiles - first + stride - 1) / stride : 0;
    if (warp == TH_PRODUCER_WARP) {
        tile_mover_any<NBUF>(p, a, tma, bufs, tile_bar, done_bar, &s_abort, s_issued, first, stride, my_tiles,
                             lane);
        tc_fence_before();
        __syncthreads();
        return;
    }
    if (tid == 0 && my_tiles > 0) {
        const uint32_t wb = (uint32_t)nst * W5;
        mbar_arrive_expect_tx(&w_bar, wb);
        bulk_g2s(wres, a.wops + a.tcs[0].wh_off, wb, &w_bar);
    }
    if (my_tiles > 0 && !mbar_wait_bounded(&w_bar, 0u, a.err)) s_abort = 1;
    const int chain = warp >> 2, slot = chain >> 1, rb = chain & 1, quarter = warp & 3;
    const uint32_t lane_base = tmem + ((uint32_t)(32 * quarter) << 16);
    const uint32_t col = (uint32_t)chain * 128u;
    const int r7 = quarter * 32 + lane;   // this thread's row within its block
    uint32_t q = 0;
    for (long long it = slot; it < my_tiles; it += 2) {
        const int b = (int)(it % NBUF);
        float2* buf = bufs + (size_t)b * TH_TILE_ELEMS;
        const bool tile_ok = wait_issued(&s_issued[b], it, a.err) &&
                             mbar_wait_bounded(&tile_bar[b], (uint32_t)((it / NBUF) & 1), a.err);
        if (sync_chain_or(chain, !tile_ok || *reinterpret_cast<volatile int*>(&s_abort) != 0)) {
            s_abort = 1;
            break;
        }
        // once per slot: block 0 starts after block 1 has issued its first MMAs
        if (it == slot && rb == 0) mbar_wait_bounded(&stag_bar[slot], 0u, a.err);
        float sc = 1.f, isc = 1.f, nin = 0.f;
        for (int s = 0; s < nst; ++s, ++q) {
            const StageH& S = sst[s];
            int g = r7;
#pragma unroll
            for (int i = 0; i < 6; ++i) g += g & S.hm[i];
            g |= rb << a.gb0;
            // one half of the row (register bit 4 = ch) -> FP16 hi/lo -> TMEM
            auto put_half = [&](int ch, float2 (&x)[16], bool first) {
                if (first) {
#pragma unroll
                    for (int v = 0; v < 16; ++v) x[v] = make_float2(x[v].x * sc, x[v].y * sc);
                    nin += row_norm2(x);
                }
                uint32_t hi[16], lo[16];
#pragma unroll
                for (int v = 0; v < 16; ++v) split_f16(x[v], hi[v], lo[v]);
                tc_st16(lane_base + col + 16u * ch, hi);
                tc_st16(lane_base + col + 32u + 16u * ch, lo);
            };
            if (s == 0) {   // the block's scale from its largest component; half 1 is kept
                float m;
                int L[16];
                {
                    stage_slots<FORM_PLAIN>(S, g, 0, L);
                    float2 x[16];
                    load_row<FORM_PLAIN>(buf, L, false, x);
                    m = row_max(x);
                }
                float2 x1[16];
                stage_slots<FORM_PLAIN>(S, g | S.sr4, 0, L);
                load_row<FORM_PLAIN>(buf, L, false, x1);
                m = warp_max(fmaxf(m, row_max(x1)));
                if (lane == 0) redm[chain][quarter] = m;
                sync_chain(chain);
                float mt = 0.f;
#pragma unroll
                for (int w = 0; w < 4; ++w) mt = fmaxf(mt, redm[chain][w]);
                tile_scale(mt, sc, isc);
                put_half(1, x1, true);
                stage_slots<FORM_PLAIN>(S, g, 0, L);
                float2 x[16];
                load_row<FORM_PLAIN>(buf, L, false, x);
                put_half(0, x, true);
            } else {
#pragma unroll
                for (int ch = 0; ch < 2; ++ch) {
                    int L[16];
                    stage_slots<FORM_PLAIN>(S, ch ? (g | S.sr4) : g, 0, L);
                    float2 x[16];
                    load_row<FORM_PLAIN>(buf, L, false, x);
                    put_half(ch, x, false);
                }
            }
            asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
            tc_fence_before();
            sync_chain(chain);
            if (quarter == 0 && elect_one()) {
                tc_fence_after();
                constexpr uint32_t idesc = f16_idesc(128, 64);
                const uint64_t dw = sw128_desc(smem_u32(wres) + (uint32_t)s * W5);
                const uint32_t d = tmem + col + 64u, ah = tmem + col, al = tmem + col + 32u;
#pragma unroll
                for (int j = 0; j < 4; ++j) tc_mma_f16_ts(d, al + 8u * j, dw + 2u * j, idesc, j);
#pragma unroll
                for (int j = 0; j < 4; ++j) tc_mma_f16_ts(d, ah + 8u * j, dw + 512u + 2u * j, idesc, 1);
#pragma unroll
                for (int j = 0; j < 4; ++j) tc_mma_f16_ts(d, ah + 8u * j, dw + 2u * j, idesc, 1);
                tc_commit(&mma_bar[chain]);
                if (it == slot && s == 0 && rb == 1) mbar_arrive(&stag_bar[slot]);
            }
            if (!mbar_wait_bounded(&mma_bar[chain], q & 1u, a.err)) s_abort = 1;
            tc_fence_after();
            float f = 1.f;
            const bool last = s == nst - 1;
            if (last) {   // unscale, restore the block norm (its rows are closed under the pass)
                float nout = 0.f;
#pragma unroll
                for (int ch = 0; ch < 2; ++ch) {
                    float y[32];
                    tc_ld32(lane_base + col + 64u + 32u * ch, y);
                    float p4[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
                    for (int v = 0; v < 32; ++v) p4[v & 3] = fmaf(y[v], y[v], p4[v & 3]);
                    nout += (p4[0] + p4[1]) + (p4[2] + p4[3]);
                }
                float ni = nin;
#pragma unroll
                for (int o = 16; o; o >>= 1) {
                    ni += __shfl_xor_sync(0xffffffffu, ni, o);
                    nout += __shfl_xor_sync(0xffffffffu, nout, o);
                }
                if (lane == 0) redn[chain][quarter] = make_float2(ni, nout);
                sync_chain(chain);
                float ti = 0.f, to = 0.f;
#pragma unroll
                for (int w = 0; w < 4; ++w) {
                    ti += redn[chain][w].x;
                    to += redn[chain][w].y;
                }
                f = norm_factor(a.renorm, ti, to, isc);
            }
#pragma unroll
            for (int ch = 0; ch < 2; ++ch) {
                float2 x[16];
                {
                    float y[32];
                    tc_ld32(lane_base + col + 64u + 32u * ch, y);
                    if (last) {   // unscale and restore the norm (the first stage keeps the scale)
#pragma unroll
                        for (int v = 0; v < 32; ++v) y[v] *= f;
                    }
#pragma unroll
                    for (int v = 0; v < 16; ++v) x[v] = make_float2(y[2 * v], y[2 * v + 1]);
                }
                int L[16];
                stage_slots<FORM_PLAIN>(S, ch ? (g | S.sr4) : g, 0, L);
                store_row<FORM_PLAIN>(buf, L, false, x);
            }
            tc_fence_before();
            sync_chain(chain);
            tc_fence_after();
        }
        fence_proxy_async_smem();   // this thread's tile writes before the tensor store reads them
        sync_chain(chain);
        if ((tid & 127) == 0) mbar_arrive(&done_bar[b]);
    }
    if (tid == 0 && s_abort && my_tiles > 0) mbar_wait_bounded(&w_bar, 0u, a.err);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TH_TMEM_COLS)
                     : "memory");
}

// ------------------------------------------------------------ host side --
size_t tch_smem_bytes(int nst, int nbuf) {
    return 1024 + (size_t)nst * TH_W_BYTES + (size_t)nbuf * TH_TILE_BYTES;
}
size_t tch5_smem_bytes(int nst) {
    return 1024 + (size_t)nst * 4 * TH_W_BYTES + 3 * (size_t)TH_TILE_BYTES;
}

template <typename K>
cudaError_t set_smem(K k, size_t bytes) {
    return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

cudaError_t set_tch_attributes() {
    const size_t s3 = tch_smem_bytes(TH_MAX_STAGES_3BUF, 3), s2 = tch_smem_bytes(TH_MAX_STAGES, 2);
    cudaError_t e = set_smem(pass_tch_lock_kernel<FORM_PLAIN, 3>, s3);
    if (e == cudaSuccess) e = set_smem(pass_tch_lock_kernel<FORM_ROT, 3>, s3);
    if (e == cudaSuccess) e = set_smem(pass_tch_lock_kernel<FORM_SWZ, 3>, s3);
    if (e == cudaSuccess) e = set_smem(pass_tch_lock_kernel<FORM_PLAIN, 2>, s2);
    if (e == cudaSuccess) e = set_smem(pass_tch_lock_kernel<FORM_ROT, 2>, s2);
    if (e == cudaSuccess) e = set_smem(pass_tch_lock_kernel<FORM_SWZ, 2>, s2);
    if (e == cudaSuccess) e = set_smem(pass_tch_group_kernel<FORM_PLAIN>, s3);
    if (e == cudaSuccess) e = set_smem(pass_tch_group_kernel<FORM_ROT>, s3);
    if (e == cudaSuccess) e = set_smem(pass_tch_group_kernel<FORM_SWZ>, s3);
    if (e == cudaSuccess) e = set_smem(pass_tch5_kernel, tch5_smem_bytes(TH_MAX_STAGES_5));
    return e;
}

// The highest tile bit >= 5 that no 5-bit stage of pass `pass` touches, or -1.
int free_block_bit(const DevPlan* dp, int pass) {
    const DevPass& P = dp->plan.passes[pass];
    uint32_t U = 0;
    for (int si = 0; si < P.stage_count; ++si)
        for (int i = 0; i < 5; ++i) U |= 1u << dp->tcs[P.stage_begin + si].rbit[i];
    for (int b = TH_TILE_BITS - 1; b >= 5; --b)
        if (!((U >> b) & 1)) return b;
    return -1;
}

// Two tile bits (>= 5) that no stage of pass `pass` touches: b0 | b1 << 8, or -1.
int free_slice_bits(const DevPlan* dp, int pass) {
    const DevPass& P = dp->plan.passes[pass];
    uint32_t U = 0;
    for (int si = 0; si < P.stage_count; ++si)
        for (int i = 0; i < 4; ++i) U |= 1u << dp->tcs[P.stage_begin + si].rbit[i];
    int g1 = -1, g0 = -1;
    for (int b = TH_TILE_BITS - 1; b >= 5 && g0 < 0; --b)
        if (!((U >> b) & 1)) {
            if (g1 < 0) g1 = b;
            else g0 = b;
        }
    return g0 >= 0 ? (g0 | (g1 << 8)) : -1;
}

}  // namespace

// ---------------------------------------- shared-memory layouts per stage --
// A lock-step stage reads rows of the swizzled tile and writes them back; the
// rows' lanes take the five lowest tile bits outside its register bits R.  A
// float2's bank slot (16 per 128 bytes) has bit 0 = position bit 0 and bit k =
// position bit k xor k + 3 (k = 1..3), so when R sits on both k and k + 3 (R =
// {2,3,4,5}, {1,2,5,6}) no lane bit reaches slot bit k and a warp's accesses take
// twice the wavefronts.  Every stage rewrites the whole tile, so each stage may
// write its register bits to new positions (the other bits keep their order and
// close up): stage s reads layout P_s and writes P_{s+1}, P_0 = P_last = the tile
// map's layout.  The planner picks each P_{s+1} greedily so that stage s's writes
// and stage s+1's reads cover every slot bit, for the whole warp and for its first
// quarter (16-byte pair accesses, tile bit 0 in R) or half (8-byte accesses).
namespace {

uint32_t lay_slot(int p) { return p == 0 ? 1u : (p <= 3 ? 1u << p : (p <= 6 ? 1u << (p - 3) : 0u)); }

int lay_rank(const uint32_t* c, int n) {
    uint32_t basis[4];
    int r = 0;
    for (int i = 0; i < n; ++i) {
        uint32_t v = c[i];
        for (int b = 0; b < r; ++b) v = std::min(v, v ^ basis[b]);
        if (v && r < 4) basis[r++] = v;
    }
    return r;
}

// 0 when accesses with register positions A (a bit set) cover every slot bit
int lay_bad(uint32_t A) {
    const bool pairs = A & 1u;
    const uint32_t need = pairs ? 0xEu : 0xFu;
    const int full = pairs ? 3 : 4, nfirst = pairs ? 3 : 4;
    uint32_t c[5];
    int nl = 0;
    for (int p = 0; p < TH_TILE_BITS && nl < 5; ++p)
        if (!((A >> p) & 1u)) c[nl++] = lay_slot(p) & need;
    return (lay_rank(c, 5) < full ? 1 : 0) + (lay_rank(c, nfirst) < full ? 1 : 0);
}

}  // namespace

// Layouts of one pass: rbit holds nst x 4 ascending tile bits; out gets nst x 8
// bytes (per stage: positions of its register bits when read, when written).
// Returns false (and writes the tile map's layout throughout) when the planner has
// nothing to gain or cannot return to the tile map's layout after the last stage.
bool lock_layouts(const uint8_t* rbit, int nst, uint8_t* out) {
    for (int s = 0; s < nst; ++s)
        for (int r = 0; r < 4; ++r) out[8 * s + r] = out[8 * s + 4 + r] = rbit[4 * s + r];
    auto regs = [&](int s) { return rbit + 4 * s; };
    int bad = 0;   // nothing to gain when the tile map's layout serves every stage
    for (int s = 0; s < nst; ++s) {
        uint32_t A = 0;
        for (int r = 0; r < 4; ++r) A |= 1u << regs(s)[r];
        bad += lay_bad(A);
    }
    if (!bad || nst < 2) return false;
    int cur[TH_TILE_BITS];   // position of each tile bit in the layout stage s reads
    for (int t = 0; t < TH_TILE_BITS; ++t) cur[t] = t;
    std::vector<uint8_t> pl8(8 * nst);
    for (int s = 0; s < nst; ++s) {
        const uint8_t* R = regs(s);
        uint32_t Rm = 0;
        for (int r = 0; r < 4; ++r) Rm |= 1u << R[r];
        int nxt[TH_TILE_BITS];
        if (s == nst - 1) {
            for (int t = 0; t < TH_TILE_BITS; ++t) nxt[t] = t;
        } else {
            // the other bits in their current order
            int others[TH_TILE_BITS], no = 0;
            for (int p = 0; p < TH_TILE_BITS; ++p)
                for (int t = 0; t < TH_TILE_BITS; ++t)
                    if (cur[t] == p && !((Rm >> t) & 1u)) others[no++] = t;
            const uint8_t* Rn = regs(s + 1);
            uint32_t Rnm = 0;
            for (int r = 0; r < 4; ++r) Rnm |= 1u << Rn[r];
            const bool has0 = Rm & 1u;
            long best = -1;
            int bestq[TH_TILE_BITS];
            // 4-subsets of positions (with 0 exactly when tile bit 0 is a register bit)
            for (uint32_t S = 0; S < (1u << TH_TILE_BITS); ++S) {
                if (__builtin_popcount(S) != 4 || ((S & 1u) != 0) != has0) continue;
                int sp[4], k = 0;
                for (int p = 0; p < TH_TILE_BITS; ++p)
                    if ((S >> p) & 1u) sp[k++] = p;
                int perm[4] = {0, 1, 2, 3};
                do {
                    int q[TH_TILE_BITS];
                    bool okp = true;
                    for (int r = 0; r < 4; ++r) {
                        q[R[r]] = sp[perm[r]];
                        if (R[r] == 0 && sp[perm[r]] != 0) okp = false;
                    }
                    if (!okp) continue;
                    for (int p = 0, o = 0; p < TH_TILE_BITS; ++p)
                        if (!((S >> p) & 1u)) q[others[o++]] = p;
                    // the last stage writes the tile map's layout: its other bits must be in order
                    if (s + 1 == nst - 1) {
                        int prev = -1;
                        bool inorder = true;
                        for (int t = 0; t < TH_TILE_BITS; ++t)
                            if (!((Rnm >> t) & 1u)) {
                                if (q[t] < prev) inorder = false;
                                prev = q[t];
                            }
                        if (!inorder) continue;
                    }
                    uint32_t A = 0, B = 0;
                    for (int t = 0; t < TH_TILE_BITS; ++t) {
                        if ((Rm >> t) & 1u) A |= 1u << q[t];
                        if ((Rnm >> t) & 1u) B |= 1u << q[t];
                    }
                    long disp = 0;
                    for (int t = 0; t < TH_TILE_BITS; ++t) disp += std::abs(q[t] - t);
                    const long score = (long)(lay_bad(A) + lay_bad(B)) * 1000 + disp;
                    if (best < 0 || score < best) {
                        best = score;
                        std::memcpy(bestq, q, sizeof q);
                    }
                } while (std::next_permutation(perm, perm + 4));
            }
            if (best < 0) return false;   // the tile map's layout is out of reach: keep it throughout
            std::memcpy(nxt, bestq, sizeof nxt);
        }
        for (int r = 0; r < 4; ++r) {
            pl8[8 * s + r] = (uint8_t)cur[R[r]];
            pl8[8 * s + 4 + r] = (uint8_t)nxt[R[r]];
        }
        std::memcpy(cur, nxt, sizeof cur);
    }
    std::memcpy(out, pl8.data(), pl8.size());
    return true;
}

void plan_lock_layouts(DevPlan* dp) {
    const Plan& pl = dp->plan;
    dp->lay.assign(dp->tcs.size() * 8, 0);
    for (size_t i = 0; i < dp->tcs.size(); ++i)
        for (int r = 0; r < 4; ++r) dp->lay[8 * i + r] = dp->lay[8 * i + 4 + r] = dp->tcs[i].rbit[r];
    for (int pass = 0; pass < (int)pl.passes.size(); ++pass) {
        const DevPass& P = pl.passes[pass];
        if (!dp->tc_pass[pass] || dp->tc5[pass] || P.m != TH_TILE_BITS || P.stage_count < 2) continue;
        if (P.stage_count <= TH_MAX_STAGES_3BUF && free_slice_bits(dp, pass) >= 0) continue;   // slice kernel
        const int nst = P.stage_count;
        std::vector<uint8_t> rb(4 * nst);
        bool four = true;
        for (int s = 0; s < nst; ++s) {
            const TcsStage& t = dp->tcs[P.stage_begin + s];
            four = four && t.nreg == 4;
            for (int r = 0; r < 4; ++r) rb[4 * s + r] = t.rbit[r];
        }
        if (four) lock_layouts(rb.data(), nst, &dp->lay[8 * P.stage_begin]);
    }
    dp->d_lay = dev_copy(dp->lay);
}

}  // namespace tcng

extern "C" tcng_status tcng_plan_lock_layouts(const unsigned char* rbit, int nst, unsigned char* out,
                                              int* relocated) {
    if (!rbit || !out || !relocated || nst < 1 || nst > 64) return TCNG_EINVAL;
    for (int s = 0; s < nst; ++s)
        for (int r = 0; r < 4; ++r)
            if (rbit[4 * s + r] >= tcng::TH_TILE_BITS || (r && rbit[4 * s + r] <= rbit[4 * s + r - 1]))
                return TCNG_EINVAL;
    *relocated = tcng::lock_layouts(rbit, nst, out) ? 1 : 0;
    return TCNG_OK;
}

namespace tcng {

bool pass_tch_eligible(const DevPlan* dp, int pass) {
    if (!dp->plan.all_unitary || !dp->tc_pass[pass]) return false;
    const DevPass& P = dp->plan.passes[pass];
    if (P.m != TH_TILE_BITS || P.stage_count < 1) return false;
    // the W operands of a pass's stages are consecutive (one bulk copy)
    const int wsz = dp->tc5[pass] ? 4 * TH_W_BYTES : TH_W_BYTES;
    for (int si = 1; si < P.stage_count; ++si)
        if (dp->tcs[P.stage_begin + si].wh_off != dp->tcs[P.stage_begin].wh_off + si * wsz) return false;
    if (dp->tc5[pass]) {   // two row blocks split by a free tile bit, plain slot reads
        if (P.stage_count > TH_MAX_STAGES_5 || free_block_bit(dp, pass) < 0) return false;
        for (int si = 0; si < P.stage_count; ++si)
            if (dp->tcs[P.stage_begin + si].nj) return false;
        return true;
    }
    if (free_slice_bits(dp, pass) >= 0 && P.stage_count <= TH_MAX_STAGES_3BUF) return true;
    return P.stage_count <= TH_MAX_STAGES;
}

cudaError_t launch_pass_tch(const DevPlan* dp, int pass, int items, const void* wops_h, unsigned* err,
                            const TmaTile& tma, bool swizzled, float2* state, const long long* item_off,
                            cudaStream_t s) {
    const DevPass& P = dp->plan.passes[pass];
    static bool attr[kMaxDeviceSlots] = {};   // the attribute is per device
    const int d = device_slot();
    if (!attr[d]) {
        cudaError_t e = set_tch_attributes();
        if (e != cudaSuccess) return e;
        attr[d] = true;
    }
    bool rot = false;   // XOR-rotated slot reads (not needed on a swizzled tile)
    for (int si = 0; si < P.stage_count; ++si) rot = rot || dp->tcs[P.stage_begin + si].nj > 0;
    rot = rot && !swizzled;
    const int form = swizzled ? FORM_SWZ : (rot ? FORM_ROT : FORM_PLAIN);
    PassTchArgs a{};
    const int grp = P.stage_count <= TH_MAX_STAGES_3BUF ? free_slice_bits(dp, pass) : -1;
    a.gb0 = grp >= 0 ? (grp & 255) : 0;
    a.gb1 = grp >= 0 ? (grp >> 8) : 0;
    a.renorm = dp->plan.all_unitary ? 1 : 0;
    a.tcs = dp->d_tcs + P.stage_begin;
    a.lay = dp->d_lay ? dp->d_lay + 8 * P.stage_begin : nullptr;
    a.wops = static_cast<const unsigned char*>(wops_h);
    const long long tpi = 1ll << (dp->plan.n - P.m);
    a.total_tiles = tpi * items;
    a.err = err;
    a.state = state;
    a.item_off = item_off;
    a.tc.nchunks = 1 << P.ngather;
    a.tc.chunk_bytes = (uint32_t)(sizeof(float2) << P.chunk);
    a.tc.tile_bytes = TH_TILE_BYTES;
    a.tc.tiles_per_item = tpi;
    a.tc.tpi_log = dp->plan.n - P.m;
    a.tc.total_tiles = a.total_tiles;
    const unsigned grid = (unsigned)std::min<long long>(a.total_tiles, num_sms());
    const int nst = P.stage_count;
    if (dp->tc5[pass]) {
        a.gb0 = free_block_bit(dp, pass);
        a.gb1 = -1;
        a.tc.nbuf = 3;
        pass_tch5_kernel<<<grid, TH_CTA_THREADS, tch5_smem_bytes(nst), s>>>(P, a, tma);
    } else if (grp >= 0) {
        a.tc.nbuf = 3;
        const size_t sm = tch_smem_bytes(nst, 3);
        if (form == FORM_SWZ) pass_tch_group_kernel<FORM_SWZ><<<grid, TH_CTA_THREADS, sm, s>>>(P, a, tma);
        else if (form == FORM_ROT) pass_tch_group_kernel<FORM_ROT><<<grid, TH_CTA_THREADS, sm, s>>>(P, a, tma);
        else pass_tch_group_kernel<FORM_PLAIN><<<grid, TH_CTA_THREADS, sm, s>>>(P, a, tma);
    } else if (nst <= TH_MAX_STAGES_3BUF) {
        a.tc.nbuf = 3;
        const size_t sm = tch_smem_bytes(nst, 3);
        if (form == FORM_SWZ) pass_tch_lock_kernel<FORM_SWZ, 3><<<grid, TH_CTA_THREADS, sm, s>>>(P, a, tma);
        else if (form == FORM_ROT) pass_tch_lock_kernel<FORM_ROT, 3><<<grid, TH_CTA_THREADS, sm, s>>>(P, a, tma);
        else pass_tch_lock_kernel<FORM_PLAIN, 3><<<grid, TH_CTA_THREADS, sm, s>>>(P, a, tma);
    } else {
        a.tc.nbuf = 2;
        const size_t sm = tch_smem_bytes(nst, 2);
        if (form == FORM_SWZ) pass_tch_lock_kernel<FORM_SWZ, 2><<<grid, TH_CTA_THREADS, sm, s>>>(P, a, tma);
        else if (form == FORM_ROT) pass_tch_lock_kernel<FORM_ROT, 2><<<grid, TH_CTA_THREADS, sm, s>>>(P, a, tma);
        else pass_tch_lock_kernel<FORM_PLAIN, 2><<<grid, TH_CTA_THREADS, sm, s>>>(P, a, tma);
    }
    count_launch();
    return cudaGetLastError();
}

}  // namespace tcng
