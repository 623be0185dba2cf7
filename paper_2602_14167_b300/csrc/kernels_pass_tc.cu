// Tile passes whose register stages run on the tensor cores (complex64).
//
// A register stage (the fused gate applications of Sec. II) moves every
// thread's 16 amplitudes -- one value of the 9 tile bits outside the stage's 4
// register bits -- through all the stage's gates.  Those gates compose to one
// 16x16 unitary U_s, so the stage is a real GEMM: the tile's 512 rows of 32
// reals (re, im of the 16 amplitudes) times W_s, the 32x32 real form of U_s^T.
//
// Per stage and 128-row slice (four warps, one per TMEM lane quarter):
//   * each thread reads its row from the shared-memory tile, splits it into
//     TF32 hi + lo parts and writes both into TMEM (the A operand);
//   * one thread issues 8 tcgen05.mma kind::tf32 (M=128, K=8): per K step one
//     N=64 MMA against [W_hi | W_lo] (a_hi*w_hi and a_hi*w_lo side by side)
//     and one N=32 MMA adding a_lo*w_hi to the small half; the halves are
//     summed in registers, so the large products accumulate on their own;
//   * the row is read back from TMEM (tcgen05.ld) and written back to the tile.
// When every gate of the plan is unitary the pass is unitary on each tile (and,
// in a grouped pass, on each slice), so after the last stage the tile's (slice's)
// norm is restored to its norm before the pass: this removes the systematic
// shrink of the round-toward-zero accumulation.
// W_s (hi and lo, 128-byte swizzled, K-major) is loaded once per CTA when one W
// set serves every tile: into the three ring slots for passes of up to three
// stages, else into an 11-slot layout with two tile buffers instead of three;
// per-item W streams from global memory (L2) through the three-slot ring, two
// stages ahead.  A seventeenth warp only moves tiles: it stores a tile once all
// four slices report it done and loads the tile two ahead into a freed buffer,
// so no compute warp waits on a TMA issue.  Rows whose register
// bits include tile bits 0..3 would put all 32 lanes on one bank: such passes
// either load the tile 128-byte swizzled (TMA) and address it through the same
// XOR map, or read their slots XOR-rotated per lane and undo the rotation in
// registers around the MMA (a separate kernel instance each).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "capi_internal.hpp"
#include "device.cuh"
#include "tc.cuh"
#include "tile_io.cuh"

namespace tcng {

constexpr int TS_THREADS = 512;                    // compute threads: 4 slices x 4 warps
constexpr int TS_CTA_THREADS = TS_THREADS + 32;    // + one producer warp (tile loads, stores)
constexpr int TS_PRODUCER_WARP = TS_THREADS / 32;
constexpr int TS_TILE_BITS = 13;
constexpr int TS_NBUF = 3;                         // tile buffers
constexpr int TS_NB = 3;                           // W ring slots
// the resident-W configuration: two tile buffers and room for the W operands of
// every stage of a pass of up to 11 stages (one W set shared by all tiles)
constexpr int TS_NBUF_RES = 2;
constexpr int TS_NB_RES = 11;
constexpr uint32_t TS_W_FLOATS = 2 * 32 * 32;      // hi + lo
constexpr uint32_t TS_W_BYTES = TS_W_FLOATS * 4;   // 8 KiB
constexpr uint32_t TS_TMEM_COLS = 512;             // 4 slices x (A hi 32 + A lo 32 + D 64)
constexpr int TS_MAX_STAGES = 64;                  // stages per pass held in shared memory

struct StageSm {            // per-stage constants, shared memory
    int sr[4];              // 1 << register tile bit i
    int hm[6];              // ~((1 << b) - 1) for the bits the row index skips (ascending)
    int gb0, gb1;           // grouped passes: tile bits fixed per 128-row slice
    int nj, renorm, tc_index, pad;
};

// ------------------------------------------------------------- prologue --
// W_s of every tensor-core stage and item: U_s = product of the stage's ops
// (FP64, from the FP64 matrix table; R register bits, so U_s is 2^R x 2^R),
// then its real form.  TF32 (H false, R = 4): hi/lo as two 32x32 K-major
// 128-byte-swizzled blocks (8 KiB per stage).  FP16 (H true): R = 4, 32 rows of
// [hi 32 | lo 32] halves, 128 bytes each (4 KiB); R = 5, the 64 rows as two
// K blocks of 64 halves, hi then lo, 8 KiB each (16 KiB).
template <bool H, int R>
__global__ void build_stage_w_kernel(const TcsStage* __restrict__ tcs, const DevOp* __restrict__ ops,
                                     const double2* __restrict__ table, long long table_stride,
                                     void* __restrict__ wops_v, long long w_item_bytes) {
    constexpr int D = 1 << R;
    const TcsStage S = tcs[blockIdx.x];
    if (S.nreg != R || (H ? S.wh_off < 0 : S.tc_index < 0)) return;
    const int item = blockIdx.y;
    __shared__ double2 U[D][D];
    const int tid = threadIdx.x, r = tid >> R, c = tid & (D - 1);
    U[r][c] = make_double2(r == c ? 1.0 : 0.0, 0.0);
    __syncthreads();
    const double2* tab = table + (long long)item * table_stride + S.mat_begin;
    for (int oi = 0; oi < S.op_count; ++oi) {
        const DevOp op = ops[S.op_begin + oi];
        const double2* M = tab + op.mat;
        double2 nv;
        if (op.kind == K_DENSE) {
            const int Dk = 1 << op.k, mask = op.mask;
            int lr = 0, j = 0;   // local index of row r
            for (int i = 0; i < R; ++i)
                if ((mask >> i) & 1) lr |= ((r >> i) & 1) << j++;
            nv = make_double2(0.0, 0.0);
            for (int l = 0; l < Dk; ++l) {
                int rr = r & ~mask, jj = 0;
                for (int i = 0; i < R; ++i)
                    if ((mask >> i) & 1) rr |= ((l >> jj++) & 1) << i;
                const double2 m = M[lr * Dk + l], u = U[rr][c];
                nv.x += m.x * u.x - m.y * u.y;
                nv.y += m.x * u.y + m.y * u.x;
            }
        } else {
            int idx = 0;   // diagonal index of row r: source j's bit of r
            if (R == 4) {
                const int nib = op.mask | (op.pad << 8);
                for (int i = 0; i < 4; ++i) {
                    const int jj = (nib >> (4 * i)) & 15;
                    if (jj) idx |= ((r >> i) & 1) << (jj - 1);
                }
            } else {
                for (int j = 0; j < op.k; ++j)
                    for (int i = 0; i < R; ++i)
                        if (S.rbit[i] == op.src[j]) idx |= ((r >> i) & 1) << j;
            }
            const double2 d = M[idx], u = U[r][c];
            nv = make_double2(d.x * u.x - d.y * u.y, d.x * u.y + d.y * u.x);
        }
        __syncthreads();
        U[r][c] = nv;
        __syncthreads();
    }
    // B operand row nn = output real 2j+b, column kk = input real 2l+a:
    // W[kk][nn] of  y_j = sum_l U[j][l] x_l  in (re, im) pairs.
    unsigned char* out = static_cast<unsigned char*>(wops_v) + (long long)item * w_item_bytes +
                         (H ? (long long)S.wh_off : (long long)S.tc_index * TS_W_BYTES);
    for (int e = tid; e < 4 * D * D; e += blockDim.x) {
        const int nn = e >> (R + 1), kk = e & (2 * D - 1);
        const int j = nn >> 1, b = nn & 1, l = kk >> 1, a = kk & 1;
        const double2 u = U[j][l];
        const double w = (a == b) ? u.x : (a ? -u.y : u.y);
        if (H) {   // hi = w rounded to FP16, lo = the rest rounded to FP16
            const __half h = __double2half(w);
            const __half lo = __double2half(w - (double)__half2float(h));
            if (R == 4) {
                *reinterpret_cast<__half*>(out + sw128_offset_h(nn, kk)) = h;
                *reinterpret_cast<__half*>(out + sw128_offset_h(nn, 32 + kk)) = lo;
            } else {
                *reinterpret_cast<__half*>(out + sw128_offset_h(nn, kk)) = h;
                *reinterpret_cast<__half*>(out + 8192 + sw128_offset_h(nn, kk)) = lo;
            }
        } else {
            const float h = tf32_round((float)w);
            const uint32_t off = sw128_offset(nn, kk, 32);
            *reinterpret_cast<float*>(out + off) = h;
            *reinterpret_cast<float*>(out + 4096 + off) = tf32_round((float)(w - (double)h));
        }
    }
}

// ------------------------------------------------------------ helpers ----
// Split of x for kind::tf32: the tensor core reads an fp32 operand as its
// leading 19 bits (sign, exponent, 10 mantissa bits: x truncated), so hi is x
// itself and lo = x - trunc(x), exact in fp32 (|lo| < 2^-10 |x|, of which the
// tensor core again keeps the leading 11 bits).  Two instructions per value.
__device__ __forceinline__ void split_tf32(float x, uint32_t& hi, uint32_t& lo) {
    hi = __float_as_uint(x);
    lo = __float_as_uint(__fsub_rn(x, __uint_as_float(__float_as_uint(x) & 0xffffe000u)));
}


__device__ __forceinline__ void tc_st32(uint32_t taddr, const uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], "
        "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
        "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(taddr),
        "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
        "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]),
        "r"(r[16]), "r"(r[17]), "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]),
        "r"(r[24]), "r"(r[25]), "r"(r[26]), "r"(r[27]), "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31])
        : "memory");
}

// D (TMEM) += A (TMEM) * B (shared-memory descriptor)
__device__ __forceinline__ void tc_mma_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t b, uint32_t idesc,
                                          int accum) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
        "r"(a_tmem), "l"(b), "r"(idesc), "r"(accum)
        : "memory");
}

// Barrier of the 512 compute threads (the producer warp never joins it).
__device__ __forceinline__ void compute_sync() {
    asm volatile("bar.sync 5, %0;" ::"n"(TS_THREADS) : "memory");
}

// a[s] holds register value s ^ tau (tau only on slots 0..nj-1): permute so
// that a[v] holds value v (the permutation is its own inverse).
__device__ __forceinline__ void unrotate(float2 (&a)[16], int tau, int nj) {
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

struct PassTcsArgs {
    int grouped;              // 1: slices run independently (see plan_tensor_stages)
    int wres;                 // 1: every stage's W loaded once (one W set for all tiles)
    int gb0, gb1;             // their fixed tile bits
    const TcsStage* tcs;      // this pass's stages
    const float* wops;        // W operands, [item][tensor-core stage]
    long long w_item_stride;  // floats per item (0: one set for all items)
    long long tiles_per_item;   // a power of two: 2^tpi_log
    int tpi_log;
    long long total_tiles;
    unsigned* err;
    float2* state;              // tile copies: state + item_off[item], in the pass's copy form
    const long long* item_off;
    TileCtx tc;
};


// ------------------------------------------------------------- kernel ----
// ROT: some stage has register bits on tile bits 0..3 (XOR-rotated reads); SWZ:
// the tile is 128-byte swizzled instead (no rotation).  The passes without such
// stages get an instance with neither.
// NBUF tile buffers, NB W slots (a ring, or every stage's W resident when a.wres).
template <bool ROT, bool SWZ, int NBUF, int NB>
__global__ void __launch_bounds__(TS_CTA_THREADS, 1)
    pass_tcs_kernel(const __grid_constant__ DevPass p, const PassTcsArgs a,
                    const __grid_constant__ TmaTile tma) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char* base = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    unsigned char* wring = base;                                            // NB x 8 KiB
    float2* bufs = reinterpret_cast<float2*>(base + NB * TS_W_BYTES);    // NBUF tiles
    constexpr int tile_elems = 1 << TS_TILE_BITS;
    __shared__ uint64_t tile_bar[NBUF], w_bar[NB], mma_bar[4];
    __shared__ uint64_t done_bar[NBUF];   // the four slices finished a tile
    __shared__ uint64_t stag_bar;            // grouped: slices 2, 3 started (once)
    __shared__ uint32_t tmem_base;
    __shared__ int s_abort;
    __shared__ float2 red[TS_THREADS / 32];
    __shared__ StageSm sst[TS_MAX_STAGES];
    // the warp index and the TMEM base are broadcast from lane 0, so the compiler
    // knows them to be warp-uniform: the MMA operands derived from them stay in
    // uniform registers (a per-thread operand costs a register move per MMA)
    const int tid = threadIdx.x, warp = __shfl_sync(0xffffffffu, tid >> 5, 0);
    const int quarter = warp & 3, slice = warp >> 2;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_base)),
                     "r"(TS_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    for (int i = tid; i < p.stage_count; i += TS_CTA_THREADS) {
        const TcsStage S = a.tcs[i];
        StageSm d;
        int skip[6], ns = 0;   // register bits (+ the slice bits of a grouped pass), ascending
        for (int r = 0; r < 4; ++r) {
            d.sr[r] = 1 << S.rbit[r];
            skip[ns++] = S.rbit[r];
        }
        if (a.grouped) {
            skip[ns++] = a.gb0;
            skip[ns++] = a.gb1;
        }
        for (int x = 1; x < ns; ++x)
            for (int y = x; y > 0 && skip[y - 1] > skip[y]; --y) {
                const int tmp = skip[y];
                skip[y] = skip[y - 1];
                skip[y - 1] = tmp;
            }
        for (int k = 0; k < 6; ++k) d.hm[k] = k < ns ? ~((1 << skip[k]) - 1) : 0;
        d.gb0 = a.gb0;
        d.gb1 = a.gb1;
        d.nj = S.nj;
        d.renorm = S.renorm;
        d.tc_index = S.tc_index;
        d.pad = 0;
        sst[i] = d;
    }
    if (tid == 0) {
        for (int i = 0; i < NBUF; ++i) mbar_init(&tile_bar[i], 1);
        for (int i = 0; i < NB; ++i) mbar_init(&w_bar[i], 1);
        for (int i = 0; i < 4; ++i) mbar_init(&mma_bar[i], 1);
        for (int i = 0; i < NBUF; ++i) mbar_init(&done_bar[i], 4);
        mbar_init(&stag_bar, 2);
        fence_mbar_init();
        s_abort = 0;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = __shfl_sync(0xffffffffu, tmem_base, 0);
    const uint32_t col_ahi = (uint32_t)slice * 128u, col_alo = col_ahi + 32u, col_d = col_ahi + 64u;
    const uint32_t lane_base = tmem + ((uint32_t)(32 * quarter) << 16);
    const uint32_t idesc64 = tf32_idesc(128, 64), idesc32 = tf32_idesc(128, 32);
    const int nst = p.stage_count;
    const long long first = blockIdx.x, stride = gridDim.x;
    const long long my_tiles = first < a.total_tiles ? (a.total_tiles - first + stride - 1) / stride : 0;
    const long long total_q = my_tiles * nst;
    if (warp == TS_PRODUCER_WARP) {   // ---------------------------- tile mover --
        // the whole warp issues the copies (the gather4 and per-chunk forms use every lane)
        const int lane = tid & 31;
        // loads run two tiles ahead: with three buffers into the one stored a tile
        // ago, with two into the one just stored (once its store has read it)
        constexpr int ahead = NBUF == 2 ? 2 : NBUF - 1;
        long long issued = 0;
        for (; issued < ahead && issued < my_tiles; ++issued)
            issue_tile_load(a.state, a.item_off, p, a.tc, first + issued * stride, bufs + issued * tile_elems,
                            &tile_bar[issued], lane, tma);
        for (long long i = 0; i < my_tiles; ++i) {
            const int b = (int)(i % NBUF);
            // lane 0 waits for the four slices (or gives up when they abort)
            uint32_t done = 0;
            if (lane == 0) {
                done = mbar_try_wait(&done_bar[b], (uint32_t)((i / NBUF) & 1));
                const unsigned long long t0 = global_ns();
                for (uint32_t k = 1; !done; ++k) {
                    if (*reinterpret_cast<volatile int*>(&s_abort)) break;
                    done = mbar_try_wait(&done_bar[b], (uint32_t)((i / NBUF) & 1));
                    if (!done && (k & 255u) == 0 && global_ns() - t0 > kWaitLimitNs) {
                        atomicOr(a.err, ERR_TIMEOUT);
                        s_abort = 1;
                        break;
                    }
                }
            }
            if (!__shfl_sync(0xffffffffu, done, 0)) break;
            issue_tile_store(a.state, a.item_off, p, a.tc, first + i * stride, bufs + (size_t)b * tile_elems,
                             lane, tma);
            if (issued < my_tiles) {
                if (NBUF == 2)
                    bulk_wait_read<0>();
                else
                    bulk_wait_read<1>();
                __syncwarp();
                const int bn = (int)(issued % NBUF);
                issue_tile_load(a.state, a.item_off, p, a.tc, first + issued * stride,
                                bufs + (size_t)bn * tile_elems, &tile_bar[bn], lane, tma);
                ++issued;
            }
        }
        bulk_wait<0>();
        // after an abort: the last loads (at most one per buffer) may still be in
        // flight; wait for them before the shared memory goes away
        if (lane == 0)
            for (long long i = issued > NBUF ? issued - NBUF : 0; i < issued; ++i)
                mbar_wait_bounded(&tile_bar[i % NBUF], (uint32_t)((i / NBUF) & 1), a.err);
        __syncwarp();
        tc_fence_before();
        __syncthreads();
        return;
    }
    // W operand producer state (thread 0): the next W operand is stage w_s of the
    // CTA's tile w_t
    long long w_issued = 0, w_t = 0;
    int w_s = 0;
    auto issue_w = [&]() {
        const long long item = (first + w_t * stride) >> a.tpi_log;
        const float* src = a.wops + item * a.w_item_stride + (long long)sst[w_s].tc_index * TS_W_FLOATS;
        const int slot = (int)(w_issued % NB);
        mbar_arrive_expect_tx(&w_bar[slot], TS_W_BYTES);
        bulk_g2s(wring + (size_t)slot * TS_W_BYTES, src, TS_W_BYTES, &w_bar[slot]);
        ++w_issued;
        if (++w_s == nst) {
            w_s = 0;
            ++w_t;
        }
    };
    if (tid == 0) {
        if (a.wres) {   // every stage's W stays resident (one set for all items)
            for (int st = 0; st < nst && my_tiles > 0; ++st) {
                mbar_arrive_expect_tx(&w_bar[st], TS_W_BYTES);
                bulk_g2s(wring + (size_t)st * TS_W_BYTES, a.wops + (long long)sst[st].tc_index * TS_W_FLOATS,
                         TS_W_BYTES, &w_bar[st]);
            }
        } else {
            while (w_issued < NB - 1 && w_issued < total_q) issue_w();
        }
    }
    // row base of each stage (fixed per thread for the whole pass), computed once in
    // the plain instance for independent-slice passes of up to three stages
    int gpre0 = 0, gpre1 = 0, gpre2 = 0;
    const bool use_gpre = !ROT && !SWZ && a.grouped && nst <= 3;
    if (use_gpre) {
        for (int s = 0; s < nst; ++s) {
            const StageSm& S = sst[s];
            int g = tid & 127;
#pragma unroll
            for (int i = 0; i < 6; ++i) g += g & S.hm[i];
            g |= (((tid >> 7) & 1) << S.gb0) | (((tid >> 8) & 1) << S.gb1);
            if (s == 0) gpre0 = g;
            else if (s == 1) gpre1 = g;
            else gpre2 = g;
        }
    }
    long long q = 0;
    long long it = 0;
    for (long long t = first; t < a.total_tiles; t += stride, ++it) {
        const int b = (int)(it % NBUF);
        float2* buf = bufs + (size_t)b * tile_elems;
        const bool tile_ok = mbar_wait_bounded(&tile_bar[b], (uint32_t)((it / NBUF) & 1), a.err);
        if (a.grouped) {
            // slices run through the tiles independently: a slice-uniform abort check
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
            // once: slices 0 and 1 start after 2 and 3 have issued their first MMAs, so
            // the two pairs stay half a stage apart (one pair's shared-memory phases
            // overlap the other's tensor-core phase)
            if (it == 0 && slice < 2) mbar_wait_bounded(&stag_bar, 0u, a.err);
        } else {
            if (!tile_ok) s_abort = 1;
            compute_sync();
            if (s_abort) break;
        }
        float nin = 0.f;   // this thread's share of the tile norm before the pass
        for (int s = 0; s < nst; ++s, ++q) {
            if (!a.wres && tid == 0 && w_issued < total_q && w_issued < q + NB) issue_w();
            const StageSm& S = sst[s];
            // this thread's row is group g = tid; slot v is read at register value v ^ tau,
            // tau = the group bits that land on tile bits >= 4 (bank-conflict-free reads)
            const int tau = (ROT && S.nj) ? (tid & 15) >> (4 - S.nj) : 0;
            int L[16];
            {
                int g;
                if (use_gpre) {
                    g = s == 0 ? gpre0 : (s == 1 ? gpre1 : gpre2);
                } else if (a.grouped) {   // slice bits of tid -> the pass's fixed tile bits
                    g = tid & 127;
#pragma unroll
                    for (int i = 0; i < 6; ++i) g += g & S.hm[i];
                    g |= (((tid >> 7) & 1) << S.gb0) | (((tid >> 8) & 1) << S.gb1);
                } else {
                    g = tid;
#pragma unroll
                    for (int i = 0; i < 4; ++i) g += g & S.hm[i];
                }
                int sr[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) sr[i] = S.sr[i];
                if (SWZ) {   // slot offset o lies at o ^ ((o >> 3) & 0xE) (linear in o)
                    g ^= (g >> 3) & 0xe;
#pragma unroll
                    for (int i = 0; i < 4; ++i) sr[i] ^= (sr[i] >> 3) & 0xe;
                }
                int stau = 0;
                if (ROT && S.nj) {
#pragma unroll
                    for (int i = 0; i < 4; ++i) stau |= ((tau >> i) & 1) ? sr[i] : 0;
                }
                L[0] = g | stau;
#pragma unroll
                for (int v = 1; v < 16; ++v)
                    L[v] = L[v & (v - 1)] ^ ((v & 1) ? sr[0] : (v & 2) ? sr[1] : (v & 4) ? sr[2] : sr[3]);
            }
            float2 x[16];
#pragma unroll
            for (int v = 0; v < 16; ++v) x[v] = buf[L[v]];
            if (ROT && S.nj) unrotate(x, tau, S.nj);
            if (S.renorm && s == 0) {   // tile norm before the pass (unitary on the tile)
                float p4[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
                for (int v = 0; v < 16; ++v) p4[v & 3] = fmaf(x[v].x, x[v].x, fmaf(x[v].y, x[v].y, p4[v & 3]));
                nin = (p4[0] + p4[1]) + (p4[2] + p4[3]);
            }
            {
                uint32_t hi[32], lo[32];
#pragma unroll
                for (int v = 0; v < 16; ++v) {
                    split_tf32(x[v].x, hi[2 * v], lo[2 * v]);
                    split_tf32(x[v].y, hi[2 * v + 1], lo[2 * v + 1]);
                }
                tc_st32(lane_base + col_ahi, hi);
                tc_st32(lane_base + col_alo, lo);
                asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
            }
            tc_fence_before();
            asm volatile("bar.sync %0, %1;" ::"r"(1 + slice), "r"(128) : "memory");
            if (quarter == 0 && elect_one()) {   // one thread of the slice's first warp
                tc_fence_after();
                const int slot = a.wres ? s : (int)(q % NB);
                const uint32_t wpar = a.wres ? 0u : (uint32_t)((q / NB) & 1);
                // resident W: only the first tile waits for it
                if ((a.wres && it > 0) || mbar_wait_bounded(&w_bar[slot], wpar, a.err)) {
                    // W slot = [W_hi (32 rows) | W_lo (32 rows)]: one N=64 MMA gives
                    // a_hi*w_hi in D[0:32] and a_hi*w_lo in D[32:64]; a_lo*w_hi joins
                    // D[32:64]; the two halves are added in registers afterwards
                    const uint64_t dw = sw128_desc(smem_u32(wring) + (uint32_t)slot * TS_W_BYTES);
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk) {   // K step kk: +32 bytes = +2 in the start field
                        tc_mma_ts(tmem + col_d, tmem + col_ahi + 8u * kk, dw + 2u * kk, idesc64, kk);
                        tc_mma_ts(tmem + col_d + 32u, tmem + col_alo + 8u * kk, dw + 2u * kk, idesc32, 1);
                    }
                } else {
                    s_abort = 1;
                }
                tc_commit(&mma_bar[slice]);
                if (a.grouped && it == 0 && s == 0 && slice >= 2) mbar_arrive(&stag_bar);
            }
            if (!mbar_wait_bounded(&mma_bar[slice], (uint32_t)(q & 1), a.err)) s_abort = 1;
            tc_fence_after();
            {
                float y[32], z[32];
                tc_ld32(lane_base + col_d, y);
                tc_ld32(lane_base + col_d + 32u, z);
#pragma unroll
                for (int v = 0; v < 16; ++v) x[v] = make_float2(y[2 * v] + z[2 * v], y[2 * v + 1] + z[2 * v + 1]);
            }
            if (S.renorm && s == nst - 1) {   // restore the tile norm after the last stage
                float p4[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
                for (int v = 0; v < 16; ++v) p4[v & 3] = fmaf(x[v].x, x[v].x, fmaf(x[v].y, x[v].y, p4[v & 3]));
                float nout = (p4[0] + p4[1]) + (p4[2] + p4[3]);
#pragma unroll
                for (int o = 16; o; o >>= 1) {
                    nin += __shfl_xor_sync(0xffffffffu, nin, o);
                    nout += __shfl_xor_sync(0xffffffffu, nout, o);
                }
                if ((tid & 31) == 0) red[warp] = make_float2(nin, nout);
                float ti = 0.f, to = 0.f;
                if (a.grouped) {   // the slice's rows are closed under the pass: its own norm
                    asm volatile("bar.sync %0, %1;" ::"r"(1 + slice), "r"(128) : "memory");
#pragma unroll
                    for (int w = 0; w < 4; ++w) {
                        const float2 r = red[4 * slice + w];
                        ti += r.x;
                        to += r.y;
                    }
                } else {
                    compute_sync();
#pragma unroll
                    for (int w = 0; w < TS_THREADS / 32; ++w) {
                        const float2 r = red[w];
                        ti += r.x;
                        to += r.y;
                    }
                }
                // sqrt(ti / to); tiles of tiny norm keep their values (ti * to, or the
                // squares themselves, would leave the FP32 range: a product state's
                // far tiles have norms far below 1e-30)
                const float f = (to > 1e-30f && ti > 1e-30f) ? sqrtf(ti) * rsqrtf(to) : 1.f;
#pragma unroll
                for (int v = 0; v < 16; ++v) x[v] = make_float2(x[v].x * f, x[v].y * f);
                nin = 0.f;
            }
            if (ROT && S.nj) unrotate(x, tau, S.nj);
#pragma unroll
            for (int v = 0; v < 16; ++v) buf[L[v]] = x[v];
            tc_fence_before();
            if (a.grouped) {   // the next stage reads only this slice's rows
                asm volatile("bar.sync %0, %1;" ::"r"(1 + slice), "r"(128) : "memory");
            } else {
                compute_sync();
            }
            tc_fence_after();
            if (!a.grouped && s_abort) break;
        }
        fence_proxy_async_smem();   // this thread's tile writes before the tensor store reads them
        if (!a.grouped && s_abort) break;
        // each slice reports the tile; the producer warp stores it once all four have
        asm volatile("bar.sync %0, %1;" ::"r"(1 + slice), "r"(128) : "memory");
        if ((tid & 127) == 0) mbar_arrive(&done_bar[b]);
    }
    if (tid == 0) {
        if (s_abort) {   // drain the W loads still in flight before the shared memory goes away
            if (a.wres) {
                for (int st = 0; st < nst; ++st) mbar_wait_bounded(&w_bar[st], 0u, a.err);
            } else {
                for (long long i = q; i < w_issued; ++i)
                    mbar_wait_bounded(&w_bar[i % NB], (uint32_t)((i / NB) & 1), a.err);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TS_TMEM_COLS)
                     : "memory");
}

// ------------------------------------------------------------ host side --
static size_t pass_tcs_smem_bytes(int nbuf, int nb) {
    return 1024 + (size_t)nb * TS_W_BYTES + (size_t)nbuf * (sizeof(float2) << TS_TILE_BITS);
}

template <int NBUF, int NB>
static cudaError_t set_pass_tcs_smem() {
    const int sm = (int)pass_tcs_smem_bytes(NBUF, NB);
    cudaError_t e = cudaFuncSetAttribute(pass_tcs_kernel<true, false, NBUF, NB>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(pass_tcs_kernel<false, false, NBUF, NB>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(pass_tcs_kernel<false, true, NBUF, NB>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    return e;
}

template <int NBUF, int NB>
static void launch_pass_tcs_cfg(bool rot, bool swizzled, unsigned grid, const DevPass& P, PassTcsArgs a,
                                const TmaTile& tma, cudaStream_t s) {
    const size_t sm = pass_tcs_smem_bytes(NBUF, NB);
    a.tc.nbuf = NBUF;
    if (rot)
        pass_tcs_kernel<true, false, NBUF, NB><<<grid, TS_CTA_THREADS, sm, s>>>(P, a, tma);
    else if (swizzled)
        pass_tcs_kernel<false, true, NBUF, NB><<<grid, TS_CTA_THREADS, sm, s>>>(P, a, tma);
    else
        pass_tcs_kernel<false, false, NBUF, NB><<<grid, TS_CTA_THREADS, sm, s>>>(P, a, tma);
}

// Which passes run their stages on the tensor cores, and the per-stage data.
// A pass qualifies when every stage has 4 register bits (TF32 or FP16 operands)
// or every stage has 5 (FP16 only) and each diagonal op reads only register bits.
void plan_tensor_stages(DevPlan* dp) {
    if (dp->tc_ready) return;
    Plan& pl = dp->plan;
    dp->tcs.assign(pl.stages.size(), TcsStage{});
    for (auto& s : dp->tcs) {
        s.tc_index = -1;
        s.wh_off = -1;
    }
    dp->tc_pass.assign(pl.passes.size(), 0);
    dp->tc5.assign(pl.passes.size(), 0);
    dp->tc_group.assign(pl.passes.size(), -1);
    dp->n_tc = 0;
    dp->n_tc32 = 0;
    dp->wh_bytes = 0;
    if (!pl.opt.unfused && !pl.opt.adjoint) {
        for (size_t pi = 0; pi < pl.passes.size(); ++pi) {
            const DevPass& P = pl.passes[pi];
            bool ok = P.m == TS_TILE_BITS && P.stage_count > 0 && P.stage_count <= TS_MAX_STAGES;
            const int R = ok ? pl.stages[P.stage_begin].nreg : 0;
            ok = ok && (R == 4 || (R == 5 && pl.all_unitary));
            for (int si = 0; ok && si < P.stage_count; ++si) {
                const DevStage& st = pl.stages[P.stage_begin + si];
                if (st.nreg != R) ok = false;
                for (uint32_t oi = 0; ok && oi < st.op_count; ++oi) {
                    const DevOp& o = pl.dops[st.op_begin + oi];
                    if (o.kind != K_DIAG) continue;
                    // foldable only if every source is a register bit
                    for (int j = 0; ok && j < o.k; ++j) {
                        bool reg = false;
                        for (int i = 0; i < R; ++i) reg = reg || st.rbit[i] == o.src[j];
                        ok = reg;
                    }
                }
            }
            if (!ok) continue;
            dp->tc_pass[pi] = 1;
            dp->tc5[pi] = R == 5 ? 1 : 0;
            // two tile bits that no stage of the pass touches (>= 5, so the lanes keep the
            // low bits): rows with fixed values of them never leave their 128-row slice
            if (R == 4) {
                uint32_t U = 0;
                for (int si = 0; si < P.stage_count; ++si)
                    for (int i = 0; i < 4; ++i) U |= 1u << pl.stages[P.stage_begin + si].rbit[i];
                int g1 = -1, g0 = -1;
                for (int b = TS_TILE_BITS - 1; b >= 5 && g0 < 0; --b)
                    if (!((U >> b) & 1)) {
                        if (g1 < 0) g1 = b;
                        else g0 = b;
                    }
                if (g0 >= 0 && P.stage_count <= TS_NB) dp->tc_group[pi] = g0 | (g1 << 8);
            }
            for (int si = 0; si < P.stage_count; ++si) {
                const DevStage& st = pl.stages[P.stage_begin + si];
                TcsStage& t = dp->tcs[P.stage_begin + si];
                int nj = 0;
                for (int i = 0; i < R; ++i) {
                    t.rbit[i] = st.rbit[i];
                    if (st.rbit[i] < 4) ++nj;
                }
                t.nj = (uint8_t)nj;
                t.nreg = (uint8_t)R;
                t.renorm = pl.all_unitary ? 1 : 0;
                t.op_begin = (int32_t)st.op_begin;
                t.op_count = (int32_t)st.op_count;
                t.mat_begin = P.mat_begin;
                if (R == 4) t.tc_index = dp->n_tc32++;
                t.wh_off = (int32_t)dp->wh_bytes;
                dp->wh_bytes += R == 5 ? 4 * TH_W_BYTES : TH_W_BYTES;
                ++dp->n_tc;
            }
        }
    }
    if (dp->n_tc) dp->d_tcs = dev_copy(dp->tcs);
    if (dp->n_tc) plan_lock_layouts(dp);
    dp->tc_ready = true;
}

cudaError_t launch_build_stage_w(const DevPlan* dp, const double2* table, long long table_stride,
                                 int items, void* wops, bool half, cudaStream_t s) {
    if (!dp->n_tc) return cudaSuccess;
    dim3 grid((unsigned)dp->tcs.size(), (unsigned)items);
    if (half) {
        build_stage_w_kernel<true, 4><<<grid, 256, 0, s>>>(dp->d_tcs, dp->d_dops, table, table_stride, wops,
                                                           dp->wh_bytes);
        count_launch();
        bool any5 = false;
        for (char c : dp->tc5) any5 = any5 || c;
        if (any5) {
            build_stage_w_kernel<true, 5><<<grid, 1024, 0, s>>>(dp->d_tcs, dp->d_dops, table, table_stride, wops,
                                                                dp->wh_bytes);
            count_launch();
        }
    } else if (dp->n_tc32) {
        build_stage_w_kernel<false, 4><<<grid, 256, 0, s>>>(dp->d_tcs, dp->d_dops, table, table_stride, wops,
                                                            (long long)dp->n_tc32 * TS_W_BYTES);
        count_launch();
    }
    return cudaGetLastError();
}

cudaError_t launch_pass_tcs(const DevPlan* dp, int pass, int items, const float* wops,
                            long long w_item_stride, unsigned* err, const TmaTile& tma, bool swizzled,
                            float2* state, const long long* item_off, cudaStream_t s) {
    const DevPass& P = dp->plan.passes[pass];
    static bool attr[kMaxDeviceSlots] = {};   // the attribute is per device
    const int d = device_slot();
    if (!attr[d]) {
        cudaError_t e = set_pass_tcs_smem<TS_NBUF, TS_NB>();
        if (e == cudaSuccess) e = set_pass_tcs_smem<TS_NBUF_RES, TS_NB_RES>();
        if (e != cudaSuccess) return e;
        attr[d] = true;
    }
    bool rot = false;   // XOR-rotated slot reads (not needed on a swizzled tile)
    for (int si = 0; si < P.stage_count; ++si) rot = rot || dp->tcs[P.stage_begin + si].nj > 0;
    rot = rot && !swizzled;
    PassTcsArgs a{};
    const int grp = dp->tc_group[pass];
    const bool w_shared = w_item_stride == 0 || items == 1;   // one W set for every tile
    a.grouped = (grp >= 0 && w_shared) ? 1 : 0;
    // lock-step passes of 4..11 stages keep every W resident with two tile buffers;
    // passes of up to three stages keep them in the ring's slots
    const bool res_cfg = w_shared && !a.grouped && P.stage_count > TS_NB && P.stage_count <= TS_NB_RES;
    a.wres = (w_shared && (P.stage_count <= TS_NB || res_cfg)) ? 1 : 0;
    a.gb0 = a.grouped ? (grp & 255) : 0;
    a.gb1 = a.grouped ? (grp >> 8) : 0;
    a.tcs = dp->d_tcs + P.stage_begin;
    a.wops = wops;
    a.w_item_stride = w_item_stride;
    a.tiles_per_item = 1ll << (dp->plan.n - P.m);
    a.tpi_log = dp->plan.n - P.m;
    a.total_tiles = a.tiles_per_item * items;
    a.err = err;
    a.state = state;
    a.item_off = item_off;
    a.tc.nchunks = 1 << P.ngather;
    a.tc.chunk_bytes = (uint32_t)(sizeof(float2) << P.chunk);
    a.tc.tile_bytes = (uint32_t)(sizeof(float2) << P.m);
    a.tc.tiles_per_item = a.tiles_per_item;
    a.tc.tpi_log = a.tpi_log;
    a.tc.total_tiles = a.total_tiles;
    const unsigned grid = (unsigned)std::min<long long>(a.total_tiles, num_sms());
    if (res_cfg)
        launch_pass_tcs_cfg<TS_NBUF_RES, TS_NB_RES>(rot, swizzled, grid, P, a, tma, s);
    else
        launch_pass_tcs_cfg<TS_NBUF, TS_NB>(rot, swizzled, grid, P, a, tma, s);
    count_launch();
    return cudaGetLastError();
}

}  // namespace tcng
