// Tile passes with the fused blocks applied on the tensor cores (complex64).
//
// Same tiles as pass_kernel (2^13 amplitudes, one TMA tensor copy in and out),
// but a dense block on k <= 4 tile bits is applied as a real GEMM over the
// tile's 2^(13-k) rows: row = the block's 2^k amplitudes as (re, im) pairs,
// times W (the real form of U^T, see kernels_tc.cu), in 128-row slices with
// tcgen05.mma kind::tf32 (M=128, N=32, K=8) and a 3-term TF32 split for fp32
// accuracy.  The slices are software-pipelined: while the tensor cores work on
// slice i, the CTA gathers and splits slice i+1 and writes slice i-1 back from
// TMEM.  Diagonal blocks are elementwise phase multiplies.
#include <cuda_runtime.h>

#include <algorithm>

#include "capi_internal.hpp"
#include "device.cuh"
#include "tc.cuh"

namespace tcng {

constexpr int PT_M = 128;
constexpr int PT_K = 32;                               // real K = 2 * 2^k padded to 32 (k <= 4)
constexpr int PT_N = 32;
constexpr uint32_t PT_A_BYTES = PT_M * PT_K * 4;       // 16 KiB per split part
constexpr uint32_t PT_B_BYTES = PT_N * PT_K * 4;       // 4 KiB per split part
constexpr uint32_t PT_B_FLOATS = 2 * PT_N * PT_K;      // hi + lo of one block
constexpr int PT_THREADS = 256;

// W^T (rows = output column 2j+b, cols = input 2l+a) of every dense block, split
// into TF32 hi/lo, in the 128-byte-swizzled K-major layout.  One CTA per block.
__global__ void build_b_operands_kernel(const TcOp* __restrict__ ops, const int* __restrict__ dense,
                                       const float2* __restrict__ table, float* __restrict__ bops) {
    const TcOp op = ops[dense[blockIdx.x]];
    const int D = 1 << op.k;
    const float2* U = table + op.mat;
    unsigned char* out = reinterpret_cast<unsigned char*>(bops + (size_t)op.slot * PT_B_FLOATS);
    for (int e = threadIdx.x; e < PT_N * PT_K; e += blockDim.x) {
        const int nn = e / PT_K, kk = e % PT_K;
        float w = 0.f;
        if (nn < 2 * D && kk < 2 * D) {
            const int j = nn >> 1, b = nn & 1, l = kk >> 1, a = kk & 1;
            const float2 u = U[j * D + l];
            w = (a == b) ? u.x : (a ? -u.y : u.y);
        }
        const float h = tf32_round(w);
        const uint32_t off = sw128_offset(nn, kk, PT_N);
        *reinterpret_cast<float*>(out + off) = h;
        *reinterpret_cast<float*>(out + PT_B_BYTES + off) = tf32_round(w - h);
    }
}

struct PassTcArgs {
    float2* state;
    const long long* item_off;
    const TcOp* ops;          // this pass's blocks
    int n_ops;
    const float2* table;      // item 0's matrix table (diagonal phases)
    const float* bops;        // B operands (8 KiB per dense block)
    long long tiles_per_item;
    long long total_tiles;
    uint32_t tile_bytes;
    unsigned* err;
};

__device__ __forceinline__ int insert_zeros_bits(int r, const uint8_t* tb, int k) {
    for (int j = 0; j < k; ++j) r = ((r >> tb[j]) << (tb[j] + 1)) | (r & ((1 << tb[j]) - 1));
    return r;
}

__global__ void __launch_bounds__(PT_THREADS, 1) pass_tc_kernel(const __grid_constant__ DevPass p,
                                                                const PassTcArgs a,
                                                                const __grid_constant__ TmaTile tma) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char* base = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    const int tile_elems = 1 << p.m;
    float2* tiles = reinterpret_cast<float2*>(base);                       // 2 x tile
    unsigned char* abuf = base + 2 * (size_t)tile_elems * sizeof(float2);  // 2 x (hi, lo)
    unsigned char* bbuf = abuf + 4 * PT_A_BYTES;                            // hi, lo
    __shared__ uint64_t tile_bar[2], mma_bar[2], b_bar;
    __shared__ uint32_t tmem_base;
    __shared__ int s_abort;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // zero the A operands once: columns beyond a block's 2^(k+1) stay 0
    for (uint32_t i = tid; i < 4 * PT_A_BYTES / 16; i += PT_THREADS)
        reinterpret_cast<float4*>(abuf)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_base)),
                     "r"(2 * PT_N)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        mbar_init(&tile_bar[0], 1);
        mbar_init(&tile_bar[1], 1);
        mbar_init(&mma_bar[0], 1);
        mbar_init(&mma_bar[1], 1);
        mbar_init(&b_bar, 1);
        fence_mbar_init();
        s_abort = 0;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;
    const uint32_t idesc = tf32_idesc(PT_M, PT_N);
    uint32_t mph[2] = {0u, 0u}, bph = 0u;
    const long long first = blockIdx.x, stride = gridDim.x;
    auto tile_coords = [&](long long t, int (&c)[5]) {
        tma_tile_coords(tma, t % a.tiles_per_item, (int)(t / a.tiles_per_item), c);
    };
    if (tid == 0)
        for (int i = 0; i < 2; ++i) {
            const long long t = first + i * stride;
            if (t < a.total_tiles) {
                int c[5];
                tile_coords(t, c);
                mbar_arrive_expect_tx(&tile_bar[i], a.tile_bytes);
                tma_load_tile(tma, tiles + (size_t)i * tile_elems, &tile_bar[i], c);
            }
        }
    int it = 0;
    for (long long t = first; t < a.total_tiles; t += stride, ++it) {
        const int bsel = it & 1;
        float2* buf = tiles + (size_t)bsel * tile_elems;
        if (!mbar_wait_bounded(&tile_bar[bsel], (uint32_t)((it >> 1) & 1), a.err)) s_abort = 1;
        __syncthreads();
        if (s_abort) break;
        const long long gbase = tile_global_base(p, t % a.tiles_per_item);
        for (int oi = 0; oi < a.n_ops && !s_abort; ++oi) {
            const TcOp op = a.ops[oi];
            if (op.kind == K_DIAG) {
                const float2* M = a.table + op.mat;
                for (int L = tid; L < tile_elems; L += PT_THREADS) {
                    int idx = 0;
                    for (int j = 0; j < op.k; ++j) idx |= src_bit(op.tb[j], L, gbase) << j;
                    buf[L] = cmul(M[idx], buf[L]);
                }
                __syncthreads();
                continue;
            }
            // ---- dense block: GEMM over the tile's rows, 128 at a time ----
            const int k = op.k, D = 1 << k;
            const int rows = tile_elems >> k;
            const int nmt = (rows + PT_M - 1) / PT_M;
            if (tid == 0) {   // this block's B operand (8 KiB) into shared memory
                mbar_arrive_expect_tx(&b_bar, 2 * PT_B_BYTES);
                bulk_g2s(bbuf, a.bops + (size_t)op.slot * PT_B_FLOATS, 2 * PT_B_BYTES, &b_bar);
            }
            for (int i = 0; i <= nmt; ++i) {
                if (i < nmt) {   // gather + split slice i into A[i & 1]
                    unsigned char* ahi = abuf + (size_t)(i & 1) * 2 * PT_A_BYTES;
                    unsigned char* alo = ahi + PT_A_BYTES;
                    for (int e = tid; e < PT_M * D; e += PT_THREADS) {
                        const int l = e / PT_M, row = e % PT_M;
                        const int r = i * PT_M + row;
                        if (r >= rows) continue;
                        int x = insert_zeros_bits(r, op.tb, k);
                        for (int j = 0; j < k; ++j)
                            if ((l >> j) & 1) x |= 1 << op.tb[j];
                        const float2 v = buf[x];
                        const float hr = tf32_round(v.x), hm = tf32_round(v.y);
                        const uint32_t o = sw128_offset(row, 2 * l, PT_M);   // re, im share a 16-B chunk
                        *reinterpret_cast<float2*>(ahi + o) = make_float2(hr, hm);
                        *reinterpret_cast<float2*>(alo + o) = make_float2(tf32_round(v.x - hr), tf32_round(v.y - hm));
                    }
                }
                fence_proxy_async_smem();
                tc_fence_before();
                __syncthreads();
                tc_fence_after();
                if (i < nmt && tid == 0) {
                    if (i == 0) {
                        if (!mbar_wait_bounded(&b_bar, bph, a.err)) s_abort = 1;
                        bph ^= 1u;
                    }
                    const uint32_t ahi = smem_u32(abuf) + (uint32_t)(i & 1) * 2 * PT_A_BYTES;
                    const uint32_t alo = ahi + PT_A_BYTES;
                    const uint32_t bhi = smem_u32(bbuf), blo = bhi + PT_B_BYTES;
                    const uint32_t acc = tmem + (uint32_t)(i & 1) * PT_N;
                    const int ksteps = (2 * D + 7) / 8;
                    // cross terms first, hi*hi last (fewer full-magnitude round-toward-zero steps)
                    for (int kk = 0; kk < ksteps; ++kk) {
                        const uint32_t ko = (uint32_t)kk * 32u;
                        tc_mma(acc, sw128_desc(ahi + ko), sw128_desc(blo + ko), idesc, kk ? 1 : 0);
                        tc_mma(acc, sw128_desc(alo + ko), sw128_desc(bhi + ko), idesc, 1);
                    }
                    for (int kk = 0; kk < ksteps; ++kk) {
                        const uint32_t ko = (uint32_t)kk * 32u;
                        tc_mma(acc, sw128_desc(ahi + ko), sw128_desc(bhi + ko), idesc, 1);
                    }
                    tc_commit(&mma_bar[i & 1]);
                }
                if (i >= 1) {   // epilogue of slice i-1
                    const int s = (i - 1) & 1;
                    if (!mbar_wait_bounded(&mma_bar[s], mph[s], a.err)) s_abort = 1;
                    mph[s] ^= 1u;
                    tc_fence_after();
                    const int q = warp & 3, half = warp >> 2;     // lane quarter, output half
                    float v[16];
                    uint32_t rr[16];
                    asm volatile(
                        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
                        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                        : "=r"(rr[0]), "=r"(rr[1]), "=r"(rr[2]), "=r"(rr[3]), "=r"(rr[4]), "=r"(rr[5]),
                          "=r"(rr[6]), "=r"(rr[7]), "=r"(rr[8]), "=r"(rr[9]), "=r"(rr[10]), "=r"(rr[11]),
                          "=r"(rr[12]), "=r"(rr[13]), "=r"(rr[14]), "=r"(rr[15])
                        : "r"(tmem + (uint32_t)s * PT_N + ((uint32_t)(32 * q) << 16) + (uint32_t)(16 * half))
                        : "memory");
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                    for (int c = 0; c < 16; ++c) v[c] = __uint_as_float(rr[c]);
                    const int row = 32 * q + lane;
                    const int r = (i - 1) * PT_M + row;
                    if (r < rows) {
                        const int x = insert_zeros_bits(r, op.tb, k);
#pragma unroll
                        for (int jj = 0; jj < 8; ++jj) {
                            const int j = 8 * half + jj;
                            if (j < D) {
                                int y = x;
                                for (int b = 0; b < k; ++b)
                                    if ((j >> b) & 1) y |= 1 << op.tb[b];
                                buf[y] = make_float2(v[2 * jj], v[2 * jj + 1]);
                            }
                        }
                    }
                    tc_fence_before();
                }
            }
            __syncthreads();   // block done: the next op sees the updated tile
        }
        if (s_abort) break;
        fence_proxy_async_smem();
        __syncthreads();
        if (tid == 0) {
            int c[5];
            tile_coords(t, c);
            tma_store_tile(tma, buf, c);
            bulk_commit();
            const long long tn = t + 2 * stride;
            if (tn < a.total_tiles) {
                bulk_wait_read<0>();
                tile_coords(tn, c);
                mbar_arrive_expect_tx(&tile_bar[bsel], a.tile_bytes);
                tma_load_tile(tma, buf, &tile_bar[bsel], c);
            }
        }
    }
    if (tid == 0) bulk_wait<0>();
    tc_fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * PT_N)
                     : "memory");
}

size_t pass_tc_smem_bytes(int m) {
    return 1024 + 2 * (sizeof(float2) << m) + 4 * PT_A_BYTES + 2 * PT_B_BYTES;
}

cudaError_t launch_build_b_operands(const TcOp* ops, const int* dense, int n_dense, const float2* table,
                                    float* bops, cudaStream_t s) {
    if (!n_dense) return cudaSuccess;
    build_b_operands_kernel<<<n_dense, 256, 0, s>>>(ops, dense, table, bops);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_pass_tc(const DevPass& p, const PassTcArgs& a, const TmaTile& tma, cudaStream_t s) {
    const size_t smem = pass_tc_smem_bytes(p.m);
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(pass_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)pass_tc_smem_bytes(13));
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const long long grid = std::min<long long>(a.total_tiles, num_sms());
    pass_tc_kernel<<<(unsigned)grid, PT_THREADS, smem, s>>>(p, a, tma);
    count_launch();
    return cudaGetLastError();
}

// ------------------------------------------------------------ host driver --
// Run a tensor-core plan (c64, one parameter set for all items).
tcng_status run_plan_tc(DevPlan* dp, float2* state, const long long* d_item_off, int items,
                        const double* params, cudaStream_t s, void* tma_base, long long item_stride) {
    Plan& pl = dp->plan;
    DeviceCtx& c = ctx();
    // host list of blocks per pass, built once
    if (dp->tc_ops.empty() && !pl.passes.empty()) {
        std::vector<TcOp> ops;
        std::vector<int> dense;
        int slot = 0;
        for (const DevPass& P : pl.passes) {
            dp->tc_begin.push_back((int)ops.size());
            for (int si = 0; si < P.stage_count; ++si) {
                const DevStage& st = pl.stages[P.stage_begin + si];
                for (uint32_t oi = 0; oi < st.op_count; ++oi) {
                    const DevOp& o = pl.dops[st.op_begin + oi];
                    TcOp t{};
                    t.kind = o.kind;
                    t.k = o.k;
                    t.mat = P.mat_begin + (int)o.mat;
                    if (o.kind == K_DENSE) {
                        if (o.k > 4) return fail(TCNG_EUNSUPPORTED, "5-qubit block: use the SIMT passes");
                        int j = 0;
                        for (int r = 0; r < st.nreg; ++r)
                            if ((o.mask >> r) & 1) t.tb[j++] = st.rbit[r];
                        t.slot = slot++;
                        dense.push_back((int)ops.size());
                    } else {
                        for (int j = 0; j < o.k; ++j) t.tb[j] = o.src[j];
                        t.slot = -1;
                    }
                    ops.push_back(t);
                }
            }
        }
        dp->tc_begin.push_back((int)ops.size());
        dp->tc_ops = ops;
        dp->tc_n_dense = slot;
        dp->d_tcops = dev_copy(ops);
        dp->d_tcdense = dev_copy(dense);
    }
    // every pass needs a tile tensor map: check them all before launching anything,
    // so that an unsupported plan falls back with the state untouched
    std::vector<TmaTile> maps(pl.passes.size());
    for (size_t pi = 0; pi < pl.passes.size(); ++pi) {
        maps[pi] = make_tma_tile(tma_base, pl.n, 8, pl.passes[pi], items, item_stride);
        if (!maps[pi].rank) return fail(TCNG_EUNSUPPORTED, "tensor-core pass needs a tile tensor map");
    }
    float2* table = static_cast<float2*>(plan_table(dp, sizeof(float2), 1));
    if (!table) return fail(TCNG_ENOMEM, "matrix table allocation failed");
    cudaError_t e;
    {
        ProfScope ps("build_matrices", s);
        e = launch_build_matrices<float2>(dp->d_bblocks, (int)pl.bblocks.size(), dp->d_bops, dp->d_pool,
                                          pl.P > 0 ? params : nullptr, pl.P, table, pl.table_size, 1, s);
    }
    if (e != cudaSuccess) return cuda_fail(e, "matrix prologue");
    float* bops = static_cast<float*>(c.scratch("tc_bops", sizeof(float) * PT_B_FLOATS * std::max(1, dp->tc_n_dense)));
    if (!bops) return fail(TCNG_ENOMEM, "B operand scratch");
    {
        ProfScope ps("build_b_operands", s);
        e = launch_build_b_operands(reinterpret_cast<const TcOp*>(dp->d_tcops), dp->d_tcdense,
                                    dp->tc_n_dense, table, bops, s);
    }
    if (e != cudaSuccess) return cuda_fail(e, "B operand prologue");
    for (size_t pi = 0; pi < pl.passes.size(); ++pi) {
        const DevPass& P = pl.passes[pi];
        const TmaTile& tma = maps[pi];
        PassTcArgs a{};
        a.state = state;
        a.item_off = d_item_off;
        a.ops = reinterpret_cast<const TcOp*>(dp->d_tcops) + dp->tc_begin[pi];
        a.n_ops = dp->tc_begin[pi + 1] - dp->tc_begin[pi];
        a.table = table;
        a.bops = bops;
        a.tiles_per_item = 1ll << (pl.n - P.m);
        a.total_tiles = a.tiles_per_item * items;
        a.tile_bytes = (uint32_t)(sizeof(float2) << P.m);
        a.err = c.err;
        ProfScope ps("pass_tc_kernel_c64", s);
        e = launch_pass_tc(P, a, tma, s);
        if (e != cudaSuccess) return cuda_fail(e, "tensor-core pass");
    }
    return TCNG_OK;
}

}  // namespace tcng
