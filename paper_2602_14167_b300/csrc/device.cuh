// Device helpers: complex arithmetic, bulk-copy (TMA) and mbarrier PTX wrappers,
// and the register-stage executor shared by the tile-pass kernels.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

#include "internal.hpp"
#include "launch.hpp"

namespace tcng {

// ------------------------------------------------------------------ errors --
enum : unsigned {
    ERR_TIMEOUT = 1u,   // a bounded mbarrier wait expired
    ERR_BAD_ITEM = 2u,  // a work item referenced an invalid structure
};
constexpr unsigned long long kWaitLimitNs = 2000000000ull;   // 2 s per wait

// ----------------------------------------------------------------- complex --
template <typename C> struct Real;
template <> struct Real<float2> { using T = float; };
template <> struct Real<double2> { using T = double; };

template <typename C> __device__ __forceinline__ C cmk(typename Real<C>::T x, typename Real<C>::T y) {
    C r; r.x = x; r.y = y; return r;
}
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
    return cmk<C>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// acc += a * b
template <typename C> __device__ __forceinline__ void cfma(C& acc, C a, C b) {
    acc.x = fma(a.x, b.x, fma(-a.y, b.y, acc.x));
    acc.y = fma(a.x, b.y, fma(a.y, b.x, acc.y));
}
template <typename C> __device__ __forceinline__ C cconj(C a) { return cmk<C>(a.x, -a.y); }

// ------------------------------------------------------------- bit helpers --
__host__ __device__ constexpr int cpopc(int v) { return v ? (v & 1) + cpopc(v >> 1) : 0; }
__host__ __device__ constexpr int cctz(int v) { return (v & 1) ? 0 : 1 + cctz(v >> 1); }
// deposit the low bits of v into the set positions of mask (compile-time friendly)
__host__ __device__ constexpr int cscatter(int v, int mask) {
    int out = 0, b = 0;
    for (int p = 0; p < 8; ++p)
        if ((mask >> p) & 1) { if ((v >> b) & 1) out |= 1 << p; ++b; }
    return out;
}
__device__ __forceinline__ int pext4(int v, int mask) {
    int out = 0, b = 0;
#pragma unroll
    for (int p = 0; p < 8; ++p)
        if ((mask >> p) & 1) { out |= ((v >> p) & 1) << b; ++b; }
    return out;
}

// ------------------------------------------------------------------- PTX --
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}
// Bounded wait: false (and error word set) if the phase did not complete in time.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, unsigned* err) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (uint32_t it = 1;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 255u) == 0 && global_ns() - t0 > kWaitLimitNs) {
            if (err) atomicOr(err, ERR_TIMEOUT);
            return false;
        }
    }
}
__device__ __forceinline__ void bulk_g2s(void* dst_smem, const void* src_gmem, uint32_t bytes,
                                         uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst_smem)),
        "l"(src_gmem), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void bulk_s2g(void* dst_gmem, const void* src_smem, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst_gmem),
                 "r"(smem_u32(src_smem)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
template <int N> __device__ __forceinline__ void bulk_wait_read() {
    asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory");
}
template <int N> __device__ __forceinline__ void bulk_wait() {
    asm volatile("cp.async.bulk.wait_group %0;" ::"n"(N) : "memory");
}

// --------------------------------------------------- TMA tensor copies --
// One multi-dimensional tensor copy of a whole tile (see TmaTile).
__device__ __forceinline__ void tma_tile_coords(const TmaTile& t, long long tile_local, int item,
                                                int (&c)[5]) {
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        c[i] = 0;
        if (i < t.rank) {
            if (t.kind[i] == 1) c[i] = (int)((tile_local >> t.shift[i]) & ((1ll << t.len[i]) - 1)) << t.lsh[i];
            else if (t.kind[i] == 2) c[i] = item;
        }
    }
}
__device__ __forceinline__ void tma_load_tile(const TmaTile& t, void* dst, uint64_t* bar, const int (&c)[5]) {
    const uint64_t map = reinterpret_cast<uint64_t>(&t.map);
    const uint32_t d = smem_u32(dst), b = smem_u32(bar);
    switch (t.rank) {
    case 1:
        asm volatile("cp.async.bulk.tensor.1d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2}], [%3];"
                     ::"r"(d), "l"(map), "r"(c[0]), "r"(b) : "memory");
        break;
    case 2:
        asm volatile("cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
                     ::"r"(d), "l"(map), "r"(c[0]), "r"(c[1]), "r"(b) : "memory");
        break;
    case 3:
        asm volatile("cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
                     ::"r"(d), "l"(map), "r"(c[0]), "r"(c[1]), "r"(c[2]), "r"(b) : "memory");
        break;
    case 4:
        asm volatile("cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];"
                     ::"r"(d), "l"(map), "r"(c[0]), "r"(c[1]), "r"(c[2]), "r"(c[3]), "r"(b) : "memory");
        break;
    default:
        asm volatile("cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5, %6}], [%7];"
                     ::"r"(d), "l"(map), "r"(c[0]), "r"(c[1]), "r"(c[2]), "r"(c[3]), "r"(c[4]), "r"(b) : "memory");
        break;
    }
}
// Four rows (r0..r3, one box each) of a 2D tensor map into consecutive shared memory.
__device__ __forceinline__ void tma_gather4(const TmaTile& t, void* dst, uint64_t* bar, int r0, int r1, int r2,
                                            int r3) {
    const uint64_t map = reinterpret_cast<uint64_t>(&t.map);
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile::gather4.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(smem_u32(dst)),
        "l"(map), "r"(0), "r"(r0), "r"(r1), "r"(r2), "r"(r3), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void tma_store_tile(const TmaTile& t, const void* src, const int (&c)[5]) {
    const uint64_t map = reinterpret_cast<uint64_t>(&t.map);
    const uint32_t sp = smem_u32(src);
    switch (t.rank) {
    case 1:
        asm volatile("cp.async.bulk.tensor.1d.global.shared::cta.tile.bulk_group [%0, {%1}], [%2];"
                     ::"l"(map), "r"(c[0]), "r"(sp) : "memory");
        break;
    case 2:
        asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.tile.bulk_group [%0, {%1, %2}], [%3];"
                     ::"l"(map), "r"(c[0]), "r"(c[1]), "r"(sp) : "memory");
        break;
    case 3:
        asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.tile.bulk_group [%0, {%1, %2, %3}], [%4];"
                     ::"l"(map), "r"(c[0]), "r"(c[1]), "r"(c[2]), "r"(sp) : "memory");
        break;
    case 4:
        asm volatile("cp.async.bulk.tensor.4d.global.shared::cta.tile.bulk_group [%0, {%1, %2, %3, %4}], [%5];"
                     ::"l"(map), "r"(c[0]), "r"(c[1]), "r"(c[2]), "r"(c[3]), "r"(sp) : "memory");
        break;
    default:
        asm volatile("cp.async.bulk.tensor.5d.global.shared::cta.tile.bulk_group [%0, {%1, %2, %3, %4, %5}], [%6];"
                     ::"l"(map), "r"(c[0]), "r"(c[1]), "r"(c[2]), "r"(c[3]), "r"(c[4]), "r"(sp) : "memory");
        break;
    }
}

// ---------------------------------------------------- tile index mapping --
// Global index (within an item) of tile offset 0: the tile number's bits are
// deposited into the global bits outside the tile.
__device__ __forceinline__ long long tile_global_base(const DevPass& p, long long tile) {
    long long base = 0;
    for (int i = 0; i < p.nrest; ++i)
        if ((tile >> i) & 1) base |= 1ll << p.rest[i];
    return base;
}
// Global offset (relative to the tile base) of chunk j (gather pattern j).
__device__ __forceinline__ long long chunk_offset(const DevPass& p, int j) {
    long long off = 0;
    for (int i = 0; i < p.ngather; ++i)
        if ((j >> i) & 1) off |= 1ll << p.gather[i];
    return off;
}
// -------------------------------------------------------- dense register op --
// a[2^R] holds the amplitudes of one group: slot s holds tile offset
// base | scatter(s ^ tau) (XOR rotation by tau spreads shared-memory banks).
// Apply a 2^K x 2^K matrix (row-major, ascending local order) on register bits
// MASK; DAG applies the conjugate transpose.
template <typename C, int R, int MASK, bool DAG>
__device__ __forceinline__ void dense_apply(C (&a)[1 << R], const C* __restrict__ M, int tau) {
    constexpr int K = cpopc(MASK);
    constexpr int D = 1 << K;
    constexpr int OMASK = ((1 << R) - 1) & ~MASK;
    constexpr int NOUT = (1 << R) >> K;
    const int t = pext4(tau, MASK);
    if constexpr (K <= 2) {
        C m[D][D];
#pragma unroll
        for (int r = 0; r < D; ++r)
#pragma unroll
            for (int c = 0; c < D; ++c) {
                if constexpr (DAG) m[r][c] = cconj(M[((c ^ t) << K) | (r ^ t)]);
                else m[r][c] = M[((r ^ t) << K) | (c ^ t)];
            }
#pragma unroll
        for (int o = 0; o < NOUT; ++o) {
            const int base = cscatter(o, OMASK);
            C v[D];
#pragma unroll
            for (int s = 0; s < D; ++s) v[s] = a[base | cscatter(s, MASK)];
#pragma unroll
            for (int r = 0; r < D; ++r) {
                C acc = cmk<C>(0, 0);
#pragma unroll
                for (int s = 0; s < D; ++s) cfma(acc, m[r][s], v[s]);
                a[base | cscatter(r, MASK)] = acc;
            }
        }
    } else {
        C v[NOUT][D];
#pragma unroll
        for (int o = 0; o < NOUT; ++o)
#pragma unroll
            for (int s = 0; s < D; ++s) v[o][s] = a[cscatter(o, OMASK) | cscatter(s, MASK)];
#pragma unroll
        for (int r = 0; r < D; ++r) {
            C acc[NOUT];
#pragma unroll
            for (int o = 0; o < NOUT; ++o) acc[o] = cmk<C>(0, 0);
#pragma unroll
            for (int s = 0; s < D; ++s) {
                C mv;
                if constexpr (DAG) mv = cconj(M[((s ^ t) << K) | (r ^ t)]);
                else mv = M[((r ^ t) << K) | (s ^ t)];
#pragma unroll
                for (int o = 0; o < NOUT; ++o) cfma(acc[o], mv, v[o][s]);
            }
#pragma unroll
            for (int o = 0; o < NOUT; ++o) a[cscatter(o, OMASK) | cscatter(r, MASK)] = acc[o];
        }
    }
}

// The same matrix on two groups at once (the adjoint sweep's psi and lambda):
// one dispatch and one decode of the matrix for both.
template <typename C, int R, int MASK, bool DAG>
__device__ __forceinline__ void dense_apply2(C (&a)[1 << R], C (&b)[1 << R], const C* __restrict__ M, int tau) {
    constexpr int K = cpopc(MASK);
    if constexpr (K <= 2) {
        constexpr int D = 1 << K;
        constexpr int OMASK = ((1 << R) - 1) & ~MASK;
        constexpr int NOUT = (1 << R) >> K;
        const int t = pext4(tau, MASK);
        C m[D][D];
#pragma unroll
        for (int r = 0; r < D; ++r)
#pragma unroll
            for (int c = 0; c < D; ++c) {
                if constexpr (DAG) m[r][c] = cconj(M[((c ^ t) << K) | (r ^ t)]);
                else m[r][c] = M[((r ^ t) << K) | (c ^ t)];
            }
#pragma unroll
        for (int o = 0; o < NOUT; ++o) {
            const int base = cscatter(o, OMASK);
            C va[D], vb[D];
#pragma unroll
            for (int s = 0; s < D; ++s) {
                va[s] = a[base | cscatter(s, MASK)];
                vb[s] = b[base | cscatter(s, MASK)];
            }
#pragma unroll
            for (int r = 0; r < D; ++r) {
                C acc_a = cmk<C>(0, 0), acc_b = cmk<C>(0, 0);
#pragma unroll
                for (int s = 0; s < D; ++s) {
                    cfma(acc_a, m[r][s], va[s]);
                    cfma(acc_b, m[r][s], vb[s]);
                }
                a[base | cscatter(r, MASK)] = acc_a;
                b[base | cscatter(r, MASK)] = acc_b;
            }
        }
    } else {
        dense_apply<C, R, MASK, DAG>(a, M, tau);
        dense_apply<C, R, MASK, DAG>(b, M, tau);
    }
}

template <typename C, int R, bool DAG, int MASK>
__device__ __forceinline__ void dense_case2(C (&a)[1 << R], C (&b)[1 << R], const C* M, int tau) {
    if constexpr (MASK < (1 << R)) dense_apply2<C, R, MASK, DAG>(a, b, M, tau);
}

template <typename C, int R, bool DAG>
__device__ __forceinline__ void dense_dispatch2(int mask, C (&a)[1 << R], C (&b)[1 << R], const C* M, int tau) {
    switch (mask) {
#define TCNG_CASE(m) case m: dense_case2<C, R, DAG, m>(a, b, M, tau); break;
        TCNG_CASE(1) TCNG_CASE(2) TCNG_CASE(3) TCNG_CASE(4) TCNG_CASE(5) TCNG_CASE(6)
        TCNG_CASE(7) TCNG_CASE(8) TCNG_CASE(9) TCNG_CASE(10) TCNG_CASE(11) TCNG_CASE(12)
        TCNG_CASE(13) TCNG_CASE(14) TCNG_CASE(15) TCNG_CASE(16) TCNG_CASE(17) TCNG_CASE(18)
        TCNG_CASE(19) TCNG_CASE(20) TCNG_CASE(21) TCNG_CASE(22) TCNG_CASE(23) TCNG_CASE(24)
        TCNG_CASE(25) TCNG_CASE(26) TCNG_CASE(27) TCNG_CASE(28) TCNG_CASE(29) TCNG_CASE(30)
        TCNG_CASE(31)
#undef TCNG_CASE
        default: break;
    }
}

template <typename C, int R, bool DAG, int MASK>
__device__ __forceinline__ void dense_case(C (&a)[1 << R], const C* M, int tau) {
    if constexpr (MASK < (1 << R)) dense_apply<C, R, MASK, DAG>(a, M, tau);
}

template <typename C, int R, bool DAG>
__device__ __forceinline__ void dense_dispatch(int mask, C (&a)[1 << R], const C* M, int tau) {
    switch (mask) {
#define TCNG_CASE(m) case m: dense_case<C, R, DAG, m>(a, M, tau); break;
        TCNG_CASE(1) TCNG_CASE(2) TCNG_CASE(3) TCNG_CASE(4) TCNG_CASE(5) TCNG_CASE(6)
        TCNG_CASE(7) TCNG_CASE(8) TCNG_CASE(9) TCNG_CASE(10) TCNG_CASE(11) TCNG_CASE(12)
        TCNG_CASE(13) TCNG_CASE(14) TCNG_CASE(15) TCNG_CASE(16) TCNG_CASE(17) TCNG_CASE(18)
        TCNG_CASE(19) TCNG_CASE(20) TCNG_CASE(21) TCNG_CASE(22) TCNG_CASE(23) TCNG_CASE(24)
        TCNG_CASE(25) TCNG_CASE(26) TCNG_CASE(27) TCNG_CASE(28) TCNG_CASE(29) TCNG_CASE(30)
        TCNG_CASE(31)
#undef TCNG_CASE
        default: break;
    }
}

// Bit of qubit source `src` for tile offset L in a tile whose global base is gbase.
__device__ __forceinline__ int src_bit(uint8_t src, int L, long long gbase) {
    return (src & kSrcBase) ? int((gbase >> (src & 63)) & 1) : ((L >> src) & 1);
}

// Phase-table index of every slot for a diagonal op: the index of slot 0 from its
// tile offset, then one XOR per slot -- flipping register bit i flips index bit
// e_i (the source fed by that register bit, from the planner's nibbles).
// L0: tile offset of slot 0.
template <int R>
__device__ __forceinline__ void diag_index0(const DevOp& op, int L0, long long gbase, int (&idx)[1 << R]) {
    int i0 = 0;
    // unrolled to the 5 source slots (compile-time indices keep op in registers)
#pragma unroll
    for (int j = 0; j < 5; ++j)
        if (j < op.k) i0 |= src_bit(op.src[j], L0, gbase) << j;
    const int nib = op.mask | (op.pad << 8);
    int e[R];
#pragma unroll
    for (int i = 0; i < R; ++i) {
        const int jj = (i < 4) ? ((nib >> (4 * i)) & 15) : 0;
        e[i] = jj ? (1 << (jj - 1)) : 0;
    }
    idx[0] = i0;
#pragma unroll
    for (int s = 1; s < (1 << R); ++s) {
        const int low = cctz(s);                   // compile-time after unrolling
        idx[s] = idx[s & (s - 1)] ^ e[low];
    }
}

template <int R>
__device__ __forceinline__ void diag_index(const DevOp& op, const int (&L)[1 << R], long long gbase,
                                           int (&idx)[1 << R]) {
    diag_index0<R>(op, L[0], gbase, idx);
}

// Slots (bit s of a mask) where source 0 / source 1 of a diagonal op is 1: slot 0's
// value from its tile offset L0, then one XOR of a constant slot pattern for each
// register bit that feeds the source.
template <int R>
__device__ __forceinline__ void src_masks(const DevOp& op, int L0, long long gbase, uint32_t& m0, uint32_t& m1) {
    constexpr uint32_t kSlots[5] = {0xAAAAAAAAu, 0xCCCCCCCCu, 0xF0F0F0F0u, 0xFF00FF00u, 0xFFFF0000u};
    m0 = src_bit(op.src[0], L0, gbase) ? 0xFFFFFFFFu : 0u;
    m1 = (op.k > 1 && src_bit(op.src[1], L0, gbase)) ? 0xFFFFFFFFu : 0u;
    const int nib = op.mask | (op.pad << 8);
#pragma unroll
    for (int i = 0; i < R && i < 4; ++i) {
        const int jj = (nib >> (4 * i)) & 15;
        if (jj == 1) m0 ^= kSlots[i];
        if (jj == 2) m1 ^= kSlots[i];
    }
}
// A lone RZ (G_Z) or RZZ (G_ZZ) takes M[0] on even and M[1] on odd parity of its
// sources: the odd slots (one mask for the parity: slot 0's from its tile offset,
// then the slot pattern of each register bit that feeds a source).
template <int R>
__device__ __forceinline__ uint32_t zpar_mask(const DevOp& op, int L0, long long gbase) {
    constexpr uint32_t kSlots[5] = {0xAAAAAAAAu, 0xCCCCCCCCu, 0xF0F0F0F0u, 0xFF00FF00u, 0xFFFF0000u};
    int p0 = src_bit(op.src[0], L0, gbase);
    if (op.k > 1) p0 ^= src_bit(op.src[1], L0, gbase);
    uint32_t m = p0 ? 0xFFFFFFFFu : 0u;
    const int nib = op.mask | (op.pad << 8);
#pragma unroll
    for (int i = 0; i < R && i < 4; ++i)
        if ((nib >> (4 * i)) & 15) m ^= kSlots[i];
    return m;
}
// A lone controlled phase (G_P11) takes M[3] on the slots where both sources are 1,
// else M[0].
template <int R>
__device__ __forceinline__ uint32_t p11_mask(const DevOp& op, int L0, long long gbase) {
    uint32_t m0, m1;
    src_masks<R>(op, L0, gbase, m0, m1);
    return m0 & m1;
}
// a[s] <- d_s a[s] with d_s = m0, or m1 on the slots of `odd`, conjugated for DAG.
template <typename C, int R, bool DAG>
__device__ __forceinline__ void zpar_apply(C (&a)[1 << R], uint32_t odd, C m0, C m1) {
    if constexpr (DAG) {
        m0 = cconj(m0);
        m1 = cconj(m1);
    }
#pragma unroll
    for (int s = 0; s < (1 << R); ++s) {
        const bool o = (odd >> s) & 1u;
        const C d = cmk<C>(o ? m1.x : m0.x, o ? m1.y : m0.y);
        a[s] = cmul(d, a[s]);
    }
}

// Diagonal op: multiply slot s by M[idx(s)].
template <typename C, int R, bool DAG>
__device__ __forceinline__ void diag_apply(C (&a)[1 << R], const DevOp& op, const C* __restrict__ M,
                                           const int (&L)[1 << R], long long gbase) {
    int idx[1 << R];
    diag_index<R>(op, L, gbase, idx);
#pragma unroll
    for (int s = 0; s < (1 << R); ++s) {
        C d = M[idx[s]];
        if constexpr (DAG) d = cconj(d);
        a[s] = cmul(d, a[s]);
    }
}

// Diagonal op on two groups with the same slot indices (psi and lambda).
template <typename C, int R, bool DAG>
__device__ __forceinline__ void diag_apply2(C (&a)[1 << R], C (&b)[1 << R], const C* __restrict__ M,
                                            const int (&idx)[1 << R]) {
#pragma unroll
    for (int s = 0; s < (1 << R); ++s) {
        C d = M[idx[s]];
        if constexpr (DAG) d = cconj(d);
        a[s] = cmul(d, a[s]);
        b[s] = cmul(d, b[s]);
    }
}

// A lone RX (IS_Y false) or RY (IS_Y true) on register bit BIT, from c = cos(t/2)
// and s = sin(t/2): U = c I - i s G (adjoint plans mark such ops with their
// generator), half the products of a general 2x2 complex matrix.  For RY a
// flipped slot order on BIT negates s (RX is symmetric under the flip).
template <typename C, int R, int BIT, bool IS_Y>
__device__ __forceinline__ void rot_apply(C (&a)[1 << R], typename Real<C>::T c, typename Real<C>::T s) {
    if constexpr (BIT < R) {
#pragma unroll
        for (int k = 0; k < (1 << R); ++k) {
            if ((k >> BIT) & 1) continue;
            const int k1 = k | (1 << BIT);
            const C a0 = a[k], a1 = a[k1];
            if constexpr (!IS_Y) {   // [[c, -i s], [-i s, c]]
                a[k] = cmk<C>(c * a0.x + s * a1.y, c * a0.y - s * a1.x);
                a[k1] = cmk<C>(c * a1.x + s * a0.y, c * a1.y - s * a0.x);
            } else {                 // [[c, -s], [s, c]]
                a[k] = cmk<C>(c * a0.x - s * a1.x, c * a0.y - s * a1.y);
                a[k1] = cmk<C>(c * a1.x + s * a0.x, c * a1.y + s * a0.y);
            }
        }
    }
}

// The same dispatched on the op's register bit; c and s from its matrix
// (RX [[c, -i s], [-i s, c]], RY [[c, -s], [s, c]], row-major).
template <typename C, int R>
__device__ __forceinline__ void rot_dispatch(const DevOp& op, C (&a)[1 << R], const C* __restrict__ M, int tau) {
    using T = typename Real<C>::T;
    const int bit = __ffs(op.mask) - 1;
    const bool is_y = op.grad == G_Y;
    const T c = M[0].x;
    const T s = is_y ? (((tau >> bit) & 1) ? -M[2].x : M[2].x) : -M[1].y;
    switch (bit) {
#define TCNG_RA(B)                                        \
    case B:                                               \
        if (is_y) rot_apply<C, R, B, true>(a, c, s);      \
        else rot_apply<C, R, B, false>(a, c, s);          \
        break;
        TCNG_RA(0) TCNG_RA(1) TCNG_RA(2) TCNG_RA(3) TCNG_RA(4)
#undef TCNG_RA
    default: break;
    }
}

// Insert a zero bit at each of the R register positions (ascending) into g.
template <int R>
__device__ __forceinline__ int insert_zero_bits(int g, const uint8_t* rbit) {
#pragma unroll
    for (int i = 0; i < R; ++i) {
        const int p = rbit[i];
        g = ((g >> p) << (p + 1)) | (g & ((1 << p) - 1));
    }
    return g;
}

// Tile offsets of the 2^R slots of group g in a stage with register bits rbit
// (slot s holds offset base | scatter(s ^ tau)).
template <int R>
__device__ __forceinline__ void group_offsets(int g, int tau, const uint8_t* rbit, int (&L)[1 << R]) {
    const int base = insert_zero_bits<R>(g, rbit);
    int sr[R];
#pragma unroll
    for (int i = 0; i < R; ++i) sr[i] = 1 << rbit[i];
    int stau = 0;
#pragma unroll
    for (int i = 0; i < R; ++i) stau |= ((tau >> i) & 1) ? sr[i] : 0;
#pragma unroll
    for (int s = 0; s < (1 << R); ++s) {
        int o = 0;
#pragma unroll
        for (int i = 0; i < R; ++i) o |= ((s >> i) & 1) ? sr[i] : 0;
        L[s] = base | (o ^ stau);
    }
}

// Stage executor: one group (2^R amplitudes) of one tile, forward direction.
// ROT: XOR-rotate the slots by the group index (only needed when the register
// bits include a bank-selecting tile bit); without it every thread reads the
// same matrix entries (shared-memory broadcast, compile-time indices).
template <typename C, int R, bool ROT>
__device__ __forceinline__ void run_stage_group(C* __restrict__ buf, const DevStage& st,
                                                const DevOp* __restrict__ ops, const C* __restrict__ mats,
                                                int g, long long gbase) {
    int L[1 << R];
    const int tau = ROT ? (g & ((1 << R) - 1)) : 0;
    group_offsets<R>(g, tau, st.rbit, L);
    C a[1 << R];
#pragma unroll
    for (int s = 0; s < (1 << R); ++s) a[s] = buf[L[s]];
    for (uint32_t i = 0; i < st.op_count; ++i) {
        const DevOp op = ops[st.op_begin + i];
        const C* M = mats + op.mat;
        if (op.kind == K_DENSE) {
            if (op.grad == G_X || op.grad == G_Y) rot_dispatch<C, R>(op, a, M, tau);   // lone RX / RY
            else dense_dispatch<C, R, false>(op.mask, a, M, tau);
        } else if (op.grad == G_Z || op.grad == G_ZZ) {   // lone RZ / RZZ
            zpar_apply<C, R, false>(a, zpar_mask<R>(op, L[0], gbase), M[0], M[1]);
        } else if (op.grad == G_P11) {                     // lone controlled phase
            zpar_apply<C, R, false>(a, p11_mask<R>(op, L[0], gbase), M[0], M[3]);
        } else {
            diag_apply<C, R, false>(a, op, M, L, gbase);
        }
    }
#pragma unroll
    for (int s = 0; s < (1 << R); ++s) buf[L[s]] = a[s];
}

// Generic stage executor working directly on the shared-memory tile, one op at
// a time (used for stages holding a 5-qubit block, which are rare: unrolling
// 32-amplitude register groups would dominate compile time).  DAG applies the
// conjugate transpose in reverse op order.  Contains barriers: call with the
// whole CTA.
template <typename C, bool DAG>
__device__ void run_stage_smem(C* __restrict__ buf, const DevStage& st, const DevOp* __restrict__ ops,
                               const C* __restrict__ mats, int tile_bits, long long gbase) {
    const int N = 1 << tile_bits;
    for (uint32_t ii = 0; ii < st.op_count; ++ii) {
        const uint32_t i = DAG ? st.op_count - 1 - ii : ii;
        const DevOp op = ops[st.op_begin + i];
        const C* M = mats + op.mat;
        if (op.kind == K_DENSE) {
            int tb[TCNG_MAX_FUSE];
            int k = 0;
            for (int r = 0; r < st.nreg; ++r)
                if ((op.mask >> r) & 1) tb[k++] = st.rbit[r];
            const int D = 1 << k;
            for (int c = threadIdx.x; c < (N >> k); c += blockDim.x) {
                int x = c;
                for (int j = 0; j < k; ++j) x = ((x >> tb[j]) << (tb[j] + 1)) | (x & ((1 << tb[j]) - 1));
                C v[32];
                for (int s = 0; s < D; ++s) {
                    int y = x;
                    for (int j = 0; j < k; ++j)
                        if ((s >> j) & 1) y |= 1 << tb[j];
                    v[s] = buf[y];
                }
                for (int r = 0; r < D; ++r) {
                    C acc = cmk<C>(0, 0);
                    for (int s = 0; s < D; ++s) {
                        const C m = DAG ? cconj(M[s * D + r]) : M[r * D + s];
                        cfma(acc, m, v[s]);
                    }
                    int y = x;
                    for (int j = 0; j < k; ++j)
                        if ((r >> j) & 1) y |= 1 << tb[j];
                    buf[y] = acc;
                }
            }
        } else {
            for (int L = threadIdx.x; L < N; L += blockDim.x) {
                int idx = 0;
#pragma unroll
                for (int j = 0; j < 5; ++j)
                    if (j < op.k) idx |= src_bit(op.src[j], L, gbase) << j;
                C d = M[idx];
                if (DAG) d = cconj(d);
                buf[L] = cmul(d, buf[L]);
            }
        }
        __syncthreads();
    }
}

// One stage over a whole tile by the CTA (no trailing barrier for register stages).
template <typename C>
__device__ __forceinline__ void run_stage(C* __restrict__ buf, const DevStage& st,
                                          const DevOp* __restrict__ ops, const C* __restrict__ mats,
                                          int tile_bits, long long gbase) {
    if (st.nreg > kRegBits) {
        run_stage_smem<C, false>(buf, st, ops, mats, tile_bits, gbase);
    } else if (st.rotate) {
        const int ngroups = 1 << (tile_bits - kRegBits);
        for (int g = threadIdx.x; g < ngroups; g += blockDim.x)
            run_stage_group<C, kRegBits, true>(buf, st, ops, mats, g, gbase);
    } else {
        const int ngroups = 1 << (tile_bits - kRegBits);
        for (int g = threadIdx.x; g < ngroups; g += blockDim.x)
            run_stage_group<C, kRegBits, false>(buf, st, ops, mats, g, gbase);
    }
}

}  // namespace tcng
