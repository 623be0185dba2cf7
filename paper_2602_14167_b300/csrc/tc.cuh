// tcgen05 helpers: 128-byte-swizzled K-major operand layout, TF32 split,
// shared-memory and instruction descriptors, MMA issue/commit, TMEM loads.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <cstdint>

#include "device.cuh"

namespace tcng {

constexpr int TC_M = 128;            // rows per tile (TMEM lanes)
constexpr int TC_K = 64;             // real K (2 * 2^k padded to 64)
constexpr int TC_N = 64;             // real N
constexpr int TC_ROWB = 128;         // bytes per row per 32-element K block (swizzle atom row)
constexpr int TC_KBLK = TC_K / 32;   // K blocks of 32 fp32
constexpr uint32_t TC_A_BYTES = TC_M * TC_K * 4;   // 32 KiB per split part
constexpr uint32_t TC_B_BYTES = TC_N * TC_K * 4;   // 16 KiB per split part

// Byte offset of element (row, kel) of a K-major, 128-byte-swizzled operand whose
// K blocks of 32 elements are stored one after another (rows x 128 B each).
__device__ __forceinline__ uint32_t sw128_offset(int row, int kel, int rows) {
    const int kb = kel >> 5, kin = kel & 31;
    const uint32_t chunk = (uint32_t)((kin >> 2) ^ (row & 7));
    return (uint32_t)kb * (uint32_t)rows * TC_ROWB + (uint32_t)(row >> 3) * 1024u +
           (uint32_t)(row & 7) * TC_ROWB + chunk * 16u + (uint32_t)(kin & 3) * 4u;
}

// The same layout for 16-bit elements: row `row` of 32 rows, element kh of the
// row's 64 halves (128 bytes).
__device__ __forceinline__ uint32_t sw128_offset_h(int row, int kh) {
    const uint32_t chunk = (uint32_t)((kh >> 3) ^ (row & 7));
    return (uint32_t)(row >> 3) * 1024u + (uint32_t)(row & 7) * TC_ROWB + chunk * 16u + (uint32_t)(kh & 7) * 2u;
}

// W operand of one FP16-split register stage: 32 rows x [hi 32 | lo 32] halves.
constexpr uint32_t TH_W_BYTES = 32 * 128;

__device__ __forceinline__ float tf32_round(float x) {
    uint32_t u = __float_as_uint(x);
    if ((u & 0x7f800000u) != 0x7f800000u) {   // finite: round to nearest even on 13 bits
        u += 0xfffu + ((u >> 13) & 1u);
        u &= 0xffffe000u;
    }
    return __uint_as_float(u);
}

// tcgen05 shared-memory matrix descriptor: K-major, 128-byte swizzle, 1024-byte
// stride between 8-row groups.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t smem_addr) {
    uint64_t d = 0;
    d |= (uint64_t)((smem_addr >> 4) & 0x3fffu);          // start address
    d |= (uint64_t)1u << 16;                               // leading byte offset (unused here)
    d |= (uint64_t)(1024u >> 4) << 32;                     // stride byte offset
    d |= (uint64_t)1u << 46;                               // fixed 0b001
    d |= (uint64_t)2u << 61;                               // 128-byte swizzle
    return d;
}

// Instruction descriptor, kind::tf32: D f32, A/B tf32, both K-major, M x N.
__host__ __device__ constexpr uint32_t tf32_idesc(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Instruction descriptor, kind::f16: D f32, A/B f16, both K-major, M x N.
__host__ __device__ constexpr uint32_t f16_idesc(int M, int N) {
    return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// D (TMEM) += A (TMEM, f16 pairs per column) * B (shared-memory descriptor, f16)
__device__ __forceinline__ void tc_mma_f16_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t b, uint32_t idesc,
                                              int accum) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
        "r"(a_tmem), "l"(b), "r"(idesc), "r"(accum)
        : "memory");
}

// 16 consecutive 32-bit TMEM columns of this warp's 32 lanes.
__device__ __forceinline__ void tc_st16(uint32_t taddr, const uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
        "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(taddr),
        "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
        "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
        : "memory");
}

__device__ __forceinline__ void tc_mma(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc, int accum) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accum)
        : "memory");
}
// One lane of a converged warp (elect.sync).  Issuing MMAs from an elected lane
// of a warp-uniform branch, with warp-uniform operands, keeps those operands in
// uniform registers.
__device__ __forceinline__ bool elect_one() {
    uint32_t p;
    asm volatile("{\n\t.reg .pred e;\n\telect.sync _|e, 0xffffffff;\n\tselp.u32 %0, 1, 0, e;\n\t}" : "=r"(p));
    return p != 0;
}
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// 32 consecutive fp32 TMEM columns of this warp's 32 lanes.
__device__ __forceinline__ void tc_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]),
          "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]),
          "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}


}  // namespace tcng
