// Batched energy + adjoint gradient: one persistent launch over B items.
//
// Paper: Sec. I.B "Paradigms" -- value_and_grad of the TFIM energy, vmapped over
// a batch of parameter sets ("thousands of independent circuit instances").
// The paper differentiates by reverse-mode AD through the tensor network; here
// the gradient comes from an adjoint sweep that keeps two states:
//   forward   psi = U_K ... U_1 |0>,
//   co-state  lambda = H psi,  E = Re <psi|lambda>,
//   reverse   for k = K..1:  g_k += Im <lambda|G_k|psi>  (U_k = exp(-i theta G_k / 2)),
//             psi <- U_k^dag psi,  lambda <- U_k^dag lambda,
// so memory is O(1) states whatever the number of parameters.
//
// Each CTA pops items from a global counter (largest n first).  States of up to
// 2^13 (complex64) / 2^12 (complex128) amplitudes live in shared memory for the
// whole item ("resident"); larger ones stream through per-CTA global scratch in
// tiles of the same size (psi and lambda tiles in the two resident buffers)
// with bulk asynchronous copies.
#include <cuda_runtime.h>

#include <algorithm>

#include "adjoint.hpp"
#include "device.cuh"

namespace tcng {

// ------------------------------------------------------------ reductions --
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <typename R>
__device__ __forceinline__ R im_conj_mul(R lx, R ly, R px, R py) {  // Im(conj(l) p)
    return lx * py - ly * px;
}

// Im<lambda|X|psi> or Im<lambda|Y|psi> of one group for a gate on register bit BIT.
template <typename C, int R, int BIT, bool is_y>
__device__ __forceinline__ typename Real<C>::T grad_xy(const C (&p)[1 << R], const C (&l)[1 << R], int flip) {
    using T = typename Real<C>::T;
    T acc = 0;
    if constexpr (BIT < R) {
#pragma unroll
        for (int s = 0; s < (1 << R); ++s) {
            if ((s >> BIT) & 1) continue;
            const int s1 = s | (1 << BIT);
            if constexpr (!is_y) {
                acc += im_conj_mul(l[s].x, l[s].y, p[s1].x, p[s1].y) +
                       im_conj_mul(l[s1].x, l[s1].y, p[s].x, p[s].y);
            } else {
                // slot s holds logical 0 unless flipped: <l|Y|p> = i [conj(l1) p0 - conj(l0) p1],
                // Im(i z) = Re(z); swapping the logical roles negates the sum
                acc += (l[s1].x * p[s].x + l[s1].y * p[s].y) - (l[s].x * p[s1].x + l[s].y * p[s1].y);
            }
        }
        if (is_y && flip) acc = -acc;
    }
    return acc;
}

// U^dag of a lone RX (IS_Y false) or RY (IS_Y true) on register bit BIT, on both
// groups: U = cos(t/2) I - i sin(t/2) G, so U^dag needs c = cos(t/2) and s =
// sin(t/2) only (half the products of a general 2x2 complex matrix).  For RY the
// caller passes -s when the slot order on BIT is flipped (RX is symmetric).
template <typename C, int R, int BIT, bool IS_Y>
__device__ __forceinline__ void rot_dag2(C (&p)[1 << R], C (&l)[1 << R], typename Real<C>::T c,
                                         typename Real<C>::T s) {
    if constexpr (BIT < R) {
#pragma unroll
        for (int k = 0; k < (1 << R); ++k) {
            if ((k >> BIT) & 1) continue;
            const int k1 = k | (1 << BIT);
#pragma unroll
            for (int w = 0; w < 2; ++w) {
                C* a = w ? l : p;
                const C a0 = a[k], a1 = a[k1];
                if constexpr (!IS_Y) {   // [[c, i s], [i s, c]]
                    a[k] = cmk<C>(c * a0.x - s * a1.y, c * a0.y + s * a1.x);
                    a[k1] = cmk<C>(c * a1.x - s * a0.y, c * a1.y + s * a0.x);
                } else {                 // [[c, s], [-s, c]]
                    a[k] = cmk<C>(c * a0.x + s * a1.x, c * a0.y + s * a1.y);
                    a[k1] = cmk<C>(c * a1.x - s * a0.x, c * a1.y - s * a0.y);
                }
            }
        }
    }
}

// Gradient term of a parameterised dense op (a lone RX or RY), then its uncompute
// on both groups, under one dispatch on the op's register bit.
template <typename C, int R>
__device__ __forceinline__ typename Real<C>::T grad_apply_xy(const DevOp& op, C (&p)[1 << R], C (&l)[1 << R],
                                                            const C* __restrict__ M, int tau) {
    using T = typename Real<C>::T;
    T acc = 0;
    const int bit = __ffs(op.mask) - 1;
    const int flip = (tau >> bit) & 1;
    const bool is_y = op.grad == G_Y;
    // the op's matrix: RX [[c, -i s], [-i s, c]], RY [[c, -s], [s, c]] (row-major)
    const T c = M[0].x;
    const T s = is_y ? (flip ? -M[2].x : M[2].x) : -M[1].y;
    switch (bit) {
#define TCNG_GA(B)                                              \
    case B:                                                     \
        if (is_y) {                                             \
            acc = grad_xy<C, R, B, true>(p, l, flip);           \
            rot_dag2<C, R, B, true>(p, l, c, s);                \
        } else {                                                \
            acc = grad_xy<C, R, B, false>(p, l, flip);          \
            rot_dag2<C, R, B, false>(p, l, c, s);               \
        }                                                       \
        break;
        TCNG_GA(0) TCNG_GA(1) TCNG_GA(2) TCNG_GA(3)
#undef TCNG_GA
    default:
        if (is_y) {
            acc = grad_xy<C, R, 4, true>(p, l, flip);
            rot_dag2<C, R, 4, true>(p, l, c, s);
        } else {
            acc = grad_xy<C, R, 4, false>(p, l, flip);
            rot_dag2<C, R, 4, false>(p, l, c, s);
        }
        break;
    }
    return acc;
}

// Gradient contribution Im<lambda|G|psi> of one group for a parameterised
// diagonal op (generator Z, ZZ or the |11><11| projector), from the op's
// phase-table index of every slot.
template <typename C, int R>
__device__ __forceinline__ typename Real<C>::T grad_part_diag(const DevOp& op, const C (&p)[1 << R],
                                                             const C (&l)[1 << R], const int (&idx)[1 << R]) {
    using T = typename Real<C>::T;
    T acc = 0;
#pragma unroll
    for (int s = 0; s < (1 << R); ++s) {
        const int b = idx[s];   // bit j = value of source j (ascending qubits)
        T w;
        if (op.grad == G_Z) w = (b & 1) ? T(-1) : T(1);
        else if (op.grad == G_ZZ) w = (__popc(b & 3) & 1) ? T(-1) : T(1);
        else w = (b == 3) ? T(1) : T(0);
        acc += w * im_conj_mul(l[s].x, l[s].y, p[s].x, p[s].y);
    }
    return acc;
}

// Reverse stage over one tile: ops in reverse order, gradient before uncompute.
// red[w][j] accumulates warp w's share of the stage's j-th gradient op.
template <typename C, int R>
__device__ void run_stage_adjoint(C* __restrict__ pbuf, C* __restrict__ lbuf, const DevStage& st,
                                  const DevOp* __restrict__ ops, const C* __restrict__ mats,
                                  int tile_bits, long long gbase, typename Real<C>::T* red,
                                  int* __restrict__ gslot) {
    using T = typename Real<C>::T;
    const int ngroups = 1 << (tile_bits - R);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int g0 = 0; g0 < ngroups; g0 += blockDim.x) {
        const int g = g0 + threadIdx.x;
        const bool active = g < ngroups;
        C p[1 << R], l[1 << R];
        const int tau = st.rotate ? (g & ((1 << R) - 1)) : 0;
        int L0 = 0;   // slot 0's offset (the diagonal ops' index); the others are recomputed for the store
        if (active) {
            int L[1 << R];
            group_offsets<R>(g, tau, st.rbit, L);
#pragma unroll
            for (int s = 0; s < (1 << R); ++s) {
                p[s] = pbuf[L[s]];
                l[s] = lbuf[L[s]];
            }
            L0 = L[0];
        } else {
#pragma unroll
            for (int s = 0; s < (1 << R); ++s) {
                p[s] = cmk<C>(0, 0);
                l[s] = cmk<C>(0, 0);
            }
        }
        // per op: one dispatch and one decode (matrix, or diagonal slot indices)
        // serve the gradient term and the uncompute of both states
        int j = 0;
        for (int i = (int)st.op_count - 1; i >= 0; --i) {
            const DevOp op = ops[st.op_begin + i];
            const C* M = mats + op.mat;
            if (op.kind == K_DENSE) {
                if (op.grad != G_NONE) {
                    T v = active ? grad_apply_xy<C, R>(op, p, l, M, tau) : T(0);
                    const T w = warp_sum(v);
                    if (lane == 0) red[warp * kMaxStageGrads + j] += w;
                    if (threadIdx.x == 0) gslot[j] = op.slot;   // the fold's accumulator slot
                    ++j;
                } else if (active) {
                    dense_dispatch2<C, R, true>(op.mask, p, l, M, tau);
                }
            } else if (op.grad == G_Z || op.grad == G_ZZ) {
                // lone RZ / RZZ: the generator's sign is the slot's source parity, and the
                // uncompute takes M[0] or M[1] by the same parity (no phase-table reads)
                const uint32_t odd = zpar_mask<R>(op, L0, gbase);
                T v = 0;
                if (active) {
#pragma unroll
                    for (int s = 0; s < (1 << R); ++s) {
                        const T w = im_conj_mul(l[s].x, l[s].y, p[s].x, p[s].y);
                        v += ((odd >> s) & 1u) ? -w : w;
                    }
                }
                const T w = warp_sum(v);
                if (lane == 0) red[warp * kMaxStageGrads + j] += w;
                if (threadIdx.x == 0) gslot[j] = op.slot;   // the fold's accumulator slot
                ++j;
                if (active) {
                    const C m0 = M[0], m1 = M[1];
                    zpar_apply<C, R, true>(p, odd, m0, m1);
                    zpar_apply<C, R, true>(l, odd, m0, m1);
                }
            } else if (op.grad == G_P11) {
                // lone controlled phase: generator |11><11| (weight 1 on the slots with both
                // sources set), uncompute by M[0] or M[3] on the same slots
                const uint32_t both = p11_mask<R>(op, L0, gbase);
                T v = 0;
                if (active) {
#pragma unroll
                    for (int s = 0; s < (1 << R); ++s)
                        if ((both >> s) & 1u) v += im_conj_mul(l[s].x, l[s].y, p[s].x, p[s].y);
                }
                const T w = warp_sum(v);
                if (lane == 0) red[warp * kMaxStageGrads + j] += w;
                if (threadIdx.x == 0) gslot[j] = op.slot;   // the fold's accumulator slot
                ++j;
                if (active) {
                    const C m0 = M[0], m1 = M[3];
                    zpar_apply<C, R, true>(p, both, m0, m1);
                    zpar_apply<C, R, true>(l, both, m0, m1);
                }
            } else {
                int idx[1 << R];
                diag_index0<R>(op, L0, gbase, idx);
                if (op.grad != G_NONE) {
                    T v = active ? grad_part_diag<C, R>(op, p, l, idx) : T(0);
                    const T w = warp_sum(v);
                    if (lane == 0) red[warp * kMaxStageGrads + j] += w;
                    if (threadIdx.x == 0) gslot[j] = op.slot;   // the fold's accumulator slot
                    ++j;
                }
                if (active) diag_apply2<C, R, true>(p, l, M, idx);
            }
        }
        if (active) {
            int L[1 << R];
            group_offsets<R>(g, tau, st.rbit, L);
#pragma unroll
            for (int s = 0; s < (1 << R); ++s) {
                pbuf[L[s]] = p[s];
                lbuf[L[s]] = l[s];
            }
        }
    }
}


// ---------------------------------------------------------- tile movement --
// Synchronous copy of one tile (chunks of 2^chunk amplitudes) between global
// and shared memory for up to two states; warp 0 issues the copies.
template <typename C>
__device__ bool tile_load(const DevPass& p, long long tile, C* const* gptr, C* const* sbuf, int nst,
                          uint64_t* bar, uint32_t* phase, unsigned* err) {
    const int lane = threadIdx.x & 31;
    if (threadIdx.x < 32) {
        const long long base = tile_global_base(p, tile);
        const uint32_t chunk_bytes = (uint32_t)(sizeof(C) << p.chunk);
        const int nchunks = 1 << p.ngather;
        if (lane == 0) mbar_arrive_expect_tx(bar, (uint32_t)(nst * (sizeof(C) << p.m)));
        __syncwarp();
        for (int s = 0; s < nst; ++s)
            for (int j = lane; j < nchunks; j += 32)
                bulk_g2s(sbuf[s] + ((long long)j << p.chunk), gptr[s] + base + chunk_offset(p, j),
                         chunk_bytes, bar);
    }
    const bool ok = mbar_wait_bounded(bar, *phase, err);
    *phase ^= 1u;
    return ok;
}

// Issue (warp 0) the copy of one tile of one state into sbuf; completion on bar.
template <typename C>
__device__ void tile_load_issue(const DevPass& p, long long tile, const C* gptr, C* sbuf, uint64_t* bar) {
    const int lane = threadIdx.x & 31;
    if (threadIdx.x < 32) {
        const long long base = tile_global_base(p, tile);
        const uint32_t chunk_bytes = (uint32_t)(sizeof(C) << p.chunk);
        const int nchunks = 1 << p.ngather;
        if (lane == 0) mbar_arrive_expect_tx(bar, (uint32_t)(sizeof(C) << p.m));
        __syncwarp();
        for (int j = lane; j < nchunks; j += 32)
            bulk_g2s(sbuf + ((long long)j << p.chunk), gptr + base + chunk_offset(p, j), chunk_bytes, bar);
    }
}

__device__ __forceinline__ void fence_proxy_async_all() {
    asm volatile("fence.proxy.async;" ::: "memory");
}

template <typename C>
__device__ void tile_store(const DevPass& p, long long tile, C* const* gptr, C* const* sbuf, int nst,
                           bool wait_read = true) {
    fence_proxy_async_smem();
    __syncthreads();
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x & 31;
        const long long base = tile_global_base(p, tile);
        const uint32_t chunk_bytes = (uint32_t)(sizeof(C) << p.chunk);
        const int nchunks = 1 << p.ngather;
        for (int s = 0; s < nst; ++s)
            for (int j = lane; j < nchunks; j += 32)
                bulk_s2g(gptr[s] + base + chunk_offset(p, j), sbuf[s] + ((long long)j << p.chunk),
                         chunk_bytes);
        bulk_commit();
        if (wait_read) bulk_wait_read<0>();   // the buffer may be refilled; the writes complete by the pass's end
    }
    __syncthreads();
}

// End of a streamed pass: this pass's tile stores complete (and ordered before
// later reads of the state) before the next pass or phase reads it.
__device__ __forceinline__ void pass_stores_done() {
    if (threadIdx.x < 32) {
        bulk_wait<0>();
        fence_proxy_async_all();
    }
}

// ------------------------------------------------------------------ kernel --
// complex64: 512 threads, one per register group of a 2^13 tile (128 registers);
// complex128 keeps 256 threads (its FP64 stages spill heavily at 128 registers).
template <typename C>
constexpr int adjoint_threads() { return sizeof(C) == 8 ? 512 : 256; }

template <typename C>
__global__ void __launch_bounds__(adjoint_threads<C>(), 1) adjoint_kernel(AdjArgs a) {
    using T = typename Real<C>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int tid = threadIdx.x;
    const int nthreads = blockDim.x;
    const int nwarps = nthreads >> 5;
    // layout: [psi tile | lam tile] (2 * 2^mres) | mats window | gacc | red (2 buffers) | gslot (2) | bar
    const int res_elems = 1 << a.res_bits;
    C* sp = reinterpret_cast<C*>(smem_raw);
    C* sl = sp + res_elems;
    C* mats = sl + res_elems;
    double* gacc = reinterpret_cast<double*>(mats + kMaxPassMat);
    T* red = reinterpret_cast<T*>(gacc + kMaxGradSlots);
    int* gslot2 = reinterpret_cast<int*>(red + 2 * 32 * kMaxStageGrads);   // 2 x kMaxStageGrads
    uint64_t* bar = reinterpret_cast<uint64_t*>(gslot2 + 2 * kMaxStageGrads);
    __shared__ int s_item;
    __shared__ double s_red[32];
    __shared__ int s_abort;
    uint32_t phase = 0;
    if (tid == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
        s_abort = 0;
    }
    __syncthreads();
    C* scratch_p = reinterpret_cast<C*>(a.scratch) + (long long)blockIdx.x * 2 * a.scratch_elems;
    C* scratch_l = scratch_p + a.scratch_elems;
    for (;;) {
        if (tid == 0) s_item = atomicAdd(a.counter, 1);
        __syncthreads();
        const int idx = s_item;
        if (idx >= a.batch || s_abort) break;
        const ItemDesc it = a.items[a.order[idx]];
        const StructDesc S = a.structs[it.s];
        const C* table = reinterpret_cast<const C*>(a.tables) + it.table_off;
        const double* coeff = a.coeffs ? a.coeffs + it.coeff_off : S.tcoef;
        const bool resident = S.resident != 0;
        const int n = S.n_eff;
        const long long N = 1ll << n;
        C* gp = resident ? nullptr : scratch_p;
        C* gl = resident ? nullptr : scratch_l;
        // ---------------- forward: psi = U |0> ----------------
        // Streamed states: the first pass makes its tiles of |0...0> in shared memory
        // (the scratch state is first written by that pass), and the tiles of a pass
        // alternate between the two buffers (lambda's is free here), so the copy of
        // tile t + 1 runs while tile t is computed.
        if (resident) {
            for (long long x = tid; x < N; x += nthreads) sp[x] = cmk<C>(x == 0 ? 1 : 0, 0);
        } else if (S.n_passes == 0) {
            for (long long x = tid; x < N; x += nthreads) gp[x] = cmk<C>(x == 0 ? 1 : 0, 0);
        }
        for (int g = tid; g < S.n_grad; g += nthreads) gacc[g] = 0.0;
        fence_proxy_async_all();   // generic writes of psi before bulk copies read it
        __syncthreads();
        for (int pi = 0; pi < S.n_passes && !s_abort; ++pi) {
            const DevPass P = S.passes[pi];
            for (int i = tid; i < P.mat_count; i += nthreads) mats[i] = table[P.mat_begin + i];
            __syncthreads();
            const long long ntiles = resident ? 1 : (1ll << (n - P.m));
            const bool make = pi == 0;   // streamed: the first pass's tiles are made, not loaded
            if (!resident && !make) tile_load_issue<C>(P, 0, gp, sp, bar);
            for (long long t = 0; t < ntiles; ++t) {
                C* cur = (!resident && (t & 1)) ? sl : sp;
                if (!resident) {
                    if (make) {
                        if (t >= 2) {   // tile t - 2's store (the older of two in flight) has read cur
                            if (tid < 32) bulk_wait_read<1>();
                            __syncthreads();
                        }
                        const long long tn = 1ll << P.m;
                        for (long long x = tid; x < tn; x += nthreads)
                            cur[x] = cmk<C>(t == 0 && x == 0 ? 1 : 0, 0);
                    } else {
                        if (!mbar_wait_bounded(bar, phase, a.err)) s_abort = 1;
                        phase ^= 1u;
                    }
                    __syncthreads();
                    if (s_abort) break;
                    if (!make && t + 1 < ntiles) {   // the other buffer, once tile t - 1's store has read it
                        if (tid < 32) bulk_wait_read<0>();
                        tile_load_issue<C>(P, t + 1, gp, (t & 1) ? sp : sl, bar);
                    }
                }
                const long long gbase = resident ? 0 : tile_global_base(P, t);
                for (int si = 0; si < P.stage_count; ++si) {
                    const DevStage st = S.stages[P.stage_begin + si];
                    run_stage<C>(cur, st, S.dops, mats, P.m, gbase);
                    __syncthreads();
                }
                if (!resident) {
                    C* gptr[1] = {gp};
                    C* sb[1] = {cur};
                    tile_store<C>(P, t, gptr, sb, 1, false);
                }
            }
            if (!resident) pass_stores_done();
            __syncthreads();
        }
        if (s_abort) break;
        const C* psi = resident ? sp : gp;
        C* lam = resident ? sl : gl;
        // optional copy of the forward state to the caller's state buffer
        if (it.psi_out_off >= 0) {
            C* out = reinterpret_cast<C*>(a.psi_out) + it.psi_out_off;
            const long long Nn = 1ll << S.n;
            for (long long x = tid; x < Nn; x += nthreads) out[x] = psi[x];
        }
        // ---------------- lambda = H psi, E = Re <psi|lambda> ----------------
        // Resident: psi is in shared memory.  Streamed: psi is read tile by tile
        // (2^res_bits contiguous amplitudes) into shared memory; partners
        // outside the tile come from global memory.
        double e_part = 0.0;
        {
            const int tb = resident ? n : a.res_bits;
            const long long tn = 1ll << tb;
            const long long ntile = resident ? 1 : (N >> tb);
            for (long long t = 0; t < ntile; ++t) {
                if (!resident) {
                    if (tid == 0) {
                        mbar_arrive_expect_tx(bar, (uint32_t)(sizeof(C) * tn));
                        bulk_g2s(sp, gp + t * tn, (uint32_t)(sizeof(C) * tn), bar);
                    }
                    if (!mbar_wait_bounded(bar, phase, a.err)) s_abort = 1;
                    phase ^= 1u;
                    __syncthreads();
                    if (s_abort) break;
                }
                for (long long xl = tid; xl < tn; xl += nthreads) {
                    const long long x = t * tn + xl;
                    T ar = 0, ai = 0;
                    for (int q = 0; q < S.n_terms; ++q) {
                        const HTerm h = S.terms[q];
                        const long long y = x ^ (long long)h.xm;
                        const C v = ((y >> tb) == t) ? sp[y & (tn - 1)] : psi[y];
                        const T c = (T)coeff[q];
                        const int sg = __popcll((unsigned long long)y & h.zm) & 1;
                        T vr = v.x, vi = v.y, tr;
                        switch (h.ny & 3) {
                        case 1: tr = -vi; vi = vr; vr = tr; break;
                        case 2: vr = -vr; vi = -vi; break;
                        case 3: tr = vi; vi = -vr; vr = tr; break;
                        default: break;
                        }
                        if (sg) { vr = -vr; vi = -vi; }
                        ar += c * vr;
                        ai += c * vi;
                    }
                    lam[x] = cmk<C>(ar, ai);
                    const C p = sp[xl];
                    e_part += (double)(p.x * ar + p.y * ai);
                }
                __syncthreads();   // tile buffer reused by the next load
            }
        }
        if (s_abort) break;
        fence_proxy_async_all();   // generic writes of lambda before bulk copies read it
        {
            double v = warp_sum(e_part);
            if ((tid & 31) == 0) s_red[tid >> 5] = v;
            __syncthreads();
            if (tid == 0) {
                double e = 0;
                for (int w = 0; w < nwarps; ++w) e += s_red[w];
                a.energy[a.order[idx]] = e;
            }
            __syncthreads();
        }
        // ---------------- reverse sweep ----------------
        if (a.want_grad) {
            for (int i = tid; i < 2 * 32 * kMaxStageGrads; i += nthreads) red[i] = T(0);
            __syncthreads();
            for (int pi = S.n_passes - 1; pi >= 0 && !s_abort; --pi) {
                const DevPass P = S.passes[pi];
                for (int i = tid; i < P.mat_count; i += nthreads) mats[i] = table[P.mat_begin + i];
                __syncthreads();
                const long long ntiles = resident ? 1 : (1ll << (n - P.m));
                C* tp = sp;
                C* tl = sl;
                for (long long t = 0; t < ntiles; ++t) {
                    if (!resident) {
                        C* gptr[2] = {gp, gl};
                        C* sb[2] = {tp, tl};
                        if (!tile_load<C>(P, t, gptr, sb, 2, bar, &phase, a.err)) s_abort = 1;
                        __syncthreads();
                        if (s_abort) break;
                    }
                    const long long gbase = resident ? 0 : tile_global_base(P, t);
                    for (int si = P.stage_count - 1; si >= 0; --si) {
                        const DevStage st = S.stages[P.stage_begin + si];
                        // two partial-sum buffers taken in turn by consecutive stages: a stage's
                        // fold reads and clears its buffer while the next stage fills the other,
                        // so one barrier per stage orders both (they are all zero here: cleared
                        // before the sweep, then by each fold)
                        T* rs = red + (si & 1) * (32 * kMaxStageGrads);
                        int* gs = gslot2 + (si & 1) * kMaxStageGrads;   // slot of the stage's j-th gradient op
                        if (st.nreg > kRegBits) {   // 5-qubit constant block: no gradient ops here
                            run_stage_smem<C, true>(tp, st, S.dops, mats, P.m, gbase);
                            run_stage_smem<C, true>(tl, st, S.dops, mats, P.m, gbase);
                        } else {
                            run_stage_adjoint<C, kRegBits>(tp, tl, st, S.dops, mats, P.m, gbase, rs, gs);
                        }
                        __syncthreads();
                        // fold this stage's gradient partials (fixed order) into gacc
                        if (tid < (int)st.n_grad) {
                            const int slot = gs[tid];
                            double s = 0;
                            for (int w = 0; w < nwarps; ++w) {
                                s += rs[w * kMaxStageGrads + tid];
                                rs[w * kMaxStageGrads + tid] = T(0);
                            }
                            gacc[slot] += s;
                        }
                    }
                    __syncthreads();
                    if (!resident) {
                        C* gptr[2] = {gp, gl};
                        C* sb[2] = {tp, tl};
                        tile_store<C>(P, t, gptr, sb, 2);
                    }
                }
                if (!resident) pass_stores_done();
                __syncthreads();
            }
            if (s_abort) break;
            // ---------------- gradient output ----------------
            double* grad = a.grad + it.grad_off;
            for (int q = tid; q < S.P; q += nthreads) grad[q] = 0.0;
            __syncthreads();
            if (tid == 0)
                for (int g = 0; g < S.n_grad; ++g) grad[S.gparam[g]] += S.gscale[g] * gacc[g];
        }
        __syncthreads();
    }
}

template <typename C>
size_t adjoint_smem_bytes(int res_bits) {
    return 2 * (sizeof(C) << res_bits) + sizeof(C) * kMaxPassMat + sizeof(double) * kMaxGradSlots +
           sizeof(typename Real<C>::T) * 2 * 32 * kMaxStageGrads + sizeof(int) * 2 * kMaxStageGrads + 16;
}

template <typename C>
cudaError_t launch_adjoint(const AdjArgs& a, int grid, cudaStream_t s) {
    const size_t smem = adjoint_smem_bytes<C>(a.res_bits);
    auto kern = adjoint_kernel<C>;
    // set once per device (the call is not legal inside every stream capture)
    static size_t set_bytes[kMaxDeviceSlots] = {};
    const int d = device_slot();
    if (set_bytes[d] < smem) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        set_bytes[d] = smem;
    }
    kern<<<grid, adjoint_threads<C>(), smem, s>>>(a);
    count_launch();
    return cudaGetLastError();
}

template cudaError_t launch_adjoint<float2>(const AdjArgs&, int, cudaStream_t);
template cudaError_t launch_adjoint<double2>(const AdjArgs&, int, cudaStream_t);
template size_t adjoint_smem_bytes<float2>(int);
template size_t adjoint_smem_bytes<double2>(int);

}  // namespace tcng
