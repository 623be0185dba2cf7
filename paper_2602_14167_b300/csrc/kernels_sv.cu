// State-vector kernels for sm_103a: matrix-builder prologue, state init,
// per-gate pair/quartet updates, pipelined tile passes, Pauli expectations,
// and H|psi>.
//
// What is computed follows the paper's circuit statement (Sec. I.B
// "Primitives": gates are local contractions on the state; expectation_ps of
// Pauli strings; the TFIM energy).  How: in-place updates of a 2^n amplitude
// vector streamed through shared memory with bulk asynchronous copies (TMA
// engine) and mbarrier completion.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <type_traits>

#include "device.cuh"
#include "gates.cuh"
#include "launch.hpp"
#include "tile_io.cuh"

namespace tcng {

// ============================================================ prologue ==

// Build every block matrix of every item from the parameters, in the block's
// ascending local order.  One CTA per (block, item); thread c builds column c.
template <typename C>
__global__ void build_matrices_kernel(const BuildBlock* __restrict__ blocks,
                                      const BuildOp* __restrict__ bops,
                                      const double2* __restrict__ pool,
                                      const double* __restrict__ params, int P,
                                      C* __restrict__ table, long long table_stride,
                                      int item_base, const long long* __restrict__ prm_off,
                                      const long long* __restrict__ tab_off, long long pool_stride) {
    const int bi = blockIdx.x;
    const int item = blockIdx.y + item_base;
    pool += (long long)item * pool_stride;   // per-item explicit matrices (0: shared pool)
    const BuildBlock blk = blocks[bi];
    const int D = 1 << blk.k;
    const double* th = params ? params + (prm_off ? prm_off[item] : (long long)item * P) : nullptr;
    __shared__ double2 opm[1024];
    double2 col[32];
    const int c = threadIdx.x;
    for (int r = 0; r < D; ++r) col[r] = make_double2(r == c ? 1.0 : 0.0, 0.0);
    for (int oi = 0; oi < blk.op_count; ++oi) {
        const BuildOp op = bops[blk.op_begin + oi];
        const int ko = op.k, dk = 1 << ko;
        double ang = op.angle0;
        if (op.param >= 0) ang += op.scale * th[op.param];
        __syncthreads();
        if (threadIdx.x == 0) gate_matrix_d(op, ang, opm, dk, pool);
        __syncthreads();
        if (c < D) {
            int qm = 0;
            for (int j = 0; j < ko; ++j) qm |= 1 << op.pos[j];
            for (int x = 0; x < D; ++x) {
                if (x & qm) continue;
                double2 v[32], w[32];
                int idx[32];
                for (int r = 0; r < dk; ++r) {
                    int y = x;
                    for (int j = 0; j < ko; ++j)
                        if ((r >> (ko - 1 - j)) & 1) y |= 1 << op.pos[j];
                    idx[r] = y;
                    v[r] = col[y];
                }
                for (int r = 0; r < dk; ++r) {
                    double2 acc = make_double2(0, 0);
                    for (int s = 0; s < dk; ++s) {
                        const double2 m = opm[r * dk + s];
                        acc.x += m.x * v[s].x - m.y * v[s].y;
                        acc.y += m.x * v[s].y + m.y * v[s].x;
                    }
                    w[r] = acc;
                }
                for (int r = 0; r < dk; ++r) col[idx[r]] = w[r];
            }
        }
    }
    if (c < D) {
        C* out = table + (tab_off ? tab_off[item] : (long long)item * table_stride) + blk.out_off;
        if (blk.diag) {
            out[c] = cmk<C>(col[c].x, col[c].y);
        } else {
            for (int r = 0; r < D; ++r) out[r * D + c] = cmk<C>(col[r].x, col[r].y);
        }
    }
}

// ============================================================== init ==
template <typename C>
__global__ void set_basis_kernel(C* __restrict__ state, const long long* __restrict__ item_off,
                                 int items) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < items) state[item_off[b]] = cmk<C>(1, 0);
}

// ==================================================== unfused per gate ==
// One index class per thread: gather 2^k amplitudes, multiply, scatter.
template <typename C>
__global__ void gate_dense_kernel(C* __restrict__ state, const long long* __restrict__ item_off,
                                  int n, int k, uint32_t qmask, const C* __restrict__ table,
                                  long long table_stride, int mat_off, long long classes) {
    const int item = blockIdx.y;
    C* psi = state + item_off[item];
    const C* M = table + (long long)item * table_stride + mat_off;
    const int D = 1 << k;
    int q[TCNG_MAX_FUSE];
    {
        int j = 0;
        for (int b = 0; b < n && j < k; ++b)
            if ((qmask >> b) & 1) q[j++] = b;
    }
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < classes;
         t += (long long)gridDim.x * blockDim.x) {
        long long x = t;
        for (int j = 0; j < k; ++j) x = ((x >> q[j]) << (q[j] + 1)) | (x & ((1ll << q[j]) - 1));
        C v[32];
        for (int s = 0; s < D; ++s) {
            long long y = x;
            for (int j = 0; j < k; ++j)
                if ((s >> j) & 1) y |= 1ll << q[j];
            v[s] = psi[y];
        }
        for (int r = 0; r < D; ++r) {
            C acc = cmk<C>(0, 0);
            for (int s = 0; s < D; ++s) cfma(acc, M[r * D + s], v[s]);
            long long y = x;
            for (int j = 0; j < k; ++j)
                if ((r >> j) & 1) y |= 1ll << q[j];
            psi[y] = acc;
        }
    }
}

// 1-qubit pair update on complex64 with 16-byte accesses: thread handles the
// two pairs (x, x+2^q) and (x+1, x+1+2^q) for even x (q >= 1).
__global__ void pair_f4_kernel(float2* __restrict__ state, const long long* __restrict__ item_off,
                               int q, const float2* __restrict__ table, long long table_stride,
                               int mat_off, long long threads_per_item) {
    const int item = blockIdx.y;
    float2* psi = state + item_off[item];
    const float2* M = table + (long long)item * table_stride + mat_off;
    const float2 m00 = M[0], m01 = M[1], m10 = M[2], m11 = M[3];
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < threads_per_item;
         t += (long long)gridDim.x * blockDim.x) {
        long long x = 2 * t;
        x = ((x >> q) << (q + 1)) | (x & ((1ll << q) - 1));
        float4* p0 = reinterpret_cast<float4*>(psi + x);
        float4* p1 = reinterpret_cast<float4*>(psi + x + (1ll << q));
        const float4 a = *p0, b = *p1;
        float2 a0 = make_float2(a.x, a.y), a1 = make_float2(a.z, a.w);
        float2 b0 = make_float2(b.x, b.y), b1 = make_float2(b.z, b.w);
        float2 r0 = cmk<float2>(0, 0), r1 = r0, s0 = r0, s1 = r0;
        cfma(r0, m00, a0); cfma(r0, m01, b0);
        cfma(s0, m10, a0); cfma(s0, m11, b0);
        cfma(r1, m00, a1); cfma(r1, m01, b1);
        cfma(s1, m10, a1); cfma(s1, m11, b1);
        *p0 = make_float4(r0.x, r0.y, r1.x, r1.y);
        *p1 = make_float4(s0.x, s0.y, s1.x, s1.y);
    }
}

// 2-qubit quartet update on complex64 with 16-byte accesses (both qubits >= 1).
// Matrix local index: bit 0 = lower qubit qa, bit 1 = higher qubit qb.
__global__ void quartet_f4_kernel(float2* __restrict__ state, const long long* __restrict__ item_off,
                                  int qa, int qb, const float2* __restrict__ table,
                                  long long table_stride, int mat_off, long long threads_per_item) {
    const int item = blockIdx.y;
    float2* psi = state + item_off[item];
    const float2* M = table + (long long)item * table_stride + mat_off;
    float2 m[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) m[i] = M[i];
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < threads_per_item;
         t += (long long)gridDim.x * blockDim.x) {
        long long x = 2 * t;
        x = ((x >> qa) << (qa + 1)) | (x & ((1ll << qa) - 1));
        x = ((x >> qb) << (qb + 1)) | (x & ((1ll << qb) - 1));
        const long long off[4] = {x, x + (1ll << qa), x + (1ll << qb), x + (1ll << qa) + (1ll << qb)};
        float2 v0[4], v1[4];
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            const float4 w = *reinterpret_cast<const float4*>(psi + off[s]);
            v0[s] = make_float2(w.x, w.y);
            v1[s] = make_float2(w.z, w.w);
        }
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            float2 r0 = cmk<float2>(0, 0), r1 = r0;
#pragma unroll
            for (int s = 0; s < 4; ++s) {
                cfma(r0, m[r * 4 + s], v0[s]);
                cfma(r1, m[r * 4 + s], v1[s]);
            }
            *reinterpret_cast<float4*>(psi + off[r]) = make_float4(r0.x, r0.y, r1.x, r1.y);
        }
    }
}

// Diagonal gate: amplitude x times table[pext(x, qubits)].
template <typename C>
__global__ void gate_diag_kernel(C* __restrict__ state, const long long* __restrict__ item_off,
                                 int k, uint32_t qmask, int n, const C* __restrict__ table,
                                 long long table_stride, int mat_off, long long N) {
    const int item = blockIdx.y;
    C* psi = state + item_off[item];
    const C* M = table + (long long)item * table_stride + mat_off;
    int q[TCNG_MAX_FUSE];
    {
        int j = 0;
        for (int b = 0; b < n && j < k; ++b)
            if ((qmask >> b) & 1) q[j++] = b;
    }
    for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < N;
         x += (long long)gridDim.x * blockDim.x) {
        int idx = 0;
        for (int j = 0; j < k; ++j) idx |= int((x >> q[j]) & 1) << j;
        psi[x] = cmul(M[idx], psi[x]);
    }
}

// ========================================================= tile passes ==
// Persistent CTAs walk tiles t = blockIdx.x + i * gridDim.x over all items.
// Three shared-memory buffers: while tile i is computed, tile i+1 is in flight
// and tile i+2 is requested as soon as the store of tile i-1 has been read out.
// Warp 0 issues the tile copies (tile_io.cuh).

template <typename C>
__global__ void __launch_bounds__(512, 1) pass_kernel(C* __restrict__ state,
                                                    const long long* __restrict__ item_off,
                                                    const __grid_constant__ DevPass p,
                                                    const DevStage* __restrict__ stages,
                                                    const DevOp* __restrict__ ops,
                                                    const C* __restrict__ table,
                                                    long long table_stride, TileCtx tc,
                                                    unsigned* __restrict__ err,
                                                    const __grid_constant__ TmaTile tma) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int tile_elems = 1 << p.m;
    C* bufs = reinterpret_cast<C*>(smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u));
    C* mats = bufs + (long long)tc.nbuf * tile_elems;
    uint64_t* bars = reinterpret_cast<uint64_t*>(mats + ((p.mat_count + 1) & ~1));
    __shared__ int s_abort;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) {
        for (int i = 0; i < tc.nbuf; ++i) mbar_init(&bars[i], 1);
        fence_mbar_init();
        s_abort = 0;
    }
    __syncthreads();
    const long long first = blockIdx.x;
    const long long stride = gridDim.x;
    if (warp == 0)
        for (int i = 0; i < tc.nbuf - 1; ++i) {
            const long long t = first + i * stride;
            if (t < tc.total_tiles)
                issue_tile_load(state, item_off, p, tc, t, bufs + (long long)i * tile_elems, &bars[i], lane, tma);
        }
    long long cur_item = -1;
    int it = 0;
    for (long long t = first; t < tc.total_tiles; t += stride, ++it) {
        const int b = it % tc.nbuf;
        C* buf = bufs + (long long)b * tile_elems;
        const long long item = (t >> tc.tpi_log);
        if (item != cur_item) {  // (re)load the matrix window of this item
            const C* src = table + item * table_stride + p.mat_begin;
            for (int i = tid; i < p.mat_count; i += blockDim.x) mats[i] = src[i];
            cur_item = item;
        }
        const bool ok = mbar_wait_bounded(&bars[b], (uint32_t)((it / tc.nbuf) & 1), err);
        if (!ok) s_abort = 1;
        __syncthreads();   // also orders the matrix window reload above before the stages
        if (s_abort) break;
        const long long gbase = tile_global_base(p, (t & (tc.tiles_per_item - 1)));
        for (int s = 0; s < p.stage_count; ++s) {
            const DevStage st = stages[p.stage_begin + s];
            run_stage<C>(buf, st, ops, mats, p.m, gbase);
            __syncthreads();
        }
        fence_proxy_async_smem();
        __syncthreads();
        if (warp == 0) {
            issue_tile_store(state, item_off, p, tc, t, buf, lane, tma);
            const long long tn = t + (long long)(tc.nbuf - 1) * stride;
            if (tn < tc.total_tiles) {
                const int bn = (it + tc.nbuf - 1) % tc.nbuf;
                bulk_wait_read<1>();
                __syncwarp();
                issue_tile_load(state, item_off, p, tc, tn, bufs + (long long)bn * tile_elems, &bars[bn], lane, tma);
            }
        }
    }
    if (warp == 0) bulk_wait<0>();
}

// ==================================================== Pauli expectation ==
// One pass over the state evaluates every term whose X bits lie in the tile:
// <P> = sum_x conj(psi[x ^ m]) i^{#Y} (-1)^{popc(x & z)} psi[x] (real part).
// This is the general form (complex128, or tiles other than 2^13); complex64
// passes over 2^13-amplitude tiles use expect_fast_kernel (kernels_expect.cu).
// The tile buffers form a ring: each warp releases a buffer through an
// mbarrier, and warp 0 refills it once every warp has.
template <typename C>
__global__ void __launch_bounds__(512, 1) expect_pass_kernel(const C* __restrict__ state,
                                                          const long long* __restrict__ item_off,
                                                          const __grid_constant__ DevPass p,
                                                          const __grid_constant__ ExpPass ep,
                                                          TileCtx tc, double* __restrict__ partial,
                                                          int n_out, unsigned* __restrict__ err,
                                                          const __grid_constant__ TmaTile tma) {
    using R = typename Real<C>::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int tile_elems = 1 << p.m;
    C* bufs = reinterpret_cast<C*>(smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u));
    uint64_t* bars = reinterpret_cast<uint64_t*>(bufs + (long long)tc.nbuf * tile_elems);
    uint64_t* ebars = bars + tc.nbuf;   // buffer released by every warp
    __shared__ double red[32][kExpTermsPerPass];
    __shared__ ExpTerm sterm[kExpTermsPerPass];   // the pass's terms, read per tile
    __shared__ int s_abort;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int item = blockIdx.y;
    for (int i = tid; i < 32 * kExpTermsPerPass; i += blockDim.x) (&red[0][0])[i] = 0.0;
    if (tid < ep.nterms) sterm[tid] = ep.t[tid];
    const int nwarps = (int)(blockDim.x >> 5);
    if (tid == 0) {
        for (int i = 0; i < tc.nbuf; ++i) {
            mbar_init(&bars[i], 1);
            mbar_init(&ebars[i], (uint32_t)nwarps);
        }
        fence_mbar_init();
        s_abort = 0;
    }
    __syncthreads();
    const long long t0 = (long long)item * tc.tiles_per_item;
    const long long t1 = t0 + tc.tiles_per_item;
    const long long first = t0 + blockIdx.x;
    const long long stride = gridDim.x;
    if (warp == 0)
        for (int i = 0; i < tc.nbuf; ++i) {
            const long long t = first + i * stride;
            if (t < t1) issue_tile_load(state, item_off, p, tc, t, bufs + (long long)i * tile_elems, &bars[i], lane, tma);
        }
    double acc[kExpTermsPerPass];
#pragma unroll
    for (int j = 0; j < kExpTermsPerPass; ++j) acc[j] = 0.0;
    int it = 0;
    for (long long t = first; t < t1; t += stride, ++it) {
        const int b = it % tc.nbuf;
        const C* buf = bufs + (long long)b * tile_elems;
        // no CTA barrier per tile: every thread waits for the tile itself, and each
        // warp releases the buffer on its own (warp 0 refills it once all have)
        if (!mbar_wait_bounded(&bars[b], (uint32_t)((it / tc.nbuf) & 1), err)) s_abort = 1;
        const long long gbase = tile_global_base(p, (t & (tc.tiles_per_item - 1)));
#pragma unroll
        for (int j = 0; j < kExpTermsPerPass; ++j) {
            if (j < ep.nterms) {
                const ExpTerm& T = ep.t[j];
                const int sgn0 = __popcll((unsigned long long)gbase & T.zm_glob) & 1;
                R part = 0;
                for (int L = tid; L < tile_elems; L += blockDim.x) {
                    const C a = buf[L];
                    const C bb = buf[L ^ (int)T.xm_tile];
                    const R wr = bb.x * a.x + bb.y * a.y;   // conj(b) * a
                    const R wi = bb.x * a.y - bb.y * a.x;
                    R v;
                    switch (T.ny & 3) {
                    case 0: v = wr; break;
                    case 1: v = -wi; break;
                    case 2: v = -wr; break;
                    default: v = wi; break;
                    }
                    const int sg = (__popc((unsigned)L & T.zm_tile) + sgn0) & 1;
                    part += sg ? -v : v;
                }
                acc[j] += (double)part;
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&ebars[b]);   // this warp is done with buf
        if (warp == 0) {
            const long long tn = t + (long long)tc.nbuf * stride;
            if (tn < t1) {
                if (!mbar_wait_bounded(&ebars[b], (uint32_t)((it / tc.nbuf) & 1), err)) s_abort = 1;
                __syncwarp();
                issue_tile_load(state, item_off, p, tc, tn, bufs + (long long)b * tile_elems, &bars[b], lane, tma);
            }
        }
        if (s_abort) break;
    }
    if (s_abort && tid == 0) {   // drain loads still in flight before the shared memory goes away
        for (int i = 0; i < tc.nbuf; ++i) {
            const long long ti = first + (long long)(it + 1 + i) * stride;
            if (ti < t1) mbar_wait_bounded(&bars[(it + 1 + i) % tc.nbuf], (uint32_t)(((it + 1 + i) / tc.nbuf) & 1), err);
        }
    }
    // deterministic block reduction: warp tree, then warps in order
#pragma unroll
    for (int j = 0; j < kExpTermsPerPass; ++j) {
        double v = acc[j];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) red[warp][j] = v;
    }
    __syncthreads();
    if (tid < ep.nterms) {
        double s = 0;
        const int nw = (blockDim.x + 31) >> 5;
        for (int w = 0; w < nw; ++w) s += red[w][tid];
        // a timed-out wait leaves the sum short: report NaN rather than a wrong value
        partial[((long long)item * n_out + ep.t[tid].out) * gridDim.x + blockIdx.x] = s_abort ? __longlong_as_double(0x7ff8000000000000ll) : s;
    }
}

// out[item][t] = sum over CTAs (fixed order); optional energy = sum_t c[item][t] out[item][t]
__global__ void expect_finalize_kernel(const double* __restrict__ partial, int nblk, int n_out,
                                       double* __restrict__ out, const double* __restrict__ coeffs,
                                       const double* __restrict__ term_coeff, double* __restrict__ energy,
                                       int items, const int* __restrict__ rows) {
    const int item = blockIdx.x;
    const long long row = rows ? rows[item] : item;
    extern __shared__ double vals[];
    for (int t = threadIdx.x; t < n_out; t += blockDim.x) {
        double s = 0;
        const double* pp = partial + ((long long)item * n_out + t) * nblk;
        for (int b = 0; b < nblk; ++b) s += pp[b];
        if (out) out[row * n_out + t] = s;
        const double c = energy ? (coeffs ? coeffs[row * n_out + t] : term_coeff[t]) : 0.0;
        vals[t] = c * s;
    }
    __syncthreads();
    if (energy && threadIdx.x == 0) {
        double e = 0;
        for (int t = 0; t < n_out; ++t) e += vals[t];
        energy[row] = e;
    }
}

// ======================================================== H |psi> ==
template <typename C>
__global__ void ham_apply_kernel(const C* __restrict__ psi_all, const long long* __restrict__ off_in,
                                 C* __restrict__ out_all, const long long* __restrict__ off_out,
                                 const HTerm* __restrict__ terms, int T, const double* __restrict__ coeffs,
                                 const double* __restrict__ term_coeff, long long N, const int* __restrict__ rows) {
    using R = typename Real<C>::T;
    const int item = blockIdx.y;
    const long long row = rows ? rows[item] : item;   // the item's coefficient row
    const C* psi = psi_all + off_in[item];
    C* out = out_all + off_out[item];
    for (long long y = blockIdx.x * (long long)blockDim.x + threadIdx.x; y < N;
         y += (long long)gridDim.x * blockDim.x) {
        R ar = 0, ai = 0;
        for (int t = 0; t < T; ++t) {
            const HTerm h = terms[t];
            const long long x = y ^ (long long)h.xm;
            const C v = psi[x];
            const R c = (R)(coeffs ? coeffs[row * T + t] : term_coeff[t]);
            const int sg = __popcll((unsigned long long)x & h.zm) & 1;
            R vr = v.x, vi = v.y, tr;
            switch (h.ny & 3) {  // multiply by i^ny
            case 1: tr = -vi; vi = vr; vr = tr; break;
            case 2: vr = -vr; vi = -vi; break;
            case 3: tr = vi; vi = -vr; vr = tr; break;
            default: break;
            }
            if (sg) { vr = -vr; vi = -vi; }
            ar += c * vr;
            ai += c * vi;
        }
        out[y] = cmk<C>(ar, ai);
    }
}

// ============================================================ launchers ==
int device_slot() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) dev = 0;
    return dev < kMaxDeviceSlots ? dev : kMaxDeviceSlots - 1;
}

static int g_num_sms[kMaxDeviceSlots] = {};
int num_sms() {
    int& n = g_num_sms[device_slot()];
    if (!n) {
        int dev = 0, v = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        n = v > 0 ? v : 148;
    }
    return n;
}

template <typename C>
cudaError_t launch_build_matrices(const BuildBlock* blocks, int n_blocks, const BuildOp* bops,
                                  const double2* pool, const double* params, int P, C* table,
                                  long long table_stride, int items, cudaStream_t s, long long pool_stride) {
    if (n_blocks == 0 || items == 0) return cudaSuccess;
    for (int i0 = 0; i0 < items; i0 += 65535) {
        dim3 grid(n_blocks, std::min(65535, items - i0));
        build_matrices_kernel<C><<<grid, 32, 0, s>>>(blocks, bops, pool, params, P, table,
                                                      table_stride, i0, nullptr, nullptr, pool_stride);
        count_launch();
    }
    return cudaGetLastError();
}

template <typename C>
cudaError_t launch_build_matrices_indexed(const BuildBlock* blocks, int n_blocks, const BuildOp* bops,
                                          const double2* pool, const double* params, C* table,
                                          const long long* prm_off, const long long* tab_off,
                                          int items, cudaStream_t s) {
    if (n_blocks == 0 || items == 0) return cudaSuccess;
    for (int i0 = 0; i0 < items; i0 += 65535) {
        dim3 grid(n_blocks, std::min(65535, items - i0));
        build_matrices_kernel<C><<<grid, 32, 0, s>>>(blocks, bops, pool, params, 0, table, 0, i0,
                                                      prm_off, tab_off, 0);
        count_launch();
    }
    return cudaGetLastError();
}

template <typename C>
cudaError_t launch_set_basis(C* state, const long long* item_off, int items, cudaStream_t s) {
    set_basis_kernel<C><<<(items + 255) / 256, 256, 0, s>>>(state, item_off, items);
    count_launch();
    return cudaGetLastError();
}

static dim3 grid_for(long long work, int items, int threads) {
    long long blocks = (work + threads - 1) / threads;
    long long cap = (long long)num_sms() * 8;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    return dim3((unsigned)blocks, (unsigned)items);
}

template <typename C>
cudaError_t launch_gate(C* state, const long long* item_off, int items, int n, const Block& blk,
                        const C* table, long long table_stride, cudaStream_t s) {
    const int k = blk.k;
    const uint32_t qmask = (uint32_t)blk.qmask;
    int q[TCNG_MAX_FUSE];
    {
        int j = 0;
        for (int b = 0; b < n && j < k; ++b)
            if ((qmask >> b) & 1) q[j++] = b;
    }
    const long long N = 1ll << n;
    if (blk.diag) {
        dim3 g = grid_for(N, items, 256);
        gate_diag_kernel<C><<<g, 256, 0, s>>>(state, item_off, k, qmask, n, table, table_stride,
                                              blk.out_off, N);
    } else if (std::is_same<C, float2>::value && k == 1 && q[0] >= 1) {
        const long long th = N >> 2;
        dim3 g = grid_for(th, items, 256);
        pair_f4_kernel<<<g, 256, 0, s>>>(reinterpret_cast<float2*>(state), item_off, q[0],
                                         reinterpret_cast<const float2*>(table), table_stride,
                                         blk.out_off, th);
    } else if (std::is_same<C, float2>::value && k == 2 && q[0] >= 1) {
        const long long th = N >> 3;
        dim3 g = grid_for(th, items, 256);
        quartet_f4_kernel<<<g, 256, 0, s>>>(reinterpret_cast<float2*>(state), item_off, q[0], q[1],
                                            reinterpret_cast<const float2*>(table), table_stride,
                                            blk.out_off, th);
    } else {
        const long long classes = N >> k;
        dim3 g = grid_for(classes, items, 256);
        gate_dense_kernel<C><<<g, 256, 0, s>>>(state, item_off, n, k, qmask, table, table_stride,
                                               blk.out_off, classes);
    }
    count_launch();
    return cudaGetLastError();
}

static TileCtx make_ctx(const DevPass& p, int n, int items, int elem_bytes, int nbuf) {
    TileCtx tc{};
    tc.nbuf = nbuf;
    tc.nchunks = 1 << p.ngather;
    tc.chunk_bytes = (uint32_t)(elem_bytes << p.chunk);
    tc.tile_bytes = (uint32_t)(elem_bytes << p.m);
    tc.tiles_per_item = 1ll << (n - p.m);
    tc.tpi_log = n - p.m;
    tc.total_tiles = tc.tiles_per_item * items;
    return tc;
}

template <typename C>
static size_t pass_smem_bytes(const DevPass& p, int nbuf) {
    return 128 + (size_t)nbuf * (sizeof(C) << p.m) + sizeof(C) * ((p.mat_count + 1) & ~1) +
           8 * (size_t)nbuf;
}

// Largest dynamic shared memory a kernel may request: the device opt-in limit
// minus the kernel's static shared memory.  Sets the attribute once.
template <typename K>
static size_t dyn_smem_limit(K kernel, bool* done, size_t* cached) {
    if (!*done) {
        int dev = 0, optin = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        cudaFuncAttributes fa{};
        cudaFuncGetAttributes(&fa, kernel);
        size_t lim = optin > (int)fa.sharedSizeBytes ? (size_t)optin - fa.sharedSizeBytes : 0;
        if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lim) !=
            cudaSuccess) {
            cudaGetLastError();
            lim = 48 * 1024 - fa.sharedSizeBytes;
        }
        *cached = lim;
        *done = true;
    }
    return *cached;
}

template <typename C>
cudaError_t launch_pass(C* state, const long long* item_off, int items, int n, const DevPass& p,
                        const DevStage* host_stages, const DevStage* stages, const DevOp* ops,
                        const C* table, long long table_stride, unsigned* err, cudaStream_t s,
                        const TmaTile* tma) {
    const int nbuf = 3;
    const size_t smem = pass_smem_bytes<C>(p, nbuf);
    (void)host_stages;
    auto kern = pass_kernel<C>;
    static bool done[kMaxDeviceSlots] = {};
    static size_t lim[kMaxDeviceSlots] = {};
    const int d = device_slot();
    if (smem > dyn_smem_limit(kern, &done[d], &lim[d])) return cudaErrorInvalidConfiguration;
    TileCtx tc = make_ctx(p, n, items, sizeof(C), nbuf);
    const int threads = std::max(32, (1 << p.m) >> kRegBits);
    int per_sm = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
    if (per_sm < 1) per_sm = 1;
    long long grid = std::min<long long>(tc.total_tiles, (long long)num_sms() * per_sm);
    const TmaTile t0{};
    kern<<<(unsigned)grid, threads, smem, s>>>(state, item_off, p, stages, ops, table, table_stride,
                                               tc, err, tma ? *tma : t0);
    count_launch();
    return cudaGetLastError();
}

template <typename C>
cudaError_t launch_expect_pass(const C* state, const long long* item_off, int items, int n,
                               const DevPass& p, const ExpPass& ep, double* partial, int n_out,
                               int nblk, unsigned* err, cudaStream_t s, const TmaTile* tma) {
    const int nbuf = 3;
    const size_t smem = 128 + (size_t)nbuf * (sizeof(C) << p.m) + 16 * nbuf;
    TileCtx tc = make_ctx(p, n, items, sizeof(C), nbuf);
    dim3 grid((unsigned)nblk, (unsigned)items);
    const TmaTile t0{};
    if constexpr (std::is_same<C, float2>::value) {   // complex64, 2^13 tiles: kernels_expect.cu
        if (p.m == 13)
            return launch_expect_fast(state, item_off, items, p, ep, tc, partial, n_out, nblk, err, s,
                                      tma ? *tma : t0);
    }
    {
        auto kern = expect_pass_kernel<C>;
        static bool done[kMaxDeviceSlots] = {};
        static size_t lim[kMaxDeviceSlots] = {};
        const int d = device_slot();
        if (smem > dyn_smem_limit(kern, &done[d], &lim[d])) return cudaErrorInvalidConfiguration;
        const int threads = std::min(512, std::max(32, 1 << p.m));
        kern<<<grid, threads, smem, s>>>(state, item_off, p, ep, tc, partial, n_out, err, tma ? *tma : t0);
    }
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_expect_finalize(const double* partial, int nblk, int n_out, double* out,
                                   const double* coeffs, const double* term_coeff, double* energy,
                                   int items, cudaStream_t s, const int* rows) {
    expect_finalize_kernel<<<items, 256, sizeof(double) * n_out, s>>>(partial, nblk, n_out, out,
                                                                      coeffs, term_coeff, energy, items, rows);
    count_launch();
    return cudaGetLastError();
}

template <typename C>
cudaError_t launch_ham_apply(const C* psi, const long long* off_in, C* out, const long long* off_out,
                             int items, int n, const HTerm* terms, int T, const double* coeffs,
                             const double* term_coeff, cudaStream_t s,
                             const int* rows) {
    const long long N = 1ll << n;
    dim3 g = grid_for(N, items, 256);
    ham_apply_kernel<C><<<g, 256, 0, s>>>(psi, off_in, out, off_out, terms, T, coeffs, term_coeff, N, rows);
    count_launch();
    return cudaGetLastError();
}

#define TCNG_INST(C)                                                                                  \
    template cudaError_t launch_build_matrices<C>(const BuildBlock*, int, const BuildOp*,             \
                                                  const double2*, const double*, int, C*, long long,  \
                                                  int, cudaStream_t, long long);                      \
    template cudaError_t launch_set_basis<C>(C*, const long long*, int, cudaStream_t);                \
    template cudaError_t launch_build_matrices_indexed<C>(const BuildBlock*, int, const BuildOp*,     \
                                                          const double2*, const double*, C*,          \
                                                          const long long*, const long long*, int,    \
                                                          cudaStream_t);                              \
    template cudaError_t launch_gate<C>(C*, const long long*, int, int, const Block&, const C*,       \
                                        long long, cudaStream_t);                                     \
    template cudaError_t launch_pass<C>(C*, const long long*, int, int, const DevPass&,               \
                                        const DevStage*, const DevStage*, const DevOp*, const C*,     \
                                        long long, unsigned*, cudaStream_t, const TmaTile*);          \
    template cudaError_t launch_expect_pass<C>(const C*, const long long*, int, int, const DevPass&,  \
                                               const ExpPass&, double*, int, int, unsigned*,          \
                                               cudaStream_t, const TmaTile*);                         \
    template cudaError_t launch_ham_apply<C>(const C*, const long long*, C*, const long long*, int,   \
                                             int, const HTerm*, int, const double*, const double*,    \
                                             cudaStream_t, const int*);
TCNG_INST(float2)
TCNG_INST(double2)

}  // namespace tcng
