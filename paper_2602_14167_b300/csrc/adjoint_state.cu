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
// ops, in the block's ascending-qubit local order) one pass over both states:
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
// Per block: 2 states read and written once (HBM-bound, 4 x state bytes);
// per-thread N partials in FP32, every 64 classes summed over the warp by a
// fixed shuffle tree into the warp's FP64 sums in shared memory (105 registers
// for complex64 with two qubits: two CTAs per SM), then a fixed-order reduction
// over warps and CTAs (bitwise reproducible).  The forward runs on the
// ordinary tile passes; lambda = H psi on the Pauli-sum kernel.
#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <stdexcept>
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

// One reverse block step over all 2^(n-K) index classes (grid-stride).
template <typename C, int K, bool GRAD>
__global__ void __launch_bounds__(kSaThreads) sa_block_kernel(C* __restrict__ psi, C* __restrict__ lam,
                                                              const C* __restrict__ U, int diag,
                                                              unsigned long long qmask, int n,
                                                              double* __restrict__ npart) {
    using R = typename Real<C>::T;
    constexpr int D = 1 << K;
    __shared__ C su[D * D];
    for (int i = threadIdx.x; i < (diag ? D : D * D); i += blockDim.x) su[i] = U[i];
    __syncthreads();
    const unsigned long long all = (n >= 64) ? ~0ull : ((1ull << n) - 1);
    const unsigned long long fm = all & ~qmask;
    long long off[D];
#pragma unroll
    for (int l = 0; l < D; ++l) off[l] = (long long)sa_pdep((unsigned long long)l, qmask);
    const long long classes = 1ll << (n - K);
    const long long stride = (long long)gridDim.x * blockDim.x;
    long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long x0 = sa_pdep((unsigned long long)j, fm);
    const unsigned long long step = sa_pdep((unsigned long long)stride, fm);
    // N partials: per thread in FP32, every 64 classes summed over the warp (fixed
    // shuffle tree) into the warp's FP64 sums in shared memory (few registers, so
    // more warps per SM hide the streaming latency)
    R nacc[GRAD ? 2 * D * D : 1];
    __shared__ double wacc[kSaThreads / 32][2 * 16];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (GRAD) {
#pragma unroll
        for (int i = 0; i < 2 * D * D; ++i) nacc[i] = 0;
        if (lane < 2 * D * D) wacc[warp][lane] = 0.0;
    }
    auto fold = [&]() {
#pragma unroll
        for (int i = 0; i < 2 * D * D; ++i) {
            R v = nacc[i];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) wacc[warp][i] += (double)v;
            nacc[i] = 0;
        }
    };
    int cnt = 0;
    for (; j < classes; j += stride) {
        C a[D], b[D], y[D], z[D];
#pragma unroll
        for (int l = 0; l < D; ++l) {
            a[l] = psi[x0 | off[l]];
            b[l] = lam[x0 | off[l]];
        }
        if (diag) {
#pragma unroll
            for (int l = 0; l < D; ++l) {   // conj(u) * v
                const C u = su[l];
                y[l] = cmk<C>(u.x * a[l].x + u.y * a[l].y, u.x * a[l].y - u.y * a[l].x);
                z[l] = cmk<C>(u.x * b[l].x + u.y * b[l].y, u.x * b[l].y - u.y * b[l].x);
            }
        } else {
#pragma unroll
            for (int l = 0; l < D; ++l) {   // y_l = sum_m conj(U[m][l]) a_m
                R yr = 0, yi = 0, zr = 0, zi = 0;
#pragma unroll
                for (int m = 0; m < D; ++m) {
                    const C u = su[m * D + l];
                    yr += u.x * a[m].x + u.y * a[m].y;
                    yi += u.x * a[m].y - u.y * a[m].x;
                    zr += u.x * b[m].x + u.y * b[m].y;
                    zi += u.x * b[m].y - u.y * b[m].x;
                }
                y[l] = cmk<C>(yr, yi);
                z[l] = cmk<C>(zr, zi);
            }
        }
        if (GRAD) {   // N[l][m] += psi_in(l) conj(lambda_out(m))
#pragma unroll
            for (int l = 0; l < D; ++l)
#pragma unroll
                for (int m = 0; m < D; ++m) {
                    nacc[2 * (l * D + m)] += y[l].x * b[m].x + y[l].y * b[m].y;
                    nacc[2 * (l * D + m) + 1] += y[l].y * b[m].x - y[l].x * b[m].y;
                }
            if (++cnt == 64) {   // warp-uniform: every lane of a warp runs the same number of classes
                fold();
                cnt = 0;
            }
        }
#pragma unroll
        for (int l = 0; l < D; ++l) {
            psi[x0 | off[l]] = y[l];
            lam[x0 | off[l]] = z[l];
        }
        x0 = ((x0 | ~fm) + step) & fm;
    }
    if (!GRAD) return;
    fold();
    __syncthreads();
    if (threadIdx.x < 2 * D * D) {
        double s = 0.0;
        for (int w = 0; w < kSaThreads / 32; ++w) s += wacc[w][threadIdx.x];
        npart[(long long)blockIdx.x * 32 + threadIdx.x] = s;
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

// N of every gradient block: the CTA partials summed in order.
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

// contrib[e] = 2 scale Re Tr(D_j N) for parameterised op e.
__global__ void sa_grad_kernel(const SaEntry* __restrict__ ents, int n_ent, const BuildOp* __restrict__ bops,
                               const double2* __restrict__ pool, const double* __restrict__ params,
                               const double* __restrict__ N, double* __restrict__ contrib) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_ent) return;
    const SaEntry en = ents[e];
    const int D = 1 << en.k;
    double2 L[16], M[16], Mp[16];
    for (int i = 0; i < D * D; ++i) L[i] = make_double2((i / D) == (i % D) ? 1.0 : 0.0, 0.0);
    const double pi = 3.14159265358979323846;
    double scale = 1.0;
    for (int o = 0; o < en.op_count; ++o) {
        const BuildOp op = bops[en.op_begin + o];
        const int dk = 1 << op.k;
        double ang = op.angle0;
        if (op.param >= 0) ang += op.scale * params[op.param];
        if (o == en.j) {   // dM/dangle from two shifted evaluations
            scale = op.scale;
            const bool cp = op.code == TCNG_CP;
            const double h = cp ? 0.5 * pi : pi, f = cp ? 0.5 : 0.25;
            gate_matrix_d(op, ang + h, M, dk, pool);
            gate_matrix_d(op, ang - h, Mp, dk, pool);
            for (int i = 0; i < dk * dk; ++i) M[i] = make_double2(f * (M[i].x - Mp[i].x), f * (M[i].y - Mp[i].y));
        } else {
            gate_matrix_d(op, ang, M, dk, pool);
        }
        sa_apply_op(L, D, op, M);
    }
    // Tr(D N) = sum_{a,b} D[b][a] N[a][b]
    const double* Nb = N + (long long)en.gblock * 32;
    double re = 0.0;
    for (int a = 0; a < D; ++a)
        for (int b = 0; b < D; ++b) {
            const double2 d = L[b * D + a];
            re += d.x * Nb[2 * (a * D + b)] - d.y * Nb[2 * (a * D + b) + 1];
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

template <typename C, int K>
cudaError_t launch_block(bool grad, C* psi, C* lam, const C* U, int diag, unsigned long long qmask, int n,
                         double* npart, int grid, cudaStream_t s) {
    if constexpr (K <= 2) {   // gradient blocks have at most two qubits
        if (grad) {
            sa_block_kernel<C, K, true><<<grid, kSaThreads, 0, s>>>(psi, lam, U, diag, qmask, n, npart);
            count_launch();
            return cudaGetLastError();
        }
    }
    (void)grad;
        sa_block_kernel<C, K, false><<<grid, kSaThreads, 0, s>>>(psi, lam, U, diag, qmask, n, npart);
    count_launch();
    return cudaGetLastError();
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
    e = launch_ham_apply<C>(static_cast<const C*>(st->buf), st->d_off + item, lam, zero, 1, n, ts->d_h,
                            (int)n_terms, coeffs, ts->d_c, s);
    if (e != cudaSuccess) return cuda_fail(e, "H apply");
    sa_dot_kernel<C><<<grid, kSaThreads, 0, s>>>(psi, lam, N, dpart);
    sa_sum_kernel<<<1, 32, 0, s>>>(dpart, grid, energy);
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
    for (int bi = (int)sp->blocks.size() - 1; bi >= 0; --bi) {
        const SaPlan::Blk& b = sp->blocks[bi];
        const bool gb = b.grad >= 0;
        double* np = gb ? npart + (size_t)b.grad * grid * 32 : nullptr;
        const C* U = table + b.out_off;
        if (b.k == 1) {
            e = launch_block<C, 1>(gb, psi, lam, U, b.diag, b.qmask, n, np, grid, s);
        } else if (b.k == 2) {
            e = launch_block<C, 2>(gb, psi, lam, U, b.diag, b.qmask, n, np, grid, s);
        } else {   // 3..5 qubits, no parameter: each state on its own
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
        }
        if (e != cudaSuccess) return cuda_fail(e, "adjoint block kernel");
    }
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
