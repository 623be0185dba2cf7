// C ABI of the simulator (declared in include/tcng.h): argument validation,
// state handles, the per-structure plan cache, and kernel orchestration.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <stdexcept>
#include <string>
#include <unordered_map>
#include <vector>

#include "capi_internal.hpp"

namespace tcng {

static std::atomic<uint64_t> g_launches{0};
static thread_local int g_count_off = 0;
void count_launch() {
    if (!g_count_off) g_launches.fetch_add(1, std::memory_order_relaxed);
}
void add_launches(uint64_t k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
LaunchCountOff::LaunchCountOff() { ++g_count_off; }
LaunchCountOff::~LaunchCountOff() { --g_count_off; }

static thread_local std::string g_err;
tcng_status fail(tcng_status s, const std::string& msg) {
    g_err = msg;
    return s;
}
tcng_status cuda_fail(cudaError_t e, const char* where) {
    cudaGetLastError();
    return fail(TCNG_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

Options g_opt;
std::mutex g_mu;

// ------------------------------------------------------------- profiling --
struct ProfRec {
    std::string name;
    cudaEvent_t e0, e1;
};
static bool g_prof = false;
static std::mutex g_prof_mu;
bool profiling_enabled() { return g_prof; }
static std::vector<ProfRec> g_prof_recs;

ProfScope::ProfScope(const char* nm, cudaStream_t st) : name(nm), s(st) {
    if (!g_prof) return;
    cudaEventCreate(&e0);
    cudaEventRecord(e0, s);
}
ProfScope::~ProfScope() {
    if (!e0) return;
    cudaEvent_t e1;
    cudaEventCreate(&e1);
    cudaEventRecord(e1, s);
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_prof_recs.push_back({name, e0, e1});
}

// ------------------------------------------------------------ device ctx --
DeviceCtx& ctx() {
    static std::map<int, std::unique_ptr<DeviceCtx>> ctxs;
    int dev = 0;
    cudaGetDevice(&dev);
    auto& p = ctxs[dev];
    if (!p) {
        p.reset(new DeviceCtx());
        p->device = dev;
        if (cudaMalloc(&p->err, sizeof(unsigned)) == cudaSuccess) {
            cudaMemset(p->err, 0, sizeof(unsigned));
        } else {
            cudaGetLastError();
            p->err = nullptr;
        }
    }
    return *p;
}

void* DeviceCtx::scratch(const std::string& name, size_t bytes) {
    auto& b = bufs[name];
    if (b.bytes < bytes) {
        if (b.ptr) {
            cudaDeviceSynchronize();
            cudaFree(b.ptr);
            b.ptr = nullptr;
            b.bytes = 0;
        }
        size_t cap = std::max(bytes, (size_t)256);
        ++gen;
        if (cudaMalloc(&b.ptr, cap) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        b.bytes = cap;
    }
    return b.ptr;
}

DevPlan::~DevPlan() {
    cudaFree(d_bblocks);
    cudaFree(d_bops);
    cudaFree(d_pool);
    cudaFree(d_stages);
    cudaFree(d_dops);
    cudaFree(d_table);
    cudaFree(d_gparam);
    cudaFree(d_gscale);
    cudaFree(d_tcs);
    cudaFree(d_lay);
}

TermSet::~TermSet() {
    cudaFree(d_h);
    cudaFree(d_c);
}

PlanOptions plan_options(tcng_dtype dt, bool adjoint) {
    PlanOptions o;
    o.fuse_width = g_opt.fuse_width;
    o.tile_bits = g_opt.tile_bits;
    if (dt == TCNG_C128) o.tile_bits = std::min(o.tile_bits, 12);
    o.chunk_bits = std::min(g_opt.chunk_bits, o.tile_bits);
    o.adjoint = adjoint ? 1 : 0;
    o.unfused = g_opt.unfused ? 1 : 0;
    o.wide = 0;
    return o;
}

// Plan options of a tcng_apply_circuit call: 32-amplitude register stages where
// they save stages when the passes will run on the FP16 tensor-core kernels
// (complex64, tensor cores and FP16 operands enabled, one W set for every tile:
// no per-item parameters).
PlanOptions apply_plan_options(tcng_dtype dt, int batch, int P) {
    PlanOptions o = plan_options(dt, false);
    o.wide = (dt == TCNG_C64 && !o.unfused && g_opt.tensor_cores != 0 && g_opt.tc_fp16 &&
              o.tile_bits == 13 && (P == 0 || batch == 1)) ? 1 : 0;
    return o;
}

// Build (or fetch) the device plan of a structure.
DevPlan* get_plan(int n, const tcng_gate* ops, size_t n_ops, const double* pool, size_t n_mat,
                  int P, const PlanOptions& o) {
    DeviceCtx& c = ctx();
    const uint64_t h = structure_hash(n, ops, n_ops, pool, n_mat, P, o);
    auto it = c.plans.find(h);
    if (it != c.plans.end()) return it->second.get();
    std::unique_ptr<DevPlan> dp(new DevPlan());
    Plan& pl = dp->plan;
    pl.n = n;
    pl.P = P;
    pl.opt = o;
    if (n < 5 && !o.adjoint) pl.opt.unfused = 1;
    pl.ops = import_ops(n, ops, n_ops, n_mat, P, pool);
    build_plan(pl);
    dp->d_bblocks = dev_copy(pl.bblocks);
    dp->d_bops = dev_copy(pl.bops);
    if (n_mat) {
        std::vector<double2> pv(n_mat);
        for (size_t i = 0; i < n_mat; ++i) pv[i] = make_double2(pool[2 * i], pool[2 * i + 1]);
        dp->d_pool = dev_copy(pv);
    }
    dp->d_stages = dev_copy(pl.stages);
    dp->d_dops = dev_copy(pl.dops);
    dp->d_gparam = dev_copy(pl.grad_param);
    dp->d_gscale = dev_copy(pl.grad_scale);
    DevPlan* raw = dp.get();
    c.plans[h] = std::move(dp);
    return raw;
}

// Device copies of a Pauli-term list (cached by content).
TermSet* get_terms(const tcng_pauli* terms, size_t n_terms, int n) {
    const uint64_t lim = (n >= 64) ? ~0ULL : ((1ULL << n) - 1);
    for (size_t t = 0; t < n_terms; ++t)
        if ((terms[t].xmask & ~lim) || (terms[t].zmask & ~lim))
            throw std::invalid_argument("Pauli mask outside the register");
    uint64_t h = 1469598103934665603ULL ^ (uint64_t)n_terms;
    const unsigned char* b = reinterpret_cast<const unsigned char*>(terms);
    for (size_t i = 0; i < sizeof(tcng_pauli) * n_terms; ++i) {
        h ^= b[i];
        h *= 1099511628211ULL;
    }
    DeviceCtx& c = ctx();
    auto it = c.terms.find(h);
    if (it != c.terms.end()) return it->second.get();
    std::unique_ptr<TermSet> ts(new TermSet());
    ts->n_terms = (int)n_terms;
    std::vector<HTerm> ht(std::max<size_t>(1, n_terms));
    std::vector<double> tc(std::max<size_t>(1, n_terms), 0.0);
    for (size_t t = 0; t < n_terms; ++t) {
        ht[t].xm = terms[t].xmask;
        ht[t].zm = terms[t].zmask;
        ht[t].ny = __builtin_popcountll(terms[t].xmask & terms[t].zmask) & 3;
        tc[t] = terms[t].coeff;
    }
    ts->d_h = dev_copy(ht);
    ts->d_c = dev_copy(tc);
    TermSet* raw = ts.get();
    c.terms[h] = std::move(ts);
    return raw;
}

// Per-item matrix table of a plan for `items` items (grown on demand).
void* plan_table(DevPlan* dp, size_t elem, int items) {
    const size_t need = std::max<size_t>(1, (size_t)dp->plan.table_size) * elem * std::max(items, 1);
    if (dp->table_bytes < need) {
        if (dp->d_table) {
            cudaDeviceSynchronize();
            cudaFree(dp->d_table);
            dp->d_table = nullptr;
            dp->table_bytes = 0;
        }
        ++ctx().gen;
        if (cudaMalloc(&dp->d_table, need) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        dp->table_bytes = need;
    }
    return dp->d_table;
}

// Run a plan on a group of items (all with n == plan.n).
template <typename C>
tcng_status run_plan(DevPlan* dp, C* state, const long long* d_item_off, int items,
                     const double* params, cudaStream_t s, void* tma_base, long long item_stride,
                     const double2* item_pool, long long pool_stride) {
    Plan& pl = dp->plan;
    // per-item matrices: from per-item parameters, or from a per-item matrix pool
    const bool per_item = pl.P > 0 || (item_pool && pool_stride > 0);
    const double2* pool = item_pool ? item_pool : dp->d_pool;
    const long long pstride = item_pool ? pool_stride : 0;
    const int tab_items = per_item ? items : 1;
    C* table = static_cast<C*>(plan_table(dp, sizeof(C), tab_items));
    if (!table) return fail(TCNG_ENOMEM, "matrix table allocation failed");
    const long long stride = per_item ? pl.table_size : 0;
    cudaError_t e;
    {
    ProfScope ps("build_matrices", s);
    e = launch_build_matrices<C>(dp->d_bblocks, (int)pl.bblocks.size(), dp->d_bops,
                                             pool, pl.P > 0 ? params : nullptr, pl.P, table,
                                             pl.table_size, tab_items, s, pstride);
    }
    if (e != cudaSuccess) return cuda_fail(e, "matrix prologue");
    if (pl.opt.unfused) {
        for (const Block& b : pl.blocks) {
            ProfScope ps(b.diag ? "gate_diag" : (b.k <= 2 ? "gate_pair_quartet" : "gate_dense"), s);
            e = launch_gate<C>(state, d_item_off, items, pl.n, b, table, stride, s);
            if (e != cudaSuccess) return cuda_fail(e, "gate kernel");
        }
    } else {
        // complex64 register stages on the tensor cores (when enabled): W operands
        // from an FP64 table of the same blocks
        const float* wops = nullptr;
        const void* wops_h = nullptr;   // FP16 operands (one W set for every tile)
        long long w_stride = 0;
        // auto: the W prologue is per item when items carry their own parameters, and
        // fewer tiles than SMs leave the tensor-core pipeline latency-bound (measured
        // slower than the SIMT stages there)
        const long long tiles = (pl.n >= 13 ? (1ll << (pl.n - 13)) : 0) * items;
        const bool tc_auto = (tab_items == 1 && tiles >= num_sms()) || tiles >= 32ll * num_sms();
        if (sizeof(C) == 8 && (g_opt.tensor_cores == 1 || (g_opt.tensor_cores == 2 && tc_auto))) {
            plan_tensor_stages(dp);
            if (dp->n_tc) {
                DeviceCtx& c = ctx();
                double2* dtab = static_cast<double2*>(
                    c.scratch("tc_table", sizeof(double2) * std::max(1, pl.table_size) * tab_items));
                float* w = static_cast<float*>(
                    c.scratch("tc_w", sizeof(float) * 2048 * (size_t)std::max(1, dp->n_tc32) * tab_items));
                if (!dtab || !w) return fail(TCNG_ENOMEM, "tensor-core operand scratch");
                ProfScope ps("build_stage_w", s);
                e = launch_build_matrices<double2>(dp->d_bblocks, (int)pl.bblocks.size(), dp->d_bops,
                                                   pool, pl.P > 0 ? params : nullptr, pl.P, dtab,
                                                   pl.table_size, tab_items, s, pstride);
                if (e == cudaSuccess) e = launch_build_stage_w(dp, dtab, stride, tab_items, w, false, s);
                // unitary plans whose tiles all share one W set also get the FP16 operands
                if (e == cudaSuccess && g_opt.tc_fp16 && pl.all_unitary && tab_items == 1) {
                    void* wh = c.scratch("tc_wh", (size_t)dp->wh_bytes);
                    if (!wh) return fail(TCNG_ENOMEM, "tensor-core operand scratch");
                    e = launch_build_stage_w(dp, dtab, stride, 1, wh, true, s);
                    wops_h = wh;
                }
                if (e != cudaSuccess) return cuda_fail(e, "tensor-core operand prologue");
                wops = w;
                w_stride = per_item ? 2048ll * dp->n_tc32 : 0;
            }
        }
        for (size_t pi = 0; pi < pl.passes.size(); ++pi) {
            const DevPass& p = pl.passes[pi];
            TmaTile tma{};
            if (tma_base && (items == 1 || item_stride > 0))
                tma = make_tma_tile(tma_base, pl.n, (int)sizeof(C), p, items, item_stride, false, true);
            if (wops && dp->tc_pass[pi]) {   // tile map, else one bulk copy per chunk
                // stages on tile bits 0..3 read conflict-free from a 128-byte swizzled tile
                bool rot = false, swz = false;
                for (int si = 0; si < p.stage_count; ++si) rot = rot || dp->tcs[p.stage_begin + si].nj > 0;
                if (rot && p.chunk >= 4 && tma.rank) {
                    const TmaTile ts = make_tma_tile(tma_base, pl.n, (int)sizeof(C), p, items, item_stride, true, true);
                    if (ts.rank) {
                        tma = ts;
                        swz = true;
                    }
                }
                if (wops_h && pass_tch_eligible(dp, (int)pi)) {
                    ProfScope ps("pass_tch_kernel_c64", s);
                    e = launch_pass_tch(dp, (int)pi, items, wops_h, ctx().err, tma, swz,
                                        reinterpret_cast<float2*>(state), d_item_off, s);
                    if (e != cudaSuccess) return cuda_fail(e, "tensor-core pass kernel");
                    continue;
                }
                if (!dp->tc5[pi]) {   // TF32 operands: 4-bit stages only
                    ProfScope ps("pass_tcs_kernel_c64", s);
                    e = launch_pass_tcs(dp, (int)pi, items, wops, w_stride, ctx().err, tma, swz,
                                        reinterpret_cast<float2*>(state), d_item_off, s);
                    if (e != cudaSuccess) return cuda_fail(e, "tensor-core pass kernel");
                    continue;
                }
            }
            ProfScope ps(sizeof(C) == 8 ? "pass_kernel_c64" : "pass_kernel_c128", s);
            e = launch_pass<C>(state, d_item_off, items, pl.n, p, pl.stages.data(), dp->d_stages,
                               dp->d_dops, table, stride, ctx().err, s, &tma);
            if (e != cudaSuccess) return cuda_fail(e, "pass kernel");
        }
    }
    return TCNG_OK;
}
template tcng_status run_plan<float2>(DevPlan*, float2*, const long long*, int, const double*, cudaStream_t,
                                      void*, long long, const double2*, long long);
template tcng_status run_plan<double2>(DevPlan*, double2*, const long long*, int, const double*, cudaStream_t,
                                       void*, long long, const double2*, long long);

// Device address of a group's first item and the spacing of its items in bytes
// (-1 if they are not equally spaced).
static void group_span(const tcng_state* st, const std::vector<int>& items, void** base, long long* stride) {
    const size_t es = st->dt == TCNG_C64 ? 8 : 16;
    *base = static_cast<char*>(st->buf) + st->off[items[0]] * es;
    *stride = items.size() > 1 ? (long long)((st->off[items[1]] - st->off[items[0]]) * es) : 0;
    for (size_t i = 1; i < items.size(); ++i)
        if ((long long)((st->off[items[i]] - st->off[items[0]]) * es) != (long long)i * *stride) {
            *stride = -1;
            return;
        }
}

// Group Pauli terms into tile passes: a term joins a pass if its X bits above
// the contiguous low bits fit the pass's gather set.
// The complex64 expectation kernel's tile bits have roles: 1..5 pick the partner
// lane, 6..9 the partner warp (a term whose lowest X bit there, with none on
// 10..12, is carried by one warp half per tile), 10..12 the partner register pair
// (the half form, half the partner reads); a term with X only on lane bits reads
// every partner pair in every warp.  The gathered qubits (tile bits chunk..12) are
// assigned to the roles to minimise the pass's term cost, by trying every split
// (at most C(10,3) x C(7,4) = 4200): per term the relative cost of its form,
// measured per term at 28 qubits: warp 39, register 49, lane 69 (Z-only terms
// and X bits on the contiguous low qubits do not depend on the order).
void order_expect_gather(const tcng_pauli* terms, const std::vector<int>& sel, int chunk, std::vector<int>& gq) {
    const int G = (int)gq.size();
    if (G > 16) return;
    auto role = [&](int i) { const int b = chunk + i; return b >= 10 ? 2 : (b >= 6 ? 1 : 0); };
    int want_reg = 0, want_warp = 0;
    for (int i = 0; i < G; ++i) {
        want_reg += role(i) == 2;
        want_warp += role(i) == 1;
    }
    // per selected X term: its X qubits among the gathered ones, as a bit set over gq
    std::vector<uint32_t> tx;
    for (int t : sel) {
        uint32_t b = 0;
        for (int i = 0; i < G; ++i) b |= (uint32_t)((terms[t].xmask >> gq[i]) & 1) << i;
        if (terms[t].xmask) tx.push_back(b);
    }
    long best = -1;
    uint32_t best_reg = 0, best_warp = 0;
    const uint32_t all = (1u << G) - 1;
    for (uint32_t rg = 0; rg <= all; ++rg) {
        if (__builtin_popcount(rg) != want_reg) continue;
        const uint32_t rest = all & ~rg;
        for (uint32_t wp = rest;; wp = (wp - 1) & rest) {   // the subsets of the rest
            if (__builtin_popcount(wp) == want_warp) {
                long c = 0;
                for (uint32_t b : tx) c += (b & rg) ? 49 : ((b & wp) ? 39 : 69);
                if (best < 0 || c < best) {
                    best = c;
                    best_reg = rg;
                    best_warp = wp;
                }
            }
            if (!wp) break;
        }
    }
    std::vector<int> reg, warp, lane;
    for (int i = 0; i < G; ++i)
        ((best_reg >> i) & 1 ? reg : (best_warp >> i) & 1 ? warp : lane).push_back(gq[i]);
    std::vector<int> out;
    size_t ir = 0, iw = 0, il = 0;
    for (int i = 0; i < G; ++i)
        out.push_back(role(i) == 2 ? reg[ir++] : role(i) == 1 ? warp[iw++] : lane[il++]);
    gq.swap(out);
}

void plan_expectation(int n, int m, int low, const tcng_pauli* terms, size_t T,
                      std::vector<DevPass>& passes, std::vector<ExpPass>& eps, std::vector<size_t>* wide) {
    const uint64_t lim = (n >= 64) ? ~0ULL : ((1ULL << n) - 1);
    for (size_t t = 0; t < T; ++t)
        if ((terms[t].xmask & ~lim) || (terms[t].zmask & ~lim))
            throw std::invalid_argument("Pauli mask outside the register");
    m = std::min(m, n);
    // at most 3 contiguous low bits: a pass then gathers up to m - 3 high qubits, so
    // fewer passes hold the same terms.  The scattered rows stream well through the
    // complex64 kernel's cp.async copies (32 qubits, 64 weight-4 strings + TFIM: 8
    // passes and a 586 ms step with 3 bits; 626 ms with 6, 650 ms with 7, 602 ms
    // with 2 (10 passes))
    constexpr int kExpLowBits = 3;
    const int low0 = std::min(std::min(low, m), kExpLowBits);
    auto mask_below = [](int b) { return b >= 64 ? ~0ULL : ((1ULL << b) - 1); };
    // a tile keeps at least its lowest qubit contiguous (16-byte copies), so a term
    // may have at most m - 1 X/Y factors above qubit 0; wider terms go to `wide`
    // (evaluated from global memory) when the caller takes them
    std::vector<char> done(T, 0);
    size_t left = T;
    if (n > m)
        for (size_t t = 0; t < T; ++t)
            if (__builtin_popcountll(terms[t].xmask & ~1ULL) > m - 1) {
                if (!wide)
                    throw std::invalid_argument("Pauli term " + std::to_string(t) + ": more than " +
                                                std::to_string(m - 1) + " X/Y factors above qubit 0");
                wide->push_back(t);
                done[t] = 1;
                --left;
            }
    // most constrained terms first (most X bits above the default contiguous bits):
    // the greedy packing then fills passes around them (results keep the input order)
    std::vector<size_t> order(T);
    for (size_t t = 0; t < T; ++t) order[t] = t;
    std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) {
        return __builtin_popcountll(terms[a].xmask & ~mask_below(low0)) >
               __builtin_popcountll(terms[b].xmask & ~mask_below(low0));
    });
    while (left) {
        // contiguous low bits of this pass: the default, or fewer when the first open
        // term has more X bits above them than the tile can gather
        int lowp = low0;
        if (n > m)
            for (size_t t : order)
                if (!done[t]) {
                    while (lowp > 1 && __builtin_popcountll(terms[t].xmask & ~mask_below(lowp)) > m - lowp)
                        --lowp;
                    break;
                }
        const int gmax = m - lowp;
        const uint64_t lowmask = mask_below(lowp);
        uint64_t G = 0;
        ExpPass ep{};
        std::vector<int> sel;
        for (size_t t : order) {
            if ((int)sel.size() >= kExpTermsPerPass) break;
            if (done[t]) continue;
            const uint64_t hi = (n <= m) ? 0 : (terms[t].xmask & ~lowmask);
            if (__builtin_popcountll(G | hi) > gmax) continue;
            G |= hi;
            sel.push_back((int)t);
        }
        if (sel.empty()) throw std::logic_error("expectation planner: no term fits a tile");
        uint64_t S;
        if (n <= m) {
            S = lim;
        } else {
            S = lowmask | G;
            for (int q = lowp; q < n && __builtin_popcountll(S) < m; ++q) S |= 1ULL << q;
        }
        DevPass dp{};
        dp.m = __builtin_popcountll(S);
        int L = 0;
        while (L < n && ((S >> L) & 1)) ++L;
        dp.chunk = std::min(L, dp.m);
        dp.ngather = dp.m - dp.chunk;
        std::vector<int> gq;   // gathered qubits, in the order of their tile bits
        int ri = 0;
        for (int q = dp.chunk; q < n; ++q) {
            if ((S >> q) & 1) gq.push_back(q);
            else dp.rest[ri++] = (uint8_t)q;
        }
        dp.nrest = ri;
        if (dp.m == 13 && dp.chunk <= 6) order_expect_gather(terms, sel, dp.chunk, gq);
        int tb[64];
        for (int q = 0; q < 64; ++q) tb[q] = -1;
        for (int q = 0; q < dp.chunk; ++q) tb[q] = q;
        for (size_t g = 0; g < gq.size(); ++g) {
            dp.gather[g] = (uint8_t)gq[g];
            tb[gq[g]] = dp.chunk + (int)g;
        }
        for (int t : sel) {
            ExpTerm et{};
            const uint64_t xm = terms[t].xmask, zm = terms[t].zmask;
            et.ny = __builtin_popcountll(xm & zm) & 3;
            et.out = t;
            for (int q = 0; q < n; ++q) {
                if ((xm >> q) & 1) et.xm_tile |= 1u << tb[q];
                if ((zm >> q) & 1) {
                    if (tb[q] >= 0) et.zm_tile |= 1u << tb[q];
                    else et.zm_glob |= 1ULL << q;
                }
            }
            ep.t[ep.nterms++] = et;
            done[t] = 1;
            --left;
        }
        passes.push_back(dp);
        eps.push_back(ep);
    }
}

}  // namespace tcng

using namespace tcng;

#define TCNG_TRY(body)                                                   \
    try {                                                                \
        body                                                             \
    } catch (const std::invalid_argument& ex) {                          \
        return fail(TCNG_EINVAL, ex.what());                             \
    } catch (const std::bad_alloc&) {                                    \
        return fail(TCNG_ENOMEM, "allocation failed");                   \
    } catch (const std::exception& ex) {                                 \
        return fail(TCNG_EINVAL, ex.what());                             \
    }

extern "C" {

const char* tcng_last_error(void) { return g_err.c_str(); }
const char* tcng_version(void) { return "tcng-b300 0.1 (sm_103a)"; }
uint64_t tcng_launch_count(void) { return g_launches.load(); }

static size_t elem_size(tcng_dtype dt) { return dt == TCNG_C64 ? 8 : 16; }

static tcng_status layout(tcng_dtype dt, int batch, const int* nq, std::vector<long long>& off,
                          size_t* bytes) {
    if (dt != TCNG_C64 && dt != TCNG_C128) return fail(TCNG_EINVAL, "bad dtype");
    if (batch < 1) return fail(TCNG_EINVAL, "batch must be >= 1");
    if (!nq) return fail(TCNG_EINVAL, "n_qubits is NULL");
    const size_t es = elem_size(dt);
    size_t pos = 0;
    off.resize(batch);
    for (int b = 0; b < batch; ++b) {
        if (nq[b] < 1 || nq[b] > TCNG_MAX_QUBITS) return fail(TCNG_EINVAL, "qubit count out of range");
        pos = (pos + 255) & ~(size_t)255;
        off[b] = (long long)(pos / es);
        pos += es << nq[b];
    }
    *bytes = pos;
    return TCNG_OK;
}

tcng_status tcng_state_bytes(tcng_dtype dt, int batch, const int* n_qubits, size_t* bytes) {
    std::vector<long long> off;
    if (!bytes) return fail(TCNG_EINVAL, "bytes is NULL");
    return layout(dt, batch, n_qubits, off, bytes);
}

tcng_status tcng_state_free(tcng_state* st) {
    if (!st) return TCNG_OK;
    if (st->owned) cudaFree(st->buf);
    cudaFree(st->d_off);
    for (auto& kv : st->groups) {
        cudaFree(kv.second.d_off);
        cudaFree(kv.second.d_items);
    }
    for (auto& kv : st->pack) cudaFree(kv.second.first);
    delete st;
    return TCNG_OK;
}

tcng_status tcng_state_reset(tcng_state* st, void* stream) {
    if (!st) return fail(TCNG_EINVAL, "state is NULL");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemsetAsync(st->buf, 0, st->bytes, s);
    if (e != cudaSuccess) return cuda_fail(e, "memset");
    if (st->dt == TCNG_C64)
        e = launch_set_basis<float2>(static_cast<float2*>(st->buf), st->d_off, st->batch, s);
    else
        e = launch_set_basis<double2>(static_cast<double2*>(st->buf), st->d_off, st->batch, s);
    if (e != cudaSuccess) return cuda_fail(e, "init kernel");
    return TCNG_OK;
}

tcng_status tcng_state_init(tcng_state** out, tcng_dtype dt, int batch, const int* n_qubits,
                            void* dev_buf, size_t buf_bytes, void* stream) {
    if (!out) return fail(TCNG_EINVAL, "out is NULL");
    *out = nullptr;
    std::vector<long long> off;
    size_t bytes = 0;
    tcng_status s = layout(dt, batch, n_qubits, off, &bytes);
    if (s) return s;
    std::lock_guard<std::mutex> lk(g_mu);
    TCNG_TRY({
        std::unique_ptr<tcng_state> st(new tcng_state());
        st->dt = dt;
        st->batch = batch;
        st->n.assign(n_qubits, n_qubits + batch);
        st->off = off;
        st->bytes = bytes;
        if (dev_buf) {
            if (buf_bytes < bytes) return fail(TCNG_ENOMEM, "caller buffer too small");
            if (reinterpret_cast<uintptr_t>(dev_buf) & 255)
                return fail(TCNG_EINVAL, "caller buffer must be 256-byte aligned");
            st->buf = dev_buf;
            st->owned = false;
        } else {
            cudaError_t e = cudaMalloc(&st->buf, bytes);
            if (e != cudaSuccess) {
                cudaGetLastError();
                return fail(TCNG_ENOMEM, std::string("state allocation: ") + cudaGetErrorString(e));
            }
            st->owned = true;
        }
        st->d_off = dev_copy(off);
        for (int b = 0; b < batch; ++b) st->groups[n_qubits[b]].items.push_back(b);
        for (auto& kv : st->groups) {
            std::vector<long long> go;
            for (int b : kv.second.items) go.push_back(off[b]);
            kv.second.d_off = dev_copy(go);
            kv.second.d_items = dev_copy(kv.second.items);
        }
        tcng_state* raw = st.release();
        s = tcng_state_reset(raw, stream);
        if (s) {
            tcng_state_free(raw);
            return s;
        }
        *out = raw;
        return TCNG_OK;
    })
}

tcng_status tcng_state_ptr(const tcng_state* st, int item, void** dev_amp, size_t* bytes) {
    if (!st || !dev_amp) return fail(TCNG_EINVAL, "null argument");
    if (item < 0 || item >= st->batch) return fail(TCNG_EINVAL, "item out of range");
    const size_t es = elem_size(st->dt);
    *dev_amp = static_cast<char*>(st->buf) + st->off[item] * es;
    if (bytes) *bytes = es << st->n[item];
    return TCNG_OK;
}

}  // extern "C"

namespace tcng {
// A batch of states smaller than a tile that all see the same gates (no
// per-item parameters) is stored back to back, so 2^(m-n) consecutive items
// form one 2^m-amplitude tile of a virtual m-qubit state whose top m - n qubits
// no gate touches (the QML batches of Sec. VII.B: B inputs, one circuit).
// Every pass then runs on full tiles -- on the tensor cores for complex64, one
// W set for the whole batch -- instead of one small tile per item.  Returns
// the number of whole virtual items (0: not packable); items past
// virtual * 2^(m-n) run the ordinary per-item path.
static long long packed_items(tcng_state* st, int m, int P, long long** d_voff) {
    if (st->groups.size() != 1 || P != 0) return 0;
    const int n = st->groups.begin()->first;
    const int es = st->dt == TCNG_C64 ? 8 : 16;
    if (n >= m || (es << n) < 256) return 0;
    for (int b = 0; b < st->batch; ++b)
        if (st->off[b] != ((long long)b << n)) return 0;
    const long long nv = ((long long)st->batch << n) >> m;
    if (nv < 1) return 0;
    auto it = st->pack.find(m);
    if (it == st->pack.end()) {
        std::vector<long long> v(nv);
        for (long long i = 0; i < nv; ++i) v[i] = i << m;
        it = st->pack.emplace(m, std::make_pair(dev_copy(v), nv)).first;
    }
    *d_voff = it->second.first;
    return it->second.second;
}
}  // namespace tcng

extern "C" {

tcng_status tcng_apply_circuit(tcng_state* st, const tcng_gate* ops, size_t n_ops,
                               const double* mat_pool, size_t n_mat, const void* params_dev, int P,
                               void* stream) {
    if (!st) return fail(TCNG_EINVAL, "state is NULL");
    if (P < 0) return fail(TCNG_EINVAL, "P < 0");
    if (P > 0 && !params_dev) return fail(TCNG_EINVAL, "params_dev is NULL");
    if (n_ops == 0) return TCNG_OK;
    std::lock_guard<std::mutex> lk(g_mu);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    TCNG_TRY({
        const PlanOptions o = apply_plan_options(st->dt, st->batch, P);
        // graph key: structure of every size class, options and every device pointer read
        uint64_t key = key_mix(options_key(), 1);
        key = key_mix(key, reinterpret_cast<uintptr_t>(st));
        key = key_mix(key, reinterpret_cast<uintptr_t>(st->buf));
        key = key_mix(key, reinterpret_cast<uintptr_t>(params_dev));
        key = key_mix(key, (uint64_t)P);
        for (auto& kv : st->groups)
            key = key_mix(key, structure_hash(kv.first, ops, n_ops, mat_pool, n_mat, P, o));
        return run_graphed(key, s, [&](cudaStream_t s) -> tcng_status {
        long long* d_voff = nullptr;
        const long long nv = o.unfused ? 0 : packed_items(st, o.tile_bits, P, &d_voff);
        int first = 0;   // first item left for the per-item path
        if (nv > 0) {
            const int n = st->groups.begin()->first;
            const int m = o.tile_bits;
            // the n-qubit plan validates every qubit against n (the virtual m-qubit
            // register would accept qubits of the neighbouring items)
            DevPlan* dq = get_plan(n, ops, n_ops, mat_pool, n_mat, 0, o);
            DevPlan* dp = get_plan(m, ops, n_ops, mat_pool, n_mat, 0, o);
            const long long vstride = (long long)(st->dt == TCNG_C64 ? 8 : 16) << m;
            tcng_status r;
            if (st->dt == TCNG_C64)
                r = run_plan<float2>(dp, static_cast<float2*>(st->buf), d_voff, (int)nv, nullptr, s, st->buf, vstride);
            else
                r = run_plan<double2>(dp, static_cast<double2*>(st->buf), d_voff, (int)nv, nullptr, s, st->buf, vstride);
            if (r) return r;
            first = (int)((nv << m) >> n);
            if (first >= st->batch) return TCNG_OK;
            const int rest = st->batch - first;
            std::vector<int> items(rest);
            for (int i = 0; i < rest; ++i) items[i] = first + i;
            void* tb = nullptr;
            long long ts = -1;
            group_span(st, items, &tb, &ts);
            if (st->dt == TCNG_C64)
                return run_plan<float2>(dq, static_cast<float2*>(st->buf), st->d_off + first, rest, nullptr, s, tb, ts);
            return run_plan<double2>(dq, static_cast<double2*>(st->buf), st->d_off + first, rest, nullptr, s, tb, ts);
        }
        for (auto& kv : st->groups) {
            const int n = kv.first;
            const int items = (int)kv.second.items.size();
            void* tb = nullptr;
            long long ts = -1;
            group_span(st, kv.second.items, &tb, &ts);
            DevPlan* dp = get_plan(n, ops, n_ops, mat_pool, n_mat, P, o);
            // Parameters are indexed by position inside the group, so a ragged
            // batch with parameters needs the items of one n to be contiguous.
            const double* prm = static_cast<const double*>(params_dev);
            if (P > 0 && st->groups.size() > 1) {
                const std::vector<int>& it = kv.second.items;
                for (size_t i = 1; i < it.size(); ++i)
                    if (it[i] != it[0] + (int)i)
                        return fail(TCNG_EUNSUPPORTED,
                                    "ragged batch with parameters needs items of equal n to be contiguous");
                prm += (size_t)it[0] * P;
            }
            tcng_status r;
            if (st->dt == TCNG_C64)
                r = run_plan<float2>(dp, static_cast<float2*>(st->buf), kv.second.d_off, items, prm, s, tb, ts);
            else
                r = run_plan<double2>(dp, static_cast<double2*>(st->buf), kv.second.d_off, items, prm, s, tb, ts);
            if (r) return r;
        }
        return TCNG_OK;
        });
    })
}

tcng_status tcng_apply_circuit_pooled(tcng_state* st, const tcng_gate* ops, size_t n_ops,
                                      const double* mat_pool, size_t n_mat, const void* item_pool_dev,
                                      size_t pool_stride, const void* params_dev, int P, void* stream) {
    if (!st) return fail(TCNG_EINVAL, "state is NULL");
    if (P < 0) return fail(TCNG_EINVAL, "P < 0");
    if (P > 0 && !params_dev) return fail(TCNG_EINVAL, "params_dev is NULL");
    if (!item_pool_dev) return fail(TCNG_EINVAL, "item_pool_dev is NULL");
    if (pool_stride < n_mat) return fail(TCNG_EINVAL, "pool_stride < n_mat");
    if (reinterpret_cast<uintptr_t>(item_pool_dev) & 15) return fail(TCNG_EINVAL, "item_pool_dev not 16-byte aligned");
    if (st->groups.size() != 1) return fail(TCNG_EUNSUPPORTED, "ragged state: call per size class");
    if (n_ops == 0) return TCNG_OK;
    std::lock_guard<std::mutex> lk(g_mu);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    TCNG_TRY({
        const PlanOptions o = plan_options(st->dt, false);
        const int n = st->groups.begin()->first;
        uint64_t key = key_mix(options_key(), 4);
        for (const void* p : {(const void*)st, (const void*)st->buf, params_dev, item_pool_dev})
            key = key_mix(key, reinterpret_cast<uintptr_t>(p));
        key = key_mix(key, ((uint64_t)pool_stride << 16) ^ (uint64_t)P);
        key = key_mix(key, structure_hash(n, ops, n_ops, mat_pool, n_mat, P, o));
        return run_graphed(key, s, [&](cudaStream_t s) -> tcng_status {
            const auto& g = st->groups.begin()->second;
            const int items = (int)g.items.size();
            void* tb = nullptr;
            long long ts = -1;
            group_span(st, g.items, &tb, &ts);
            DevPlan* dp = get_plan(n, ops, n_ops, mat_pool, n_mat, P, o);
            const double* prm = static_cast<const double*>(params_dev);
            const double2* pool = static_cast<const double2*>(item_pool_dev);
            if (st->dt == TCNG_C64)
                return run_plan<float2>(dp, static_cast<float2*>(st->buf), g.d_off, items, prm, s, tb, ts, pool,
                                        (long long)pool_stride);
            return run_plan<double2>(dp, static_cast<double2*>(st->buf), g.d_off, items, prm, s, tb, ts, pool,
                                     (long long)pool_stride);
        });
    })
}

// ------------------------------------------------------------ expectations --
static tcng_status expect_impl(const tcng_state* st, const tcng_pauli* terms, size_t n_terms,
                               double* out_dev, const double* coeffs_dev, double* energy_dev,
                               cudaStream_t s) {
    if (!st) return fail(TCNG_EINVAL, "state is NULL");
    if (n_terms == 0) return TCNG_OK;
    if (!terms) return fail(TCNG_EINVAL, "terms is NULL");
    if (n_terms > 4096) return fail(TCNG_EINVAL, "at most 4096 terms per call");
    std::lock_guard<std::mutex> lk(g_mu);
    TCNG_TRY({
        DeviceCtx& c = ctx();
        const PlanOptions o = plan_options(st->dt, false);
        const bool ragged = st->groups.size() > 1;
        // one size class at a time (a ragged batch has several); results go to the
        // classes' batch rows
        for (const auto& kv : st->groups) {
            const int n = kv.first;
            const tcng_state::Group& grp = kv.second;
            const int items = (int)grp.items.size();
            std::vector<DevPass> passes;
            std::vector<ExpPass> eps;
            std::vector<size_t> wide;   // strings wider than a tile: one global-memory pass each
            plan_expectation(n, o.tile_bits, o.chunk_bits, terms, n_terms, passes, eps, &wide);
            TermSet* ts = get_terms(terms, n_terms, n);
            const int m = passes.empty() ? std::min(o.tile_bits, n) : passes[0].m;
            const long long tpi = 1ll << (n - m);
            const long long want = (num_sms() + items - 1) / items;
            const int nblk = (int)std::max<long long>(1, std::min<long long>(tpi, want));
            double* partial = static_cast<double*>(
                c.scratch("exp_partial", sizeof(double) * (size_t)items * n_terms * nblk));
            if (!partial) return fail(TCNG_ENOMEM, "expectation scratch");
            void* tbase = nullptr;
            long long tstride = -1;
            group_span(st, grp.items, &tbase, &tstride);
            const int es = st->dt == TCNG_C64 ? 8 : 16;
            for (size_t i = 0; i < passes.size(); ++i) {
                cudaError_t e;
                // one tensor copy per tile where the pass's bit runs fit a tensor map
                TmaTile tma{};
                if (items == 1 || tstride > 0) {
                    tma = make_tma_tile(tbase, n, es, passes[i], items, tstride);
                    if (!tma.rank)   // scattered gather bits: four chunks per gather4 copy
                        tma = make_tma_gather4(tbase, st->off[grp.items[0]], n, es, passes[i], items, tstride);
                }
                ProfScope ps(st->dt == TCNG_C64 ? "expect_pass_c64" : "expect_pass_c128", s);
                if (st->dt == TCNG_C64)
                    e = launch_expect_pass<float2>(static_cast<const float2*>(st->buf), grp.d_off, items, n,
                                                   passes[i], eps[i], partial, (int)n_terms, nblk, c.err, s, &tma);
                else
                    e = launch_expect_pass<double2>(static_cast<const double2*>(st->buf), grp.d_off, items, n,
                                                    passes[i], eps[i], partial, (int)n_terms, nblk, c.err, s,
                                                    &tma);
                if (e != cudaSuccess) return cuda_fail(e, "expectation pass");
            }
            for (size_t w : wide) {
                ProfScope ps("expect_wide", s);
                cudaError_t e;
                if (st->dt == TCNG_C64)
                    e = launch_expect_wide<float2>(static_cast<const float2*>(st->buf), grp.d_off, items, n,
                                                   terms[w], (int)w, partial, (int)n_terms, nblk, s);
                else
                    e = launch_expect_wide<double2>(static_cast<const double2*>(st->buf), grp.d_off, items, n,
                                                    terms[w], (int)w, partial, (int)n_terms, nblk, s);
                if (e != cudaSuccess) return cuda_fail(e, "wide expectation pass");
            }
            ProfScope ps("expect_finalize", s);
            cudaError_t e = launch_expect_finalize(partial, nblk, (int)n_terms, out_dev, coeffs_dev, ts->d_c,
                                                   energy_dev, items, s, ragged ? grp.d_items : nullptr);
            if (e != cudaSuccess) return cuda_fail(e, "expectation finalize");
        }
        return TCNG_OK;
    })
}

tcng_status tcng_expect_pauli(const tcng_state* st, const tcng_pauli* terms, size_t n_terms,
                              double* out_dev, void* stream) {
    if (!out_dev) return fail(TCNG_EINVAL, "out_dev is NULL");
    return expect_impl(st, terms, n_terms, out_dev, nullptr, nullptr, static_cast<cudaStream_t>(stream));
}

tcng_status tcng_expect_energy(const tcng_state* st, const tcng_pauli* terms, size_t n_terms,
                               const double* coeffs_dev, double* out_dev, double* energy_dev,
                               void* stream) {
    if (!out_dev || !energy_dev) return fail(TCNG_EINVAL, "out_dev or energy_dev is NULL");
    return expect_impl(st, terms, n_terms, out_dev, coeffs_dev, energy_dev,
                       static_cast<cudaStream_t>(stream));
}

tcng_status tcng_energy(const tcng_state* st, const tcng_pauli* terms, size_t n_terms,
                        const double* coeffs_dev, double* energy_dev, void* stream) {
    if (!energy_dev) return fail(TCNG_EINVAL, "energy_dev is NULL");
    return expect_impl(st, terms, n_terms, nullptr, coeffs_dev, energy_dev,
                       static_cast<cudaStream_t>(stream));
}

tcng_status tcng_hamiltonian_apply(const tcng_state* st, const tcng_pauli* terms, size_t n_terms,
                                   const double* coeffs_dev, tcng_state* out, void* stream) {
    if (!st || !out || (!terms && n_terms)) return fail(TCNG_EINVAL, "null argument");
    if (out->dt != st->dt || out->batch != st->batch || out->n != st->n)
        return fail(TCNG_EINVAL, "output state shape differs");
    std::lock_guard<std::mutex> lk(g_mu);
    TCNG_TRY({
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        const bool ragged = st->groups.size() > 1;
        for (const auto& kv : st->groups) {   // one size class at a time
            const int n = kv.first;
            const tcng_state::Group& gi = kv.second;
            const tcng_state::Group& go = out->groups.at(n);
            TermSet* ts = get_terms(terms, n_terms, n);
            const int items = (int)gi.items.size();
            const int* rows = ragged ? gi.d_items : nullptr;
            cudaError_t e;
            if (st->dt == TCNG_C64)
                e = launch_ham_apply<float2>(static_cast<const float2*>(st->buf), gi.d_off,
                                             static_cast<float2*>(out->buf), go.d_off, items, n, ts->d_h,
                                             (int)n_terms, coeffs_dev, ts->d_c, s, rows);
            else
                e = launch_ham_apply<double2>(static_cast<const double2*>(st->buf), gi.d_off,
                                              static_cast<double2*>(out->buf), go.d_off, items, n, ts->d_h,
                                              (int)n_terms, coeffs_dev, ts->d_c, s, rows);
            if (e != cudaSuccess) return cuda_fail(e, "H apply");
        }
        return TCNG_OK;
    })
}

tcng_status tcng_set_option(tcng_option opt, int value) {
    std::lock_guard<std::mutex> lk(g_mu);
    switch (opt) {
    case TCNG_OPT_FUSE_WIDTH:
        if (value < 1 || value > TCNG_MAX_FUSE) return fail(TCNG_EINVAL, "fuse width 1..5");
        g_opt.fuse_width = value;
        return TCNG_OK;
    case TCNG_OPT_TILE_BITS:
        if (value < 5 || value > 13) return fail(TCNG_EINVAL, "tile bits 5..13");
        g_opt.tile_bits = value;
        return TCNG_OK;
    case TCNG_OPT_CHUNK_BITS:
        if (value < 1 || value > 13) return fail(TCNG_EINVAL, "chunk bits 1..13");
        g_opt.chunk_bits = value;
        return TCNG_OK;
    case TCNG_OPT_USE_GRAPHS:
        g_opt.use_graphs = value ? 1 : 0;
        return TCNG_OK;
    case TCNG_OPT_UNFUSED:
        g_opt.unfused = value ? 1 : 0;
        return TCNG_OK;
    case TCNG_OPT_TENSOR_CORES:
        if (value < 0 || value > 2) return fail(TCNG_EINVAL, "tensor-core option is 0, 1 or 2");
        g_opt.tensor_cores = value;
        return TCNG_OK;
    case TCNG_OPT_STATE_ADJOINT_N:
        if (value < 1 || value > TCNG_MAX_QUBITS + 1) return fail(TCNG_EINVAL, "state-pass adjoint n is 1..35");
        g_opt.state_adjoint_n = value;
        return TCNG_OK;
    case TCNG_OPT_TC_FP16:
        g_opt.tc_fp16 = value ? 1 : 0;
        return TCNG_OK;
    case TCNG_OPT_STATE_ADJOINT_SMALL:
        g_opt.state_adjoint_small = value ? 1 : 0;
        return TCNG_OK;
    }
    return fail(TCNG_EINVAL, "unknown option");
}

tcng_status tcng_get_option(tcng_option opt, int* value) {
    if (!value) return fail(TCNG_EINVAL, "value is NULL");
    switch (opt) {
    case TCNG_OPT_FUSE_WIDTH: *value = g_opt.fuse_width; return TCNG_OK;
    case TCNG_OPT_TILE_BITS: *value = g_opt.tile_bits; return TCNG_OK;
    case TCNG_OPT_CHUNK_BITS: *value = g_opt.chunk_bits; return TCNG_OK;
    case TCNG_OPT_USE_GRAPHS: *value = g_opt.use_graphs; return TCNG_OK;
    case TCNG_OPT_UNFUSED: *value = g_opt.unfused; return TCNG_OK;
    case TCNG_OPT_TENSOR_CORES: *value = g_opt.tensor_cores; return TCNG_OK;
    case TCNG_OPT_STATE_ADJOINT_N: *value = g_opt.state_adjoint_n; return TCNG_OK;
    case TCNG_OPT_TC_FP16: *value = g_opt.tc_fp16; return TCNG_OK;
    case TCNG_OPT_STATE_ADJOINT_SMALL: *value = g_opt.state_adjoint_small; return TCNG_OK;
    }
    return fail(TCNG_EINVAL, "unknown option");
}

tcng_status tcng_sync_status(void) {
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "synchronize");
    DeviceCtx& c = ctx();
    unsigned h = 0;
    if (c.err) {
        cudaMemcpy(&h, c.err, sizeof(unsigned), cudaMemcpyDeviceToHost);
        if (h) {
            cudaMemset(c.err, 0, sizeof(unsigned));
            if (h & ERR_TIMEOUT_FLAG) return fail(TCNG_ETIMEOUT, "a device-side wait timed out");
            return fail(TCNG_EINVAL, "device reported an invalid work item");
        }
    }
    return TCNG_OK;
}

tcng_status tcng_profile_enable(int on) {
    g_prof = on != 0;
    return TCNG_OK;
}

tcng_status tcng_profile_read(char* buf, size_t len, int reset) {
    if (!buf || !len) return fail(TCNG_EINVAL, "buffer is NULL");
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "synchronize");
    std::lock_guard<std::mutex> lk(g_prof_mu);
    std::map<std::string, std::pair<long, double>> agg;
    for (const ProfRec& r : g_prof_recs) {
        float ms = 0;
        cudaEventElapsedTime(&ms, r.e0, r.e1);
        auto& a = agg[r.name];
        a.first += 1;
        a.second += ms;
    }
    std::string out;
    char line[256];
    for (auto& kv : agg) {
        snprintf(line, sizeof line, "%s %ld %.6f\n", kv.first.c_str(), kv.second.first, kv.second.second);
        out += line;
    }
    snprintf(buf, len, "%s", out.c_str());
    if (reset) {
        for (ProfRec& r : g_prof_recs) {
            cudaEventDestroy(r.e0);
            cudaEventDestroy(r.e1);
        }
        g_prof_recs.clear();
    }
    return TCNG_OK;
}

const char* tcng_describe_plan(int n, const tcng_gate* ops, size_t n_ops, const double* mat_pool,
                               size_t n_mat, int P, int adjoint) {
    static thread_local std::string out;
    try {
        Plan pl;
        pl.n = n;
        pl.P = P;
        // the plan a one-item complex64 tcng_apply_circuit would run (or the adjoint's)
        pl.opt = adjoint ? plan_options(TCNG_C64, true) : apply_plan_options(TCNG_C64, 1, P);
        if (n < 5 && !adjoint) pl.opt.unfused = 1;
        pl.ops = import_ops(n, ops, n_ops, n_mat, P, mat_pool);
        build_plan(pl);
        out = describe_plan(pl);
    } catch (const std::exception& ex) {
        out = std::string("error: ") + ex.what();
    }
    return out.c_str();
}

tcng_status tcng_marginal_probs(const tcng_state* st, const int* qubits, int k, double* out_dev,
                                void* stream) {
    if (!st || !qubits || !out_dev) return fail(TCNG_EINVAL, "null argument");
    if (k < 1 || k > 10) return fail(TCNG_EINVAL, "k must be 1..10");
    if (st->groups.size() != 1) return fail(TCNG_EUNSUPPORTED, "ragged state: call per size class");
    const int n = st->n[0];
    uint64_t seen = 0;
    for (int i = 0; i < k; ++i) {
        if (qubits[i] < 0 || qubits[i] >= n) return fail(TCNG_EINVAL, "qubit out of range");
        if ((seen >> qubits[i]) & 1) return fail(TCNG_EINVAL, "repeated qubit");
        seen |= 1ull << qubits[i];
    }
    std::lock_guard<std::mutex> lk(g_mu);
    TCNG_TRY({
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        const int items = st->batch;
        const int splits = marginal_splits(items, n, k);
        double* partial = nullptr;
        if (splits > 1) {
            partial = static_cast<double*>(
                ctx().scratch("marginal", sizeof(double) * ((size_t)items << k) * splits));
            if (!partial) return fail(TCNG_ENOMEM, "marginal scratch");
        }
        ProfScope ps("marginal_probs", s);
        cudaError_t e;
        if (st->dt == TCNG_C64)
            e = launch_marginal<float2>(static_cast<const float2*>(st->buf), st->d_off, items, n, qubits, k,
                                        out_dev, partial, splits, s);
        else
            e = launch_marginal<double2>(static_cast<const double2*>(st->buf), st->d_off, items, n, qubits, k,
                                         out_dev, partial, splits, s);
        if (e != cudaSuccess) return cuda_fail(e, "marginal kernel");
        return TCNG_OK;
    })
}

tcng_status tcng_measure(tcng_state* st, const uint64_t* mask_dev, const double* u_dev, int8_t* outcome_dev,
                         double* logp_dev, void* stream) {
    if (!st || !mask_dev || !u_dev || !outcome_dev) return fail(TCNG_EINVAL, "null argument");
    if (st->groups.size() != 1) return fail(TCNG_EUNSUPPORTED, "ragged state: call per size class");
    std::lock_guard<std::mutex> lk(g_mu);
    TCNG_TRY({
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        const int n = st->n[0];
        const int items = st->batch;
        const int splits = measure_splits(items, n);
        DeviceCtx& c = ctx();
        double* hist = static_cast<double*>(c.scratch("meas_hist", sizeof(double) * 1024 * (size_t)items * splits));
        void* proj = c.scratch("meas_proj", measure_proj_bytes(items));
        if (!hist || !proj) return fail(TCNG_ENOMEM, "measurement scratch");
        ProfScope ps("measure", s);
        cudaError_t e;
        const auto* mk = reinterpret_cast<const unsigned long long*>(mask_dev);
        auto* oc = reinterpret_cast<signed char*>(outcome_dev);
        if (st->dt == TCNG_C64)
            e = launch_measure<float2>(static_cast<float2*>(st->buf), st->d_off, items, n, mk, u_dev, oc, logp_dev,
                                       hist, splits, proj, s);
        else
            e = launch_measure<double2>(static_cast<double2*>(st->buf), st->d_off, items, n, mk, u_dev, oc,
                                        logp_dev, hist, splits, proj, s);
        if (e != cudaSuccess) return cuda_fail(e, "measurement kernels");
        return TCNG_OK;
    })
}

}  // extern "C"
