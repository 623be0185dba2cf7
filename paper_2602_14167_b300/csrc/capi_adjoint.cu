// C ABI: batched energy + adjoint gradient (tcng_energy_grad, tcng_energy_grad_ragged).
//
// Host side of the persistent launch: one plan per circuit structure (adjoint
// mode: parameterised gates stay single blocks), per-item matrix tables built
// by the indexed prologue, a work order (largest n first), per-CTA scratch for
// streamed states, and the launch itself.  The descriptor arrays are cached by
// a hash of the batch layout, so a repeated call with the same structures only
// re-runs the prologue and the persistent kernel.
#include <cuda_runtime.h>
#include <cmath>

#include <algorithm>
#include <numeric>
#include <stdexcept>
#include <string>
#include <vector>

#include "adjoint.hpp"
#include "capi_internal.hpp"

namespace tcng {

struct AdjLayout {
    std::vector<DevPlan*> plans;
    std::vector<TermSet*> termsets;
    std::vector<StructDesc> hs;        // host copies
    std::vector<int> item_struct;
    std::vector<long long> prm_off, coeff_off, tab_off;
    std::vector<std::vector<int>> struct_items;
    StructDesc* d_structs = nullptr;
    ItemDesc* d_items = nullptr;
    int* d_order = nullptr;
    DevPass** d_passes = nullptr;      // per structure
    std::vector<DevPass*> pass_bufs;
    std::vector<long long*> d_prm_off, d_tab_off;   // per structure, its items
    long long table_elems = 0;
    int res_bits = 0;
    int max_stream_n = 0;
    ~AdjLayout() {
        cudaFree(d_structs);
        cudaFree(d_items);
        cudaFree(d_order);
        for (DevPass* p : pass_bufs) cudaFree(p);
        for (long long* p : d_prm_off) cudaFree(p);
        for (long long* p : d_tab_off) cudaFree(p);
    }
};

static std::unordered_map<uint64_t, std::unique_ptr<AdjLayout>>& layouts() {
    static std::unordered_map<uint64_t, std::unique_ptr<AdjLayout>> m;
    return m;
}

static uint64_t fnv(uint64_t h, const void* p, size_t len) {
    const unsigned char* b = static_cast<const unsigned char*>(p);
    for (size_t i = 0; i < len; ++i) {
        h ^= b[i];
        h *= 1099511628211ULL;
    }
    return h;
}

static AdjLayout* get_layout(const tcng_problem* probs, int n_probs, const int* item_problem,
                             int batch, tcng_dtype dt, const long long* psi_off) {
    const PlanOptions base = plan_options(dt, true);
    const int res_bits = dt == TCNG_C64 ? 13 : 12;
    const int stream_tile = res_bits;   // streamed psi and lambda tiles use the two resident buffers
    uint64_t h = 1469598103934665603ULL;
    std::vector<uint64_t> shash(n_probs);
    for (int s = 0; s < n_probs; ++s) {
        const tcng_problem& p = probs[s];
        if (p.n < 1 || p.n > 20) throw std::invalid_argument("adjoint: qubit count must be 1..20");
        if (p.P < 0) throw std::invalid_argument("adjoint: P < 0");
        shash[s] = structure_hash(p.n, p.ops, p.n_ops, p.mat_pool, p.n_mat, p.P, base);
        shash[s] = fnv(shash[s], p.H, sizeof(tcng_pauli) * p.n_terms);
        h = fnv(h, &shash[s], 8);
    }
    h = fnv(h, item_problem, sizeof(int) * batch);
    h = fnv(h, &dt, sizeof dt);
    const int has_psi = psi_off ? 1 : 0;
    h = fnv(h, &has_psi, sizeof has_psi);
    if (psi_off) h = fnv(h, psi_off, sizeof(long long) * batch);
    h = fnv(h, &base, sizeof base);
    auto& L = layouts();
    auto it = L.find(h);
    if (it != L.end()) return it->second.get();

    std::unique_ptr<AdjLayout> lay(new AdjLayout());
    lay->res_bits = res_bits;
    lay->struct_items.resize(n_probs);
    for (int s = 0; s < n_probs; ++s) {
        const tcng_problem& p = probs[s];
        const int n_eff = std::max(p.n, 5);
        const bool resident = n_eff <= res_bits;
        import_ops(p.n, p.ops, p.n_ops, p.n_mat, p.P, p.mat_pool);   // validate against the real n
        PlanOptions o = base;
        o.tile_bits = resident ? n_eff : stream_tile;
        o.chunk_bits = std::min(o.chunk_bits, o.tile_bits);
        o.unfused = 0;
        DevPlan* dp = get_plan(n_eff, p.ops, p.n_ops, p.mat_pool, p.n_mat, p.P, o);
        TermSet* ts = get_terms(p.H, p.n_terms, p.n);
        lay->plans.push_back(dp);
        lay->termsets.push_back(ts);
        if (!resident) lay->max_stream_n = std::max(lay->max_stream_n, n_eff);
        StructDesc sd{};
        sd.n = p.n;
        sd.n_eff = n_eff;
        sd.resident = resident ? 1 : 0;
        sd.P = p.P;
        sd.n_terms = (int)p.n_terms;
        sd.n_passes = (int)dp->plan.passes.size();
        sd.n_grad = dp->plan.n_grad;
        sd.table_size = dp->plan.table_size;
        DevPass* dpass = dev_copy(dp->plan.passes);
        lay->pass_bufs.push_back(dpass);
        sd.passes = dpass;
        sd.stages = dp->d_stages;
        sd.dops = dp->d_dops;
        sd.terms = ts->d_h;
        sd.tcoef = ts->d_c;
        sd.gparam = dp->d_gparam;
        sd.gscale = dp->d_gscale;
        lay->hs.push_back(sd);
    }
    std::vector<ItemDesc> items(batch);
    long long po = 0, co = 0, to = 0;
    lay->prm_off.resize(batch);
    lay->coeff_off.resize(batch);
    lay->tab_off.resize(batch);
    for (int b = 0; b < batch; ++b) {
        const int s = item_problem[b];
        if (s < 0 || s >= n_probs) throw std::invalid_argument("item_problem out of range");
        ItemDesc d{};
        d.s = s;
        d.param_off = po;
        d.coeff_off = co;
        d.grad_off = po;
        d.table_off = to;
        d.psi_out_off = psi_off ? psi_off[b] : -1;
        lay->prm_off[b] = po;
        lay->coeff_off[b] = co;
        lay->tab_off[b] = to;
        po += probs[s].P;
        co += (long long)probs[s].n_terms;
        to += std::max(1, lay->hs[s].table_size);
        items[b] = d;
        lay->struct_items[s].push_back(b);
    }
    lay->table_elems = to;
    std::vector<int> order(batch);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        return lay->hs[items[a].s].n_eff > lay->hs[items[b].s].n_eff;
    });
    for (int s = 0; s < n_probs; ++s) {
        std::vector<long long> pv, tv;
        for (int b : lay->struct_items[s]) {
            pv.push_back(lay->prm_off[b]);
            tv.push_back(lay->tab_off[b]);
        }
        lay->d_prm_off.push_back(dev_copy(pv));
        lay->d_tab_off.push_back(dev_copy(tv));
    }
    lay->d_structs = dev_copy(lay->hs);
    lay->d_items = dev_copy(items);
    lay->d_order = dev_copy(order);
    AdjLayout* raw = lay.get();
    L[h] = std::move(lay);
    return raw;
}

template <typename C>
static tcng_status run_adjoint(AdjLayout* lay, int batch, const double* params, const double* coeffs,
                               double* energy, double* grad, void* psi_out, bool want_grad,
                               cudaStream_t s) {
    DeviceCtx& c = ctx();
    C* tables = static_cast<C*>(c.scratch("adj_tables", sizeof(C) * std::max<long long>(1, lay->table_elems)));
    if (!tables) return fail(TCNG_ENOMEM, "adjoint matrix tables");
    for (size_t si = 0; si < lay->plans.size(); ++si) {
        const int cnt = (int)lay->struct_items[si].size();
        if (!cnt) continue;
        DevPlan* dp = lay->plans[si];
        ProfScope ps("build_matrices", s);
        cudaError_t e = launch_build_matrices_indexed<C>(dp->d_bblocks, (int)dp->plan.bblocks.size(),
                                                         dp->d_bops, dp->d_pool, params, tables,
                                                         lay->d_prm_off[si], lay->d_tab_off[si], cnt, s);
        if (e != cudaSuccess) return cuda_fail(e, "adjoint prologue");
    }
    const int grid = std::min(batch, num_sms());
    const long long selems = lay->max_stream_n ? (1ll << lay->max_stream_n) : 0;
    void* scratch = nullptr;
    if (selems) {
        scratch = c.scratch("adj_states", sizeof(C) * 2 * selems * grid);
        if (!scratch) return fail(TCNG_ENOMEM, "adjoint state scratch");
    }
    int* counter = static_cast<int*>(c.scratch("adj_counter", sizeof(int)));
    if (!counter) return fail(TCNG_ENOMEM, "adjoint counter");
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(int), s);
    if (e != cudaSuccess) return cuda_fail(e, "counter reset");
    AdjArgs a{};
    a.structs = lay->d_structs;
    a.items = lay->d_items;
    a.order = lay->d_order;
    a.batch = batch;
    a.res_bits = lay->res_bits;
    a.want_grad = want_grad ? 1 : 0;
    a.counter = counter;
    a.tables = tables;
    a.coeffs = coeffs;
    a.energy = energy;
    a.grad = grad;
    a.psi_out = psi_out;
    a.scratch = scratch;
    a.scratch_elems = selems;
    a.err = c.err;
    ProfScope ps(sizeof(C) == 8 ? "adjoint_kernel_c64" : "adjoint_kernel_c128", s);
    e = launch_adjoint<C>(a, grid, s);
    if (e != cudaSuccess) return cuda_fail(e, "adjoint kernel");
    return TCNG_OK;
}

// Cost model of the two adjoint paths for a batch of one size class (measured on
// a B300, TFIM ring ansatz, 12 layers): the per-item kernel runs one item per
// CTA, so its time is ceil(batch / SMs) x t_item(n); the state-pass adjoint takes
// the items one after another on the whole GPU, batch x t_state(n).  t_item /
// t_state: complex64 about 1.8 x 1.95^(n - 14) (0.74 / 1.0 ms at 12 qubits, 9.5 /
// 1.4 at 16, 197 / 2.1 at 20 for one item); complex128 about 4.8 x 2^(n - 14), at
// most 99 (37.6 / 7.8 ms at 14, 770 / 10.1 at 18, 3422 / 34.6 at 20).
bool state_path_faster(int n, int batch, int sms, bool c128) {
    if (n < 14) return false;
    const double ratio = c128 ? std::min(99.0, 4.8 * std::pow(2.0, n - 14)) : 1.8 * std::pow(1.95, n - 14);
    const double waves = (double)((batch + sms - 1) / std::max(1, sms));
    return (double)batch < waves * ratio;
}

}  // namespace tcng

using namespace tcng;

extern "C" {

tcng_status tcng_energy_grad(tcng_state* st, const tcng_gate* ops, size_t n_ops,
                             const double* mat_pool, size_t n_mat, const void* params_dev, int P,
                             const tcng_pauli* H, size_t n_terms, const double* coeffs_dev,
                             double* energy_dev, double* grad_dev, void* stream) {
    if (!st || !energy_dev) return fail(TCNG_EINVAL, "null argument");
    if (P > 0 && (!params_dev || !grad_dev)) return fail(TCNG_EINVAL, "params_dev/grad_dev is NULL");
    if (st->groups.size() != 1)
        return fail(TCNG_EUNSUPPORTED, "ragged state: use tcng_energy_grad_ragged");
    std::lock_guard<std::mutex> lk(g_mu);
    try {
        // single large states, and circuits with Pauli-word rotation parameters,
        // take the state-pass adjoint (one pass over psi and lambda per fused run of blocks)
        bool state_path = st->n[0] >= g_opt.state_adjoint_n ||
                          (g_opt.state_adjoint_small &&
                           state_path_faster(st->n[0], st->batch, num_sms(), st->dt == TCNG_C128));
        for (size_t i = 0; i < n_ops && !state_path; ++i)
            state_path = ops && ops[i].op == TCNG_RP && ops[i].param >= 0;
        if (state_path) {
            const double* prm = static_cast<const double*>(params_dev);
            uint64_t key = key_mix(options_key(), 5);
            for (const void* p : {(const void*)st, (const void*)st->buf, params_dev, (const void*)coeffs_dev,
                                  (const void*)energy_dev, (const void*)grad_dev})
                key = key_mix(key, reinterpret_cast<uintptr_t>(p));
            key = key_mix(key, structure_hash(st->n[0], ops, n_ops, mat_pool, n_mat, P, plan_options(st->dt, false)));
            for (size_t t = 0; t < n_terms; ++t)
                key = key_mix(key_mix(key, H[t].xmask ^ (H[t].zmask << 1)), (uint64_t)t);
            return run_graphed(key, static_cast<cudaStream_t>(stream), [&](cudaStream_t s) -> tcng_status {
                for (int b = 0; b < st->batch; ++b) {
                    const tcng_status r =
                        st->dt == TCNG_C64
                            ? run_state_adjoint<float2>(st, b, ops, n_ops, mat_pool, n_mat, prm + (size_t)b * P, P,
                                                        H, n_terms, coeffs_dev ? coeffs_dev + (size_t)b * n_terms : nullptr,
                                                        energy_dev + b, P > 0 ? grad_dev + (size_t)b * P : nullptr, s)
                            : run_state_adjoint<double2>(st, b, ops, n_ops, mat_pool, n_mat, prm + (size_t)b * P, P,
                                                         H, n_terms, coeffs_dev ? coeffs_dev + (size_t)b * n_terms : nullptr,
                                                         energy_dev + b, P > 0 ? grad_dev + (size_t)b * P : nullptr, s);
                    if (r) return r;
                }
                return TCNG_OK;
            });
        }
        tcng_problem pr{};
        pr.n = st->n[0];
        pr.ops = ops;
        pr.n_ops = n_ops;
        pr.mat_pool = mat_pool;
        pr.n_mat = n_mat;
        pr.P = P;
        pr.H = H;
        pr.n_terms = n_terms;
        std::vector<int> ip(st->batch, 0);
        AdjLayout* lay = get_layout(&pr, 1, ip.data(), st->batch, st->dt, st->off.data());
        const double* prm = static_cast<const double*>(params_dev);
        uint64_t key = key_mix(options_key(), 2);
        for (const void* p : {(const void*)lay, (const void*)st->buf, params_dev, (const void*)coeffs_dev,
                              (const void*)energy_dev, (const void*)grad_dev})
            key = key_mix(key, reinterpret_cast<uintptr_t>(p));
        key = key_mix(key, ((uint64_t)st->batch << 32) | (uint32_t)P);
        const tcng_dtype dt = st->dt;
        const int batch = st->batch;
        void* buf = st->buf;
        return run_graphed(key, static_cast<cudaStream_t>(stream), [&](cudaStream_t s) -> tcng_status {
            if (dt == TCNG_C64)
                return run_adjoint<float2>(lay, batch, prm, coeffs_dev, energy_dev, grad_dev, buf, P > 0, s);
            return run_adjoint<double2>(lay, batch, prm, coeffs_dev, energy_dev, grad_dev, buf, P > 0, s);
        });
    } catch (const std::invalid_argument& ex) {
        return fail(TCNG_EINVAL, ex.what());
    } catch (const std::bad_alloc&) {
        return fail(TCNG_ENOMEM, "allocation failed");
    } catch (const std::exception& ex) {
        return fail(TCNG_EINVAL, ex.what());
    }
}

tcng_status tcng_energy_grad_ragged(const tcng_problem* problems, int n_problems,
                                    const int* item_problem, int batch, const double* params_dev,
                                    const double* coeffs_dev, double* energy_dev, double* grad_dev,
                                    void* stream) {
    if (!problems || n_problems < 1 || !item_problem || batch < 1 || !energy_dev)
        return fail(TCNG_EINVAL, "null or empty argument");
    bool any_p = false;
    for (int s = 0; s < n_problems; ++s) any_p = any_p || problems[s].P > 0;
    if (any_p && (!params_dev || !grad_dev)) return fail(TCNG_EINVAL, "params_dev/grad_dev is NULL");
    for (int s = 0; s < n_problems; ++s)
        for (size_t i = 0; i < problems[s].n_ops; ++i)
            if (problems[s].ops && problems[s].ops[i].op == TCNG_RP && problems[s].ops[i].param >= 0)
                return fail(TCNG_EUNSUPPORTED, "ragged batches: RP parameters need tcng_energy_grad");
    std::lock_guard<std::mutex> lk(g_mu);
    try {
        AdjLayout* lay = get_layout(problems, n_problems, item_problem, batch, TCNG_C64, nullptr);
        uint64_t key = key_mix(options_key(), 3);
        for (const void* p : {(const void*)lay, (const void*)params_dev, (const void*)coeffs_dev,
                              (const void*)energy_dev, (const void*)grad_dev})
            key = key_mix(key, reinterpret_cast<uintptr_t>(p));
        key = key_mix(key, (uint64_t)batch);
        return run_graphed(key, static_cast<cudaStream_t>(stream), [&](cudaStream_t s) -> tcng_status {
            return run_adjoint<float2>(lay, batch, params_dev, coeffs_dev, energy_dev, grad_dev, nullptr,
                                       any_p, s);
        });
    } catch (const std::invalid_argument& ex) {
        return fail(TCNG_EINVAL, ex.what());
    } catch (const std::bad_alloc&) {
        return fail(TCNG_ENOMEM, "allocation failed");
    } catch (const std::exception& ex) {
        return fail(TCNG_EINVAL, ex.what());
    }
}

}  // extern "C"
