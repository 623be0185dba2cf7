// Host planner: IR validation, gate fusion, tile-pass scheduling, stage building.
//
// The paper compiles a circuit once per structure (Sec. I.B "Paradigms: JIT",
// the contraction path and gradient graph are traced once); the analogue here is
// a plan built once per structure hash and cached by the C ABI layer.
#include <algorithm>
#include <functional>
#include <unordered_map>
#include <cmath>
#include <cstring>
#include <sstream>
#include <stdexcept>

#include "internal.hpp"

namespace tcng {

static int popc64(uint64_t v) { return __builtin_popcountll(v); }

static int op_arity(int code, int nq) {
    switch (code) {
    case TCNG_I: case TCNG_X: case TCNG_Y: case TCNG_Z: case TCNG_H: case TCNG_S: case TCNG_T:
    case TCNG_RX: case TCNG_RY: case TCNG_RZ: case TCNG_U1:
        return 1;
    case TCNG_CX: case TCNG_CZ: case TCNG_CP: case TCNG_SWAP: case TCNG_RZZ: case TCNG_U2:
        return 2;
    case TCNG_UK: case TCNG_RP:
        return (nq >= 1 && nq <= TCNG_MAX_FUSE) ? nq : -1;
    default:
        return -1;
    }
}

static bool is_param_code(int code) {
    return code == TCNG_RX || code == TCNG_RY || code == TCNG_RZ || code == TCNG_RZZ ||
           code == TCNG_CP || code == TCNG_RP;
}

std::vector<HostOp> import_ops(int n, const tcng_gate* ops, size_t n_ops, size_t n_mat, int P,
                               const double* pool) {
    if (n < 1 || n > TCNG_MAX_QUBITS) throw std::invalid_argument("qubit count out of range");
    if (n_ops && !ops) throw std::invalid_argument("ops is NULL");
    if (n_mat && !pool) throw std::invalid_argument("mat_pool is NULL");
    std::vector<HostOp> out;
    out.reserve(n_ops);
    for (size_t i = 0; i < n_ops; ++i) {
        const tcng_gate& g = ops[i];
        HostOp h{};
        h.code = g.op;
        h.k = op_arity(g.op, g.nq);
        std::ostringstream where;
        where << "gate " << i << ": ";
        if (h.k < 0) throw std::invalid_argument(where.str() + "unknown op or bad nq");
        if (g.nq != h.k) throw std::invalid_argument(where.str() + "nq does not match op");
        for (int j = 0; j < h.k; ++j) {
            h.q[j] = g.q[j];
            if (g.q[j] < 0 || g.q[j] >= n) throw std::invalid_argument(where.str() + "qubit out of range");
            for (int l = 0; l < j; ++l)
                if (g.q[l] == g.q[j]) throw std::invalid_argument(where.str() + "repeated qubit");
        }
        h.param = g.param < 0 ? -1 : g.param;
        if (g.param >= P) throw std::invalid_argument(where.str() + "param index >= P");
        if (g.param >= 0 && !is_param_code(g.op))
            throw std::invalid_argument(where.str() + "only RX/RY/RZ/RZZ/CP/RP take a parameter");
        h.scale = g.scale;
        h.angle0 = g.angle0;
        if (!std::isfinite(g.scale) || !std::isfinite(g.angle0))
            throw std::invalid_argument(where.str() + "non-finite angle");
        h.mat_off = -1;
        h.unitary = true;
        if (g.op == TCNG_U1 || g.op == TCNG_U2 || g.op == TCNG_UK) {
            int64_t need = int64_t(1) << (2 * h.k);
            if (g.mat_off < 0 || size_t(g.mat_off + need) > n_mat)
                throw std::invalid_argument(where.str() + "matrix outside the pool");
            h.mat_off = g.mat_off;
        }
        if (g.op == TCNG_RP) {   // mat_off holds the Pauli word, 2 bits per qubit
            if (g.mat_off < 0 || g.mat_off >= (int64_t(1) << (2 * h.k)))
                throw std::invalid_argument(where.str() + "Pauli word out of range");
            h.mat_off = g.mat_off;
        }
        switch (g.op) {
        case TCNG_I: case TCNG_Z: case TCNG_S: case TCNG_T: case TCNG_RZ: case TCNG_CZ:
        case TCNG_CP: case TCNG_RZZ:
            h.diag = true;
            break;
        case TCNG_RP: {   // diagonal iff every factor is I or Z
            bool dg = true;
            for (int j = 0; j < h.k; ++j) {
                const int w = (int)((g.mat_off >> (2 * j)) & 3);
                dg = dg && (w == 0 || w == 3);
            }
            h.diag = dg;
            break;
        }
        case TCNG_U1: case TCNG_U2: case TCNG_UK: {
            int d = 1 << h.k;
            bool dg = true;
            for (int r = 0; r < d && dg; ++r)
                for (int c = 0; c < d; ++c)
                    if (r != c && (pool[2 * (h.mat_off + r * d + c)] != 0.0 ||
                                   pool[2 * (h.mat_off + r * d + c) + 1] != 0.0)) {
                        dg = false;
                        break;
                    }
            h.diag = dg;
            // unitary to 1e-9 (U^dagger U = I); only then may row norms be restored
            double dev = 0.0;
            for (int r = 0; r < d; ++r)
                for (int c = 0; c < d; ++c) {
                    double re = 0.0, im = 0.0;
                    for (int l = 0; l < d; ++l) {
                        const double* a = pool + 2 * (h.mat_off + l * d + r);
                        const double* b = pool + 2 * (h.mat_off + l * d + c);
                        re += a[0] * b[0] + a[1] * b[1];
                        im += a[0] * b[1] - a[1] * b[0];
                    }
                    dev = std::max(dev, std::hypot(re - (r == c ? 1.0 : 0.0), im));
                }
            h.unitary = dev < 1e-9;
            break;
        }
        default:
            h.diag = false;
        }
        out.push_back(h);
    }
    return out;
}

uint64_t structure_hash(int n, const tcng_gate* ops, size_t n_ops, const double* pool,
                        size_t n_mat, int P, const PlanOptions& opt) {
    uint64_t h = 1469598103934665603ULL;
    auto mix = [&](const void* p, size_t len) {
        const unsigned char* b = static_cast<const unsigned char*>(p);
        for (size_t i = 0; i < len; ++i) {
            h ^= b[i];
            h *= 1099511628211ULL;
        }
    };
    mix(&n, sizeof n);
    mix(&P, sizeof P);
    mix(&opt, sizeof opt);
    mix(&n_ops, sizeof n_ops);
    for (size_t i = 0; i < n_ops; ++i) {
        const tcng_gate& g = ops[i];
        mix(&g.op, 2);
        mix(&g.nq, 1);
        mix(g.q, sizeof(int32_t) * 5);
        mix(&g.param, 4);
        mix(&g.scale, 8);
        mix(&g.angle0, 8);
        mix(&g.mat_off, 8);
    }
    mix(&n_mat, sizeof n_mat);
    if (n_mat) mix(pool, sizeof(double) * 2 * n_mat);
    return h;
}

// ---------------------------------------------------------------- fusion --
// Order-preserving greedy fusion: a gate joins the most recent block touching
// any of its qubits if the union stays within the width; since that block is
// the latest on every qubit of the gate, the gate only moves across blocks on
// disjoint qubits, which commute with it.
static void fuse(Plan& plan) {
    const PlanOptions& o = plan.opt;
    std::vector<int> last(64, -1);
    std::vector<char> closed;
    plan.blocks.clear();
    for (int i = 0; i < (int)plan.ops.size(); ++i) {
        const HostOp& op = plan.ops[i];
        uint64_t qm = 0;
        int B = -1;
        for (int j = 0; j < op.k; ++j) {
            qm |= 1ULL << op.q[j];
            B = std::max(B, last[op.q[j]]);
        }
        bool lone = o.adjoint && op.param >= 0;
        bool join = !o.unfused && !lone && B >= 0 && !closed[B] &&
                    popc64(plan.blocks[B].qmask | qm) <= o.fuse_width;
        if (join) {
            Block& b = plan.blocks[B];
            b.qmask |= qm;
            b.ops.push_back(i);
            b.diag = b.diag && op.diag;
        } else {
            Block b;
            b.qmask = qm;
            b.ops.push_back(i);
            b.diag = op.diag;
            if (lone) {
                b.param_single = true;
                b.param = op.param;
                b.scale = op.scale;
                switch (op.code) {
                case TCNG_RX: b.grad = G_X; b.grad_factor = 1.0; break;
                case TCNG_RY: b.grad = G_Y; b.grad_factor = 1.0; break;
                case TCNG_RZ: b.grad = G_Z; b.grad_factor = 1.0; break;
                case TCNG_RZZ: b.grad = G_ZZ; b.grad_factor = 1.0; break;
                case TCNG_CP: b.grad = G_P11; b.grad_factor = -2.0; break;
                default: break;
                }
            }
            plan.blocks.push_back(b);
            closed.push_back(lone || o.unfused ? 1 : 0);
            B = (int)plan.blocks.size() - 1;
        }
        for (int j = 0; j < op.k; ++j) last[op.q[j]] = B;
    }
    for (Block& b : plan.blocks) {
        b.k = popc64(b.qmask);
        b.size = b.diag ? (1 << b.k) : (1 << (2 * b.k));
    }
}

// Predecessor blocks (the previous block on each qubit).
static std::vector<std::vector<int>> block_deps(const Plan& plan) {
    std::vector<std::vector<int>> deps(plan.blocks.size());
    std::vector<int> last(64, -1);
    for (int b = 0; b < (int)plan.blocks.size(); ++b) {
        uint64_t m = plan.blocks[b].qmask;
        while (m) {
            int q = __builtin_ctzll(m);
            m &= m - 1;
            if (last[q] >= 0 &&
                std::find(deps[b].begin(), deps[b].end(), last[q]) == deps[b].end())
                deps[b].push_back(last[q]);
            last[q] = b;
        }
    }
    return deps;
}

// Simulate one pass with gather set G (bits >= low): which unplaced blocks run.
static std::vector<int> simulate_pass(const Plan& plan, const std::vector<std::vector<int>>& deps,
                                      const std::vector<char>& placed, uint64_t S_fixed,
                                      uint64_t* Gio, int gmax, bool grow, int low,
                                      int mat_budget) {
    uint64_t G = *Gio;
    uint64_t lowmask = (low >= 64) ? ~0ULL : ((1ULL << low) - 1);
    std::vector<char> inpass(plan.blocks.size(), 0);
    std::vector<int> taken;
    int mat = 0;
    for (int b = 0; b < (int)plan.blocks.size(); ++b) {
        if (placed[b]) continue;
        bool ok = true;
        for (int d : deps[b])
            if (!placed[d] && !inpass[d]) { ok = false; break; }
        if (!ok) continue;
        const Block& blk = plan.blocks[b];
        if (mat + blk.size > mat_budget) break;
        if (!blk.diag) {
            uint64_t hi = blk.qmask & ~lowmask & ~S_fixed;
            if ((hi & ~G) != 0) {
                if (!grow || popc64(G | hi) > gmax) continue;
                G |= hi;
            }
        }
        inpass[b] = 1;
        taken.push_back(b);
        mat += blk.size;
    }
    *Gio = G;
    return taken;
}

static int pass_work(const Plan& plan, const std::vector<int>& taken) {
    int w = 0;
    for (int b : taken) w += plan.blocks[b].diag ? 1 : 8;
    return w;
}

void build_plan(Plan& plan) {
    const PlanOptions& o = plan.opt;
    const int n = plan.n;
    plan.all_unitary = true;
    for (const HostOp& h : plan.ops) plan.all_unitary = plan.all_unitary && h.unitary;
    fuse(plan);
    plan.passes.clear();
    plan.stages.clear();
    plan.dops.clear();
    plan.pass_blocks.clear();
    plan.pass_block_begin.clear();
    plan.grad_param.clear();
    plan.grad_scale.clear();
    plan.n_grad = 0;
    if (o.unfused) {
        int off = 0;
        for (Block& b : plan.blocks) {
            b.out_off = off;
            off += b.size;
        }
        plan.table_size = off;
    } else {
        const int m = std::min(o.tile_bits, n);
        const int low = std::min(o.chunk_bits, m);
        const int gmax = m - low;
        if (m < kRegBits + 1) throw std::invalid_argument("state too small for tile passes");
        auto deps = block_deps(plan);
        std::vector<char> placed(plan.blocks.size(), 0);
        size_t n_placed = 0;
        int off = 0;
        const int budget = kMaxPassMat;
        for (const Block& b : plan.blocks)
            if (b.size > budget) throw std::invalid_argument("fused block too large");
        while (n_placed < plan.blocks.size()) {
            uint64_t bestG = 0;
            std::vector<int> best;
            int bestw = -1;
            if (n <= m) {
                bestG = 0;
                best = simulate_pass(plan, deps, placed, ~0ULL, &bestG, 0, false, 64, budget);
            } else {
                // candidate 1: grow from the frontier
                uint64_t G = 0;
                auto t = simulate_pass(plan, deps, placed, 0, &G, gmax, true, low, budget);
                int w = pass_work(plan, t);
                if (w > bestw) { bestw = w; best = t; bestG = G; }
                // candidates 2: contiguous windows of gather bits
                for (int a = low; a + gmax <= n; ++a) {
                    uint64_t Gw = (gmax >= 64 ? ~0ULL : ((1ULL << gmax) - 1)) << a;
                    auto tw = simulate_pass(plan, deps, placed, 0, &Gw, gmax, false, low, budget);
                    int ww = pass_work(plan, tw);
                    if (ww > bestw) { bestw = ww; best = tw; bestG = Gw; }
                }
            }
            if (best.empty()) throw std::runtime_error("planner made no progress");
            // tile qubit set S: low bits + gather, padded with the smallest free bits
            uint64_t S;
            if (n <= m) {
                S = (n >= 64) ? ~0ULL : ((1ULL << n) - 1);
            } else {
                S = ((1ULL << low) - 1) | bestG;
                for (int q = low; q < n && popc64(S) < m; ++q) S |= 1ULL << q;
            }
            DevPass dp{};
            dp.m = popc64(S);
            int tb_of_q[64];
            for (int q = 0; q < 64; ++q) tb_of_q[q] = -1;
            {
                int i = 0;
                for (int q = 0; q < n; ++q)
                    if ((S >> q) & 1) tb_of_q[q] = i++;
                int L = 0;
                while (L < n && ((S >> L) & 1)) ++L;
                dp.chunk = std::min(L, dp.m);
                dp.ngather = dp.m - dp.chunk;
                if (dp.ngather > kMaxGather) throw std::invalid_argument("too many gather bits");
                int gi = 0, ri = 0;
                for (int q = dp.chunk; q < n; ++q) {
                    if ((S >> q) & 1) dp.gather[gi++] = (uint8_t)q;
                    else dp.rest[ri++] = (uint8_t)q;
                }
                dp.nrest = ri;
            }
            plan.pass_block_begin.push_back((int)plan.pass_blocks.size());
            dp.mat_begin = off;
            const std::vector<int>& pass_list = best;
            for (int b : pass_list) {
                placed[b] = 1;
                ++n_placed;
            }
            // ---- stages: list scheduling with register-set affinity ----
            // schedule(SB, out): the pass's blocks into register stages of SB tile bits
            // (kMaxRegBits for a stage that holds a 5-qubit block); records each
            // stage's register set (padded with the highest free tile bits) and blocks
            struct Staged {
                uint32_t R;
                int cap;
                std::vector<int> blocks;
            };
            std::vector<std::vector<int>> pdeps(plan.blocks.size());
            {
                std::vector<char> inp(plan.blocks.size(), 0);
                for (int b : pass_list) inp[b] = 1;
                for (int b : pass_list)
                    for (int d : deps[b])
                        if (inp[d]) pdeps[b].push_back(d);
            }
            // tile-bit mask of each block of the pass
            std::vector<uint32_t> tbm_of(plan.blocks.size(), 0);
            for (int b : pass_list) {
                uint64_t qm = plan.blocks[b].qmask;
                while (qm) {
                    int q = __builtin_ctzll(qm);
                    qm &= qm - 1;
                    tbm_of[b] |= 1u << tb_of_q[q];
                }
            }
            auto schedule = [&](const int SB, std::vector<Staged>& out) {
            std::vector<char> done(plan.blocks.size(), 0);
            size_t left = pass_list.size();
            uint32_t Rset = 0;  // tile-bit mask
            int Rcap = SB;
            int cur_grads = 0;
            std::vector<int> cur;
            auto close_stage = [&]() {
                if (cur.empty()) return;
                // pad register set with the highest free tile bits
                for (int tb = dp.m - 1; tb >= 0 && __builtin_popcount(Rset) < Rcap; --tb)
                    Rset |= 1u << tb;
                out.push_back(Staged{Rset, Rcap, cur});
                cur.clear();
                Rset = 0;
                Rcap = SB;
                cur_grads = 0;
            };
            bool small_blocks = !o.adjoint;   // the register-set search below: <= SB-qubit blocks
            for (int b : pass_list)
                if (!plan.blocks[b].diag && __builtin_popcount(tbm_of[b]) > SB) small_blocks = false;
            // Register sets of the stages: for passes of up to 12 dense blocks, the
            // fewest stages (a stage costs about the same whatever it holds on the
            // tensor-core passes).  A stage with register set R takes every block that
            // becomes ready and fits R (taking more never hurts the rest), so the search
            // runs over sets of placed blocks, memoised; ties prefer sets without tile
            // bits 0..3 (no slot rotation).  Larger passes grow stages greedily.
            std::vector<int> dense_ids;   // pass blocks by local index
            for (int b : pass_list) dense_ids.push_back(b);
            const int nbk = (int)dense_ids.size();
            int n_dense_pass = 0;
            for (int b : pass_list) n_dense_pass += plan.blocks[b].diag ? 0 : 1;
            bool search = small_blocks && nbk <= 64 && n_dense_pass <= 12;
            std::vector<uint64_t> pdep_mask(nbk, 0);
            {
                std::vector<int> local(plan.blocks.size(), -1);
                for (int i = 0; i < nbk; ++i) local[dense_ids[i]] = i;
                for (int i = 0; i < nbk; ++i)
                    for (int d : pdeps[dense_ids[i]]) pdep_mask[i] |= 1ULL << local[d];
            }
            const uint64_t all_mask = nbk >= 64 ? ~0ULL : ((1ULL << nbk) - 1);
            auto closure = [&](uint64_t dm, uint32_t R) {
                for (bool prog = true; prog;) {
                    prog = false;
                    for (int i = 0; i < nbk; ++i) {
                        if ((dm >> i) & 1) continue;
                        if ((pdep_mask[i] & ~dm) != 0) continue;
                        const int b = dense_ids[i];
                        if (plan.blocks[b].diag || (tbm_of[b] & ~R) == 0) {
                            dm |= 1ULL << i;
                            prog = true;
                        }
                    }
                }
                return dm;
            };
            // Tie-break between stagings of equal length: the shared-memory bank
            // conflicts of the stages.  A stage on tile bits 0..3 reads its slots from a
            // 128-byte-swizzled tile, where a float2's bank slot (16 per 128 bytes) has bit
            // 0 = tile bit 0 and bit k = tile bit k xor tile bit k + 3 (k = 1..3); a warp's
            // lanes take the five lowest tile bits outside R, and 16-byte pair reads (tile
            // bit 0 in R) need only slot bits 1..3.  Each slot bit the lanes miss doubles
            // the wavefronts.  Stages off tile bits 0..3 cost nothing.
            auto stage_cost = [&](uint32_t R) -> int {
                if (!(R & 0xFu)) return 0;
                const uint32_t need_mask = (R & 1u) ? 0xEu : 0xFu;
                uint32_t basis[4] = {0, 0, 0, 0};
                int rank = 0, nl = 0;
                for (int tb = 0; tb < dp.m && nl < 5; ++tb) {
                    if ((R >> tb) & 1) continue;
                    ++nl;
                    uint32_t v = tb == 0 ? 1u : (tb <= 3 ? 1u << tb : (tb <= 6 ? 1u << (tb - 3) : 0u));
                    v &= need_mask;
                    for (int b = 3; b >= 0 && v; --b) {
                        if (!((v >> b) & 1)) continue;
                        if (basis[b]) {
                            v ^= basis[b];
                        } else {
                            basis[b] = v;
                            ++rank;
                            v = 0;
                        }
                    }
                }
                return 1 + 4 * (__builtin_popcount(need_mask) - rank);
            };
            struct Best {
                int stages, cost;
                uint32_t R;
            };
            std::unordered_map<uint64_t, Best> memo;
            std::function<std::pair<int, int>(uint64_t)> solve = [&](uint64_t dm) -> std::pair<int, int> {
                if ((dm & all_mask) == all_mask) return {0, 0};
                if (memo.size() > 20000) {   // too many reachable states: greedy instead
                    search = false;
                    return {0, 0};
                }
                auto it = memo.find(dm);
                if (it != memo.end()) return {it->second.stages, it->second.cost};
                uint32_t touch = 0;
                for (int i = 0; i < nbk; ++i)
                    if (!((dm >> i) & 1) && !plan.blocks[dense_ids[i]].diag) touch |= tbm_of[dense_ids[i]];
                std::vector<int> bits;
                for (int tb = 0; tb < dp.m; ++tb)
                    if ((touch >> tb) & 1) bits.push_back(tb);
                std::vector<uint32_t> cands;
                if ((int)bits.size() <= SB) {
                    cands.push_back(touch);
                } else {   // every SB-subset of the touched bits
                    const int nb = (int)bits.size();
                    for (uint32_t sel = 0; sel < (1u << nb); ++sel) {
                        if (__builtin_popcount(sel) != SB) continue;
                        uint32_t R = 0;
                        for (int i = 0; i < nb; ++i)
                            if ((sel >> i) & 1) R |= 1u << bits[i];
                        cands.push_back(R);
                    }
                }
                Best best{1 << 20, 1 << 30, 0};
                std::vector<std::pair<uint64_t, int>> seen;   // state reached, cost of the stage
                for (uint32_t R : cands) {
                    const uint64_t nd = closure(dm, R);
                    if (nd == dm) continue;
                    const int c = stage_cost(R);
                    bool dup = false;
                    for (const auto& x : seen) dup = dup || (x.first == nd && x.second <= c);
                    if (dup) continue;
                    seen.push_back({nd, c});
                    const std::pair<int, int> r = solve(nd);
                    const int v = 1 + r.first, vc = c + r.second;
                    if (v < best.stages || (v == best.stages && vc < best.cost)) best = Best{v, vc, R};
                }
                memo[dm] = best;
                return {best.stages, best.cost};
            };
            auto choose_set = [&]() -> uint32_t {
                if (!search) return 0;
                uint64_t dm = 0;
                for (int i = 0; i < nbk; ++i)
                    if (done[dense_ids[i]]) dm |= 1ULL << i;
                solve(dm);
                if (!search) return 0;
                auto it = memo.find(dm);
                return it == memo.end() ? 0 : it->second.R;
            };
            uint32_t Rfix = 0;   // chosen register set of the open stage (0: grow greedily)
            while (left) {
                if (cur.empty() && small_blocks) Rfix = choose_set();
                int pick = -1;
                for (int b : pass_list) {
                    if (done[b]) continue;
                    bool ready = true;
                    for (int d : pdeps[b])
                        if (!done[d]) { ready = false; break; }
                    if (!ready) continue;
                    const Block& blk = plan.blocks[b];
                    if (Rfix && !blk.diag) {
                        if ((tbm_of[b] & ~Rfix) == 0) {
                            pick = b;
                            Rset = Rfix;
                            break;
                        }
                        continue;
                    }
                    if (o.adjoint && blk.param_single &&
                        (cur_grads >= kMaxStageGrads || Rcap > kRegBits))
                        continue;   // gradient ops stay in 16-amplitude register stages
                    if (blk.diag) { pick = b; break; }
                    const uint32_t tbm = tbm_of[b];
                    // a 5-qubit block opens a 32-amplitude stage of its own bits
                    if (cur.empty() && __builtin_popcount(tbm) > SB) Rcap = kMaxRegBits;
                    if (__builtin_popcount(Rset | tbm) <= Rcap) {
                        pick = b;
                        Rset |= tbm;
                        break;
                    }
                }
                if (pick < 0) {
                    if (cur.empty()) throw std::runtime_error("planner: no ready block fits");
                    close_stage();
                    continue;
                }
                done[pick] = 1;
                cur.push_back(pick);
                if (plan.blocks[pick].param_single) ++cur_grads;
                --left;
            }
            close_stage();
            };
            std::vector<Staged> staged, wide;
            schedule(kRegBits, staged);
            // 32-amplitude stages where they take fewer stages: unitary passes of one
            // or two such stages off tile bits 0..3 that leave a tile bit >= 5 untouched
            // (the FP16 tensor-core kernel for these runs two independent row blocks)
            if (o.wide && plan.all_unitary && !o.adjoint && dp.m == 13 && staged.size() > 1) {
                schedule(kMaxRegBits, wide);
                uint32_t U = 0;
                bool ok = !wide.empty() && wide.size() <= 2 && wide.size() < staged.size();
                for (const Staged& w : wide) {
                    U |= w.R;
                    ok = ok && w.cap == kMaxRegBits;
                }
                ok = ok && (U & 0xFu) == 0 && (U >> 5) != ((1u << (dp.m - 5)) - 1);
                if (ok) staged.swap(wide);
            }
            // plans for the FP16 tensor-core passes keep every stage's W resident: a
            // longer pass ends after kMaxWideStages stages and its later blocks wait
            // for the next pass (the stages are in dependency order, so the blocks
            // kept never need one left out)
            if (o.wide && plan.all_unitary && !o.adjoint && (int)staged.size() > kMaxWideStages) {
                for (size_t k = kMaxWideStages; k < staged.size(); ++k)
                    for (int b : staged[k].blocks) {
                        placed[b] = 0;
                        --n_placed;
                    }
                staged.resize(kMaxWideStages);
            }
            dp.stage_begin = (int)plan.stages.size();
            for (const Staged& sg : staged) {
                DevStage st{};
                const uint32_t Rset = sg.R;
                st.nreg = (uint8_t)sg.cap;
                // shared-memory banks are picked by tile bits 0..3 (8-byte amplitudes): only then
                // do the slots need the per-group XOR rotation
                st.rotate = (Rset & 0xFu) ? 1 : 0;
                int ri = 0;
                int reg_of_tb[kMaxTileBits + 2];
                for (int tb = 0; tb < dp.m; ++tb) {
                    reg_of_tb[tb] = -1;
                    if ((Rset >> tb) & 1) {
                        st.rbit[ri] = (uint8_t)tb;
                        reg_of_tb[tb] = ri++;
                    }
                }
                st.op_begin = (uint32_t)plan.dops.size();
                for (int b : sg.blocks) {
                    Block& blk = plan.blocks[b];
                    blk.out_off = off;
                    off += blk.size;
                    plan.pass_blocks.push_back(b);
                    DevOp d{};
                    d.k = (uint8_t)blk.k;
                    d.mat = (uint32_t)(blk.out_off - dp.mat_begin);
                    int j = 0;
                    uint64_t qm = blk.qmask;
                    if (blk.diag) {
                        d.kind = K_DIAG;
                        uint16_t nib = 0;
                        while (qm) {
                            int q = __builtin_ctzll(qm);
                            qm &= qm - 1;
                            d.src[j] = (tb_of_q[q] >= 0) ? (uint8_t)tb_of_q[q]
                                                         : (uint8_t)(kSrcBase | q);
                            if (tb_of_q[q] >= 0 && reg_of_tb[tb_of_q[q]] >= 0 &&
                                reg_of_tb[tb_of_q[q]] < kRegBits)
                                nib |= (uint16_t)((j + 1) << (4 * reg_of_tb[tb_of_q[q]]));
                            ++j;
                        }
                        d.mask = (uint8_t)(nib & 0xFF);
                        d.pad = (uint8_t)(nib >> 8);
                    } else {
                        d.kind = K_DENSE;
                        while (qm) {
                            int q = __builtin_ctzll(qm);
                            qm &= qm - 1;
                            int r = reg_of_tb[tb_of_q[q]];
                            if (r < 0) throw std::runtime_error("planner: block outside stage");
                            d.mask |= (uint8_t)(1u << r);
                        }
                    }
                    if (o.adjoint && blk.param_single) {
                        d.grad = (uint8_t)blk.grad;
                        if (plan.n_grad >= kMaxGradSlots)
                            throw std::invalid_argument("adjoint: at most 2048 parameterised gates per circuit");
                        d.slot = (uint16_t)plan.n_grad++;
                        ++st.n_grad;
                        plan.grad_param.push_back(blk.param);
                        plan.grad_scale.push_back(blk.grad_factor * blk.scale);
                    }
                    plan.dops.push_back(d);
                }
                st.op_count = (uint32_t)(plan.dops.size() - st.op_begin);
                plan.stages.push_back(st);
            }
            dp.stage_count = (int)plan.stages.size() - dp.stage_begin;
            dp.mat_count = off - dp.mat_begin;
            plan.passes.push_back(dp);
        }
        plan.table_size = off;
    }
    // ---- prologue descriptors ----
    plan.bops.clear();
    plan.bblocks.clear();
    for (const Block& b : plan.blocks) {
        BuildBlock bb{};
        bb.k = b.k;
        bb.diag = b.diag ? 1 : 0;
        bb.op_begin = (int)plan.bops.size();
        bb.op_count = (int)b.ops.size();
        bb.out_off = b.out_off;
        for (int oi : b.ops) {
            const HostOp& op = plan.ops[oi];
            BuildOp bo{};
            bo.code = (uint8_t)op.code;
            bo.k = (uint8_t)op.k;
            for (int j = 0; j < op.k; ++j)
                bo.pos[j] = (uint8_t)popc64(b.qmask & ((1ULL << op.q[j]) - 1));
            bo.param = op.param;
            bo.scale = op.scale;
            bo.angle0 = op.angle0;
            bo.pool_off = op.mat_off;
            plan.bops.push_back(bo);
        }
        plan.bblocks.push_back(bb);
    }
}

std::string describe_plan(const Plan& plan) {
    std::ostringstream s;
    s << "n=" << plan.n << " ops=" << plan.ops.size() << " blocks=" << plan.blocks.size()
      << " passes=" << plan.passes.size() << " stages=" << plan.stages.size()
      << " table=" << plan.table_size << " grads=" << plan.n_grad << "\n";
    for (size_t p = 0; p < plan.passes.size(); ++p) {
        const DevPass& d = plan.passes[p];
        s << " pass " << p << ": m=" << d.m << " chunk=" << d.chunk << " gather=[";
        for (int i = 0; i < d.ngather; ++i) s << (i ? "," : "") << int(d.gather[i]);
        s << "] stages=" << d.stage_count << " mats=" << d.mat_count << " regs=";
        for (int i = 0; i < d.stage_count; ++i) {   // register tile bits and op count per stage
            const DevStage& st = plan.stages[d.stage_begin + i];
            s << (i ? " " : "") << "{";
            for (int r = 0; r < st.nreg; ++r) s << (r ? "," : "") << int(st.rbit[r]);
            s << "}x" << st.op_count;
        }
        s << "\n";
    }
    return s.str();
}

}  // namespace tcng
