// Host-side state of the C ABI layer (shared by the host .cu files).
#pragma once

#include <cuda_runtime.h>

#include <functional>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <unordered_map>
#include <vector>

#include "internal.hpp"
#include "launch.hpp"

struct tcng_state {
    struct Group {
        std::vector<int> items;
        long long* d_off = nullptr;   // device element offsets of the group's items
        int* d_items = nullptr;       // device batch indices of the group's items
    };
    tcng_dtype dt = TCNG_C64;
    int batch = 0;
    std::vector<int> n;
    std::vector<long long> off;       // element offset of each item
    size_t bytes = 0;
    void* buf = nullptr;
    bool owned = false;
    long long* d_off = nullptr;
    std::map<int, Group> groups;      // items by qubit count
    // packed views of a batch of small states: tile bits m -> device offsets of the
    // virtual 2^m-amplitude items (2^(m-n) consecutive items each) and their count
    std::map<int, std::pair<long long*, long long>> pack;
};

namespace tcng {

constexpr unsigned ERR_TIMEOUT_FLAG = 1u;

struct Options {
    int fuse_width = 2;
    int tile_bits = 13;
    int chunk_bits = 7;
    int use_graphs = 1;
    int unfused = 0;
    int tensor_cores = 2;     // 0 off, 1 on, 2 auto
    int state_adjoint_n = 21; // tcng_energy_grad: states of >= this many qubits use the state-pass adjoint
    int tc_fp16 = 1;          // 1: FP16-split tensor-core passes where eligible, 0: TF32 split only
    int state_adjoint_small = 1;   // 1: small batches below state_adjoint_n take the state pass
                                   // when the cost model says it is faster
};
extern Options g_opt;
extern std::mutex g_mu;

struct DevPlan {
    Plan plan;
    BuildBlock* d_bblocks = nullptr;
    BuildOp* d_bops = nullptr;
    double2* d_pool = nullptr;
    DevStage* d_stages = nullptr;
    DevOp* d_dops = nullptr;
    int* d_gparam = nullptr;
    double* d_gscale = nullptr;
    void* d_table = nullptr;
    size_t table_bytes = 0;
    // tensor-core register stages (complex64)
    bool tc_ready = false;
    std::vector<TcsStage> tcs;        // per plan stage
    std::vector<char> tc_pass;        // per pass: 1 = run on the tensor cores
    std::vector<char> tc5;            // per pass: its stages have 5 register bits (FP16 only)
    std::vector<int> tc_group;        // per pass: slice tile bits (b0 | b1 << 8), -1 = none
    int n_tc = 0;                     // tensor-core stages
    int n_tc32 = 0;                   // ... with TF32 W operands (4-bit stages; 8 KiB each per item)
    long long wh_bytes = 0;           // FP16 W operand bytes per item
    TcsStage* d_tcs = nullptr;
    // FP16 lock-step passes on the swizzled tile: per stage, the shared-memory bit
    // positions of its four register bits when read and when written (rpos[4], wpos[4])
    std::vector<uint8_t> lay;
    uint8_t* d_lay = nullptr;
    ~DevPlan();
};

struct TermSet {
    int n_terms = 0;
    HTerm* d_h = nullptr;
    double* d_c = nullptr;
    ~TermSet();
};

struct DeviceCtx {
    struct Buf {
        void* ptr = nullptr;
        size_t bytes = 0;
    };
    int device = 0;
    unsigned* err = nullptr;
    std::unordered_map<uint64_t, std::unique_ptr<DevPlan>> plans;
    std::unordered_map<uint64_t, std::unique_ptr<TermSet>> terms;
    std::map<std::string, Buf> bufs;
    void* scratch(const std::string& name, size_t bytes);
    // allocation generation: bumped whenever a scratch buffer or matrix table
    // moves, which invalidates every recorded graph
    uint64_t gen = 0;
    // recorded launch sequences (one CUDA graph per structure and pointer set)
    struct GraphEntry {
        int seen = 0;
        bool bad = false;
        cudaGraphExec_t exec = nullptr;
        int kernels = 0;
        ~GraphEntry();
    };
    std::unordered_map<uint64_t, std::unique_ptr<GraphEntry>> graphs;
    uint64_t graph_gen = 0;
    cudaStream_t capture_stream = nullptr;
};

// Event-timed scope around one kernel launch (active only when profiling is on).
struct ProfScope {
    ProfScope(const char* name, cudaStream_t s);
    ~ProfScope();
    const char* name;
    cudaStream_t s;
    cudaEvent_t e0 = nullptr;
};

DeviceCtx& ctx();
bool profiling_enabled();
void add_launches(uint64_t k);
// While alive, launches on this thread are not counted (they are being recorded).
struct LaunchCountOff {
    LaunchCountOff();
    ~LaunchCountOff();
};
// CUDA graph per structure (graphs.cu): key_mix folds values into a key;
// options_key() covers every option a launch sequence depends on; run_graphed
// runs body eagerly, records it, or replays the recording (see graphs.cu).
uint64_t key_mix(uint64_t h, uint64_t v);
uint64_t options_key();
tcng_status run_graphed(uint64_t key, cudaStream_t s, const std::function<tcng_status(cudaStream_t)>& body);
tcng_status fail(tcng_status s, const std::string& msg);
tcng_status cuda_fail(cudaError_t e, const char* where);
PlanOptions plan_options(tcng_dtype dt, bool adjoint);
PlanOptions apply_plan_options(tcng_dtype dt, int batch, int P);
DevPlan* get_plan(int n, const tcng_gate* ops, size_t n_ops, const double* pool, size_t n_mat, int P,
                  const PlanOptions& o);
void* plan_table(DevPlan* dp, size_t elem, int items);
TermSet* get_terms(const tcng_pauli* terms, size_t n_terms, int n);
void plan_expectation(int n, int m, int low, const tcng_pauli* terms, size_t T,
                      std::vector<DevPass>& passes, std::vector<ExpPass>& eps, std::vector<size_t>* wide = nullptr);
// tma_base: device address of the group's first item and item_stride its spacing
// in bytes (< 0: items not equally spaced -> per-chunk bulk copies).
template <typename C>
tcng_status run_plan(DevPlan* dp, C* state, const long long* d_item_off, int items,
                     const double* params, cudaStream_t s, void* tma_base = nullptr,
                     long long item_stride = -1, const double2* item_pool = nullptr,
                     long long pool_stride = 0);

// State-pass adjoint of one item (adjoint_state.cu): params/coeffs/energy/grad
// point at the item's rows (coeffs may be NULL: the terms' own coefficients).
template <typename C>
tcng_status run_state_adjoint(tcng_state* st, int item, const tcng_gate* ops, size_t n_ops, const double* pool,
                              size_t n_mat, const double* params, int P, const tcng_pauli* H, size_t n_terms,
                              const double* coeffs, double* energy, double* grad, cudaStream_t s);

// Tensor-core register stages (kernels_pass_tc.cu).
void plan_tensor_stages(DevPlan* dp);
void plan_lock_layouts(DevPlan* dp);   // fills lay / d_lay (kernels_pass_tch.cu)
cudaError_t launch_build_stage_w(const DevPlan* dp, const double2* table, long long table_stride,
                                 int items, void* wops, bool half, cudaStream_t s);
// FP16-split tensor-core passes (unitary plans, one W set for every tile):
// whether pass `pass` can run them, and the launch.
bool pass_tch_eligible(const DevPlan* dp, int pass);
// One Pauli string with more X/Y factors than a tile gathers, straight from
// global memory (kernels_expect_wide.cu): partial[(item * n_out + out) * nblk + blk].
template <typename C>
cudaError_t launch_expect_wide(const C* state, const long long* item_off, int items, int n, const tcng_pauli& t,
                               int out, double* partial, int n_out, int nblk, cudaStream_t s);
cudaError_t launch_pass_tch(const DevPlan* dp, int pass, int items, const void* wops_h, unsigned* err,
                            const TmaTile& tma, bool swizzled, float2* state, const long long* item_off,
                            cudaStream_t s);
cudaError_t launch_pass_tcs(const DevPlan* dp, int pass, int items, const float* wops,
                            long long w_item_stride, unsigned* err, const TmaTile& tma, bool swizzled,
                            float2* state, const long long* item_off, cudaStream_t s);

// Synchronous upload of a host vector (used once per structure); throws bad_alloc.

template <typename T>
T* dev_copy(const std::vector<T>& v) {
    if (v.empty()) return nullptr;
    T* p = nullptr;
    if (cudaMalloc(&p, sizeof(T) * v.size()) != cudaSuccess) {
        cudaGetLastError();
        throw std::bad_alloc();
    }
    cudaMemcpy(p, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice);
    return p;
}

}  // namespace tcng
