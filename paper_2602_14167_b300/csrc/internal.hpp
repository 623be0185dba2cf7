// Internal data structures shared by the host planner (plan.cu) and the kernels.
//
// A circuit is compiled into a *plan*:
//   blocks  -- consecutive gates fused into one matrix on <= TCNG_MAX_FUSE qubits
//              (diagonal blocks store only their diagonal);
//   passes  -- one streaming sweep over the state: a shared-memory tile holds
//              2^m amplitudes (the low `chunk` bits contiguous plus gathered
//              high bits) and every block whose qubits lie in the tile is applied
//              to it (diagonal blocks are applied in any pass);
//   stages  -- inside a pass, each thread holds 2^R amplitudes in registers that
//              span R tile bits and applies every block on those bits before the
//              tile is shuffled through shared memory to the next stage.
// Block matrices are built on the device from the parameters by a prologue
// kernel, in "ascending" local order: bit j of the local index is the j-th
// smallest qubit of the block.
#pragma once

#include <cstdint>
#include <cstddef>
#include <string>
#include <vector>

#include "../../include/tcng.h"

namespace tcng {

constexpr int kRegBits = 4;          // R of an ordinary stage: 16 amplitudes per thread
constexpr int kMaxRegBits = 5;       // R of a stage holding a 5-qubit block: 32 amplitudes
constexpr int kMaxTileBits = 14;
constexpr int kMaxPassMat = 2048;    // complex entries of block matrices per pass (smem)
constexpr int kMaxWideStages = 22;   // FP16 tensor-core passes: stages whose W stay resident
constexpr int kMaxGather = 12;
constexpr int kMaxStageGrads = 32;   // adjoint: parameterised ops per stage
constexpr int kMaxGradSlots = 2048;  // adjoint: parameterised ops per circuit

// ---- device program ---------------------------------------------------------
enum OpKind : uint8_t {
    K_DENSE = 0,   // dense 2^k x 2^k matrix on register bits `mask`
    K_DIAG = 1,    // diagonal of 2^k entries on qubit sources src[0..k)
};

enum GradKind : uint8_t {
    G_NONE = 0,
    G_X = 1,       // generator X on the (single) register bit of the op
    G_Y = 2,       // generator Y
    G_Z = 3,       // generator Z on src[0]          (diagonal op)
    G_ZZ = 4,      // generator Z(x)Z on src[0], src[1]
    G_P11 = 5,     // projector |11><11| on src[0], src[1]
};

// Qubit source of a diagonal op: bit 7 set -> bit (src & 63) of the tile's global
// base index; else tile bit (src & 63).
constexpr uint8_t kSrcBase = 0x80;

struct DevOp {               // 16 bytes
    uint8_t kind;            // OpKind
    uint8_t k;               // qubits
    uint8_t mask;            // K_DENSE: register-bit mask (popcount k); K_DIAG: see pad
    uint8_t grad;            // GradKind (adjoint plans only)
    uint8_t src[5];          // K_DIAG: qubit sources (ascending qubit order)
    uint8_t pad;             // K_DIAG: (pad << 8 | mask) holds one nibble per register bit i:
                             //   j + 1 if register bit i is source j, else 0
    uint16_t slot;           // adjoint: gradient slot of a parameterised op
    uint32_t mat;            // complex offset inside the pass's matrix window
};
static_assert(sizeof(DevOp) == 16, "DevOp layout");

struct DevStage {            // 20 bytes
    uint8_t rbit[kMaxRegBits];  // tile bit of register bit i (ascending)
    uint8_t nreg;            // R: 4, or 5 for a stage holding a 5-qubit block
    uint8_t rotate;          // 1: slots XOR-rotated per group (register bits include tile bits 0..3)
    uint8_t pad;
    uint32_t op_begin;
    uint32_t op_count;
    uint32_t n_grad;         // adjoint: parameterised ops in this stage
};

struct DevPass {
    int32_t m;               // tile bits
    int32_t chunk;           // contiguous low bits of the tile (copy unit 2^chunk)
    int32_t ngather;         // tile bits above chunk
    int32_t nrest;           // global bits outside the tile
    uint8_t gather[kMaxGather + 4];  // global bit of tile bit chunk+i
    uint8_t rest[40];        // global bits outside the tile, ascending
    int32_t stage_begin;
    int32_t stage_count;
    int32_t mat_begin;       // complex offset of this pass's matrix window (per item)
    int32_t mat_count;
};

// ---- tensor-core register stages ----------------------------------------------
struct TcsStage {             // one register stage run as a 16x16 (32x32) GEMM (28 bytes)
    uint8_t rbit[5];          // tile bit of register bit i (ascending)
    uint8_t nj;               // register bits 0..nj-1 lie on tile bits 0..3 (XOR-rotated reads)
    uint8_t renorm;           // 1: every gate is unitary, restore the tile norm after the pass
    uint8_t nreg;             // register bits: 4 (16 amplitudes per row) or 5 (32)
    int32_t op_begin;         // the stage's ops (DevOp) for the matrix prologue
    int32_t op_count;
    int32_t mat_begin;        // the pass's matrix window in the item's table
    int32_t tc_index;         // TF32 W operand index, -1: not a tensor-core stage
    int32_t wh_off;           // byte offset of the FP16 W operand (4 KiB, or 16 KiB for 5 bits)
};
static_assert(sizeof(TcsStage) == 28, "TcsStage layout");

// ---- matrix-builder prologue -----------------------------------------------
struct BuildOp {             // one gate inside a block (40 bytes)
    uint8_t code;            // tcng_op
    uint8_t k;               // qubits of the gate
    uint8_t pos[5];          // position of gate qubit j inside the block's ascending list
    uint8_t pad;
    int32_t param;
    int32_t pad2;
    double scale;
    double angle0;
    int64_t pool_off;        // complex offset into the device matrix pool, -1 none
};

struct BuildBlock {          // 32 bytes
    int32_t k;               // block qubits
    int32_t diag;            // 1: diagonal only (2^k entries), 0: dense (4^k)
    int32_t op_begin;
    int32_t op_count;
    int32_t out_off;         // complex offset into the per-item matrix table
    int32_t pad[3];
};

// ---- host-side plan ---------------------------------------------------------
struct HostOp {
    int code, k;
    int q[5];
    int param;
    double scale, angle0;
    int64_t mat_off;
    bool diag;
    bool unitary;                // explicit matrices: checked on import; named gates: true
};

struct Block {
    uint64_t qmask = 0;          // qubits
    std::vector<int> ops;        // indices into HostOp list, in order
    bool diag = true;
    bool param_single = false;   // adjoint: a lone parameterised gate
    int k = 0;
    int out_off = 0;             // complex offset in the per-item table
    int size = 0;                // complex entries (2^k diag or 4^k dense)
    GradKind grad = G_NONE;      // generator of the lone parameterised gate
    double grad_factor = 0.0;    // dE/dtheta = factor * scale * Im<lam|G|psi>
    int param = -1;
    double scale = 0.0;
};

struct PlanOptions {
    int fuse_width = 2;          // max qubits per fused block
    int tile_bits = 13;          // m
    int chunk_bits = 7;          // c (lowest contiguous bits)
    int adjoint = 0;             // parameterised gates stay single blocks
    int unfused = 0;             // one block per gate, no passes
    int wide = 0;                // 32-amplitude register stages where they save stages
                                 // (complex64 tensor-core passes with FP16 operands)
};

struct Plan {
    int n = 0;
    PlanOptions opt;
    std::vector<HostOp> ops;
    std::vector<Block> blocks;
    int table_size = 0;          // complex entries per item
    // device program (host copies)
    std::vector<BuildOp> bops;
    std::vector<BuildBlock> bblocks;
    std::vector<DevPass> passes;
    std::vector<DevStage> stages;
    std::vector<DevOp> dops;
    std::vector<int> pass_blocks;      // block ids per pass, concatenated (for inspection)
    std::vector<int> pass_block_begin; // offsets into pass_blocks
    int n_grad = 0;                    // adjoint: number of gradient slots
    std::vector<int> grad_param;       // slot -> param index
    std::vector<double> grad_scale;    // slot -> factor * scale
    int P = 0;
    bool all_unitary = true;           // every op's matrix is unitary
};

// Validate the IR and build HostOps (throws std::invalid_argument).
std::vector<HostOp> import_ops(int n, const tcng_gate* ops, size_t n_ops, size_t n_mat, int P,
                               const double* pool);
// Build the full plan.
void build_plan(Plan& plan);
// Hash of the structure (everything but parameter values).
uint64_t structure_hash(int n, const tcng_gate* ops, size_t n_ops, const double* pool,
                        size_t n_mat, int P, const PlanOptions& opt);
std::string describe_plan(const Plan& plan);

}  // namespace tcng
