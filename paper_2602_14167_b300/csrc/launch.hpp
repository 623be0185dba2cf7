// Kernel launchers (defined in the .cu files, called by the C ABI layer).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include "internal.hpp"

namespace tcng {

void count_launch();
int num_sms();
// Per-device caches (kernel attributes, SM counts) are indexed by this slot:
// the current device's index, 0 .. kMaxDeviceSlots - 1.
constexpr int kMaxDeviceSlots = 64;
int device_slot();

struct ExpTerm {
    uint32_t xm_tile;   // X mask in tile bits
    uint32_t zm_tile;   // Z mask in tile bits
    uint64_t zm_glob;   // Z mask on global bits outside the tile
    int32_t ny;         // number of Y factors mod 4
    int32_t out;        // output column
};
// Expectation tiles are read by 512 threads, 16 amplitudes each: element i of
// thread t is tile offset t + 512 i, so the Z parity of an element splits into
// a per-thread part (zm_tile & 511) and a per-slot part (bit i of slot_sign).
constexpr int kExpThreads = 512;
constexpr int kExpSlots = 16;
constexpr int kExpTermsPerPass = 16;
struct ExpPass {
    int nterms;
    ExpTerm t[kExpTermsPerPass];
};
// One multi-dimensional TMA tensor copy per tile: the n index bits split into
// runs; tile runs are box dimensions (<= 256 elements), rest runs and the item
// index are box-1 dimensions addressed by coordinates.
struct alignas(64) TmaTile {
    CUtensorMap map;
    int32_t rank;              // 0: no tile map (gather4 map or per-chunk bulk copies)
    int8_t kind[5];            // 0 tile run (coordinate 0), 1 rest run, 2 item
    int8_t shift[5];           // rest run: first bit of the tile number it takes
    int8_t len[5];             // rest run: number of bits
    int8_t lsh[5];             // rest run: tile bits below it in the same dimension (the
                               // box covers them; the coordinate is the rest bits << lsh)
    int8_t g4;                 // rank 0: map is a 2D [rows x 2^g4rb] gather4 map
    long long g4base;          // gather4: element offset of the map's first row
    int32_t g4rb;              // gather4: log2 amplitudes per row (<= chunk)
};

// Build the tensor map of a pass (returns rank 0 if the pass needs > 5 dims or
// the encoder rejects it).  items > 1 needs equally spaced items (stride bytes).
// sw128: the tile lands in shared memory with the 128-byte swizzle (rows of 128
// bytes whose 16-byte chunk index is XORed with the row index mod 8); needs a
// 1024-byte aligned destination and a low chunk of at least 128 bytes.
// merge: where the plain form needs more than five dimensions, give the rest run
// above each tile run the dimension of that run's last piece (the box covers the
// tile bits at its bottom), which needs one dimension per tile run.
TmaTile make_tma_tile(void* base, int n, int elem_bytes, const DevPass& p, int items,
                      long long item_stride_bytes, bool sw128 = false, bool merge = false);
// A pass's tiles as rows of one chunk (2^chunk amplitudes, at most 256 8-byte
// elements), four arbitrary rows per tile::gather4 copy (for passes whose bit
// runs need more than five tensor dimensions).  base_elems: element offset of
// base within the state buffer.  Returns g4 = 0 if the pass does not fit
// (larger chunks, fewer than 4 chunks per tile, unequal item spacing).
TmaTile make_tma_gather4(void* base, long long base_elems, int n, int elem_bytes, const DevPass& p,
                         int items, long long item_stride_bytes);

struct HTerm {
    uint64_t xm, zm;
    int32_t ny;
    int32_t pad;
};

template <typename C>
cudaError_t launch_build_matrices(const BuildBlock* blocks, int n_blocks, const BuildOp* bops,
                                  const double2* pool, const double* params, int P, C* table,
                                  long long table_stride, int items, cudaStream_t s,
                                  long long pool_stride = 0);
template <typename C>
cudaError_t launch_build_matrices_indexed(const BuildBlock* blocks, int n_blocks, const BuildOp* bops,
                                          const double2* pool, const double* params, C* table,
                                          const long long* prm_off, const long long* tab_off,
                                          int items, cudaStream_t s);
template <typename C>
cudaError_t launch_set_basis(C* state, const long long* item_off, int items, cudaStream_t s);
template <typename C>
cudaError_t launch_gate(C* state, const long long* item_off, int items, int n, const Block& blk,
                        const C* table, long long table_stride, cudaStream_t s);
template <typename C>
cudaError_t launch_pass(C* state, const long long* item_off, int items, int n, const DevPass& p,
                        const DevStage* host_stages, const DevStage* stages, const DevOp* ops,
                        const C* table, long long table_stride, unsigned* err, cudaStream_t s,
                        const TmaTile* tma = nullptr);
template <typename C>
cudaError_t launch_expect_pass(const C* state, const long long* item_off, int items, int n,
                               const DevPass& p, const ExpPass& ep, double* partial, int n_out,
                               int nblk, unsigned* err, cudaStream_t s, const TmaTile* tma = nullptr);
// Probabilities of k <= 10 qubits (kernels_measure.cu); partial holds
// items * 2^k * splits doubles when splits > 1.
template <typename C>
cudaError_t launch_marginal(const C* state, const long long* item_off, int items, int n, const int* q, int k,
                            double* out, double* partial, int splits, cudaStream_t s);
int marginal_splits(int items, int n, int k);
// Projective measurement of per-item qubit sets (kernels_measure.cu): hist holds
// items * 1024 * splits doubles, proj measure_proj_bytes(items) bytes.
template <typename C>
cudaError_t launch_measure(C* state, const long long* item_off, int items, int n,
                           const unsigned long long* mask, const double* u, signed char* outcome, double* logp,
                           double* hist, int splits, void* proj, cudaStream_t s);
size_t measure_proj_bytes(int items);
int measure_splits(int items, int n);
// rows: batch row of each item (out, coefficients, energy), or NULL for item i -> row i
cudaError_t launch_expect_finalize(const double* partial, int nblk, int n_out, double* out,
                                   const double* coeffs, const double* term_coeff, double* energy,
                                   int items, cudaStream_t s, const int* rows = nullptr);
template <typename C>
cudaError_t launch_ham_apply(const C* psi, const long long* off_in, C* out, const long long* off_out,
                             int items, int n, const HTerm* terms, int T, const double* coeffs,
                             const double* term_coeff, cudaStream_t s, const int* rows = nullptr);

}  // namespace tcng
