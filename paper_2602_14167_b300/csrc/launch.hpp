// Kernel launchers (defined in the .cu files, called by the C ABI layer).
#pragma once

#include <cuda_runtime.h>

#include "internal.hpp"

namespace tcng {

void count_launch();
int num_sms();

struct ExpTerm {
    uint32_t xm_tile;   // X mask in tile bits
    uint32_t zm_tile;   // Z mask in tile bits
    uint64_t zm_glob;   // Z mask on global bits outside the tile
    int32_t ny;         // number of Y factors mod 4
    int32_t out;        // output column
};
constexpr int kExpTermsPerPass = 16;
struct ExpPass {
    int nterms;
    ExpTerm t[kExpTermsPerPass];
};
struct HTerm {
    uint64_t xm, zm;
    int32_t ny;
    int32_t pad;
};

template <typename C>
cudaError_t launch_build_matrices(const BuildBlock* blocks, int n_blocks, const BuildOp* bops,
                                  const double2* pool, const double* params, int P, C* table,
                                  long long table_stride, int items, cudaStream_t s);
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
                        const C* table, long long table_stride, unsigned* err, cudaStream_t s);
template <typename C>
cudaError_t launch_expect_pass(const C* state, const long long* item_off, int items, int n,
                               const DevPass& p, const ExpPass& ep, double* partial, int n_out,
                               int nblk, unsigned* err, cudaStream_t s);
cudaError_t launch_expect_finalize(const double* partial, int nblk, int n_out, double* out,
                                   const double* coeffs, const double* term_coeff, double* energy,
                                   int items, cudaStream_t s);
template <typename C>
cudaError_t launch_ham_apply(const C* psi, const long long* off_in, C* out, const long long* off_out,
                             int items, int n, const HTerm* terms, int T, const double* coeffs,
                             const double* term_coeff, cudaStream_t s);

}  // namespace tcng
