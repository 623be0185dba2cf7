// Descriptors of the batched energy/adjoint-gradient launch.
#pragma once

#include <cuda_runtime.h>

#include "internal.hpp"
#include "launch.hpp"

namespace tcng {

struct StructDesc {            // one circuit structure of the batch (device copy)
    int32_t n;                 // qubits of the problem
    int32_t n_eff;             // qubits simulated (>= 5; extra qubits stay |0>)
    int32_t resident;          // 1: whole state in shared memory
    int32_t P;                 // parameters per item
    int32_t n_terms;
    int32_t n_passes;
    int32_t n_grad;
    int32_t table_size;
    const DevPass* passes;
    const DevStage* stages;
    const DevOp* dops;
    const HTerm* terms;
    const double* tcoef;       // terms' own coefficients
    const int* gparam;         // gradient slot -> parameter index
    const double* gscale;      // gradient slot -> factor * scale
};

struct ItemDesc {
    int32_t s;                 // structure
    int32_t pad;
    long long param_off;       // offset of the item's parameters
    long long coeff_off;       // offset of the item's coefficients
    long long grad_off;        // offset of the item's gradient row
    long long table_off;       // element offset of the item's matrix table
    long long psi_out_off;     // element offset of the forward state copy, -1 none
};

struct AdjArgs {
    const StructDesc* structs;
    const ItemDesc* items;
    const int* order;          // processing order (largest n first)
    int batch;
    int res_bits;              // resident-state capacity (log2 amplitudes)
    int want_grad;
    int* counter;              // work queue head (zeroed before launch)
    const void* tables;        // per-item block matrices
    const double* coeffs;      // per-item coefficients or NULL
    double* energy;            // [batch]
    double* grad;              // packed like params
    void* psi_out;             // forward-state copies or NULL
    void* scratch;             // per-CTA psi/lambda for streamed items
    long long scratch_elems;   // amplitudes per state per CTA
    unsigned* err;
};

template <typename C>
cudaError_t launch_adjoint(const AdjArgs& a, int grid, cudaStream_t s);
template <typename C>
size_t adjoint_smem_bytes(int res_bits);

}  // namespace tcng
