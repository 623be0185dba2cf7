// Host side of the tile tensor maps (cuTensorMapEncodeTiled through the
// runtime's driver entry point, so the library needs no libcuda link).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>
#include <vector>

#include "launch.hpp"

namespace tcng {

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            cudaGetLastError();
    });
    return fn;
}

TmaTile make_tma_tile(void* base, int n, int elem_bytes, const DevPass& p, int items,
                      long long item_stride_bytes, bool sw128, bool merge) {
    if (merge) {   // the plain form first; the merged one only where it needs too many dimensions
        TmaTile t0 = make_tma_tile(base, n, elem_bytes, p, items, item_stride_bytes, sw128, false);
        if (t0.rank) return t0;
    }
    TmaTile t;
    std::memset(&t, 0, sizeof t);
    auto fn = encode_fn();
    if (!fn) return t;
    // membership of each index bit in the tile
    // the tensor map lays the tile out in ascending global bit order: a pass whose
    // gathered qubits take their tile bits in another order has no tile map
    for (int i = 1; i < p.ngather; ++i)
        if (p.gather[i] <= p.gather[i - 1]) return TmaTile{};
    std::vector<int> in_tile(n, 0);
    for (int q = 0; q < p.chunk; ++q) in_tile[q] = 1;
    for (int i = 0; i < p.ngather; ++i) in_tile[p.gather[i]] = 1;
    const int e = elem_bytes / 8;          // 8-byte elements per amplitude
    cuuint64_t gdim[5], gstride[5];
    cuuint32_t box[5], estr[5];
    int rank = 0, rest_seen = 0;
    for (int q = 0; q < n;) {
        const int tile = in_tile[q];
        int len = 1;
        while (q + len < n && in_tile[q + len] == tile) ++len;
        // merge: the rest run above a tile run shares the dimension of the tile
        // run's last piece (box = the tile bits, coordinate = the rest bits << them)
        int above = 0;
        if (merge && tile && q + len < n) {
            while (q + len + above < n && !in_tile[q + len + above]) ++above;
        }
        // split tile runs so every box dimension stays <= 256 elements
        int done = 0;
        while (done < len) {
            int piece = len - done;
            if (tile) {
                // sw128: the innermost box dimension is one 128-byte swizzle row
                const int cap = (rank == 0) ? (sw128 ? (e == 1 ? 4 : 3) : (e == 1 ? 8 : 7)) : 8;
                if (piece > cap) piece = cap;
            }
            if (rank == 5) return TmaTile{};   // too many dimensions
            const int start = q + done;
            const bool last_piece = done + piece == len;
            const int extra = (tile && last_piece) ? above : 0;   // merged rest bits
            const cuuint64_t ext = 1ull << (piece + extra);
            gdim[rank] = (rank == 0) ? ext * e : ext;
            if (rank > 0) gstride[rank - 1] = (cuuint64_t)elem_bytes << start;
            box[rank] = tile ? (cuuint32_t)((1ull << piece) * (rank == 0 ? e : 1)) : 1;
            estr[rank] = 1;
            if (extra) {
                t.kind[rank] = 1;
                t.shift[rank] = (int8_t)rest_seen;
                t.len[rank] = (int8_t)extra;
                t.lsh[rank] = (int8_t)(piece + (rank == 0 && e == 2 ? 1 : 0));
                rest_seen += extra;
            } else {
                t.kind[rank] = tile ? 0 : 1;
                t.shift[rank] = (int8_t)(tile ? 0 : rest_seen);
                t.len[rank] = (int8_t)(tile ? 0 : piece);
                t.lsh[rank] = 0;
                if (!tile) rest_seen += piece;
            }
            if (rank == 0 && !tile) return TmaTile{};   // bit 0 is always a tile bit
            ++rank;
            done += piece;
        }
        q += len + (tile ? above : 0);
    }
    if (items > 1) {
        if (rank == 5) return TmaTile{};
        gdim[rank] = (cuuint64_t)items;
        gstride[rank - 1] = (cuuint64_t)item_stride_bytes;
        box[rank] = 1;
        estr[rank] = 1;
        t.kind[rank] = 2;
        ++rank;
    }
    CUresult r = fn(&t.map, CU_TENSOR_MAP_DATA_TYPE_INT64, (cuuint32_t)rank, base, gdim, gstride, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, sw128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return TmaTile{};
    t.rank = rank;
    return t;
}

TmaTile make_tma_gather4(void* base, long long base_elems, int n, int elem_bytes, const DevPass& p,
                         int items, long long item_stride_bytes) {
    TmaTile t;
    std::memset(&t, 0, sizeof t);
    auto fn = encode_fn();
    const int e = elem_bytes / 8;
    // one chunk per row, at most 256 8-byte elements (measured: splitting larger
    // chunks into several gathered rows is slower than their per-chunk bulk copies)
    const int rb = p.chunk;
    const long long row_elems = 1ll << rb;
    if (!fn || row_elems * e > 256 || (p.m - rb) < 2) return t;
    if (items > 1 && (item_stride_bytes <= 0 || item_stride_bytes % (row_elems * elem_bytes))) return t;
    const long long span = (items > 1 ? (long long)(items - 1) * (item_stride_bytes / elem_bytes) : 0) + (1ll << n);
    cuuint64_t gdim[2] = {(cuuint64_t)(row_elems * e), (cuuint64_t)(span / row_elems)};
    cuuint64_t gstride[1] = {(cuuint64_t)(row_elems * elem_bytes)};
    cuuint32_t box[2] = {(cuuint32_t)(row_elems * e), 1};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(&t.map, CU_TENSOR_MAP_DATA_TYPE_INT64, 2, base, gdim, gstride, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return TmaTile{};
    t.rank = 0;
    t.g4 = 1;
    t.g4base = base_elems;
    t.g4rb = rb;
    return t;
}

}  // namespace tcng
