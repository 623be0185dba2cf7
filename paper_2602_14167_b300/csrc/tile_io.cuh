// Tile copies between the state and shared memory for the tile-pass kernels:
// one tensor copy per tile (tile map), four rows per tile::gather4 copy, or one
// bulk copy per contiguous chunk of 2^chunk amplitudes.  One warp issues them
// (all 32 lanes take part in the gather4 and per-chunk forms).
#pragma once

#include <cuda_runtime.h>

#include "device.cuh"
#include "launch.hpp"

namespace tcng {

struct TileCtx {
    int nbuf;
    int nchunks;
    uint32_t chunk_bytes;
    uint32_t tile_bytes;
    long long tiles_per_item;   // a power of two: 2^tpi_log
    int tpi_log;
    long long total_tiles;
};

template <typename C>
__device__ __forceinline__ void issue_tile_load(const C* state, const long long* item_off,
                                                const DevPass& p, const TileCtx& tc, long long tile,
                                                C* buf, uint64_t* bar, int lane, const TmaTile& tma) {
    const long long item = (tile >> tc.tpi_log);
    if (tma.rank) {   // one tensor copy for the whole tile
        if (lane == 0) {
            int c[5];
            tma_tile_coords(tma, (tile & (tc.tiles_per_item - 1)), (int)item, c);
            mbar_arrive_expect_tx(bar, tc.tile_bytes);
            tma_load_tile(tma, buf, bar, c);
        }
        return;
    }
    const long long base = tile_global_base(p, (tile & (tc.tiles_per_item - 1)));
    if (tma.g4) {   // four rows of 2^g4rb amplitudes per tile::gather4 copy, in tile order
        const long long b0 = item_off[item] - tma.g4base + base;
        const int rb = tma.g4rb, sub = p.chunk - rb;   // rows per chunk: 2^sub
        if (lane == 0) mbar_arrive_expect_tx(bar, tc.tile_bytes);
        __syncwarp();
        for (int k = lane; k < ((1 << p.m) >> (rb + 2)); k += 32) {
            int r[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int row = 4 * k + q;   // chunk row >> sub, piece row & (2^sub - 1)
                r[q] = (int)((b0 + chunk_offset(p, row >> sub) + ((long long)(row & ((1 << sub) - 1)) << rb)) >> rb);
            }
            tma_gather4(tma, buf + ((long long)(4 * k) << rb), bar, r[0], r[1], r[2], r[3]);
        }
        return;
    }
    const C* src = state + item_off[item] + base;
    if (lane == 0) mbar_arrive_expect_tx(bar, tc.tile_bytes);
    __syncwarp();
    for (int j = lane; j < tc.nchunks; j += 32)
        bulk_g2s(buf + ((long long)j << p.chunk), src + chunk_offset(p, j), tc.chunk_bytes, bar);
}

template <typename C>
__device__ __forceinline__ void issue_tile_store(C* state, const long long* item_off, const DevPass& p,
                                                 const TileCtx& tc, long long tile, const C* buf,
                                                 int lane, const TmaTile& tma) {
    const long long item = (tile >> tc.tpi_log);
    if (tma.rank) {
        if (lane == 0) {
            int c[5];
            tma_tile_coords(tma, (tile & (tc.tiles_per_item - 1)), (int)item, c);
            tma_store_tile(tma, buf, c);
        }
        bulk_commit();
        return;
    }
    const long long base = tile_global_base(p, (tile & (tc.tiles_per_item - 1)));
    C* dst = state + item_off[item] + base;
    for (int j = lane; j < tc.nchunks; j += 32)
        bulk_s2g(dst + chunk_offset(p, j), buf + ((long long)j << p.chunk), tc.chunk_bytes);
    bulk_commit();
}

// The complex64 expectation pass over 2^13-amplitude tiles (kernels_expect.cu).
size_t expect_fast_smem_bytes();
cudaError_t launch_expect_fast(const float2* state, const long long* item_off, int items, const DevPass& p,
                               const ExpPass& ep, const TileCtx& tc, double* partial, int n_out, int nblk,
                               unsigned* err, cudaStream_t s, const TmaTile& tma);

}  // namespace tcng
