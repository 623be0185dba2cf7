// Autotuner: choose fusion width, tile bits and chunk bits for the tile passes.
//
// Candidates are timed with CUDA events on a synthetic brickwork of n qubits
// (dense 2-qubit blocks built from RY/RZ/CX gates with fixed angles, plus an RZ
// layer, the shape of the paper's SU(4) brickwork circuits) applied to `batch`
// states of the requested dtype.  The best candidate becomes the process-wide
// option set and is appended to cache_path as one line
//   "n dtype batch fuse_width tile_bits chunk_bits ms".
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <fstream>
#include <sstream>
#include <string>
#include <vector>

#include "capi_internal.hpp"

using namespace tcng;

static std::vector<tcng_gate> synthetic_brickwork(int n, int depth) {
    std::vector<tcng_gate> g;
    auto add = [&](int op, int nq, int q0, int q1, double ang) {
        tcng_gate x{};
        x.op = (uint16_t)op;
        x.nq = (uint8_t)nq;
        for (int j = 0; j < 5; ++j) x.q[j] = -1;
        x.q[0] = q0;
        if (nq == 2) x.q[1] = q1;
        x.param = -1;
        x.scale = 1.0;
        x.angle0 = ang;
        x.mat_off = -1;
        g.push_back(x);
    };
    for (int t = 0; t < depth; ++t) {
        for (int i = t % 2; i + 1 < n; i += 2) {
            add(TCNG_RY, 1, i, -1, 0.3 + 0.01 * i);
            add(TCNG_RY, 1, i + 1, -1, -0.7);
            add(TCNG_CX, 2, i, i + 1, 0);
            add(TCNG_RZ, 1, i + 1, -1, 0.9);
            add(TCNG_CX, 2, i + 1, i, 0);
            add(TCNG_RY, 1, i, -1, 0.4);
        }
        for (int q = 0; q < n; ++q) add(TCNG_RZ, 1, q, -1, 0.1 * q);
    }
    return g;
}

extern "C" tcng_status tcng_autotune(int n, tcng_dtype dt, int batch, const char* cache_path) {
    if (n < 5 || n > TCNG_MAX_QUBITS || batch < 1) return fail(TCNG_EINVAL, "need n >= 5 and batch >= 1");
    if (dt != TCNG_C64 && dt != TCNG_C128) return fail(TCNG_EINVAL, "bad dtype");
    if (cache_path) {
        std::ifstream in(cache_path);
        std::string line;
        while (std::getline(in, line)) {
            std::istringstream ss(line);
            int cn, cd, cb, fw, tb, cbits;
            double ms;
            if (ss >> cn >> cd >> cb >> fw >> tb >> cbits >> ms && cn == n && cd == (int)dt && cb == batch) {
                std::lock_guard<std::mutex> lk(g_mu);
                g_opt.fuse_width = fw;
                g_opt.tile_bits = tb;
                g_opt.chunk_bits = cbits;
                return TCNG_OK;
            }
        }
    }
    const Options saved = g_opt;
    std::vector<int> nq(batch, n);
    tcng_state* st = nullptr;
    tcng_status s = tcng_state_init(&st, dt, batch, nq.data(), nullptr, 0, nullptr);
    if (s) return s;
    const std::vector<tcng_gate> g = synthetic_brickwork(n, 6);
    const int tmax = dt == TCNG_C64 ? 13 : 12;
    int best_fw = saved.fuse_width, best_tb = saved.tile_bits, best_cb = saved.chunk_bits;
    double best = 1e300;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    for (int fw = 1; fw <= 3; ++fw)
        for (int tb = tmax - 2; tb <= tmax; ++tb)
            for (int cb = 5; cb <= 8; ++cb) {
                {
                    std::lock_guard<std::mutex> lk(g_mu);
                    g_opt.fuse_width = fw;
                    g_opt.tile_bits = tb;
                    g_opt.chunk_bits = cb;
                    g_opt.unfused = 0;
                }
                s = tcng_apply_circuit(st, g.data(), g.size(), nullptr, 0, nullptr, 0, nullptr);   // plan + warm-up
                if (s) continue;
                cudaEventRecord(e0);
                for (int r = 0; r < 2; ++r) tcng_apply_circuit(st, g.data(), g.size(), nullptr, 0, nullptr, 0, nullptr);
                cudaEventRecord(e1);
                if (cudaEventSynchronize(e1) != cudaSuccess) {
                    cudaGetLastError();
                    continue;
                }
                float ms = 0;
                cudaEventElapsedTime(&ms, e0, e1);
                if (ms < best) {
                    best = ms;
                    best_fw = fw;
                    best_tb = tb;
                    best_cb = cb;
                }
            }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    tcng_state_free(st);
    {
        std::lock_guard<std::mutex> lk(g_mu);
        g_opt = saved;
        g_opt.fuse_width = best_fw;
        g_opt.tile_bits = best_tb;
        g_opt.chunk_bits = best_cb;
    }
    if (best >= 1e300) return fail(TCNG_ECUDA, "no candidate ran");
    if (cache_path) {
        std::ofstream out(cache_path, std::ios::app);
        out << n << " " << (int)dt << " " << batch << " " << best_fw << " " << best_tb << " " << best_cb
            << " " << best / 2 << "\n";
    }
    return tcng_sync_status();
}
