// One CUDA graph per circuit structure (option TCNG_OPT_USE_GRAPHS).
//
// The paper compiles a circuit once (jit) and re-runs the compiled program for
// new parameter values (Sec. I.B "Paradigms").  Here the launch sequence of a
// call -- the matrix prologue, every tile pass, the adjoint launch -- depends
// only on the structure (plan), the options and the device pointers passed in;
// parameters, coefficients and states are read from device memory when the
// kernels run.  So the sequence is recorded once into a CUDA graph and
// replayed: the first call of a key runs eagerly (building plans and sizing
// scratch), the second records the sequence on a private capture stream,
// instantiates it and launches it on the caller's stream, later calls only
// launch the instantiated graph.
//
// The key mixes the structure hash with every device pointer and option the
// launches read, and with the device context's allocation generation: a scratch
// buffer or matrix table that grows invalidates every recorded graph.  Calls
// made while the caller's stream is itself being captured, or while kernel
// profiling is on, run eagerly (the caller's capture then records them).
#include <cuda_runtime.h>

#include "capi_internal.hpp"

namespace tcng {

uint64_t key_mix(uint64_t h, uint64_t v) {
    // splitmix64 finaliser of (h ^ v), then combined with h
    uint64_t z = h ^ (v + 0x9e3779b97f4a7c15ULL + (h << 6) + (h >> 2));
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

uint64_t options_key() {
    uint64_t h = 0x74636e67ULL;
    h = key_mix(h, (uint64_t)g_opt.fuse_width);
    h = key_mix(h, (uint64_t)g_opt.tile_bits);
    h = key_mix(h, (uint64_t)g_opt.chunk_bits);
    h = key_mix(h, (uint64_t)g_opt.unfused);
    h = key_mix(h, (uint64_t)g_opt.tensor_cores);
    h = key_mix(h, (uint64_t)g_opt.tc_fp16);
    return h;
}

DeviceCtx::GraphEntry::~GraphEntry() {
    if (exec) cudaGraphExecDestroy(exec);
}

static void clear_graphs(DeviceCtx& c) {
    c.graphs.clear();
    c.graph_gen = c.gen;
}

tcng_status run_graphed(uint64_t key, cudaStream_t s, const std::function<tcng_status(cudaStream_t)>& body) {
    if (!g_opt.use_graphs || profiling_enabled()) return body(s);
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) {
        cudaGetLastError();
        return body(s);
    }
    if (cs != cudaStreamCaptureStatusNone) return body(s);
    DeviceCtx& c = ctx();
    if (c.graph_gen != c.gen) clear_graphs(c);
    std::unique_ptr<DeviceCtx::GraphEntry>& slot = c.graphs[key];
    if (!slot) slot.reset(new DeviceCtx::GraphEntry());
    DeviceCtx::GraphEntry& g = *slot;
    if (g.exec) {
        const cudaError_t e = cudaGraphLaunch(g.exec, s);
        if (e != cudaSuccess) return cuda_fail(e, "graph launch");
        add_launches(g.kernels);
        return TCNG_OK;
    }
    if (g.bad || g.seen == 0) {   // first call: eager (plans, scratch, attributes)
        g.seen = 1;
        return body(s);
    }
    if (!c.capture_stream) {
        if (cudaStreamCreateWithFlags(&c.capture_stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            c.capture_stream = nullptr;
            g.bad = true;
            return body(s);
        }
    }
    const uint64_t gen0 = c.gen;
    cudaError_t e = cudaStreamBeginCapture(c.capture_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        cudaGetLastError();
        g.bad = true;
        return body(s);
    }
    tcng_status st;
    try {
        LaunchCountOff off;   // recorded launches do not run
        st = body(c.capture_stream);
    } catch (...) {
        cudaGraph_t dropped = nullptr;
        cudaStreamEndCapture(c.capture_stream, &dropped);
        if (dropped) cudaGraphDestroy(dropped);
        cudaGetLastError();
        g.bad = true;
        throw;
    }
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(c.capture_stream, &graph);
    if (st != TCNG_OK || e != cudaSuccess || !graph || c.gen != gen0) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        g.bad = true;        // not recordable (or scratch moved while recording): stay eager
        return body(s);
    }
    size_t n_nodes = 0;
    cudaGraphGetNodes(graph, nullptr, &n_nodes);
    std::vector<cudaGraphNode_t> nodes(n_nodes);
    int kernels = 0;
    if (n_nodes && cudaGraphGetNodes(graph, nodes.data(), &n_nodes) == cudaSuccess) {
        for (size_t i = 0; i < n_nodes; ++i) {
            cudaGraphNodeType t;
            if (cudaGraphNodeGetType(nodes[i], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++kernels;
        }
    }
    e = cudaGraphInstantiate(&g.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        cudaGetLastError();
        g.exec = nullptr;
        g.bad = true;
        return body(s);
    }
    g.kernels = kernels;
    e = cudaGraphLaunch(g.exec, s);
    if (e != cudaSuccess) return cuda_fail(e, "graph launch");
    add_launches(g.kernels);
    return TCNG_OK;
}

}  // namespace tcng
