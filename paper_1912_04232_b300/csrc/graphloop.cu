// graphloop.cu -- device-controlled loops as CUDA graphs for the host-side
// step loops (gradient descent, FIRE, flocking): WHILE(iteration < n) { body }, the body
// captured from the caller's kernels, with the neighbor-list rebuild chain
// under an IF node whose condition a one-thread kernel takes from the
// device rebuild flag.  An idle rebuild chain then costs nothing, and the
// host issues one graph launch instead of a dozen kernels per step.
// Executable graphs are cached by the caller's key (all arguments by value)
// and device, like the NVE graph.
#include <cstring>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"

namespace jmd {

int g_loop_graphs = 1;

__global__ void k_loop_counter_init(uint32_t *ctl, uint32_t n)
{
    count_launch();
    ctl[CTL_ITER] = 0u;
    ctl[CTL_NITER] = n;
}

__global__ void k_loop_tick(uint32_t *ctl, unsigned long long cond_while)
{
    count_launch();
    const uint32_t it = ctl[CTL_ITER] + 1u;
    ctl[CTL_ITER] = it;
    cudaGraphSetConditional((cudaGraphConditionalHandle)cond_while, it < ctl[CTL_NITER] ? 1u : 0u);
}

__global__ void k_if_from_flag(const uint32_t *ctl, unsigned long long cond_if)
{
    count_launch();
    cudaGraphSetConditional((cudaGraphConditionalHandle)cond_if,
                            *(const volatile uint32_t *)&ctl[CTL_REBUILD] ? 1u : 0u);
}

static cudaGraphNodeParams *cleared(unsigned char *raw)
{
    memset(raw, 0, sizeof(cudaGraphNodeParams));
    return reinterpret_cast<cudaGraphNodeParams *>(raw);
}

md_status LoopBuilder::rebuild_if(const NbrArgs &na, int ncell_total)
{
    cudaGraphConditionalHandle h;
    JMD_CUDA_TRY(cudaGraphConditionalHandleCreate(&h, graph, 0u, cudaGraphCondAssignDefault));
    k_if_from_flag<<<1, 1, 0, cs>>>(ctl, (unsigned long long)h);
    cudaStreamCaptureStatus cst;
    cudaGraph_t cg = nullptr;
    const cudaGraphNode_t *deps = nullptr;
    size_t nd = 0;
    JMD_CUDA_TRY(cudaStreamGetCaptureInfo(cs, &cst, nullptr, &cg, &deps, nullptr, &nd));
    alignas(cudaGraphNodeParams) unsigned char raw[sizeof(cudaGraphNodeParams)];
    cudaGraphNodeParams *ip = cleared(raw);
    ip->type = cudaGraphNodeTypeConditional;
    ip->conditional.handle = h;
    ip->conditional.type = cudaGraphCondTypeIf;
    ip->conditional.size = 1;
    cudaGraphNode_t in;
    JMD_CUDA_TRY(cudaGraphAddNode(&in, cg, deps, nullptr, nd, ip));
    JMD_CUDA_TRY(cudaStreamUpdateCaptureDependencies(cs, &in, nullptr, 1, cudaStreamSetCaptureDependencies));
    cudaGraph_t ibody = ip->conditional.phGraph_out[0];
    JMD_CUDA_TRY(cudaStreamBeginCaptureToGraph(cs2, ibody, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    NbrArgs a = na;
    a.gated = 0;
    enqueue_rebuild_chain(a, ncell_total, cs2);
    JMD_CUDA_TRY(cudaStreamEndCapture(cs2, &ibody));
    return MD_OK;
}

struct CachedLoop {
    std::vector<unsigned char> key;
    int device;
    cudaGraphExec_t exec;
};
static std::vector<CachedLoop> g_loops;
static std::mutex g_loops_mu;

md_status run_graph_loop(const void *key, size_t key_bytes, uint32_t *ctl, int niter,
                         const std::function<md_status(LoopBuilder &)> &body, cudaStream_t st)
{
    if (niter <= 0) return MD_OK;
    int dev = 0;
    JMD_CUDA_TRY(cudaGetDevice(&dev));
    cudaGraphExec_t ex = nullptr;
    std::lock_guard<std::mutex> lk(g_loops_mu);
    for (auto &e : g_loops)
        if (e.device == dev && e.key.size() == key_bytes && memcmp(e.key.data(), key, key_bytes) == 0) ex = e.exec;
    if (!ex) {
        LoopBuilder b;
        b.ctl = ctl;
        JMD_CUDA_TRY(cudaGraphCreate(&b.graph, 0));
        cudaGraphConditionalHandle hw;
        JMD_CUDA_TRY(cudaGraphConditionalHandleCreate(&hw, b.graph, 1u, cudaGraphCondAssignDefault));
        alignas(cudaGraphNodeParams) unsigned char raw[sizeof(cudaGraphNodeParams)];
        cudaGraphNodeParams *wp = cleared(raw);
        wp->type = cudaGraphNodeTypeConditional;
        wp->conditional.handle = hw;
        wp->conditional.type = cudaGraphCondTypeWhile;
        wp->conditional.size = 1;
        cudaGraphNode_t wn;
        JMD_CUDA_TRY(cudaGraphAddNode(&wn, b.graph, nullptr, nullptr, 0, wp));
        cudaGraph_t wbody = wp->conditional.phGraph_out[0];
        JMD_CUDA_TRY(cudaStreamCreateWithFlags(&b.cs, cudaStreamNonBlocking));
        JMD_CUDA_TRY(cudaStreamCreateWithFlags(&b.cs2, cudaStreamNonBlocking));
        JMD_CUDA_TRY(cudaStreamBeginCaptureToGraph(b.cs, wbody, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
        md_status s = body(b);
        k_loop_tick<<<1, 1, 0, b.cs>>>(ctl, (unsigned long long)hw);
        cudaError_t ce = cudaStreamEndCapture(b.cs, &wbody);
        cudaStreamDestroy(b.cs2);
        cudaStreamDestroy(b.cs);
        if (s != MD_OK) return s;
        if (ce != cudaSuccess) return MD_ERR_CUDA;
        JMD_CUDA_TRY(cudaGraphInstantiate(&ex, b.graph, 0));
        CachedLoop c;
        c.key.assign((const unsigned char *)key, (const unsigned char *)key + key_bytes);
        c.device = dev;
        c.exec = ex;
        g_loops.push_back(c);
    }
    k_loop_counter_init<<<1, 1, 0, st>>>(ctl, (uint32_t)niter);
    JMD_CUDA_TRY(cudaGraphLaunch(ex, st));
    JMD_CUDA_TRY(cudaGetLastError());
    return MD_OK;
}

// A whole host-driven call as one graph: the launches of `body` (kernels,
// device-to-device copies and sets on the stream it is given) captured once
// on a private stream per argument key and device, then replayed with one
// graph launch on the caller's stream.  For calls whose launch sequence is
// fixed by their arguments (the adjoints: fixed step counts and checkpoint
// schedule); each replay runs the same kernels in the same order.
struct CachedCall {
    std::vector<unsigned char> key;
    int device;
    cudaGraphExec_t exec;
};
static std::vector<CachedCall> g_calls;
static const size_t CALLS_CACHED = 32;
static std::mutex g_calls_mu;

md_status run_captured_call(const void *key, size_t key_bytes, const std::function<md_status(cudaStream_t)> &body,
                            cudaStream_t st)
{
    int dev = 0;
    JMD_CUDA_TRY(cudaGetDevice(&dev));
    cudaGraphExec_t ex = nullptr;
    std::lock_guard<std::mutex> lk(g_calls_mu);
    for (auto &e : g_calls)
        if (e.device == dev && e.key.size() == key_bytes && memcmp(e.key.data(), key, key_bytes) == 0) ex = e.exec;
    if (!ex) {
        cudaStream_t cs = nullptr;
        JMD_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        cudaGraph_t g = nullptr;
        cudaError_t ce = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed);
        md_status s = ce == cudaSuccess ? body(cs) : MD_ERR_CUDA;
        cudaError_t ee = cudaStreamEndCapture(cs, &g);
        cudaStreamDestroy(cs);
        if (s == MD_OK && (ce != cudaSuccess || ee != cudaSuccess)) s = MD_ERR_CUDA;
        if (s == MD_OK && cudaGraphInstantiate(&ex, g, 0) != cudaSuccess) s = MD_ERR_CUDA;
        if (g) cudaGraphDestroy(g);
        if (s != MD_OK) {
            cudaGetLastError();
            return s;
        }
        // at most CALLS_CACHED graphs (a parameter sweep makes one per
        // value): the oldest is destroyed once the device is idle, so no
        // launch of it can still be pending on any stream
        if (g_calls.size() >= CALLS_CACHED) {
            JMD_CUDA_TRY(cudaDeviceSynchronize());
            cudaGraphExecDestroy(g_calls.front().exec);
            g_calls.erase(g_calls.begin());
        }
        CachedCall c;
        c.key.assign((const unsigned char *)key, (const unsigned char *)key + key_bytes);
        c.device = dev;
        c.exec = ex;
        g_calls.push_back(c);
    }
    JMD_CUDA_TRY(cudaGraphLaunch(ex, st));
    return MD_OK;
}

}  // namespace jmd

extern "C" md_status md_set_loop_graphs(int on)
{
    if (on != 0 && on != 1) return MD_ERR_INVALID;
    jmd::g_loop_graphs = on;
    return MD_OK;
}
