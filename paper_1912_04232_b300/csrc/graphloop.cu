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

}  // namespace jmd

extern "C" md_status md_set_loop_graphs(int on)
{
    if (on != 0 && on != 1) return MD_ERR_INVALID;
    jmd::g_loop_graphs = on;
    return MD_OK;
}
