// nbr_noalloc.cu -- a neighbor-list build whose scratch lives in a fixed,
// library-owned device array instead of a caller buffer.
//
// Some callers cannot hand the library a workspace: a host program that
// passes only its own input and output buffers through a plugin interface
// and forbids any other device allocation, or a latency-critical loop that
// must not pay cudaMalloc's implicit device synchronisation.  For them this
// entry point runs the ordinary rebuild chain (the same kernels as
// md_neighbor_list_build) on scratch carved out of the file-scope array
// below.  It calls no cudaMalloc, cudaFree or allocating library routine.
#include "common.cuh"
#include "kernels.cuh"

namespace jmd {

// The static scratch pool.  Every GPU that loads libjmd holds these bytes
// until the process exits.  In host code `g_nbr_scratch` names a host-side
// stand-in, not device memory, so its device address comes from
// cudaGetSymbolAddress and is passed to the kernels.
constexpr size_t kNoallocScratchBytes = 4u << 20;   // 4 MiB
static __device__ __align__(256) unsigned char g_nbr_scratch[kNoallocScratchBytes];

constexpr int kMaxDevices = 64;
static void *g_scratch_ptr[kMaxDevices];   // last address seen per device, NULL = never looked up

// The pool's device address for the current device.  Outside stream
// capture it is looked up on every call, so a module reloaded after
// cudaDeviceReset (or a re-created primary context) is never written
// through a stale pointer.  While `stream` is being captured the address
// seen by the last uncaptured call is reused (the lookup may load the
// module, which a capture does not allow); a library used across a device
// reset must therefore make one uncaptured call before capturing again.
static md_status scratch_for_current_device(cudaStream_t stream, void **out)
{
    int dev = 0;
    JMD_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return MD_ERR_INVALID;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(stream, &cs) != cudaSuccess) {
        // the legacy stream while another stream captures: treat as captured
        (void)cudaGetLastError();
        cs = cudaStreamCaptureStatusActive;
    }
    if (cs == cudaStreamCaptureStatusNone || !g_scratch_ptr[dev]) {
        void *p = nullptr;
        JMD_CUDA_TRY(cudaGetSymbolAddress(&p, g_nbr_scratch));
        if (!p) return MD_ERR_CUDA;
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return MD_OK;
}

}  // namespace jmd

using namespace jmd;

extern "C" size_t md_noalloc_scratch_bytes(void) { return kNoallocScratchBytes; }

extern "C" md_status md_neighbor_list_build_noalloc(const md_space *s, const float *d_r, int N, float r_cut,
                                                    float skin, int cap, int32_t *d_nbr, int32_t *d_cnt,
                                                    uint32_t *d_status, md_stream_t stream)
{
    if (!s || !d_r || !d_nbr || !d_cnt) return MD_ERR_INVALID;
    md_nbr nb;
    md_status st = md_nbr_plan(s, N, r_cut, skin, cap, &nb);
    if (st != MD_OK) return st;
    // the positions at build time (rref) sit after the workspace proper
    size_t ws = align256(nb.ws_bytes);
    size_t need = ws + sizeof(float4) * (size_t)N;
    if (need > kNoallocScratchBytes) return MD_ERR_INVALID;   // N or the cell grid too large for the pool
    void *base = nullptr;
    st = scratch_for_current_device((cudaStream_t)stream, &base);
    if (st != MD_OK) return st;
    float *rref = (float *)((char *)base + ws);
    // md_nbr_bind clears the control words and the cell histogram, which
    // must start at zero; the rest of the pool is overwritten by the build.
    st = md_nbr_bind(&nb, d_nbr, d_cnt, rref, base, stream);
    if (st != MD_OK) return st;
    return md_neighbor_list_build(s, d_r, &nb, d_status, stream);
}
