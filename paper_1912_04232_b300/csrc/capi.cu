// capi.cu -- periodic space, status and accounting entry points.
#include <cmath>

#include "common.cuh"
#include "kernels.cuh"

namespace jmd {
static launch_reader_t g_readers[64];
static int g_nreaders = 0;
void register_launch_reader(launch_reader_t f)
{
    if (g_nreaders < 64) g_readers[g_nreaders++] = f;
}
}  // namespace jmd

using namespace jmd;

extern "C" md_status md_space_periodic(int dim, const double *box, md_space *out)
{
    if (!box || !out || (dim != 2 && dim != 3)) return MD_ERR_INVALID;
    md_space s;
    memset(&s, 0, sizeof(s));
    s.dim = dim;
    for (int k = 0; k < 3; ++k) {
        double L = k < dim ? box[k] : 1.0;
        if (!(L > 0.0) || !std::isfinite(L)) return MD_ERR_INVALID;
        s.L64[k] = L;
        s.L[k] = (float)L;
        s.Linv[k] = (float)(1.0 / L);
    }
    *out = s;
    return MD_OK;
}

extern "C" md_status md_status_poll(const uint32_t *d_status, uint32_t *h_status, md_stream_t stream)
{
    if (!d_status || !h_status) return MD_ERR_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    JMD_CUDA_TRY(cudaMemcpyAsync(h_status, d_status, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    JMD_CUDA_TRY(cudaStreamSynchronize(st));
    return MD_OK;
}

extern "C" uint64_t md_launch_count(void)
{
    if (cudaDeviceSynchronize() != cudaSuccess) return 0;
    unsigned long long v = 0;
    for (int k = 0; k < g_nreaders; ++k) v += g_readers[k]();
    return (uint64_t)v;
}

extern "C" const char *md_version(void) { return "jmd-b300 0.1 (sm_103a)"; }

// Bounded device wait: spin on *flag until it becomes nonzero or `limit`
// polls have passed; on running out, raise MD_ERR_TIMEOUT and return.  The
// library's waits (tensor-core MMA completion) follow the same rule; this
// entry point lets a test exercise the timeout path on a flag nothing sets.
__global__ void k_bounded_wait(const volatile uint32_t *flag, unsigned long long limit, uint32_t *status)
{
    count_launch();
    unsigned long long it = 0;
    while (*flag == 0u) {
        if (++it > limit) {
            raise_status(status, MD_ERR_TIMEOUT);
            return;
        }
        __nanosleep(100);
    }
}

extern "C" md_status md_bounded_wait(const uint32_t *d_flag, uint64_t limit, uint32_t *d_status, md_stream_t stream)
{
    if (!d_flag || !d_status || limit > (1ull << 24)) return MD_ERR_INVALID;
    k_bounded_wait<<<1, 1, 0, (cudaStream_t)stream>>>(d_flag, (unsigned long long)limit, d_status);
    JMD_CUDA_TRY(cudaGetLastError());
    return MD_OK;
}

// FP32 FMA throughput probe, the denominator of the ALU-bound rooflines:
// every thread runs FMA_CHAINS independent recurrences x <- x*a + b, enough
// independent work per warp to cover the FMA latency on every FP32 lane.
// The sums are stored so that no chain can be dropped.
#define FMA_CHAINS 8
__global__ void __launch_bounds__(1024) k_fma_probe(float *out, int iters, float a, float b)
{
    float x[FMA_CHAINS];
#pragma unroll
    for (int k = 0; k < FMA_CHAINS; ++k) x[k] = 1e-3f * (float)(threadIdx.x + k);
#pragma unroll 8
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < FMA_CHAINS; ++k) x[k] = fmaf(x[k], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < FMA_CHAINS; ++k) s += x[k];
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

extern "C" md_status md_fma_probe(float *d_out, int blocks, int threads, int iters, uint64_t *flops,
                                  md_stream_t stream)
{
    if (!d_out || blocks <= 0 || threads < 32 || threads > 1024 || threads % 32 || iters <= 0)
        return MD_ERR_INVALID;
    k_fma_probe<<<blocks, threads, 0, (cudaStream_t)stream>>>(d_out, iters, 0.999f, 1e-3f);
    JMD_CUDA_TRY(cudaGetLastError());
    if (flops) *flops = 2ull * FMA_CHAINS * (uint64_t)iters * (uint64_t)threads * (uint64_t)blocks;
    return MD_OK;
}
