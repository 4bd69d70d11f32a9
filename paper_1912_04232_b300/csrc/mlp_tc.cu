// mlp_tc.cu -- the per-atom network of the learned potential on the 5th-
// generation tensor cores (tcgen05, BF16 operands, FP32 accumulation in
// tensor memory): energy E_i and input gradient dE_i/dG_i for tiles of 128
// atoms (Sec. 4.1 deployment; same network as mlp.cu).
//
// Per tile (one CTA of 4 warps; thread t owns row/atom t of the tile, which
// is TMEM lane t):
//   MMA1  D1 = X  W1^T        [128 x 16] x [16 x 64]     (a1 = D1 + b1)
//   MMA2  D2 = H1 W2^T        [128 x 64] x [64 x 64]     (a2 = D2 + b2, E = w3 . silu(a2) + b3)
//   MMA3  D3 = G2 W2          [128 x 64] x [64 x 64]     (G2 = w3 * silu'(a2))
//   MMA4  D4 = G1 W1          [128 x 64] x [64 x 16]     (G1 = D3 * silu'(a1); dE/dx = D4)
// A operands are written by the threads (BF16) into shared memory in the
// canonical K-major, no-swizzle layout (8-row x 16-byte core matrices; K-
// adjacent core matrices 128 B apart, 8-row groups K/8 * 128 B apart); the
// weights are staged once per CTA in the same layout.  One elected thread
// issues the MMAs and commits them to an mbarrier; every wait is bounded
// and reports MD_ERR_TIMEOUT instead of hanging.
#include <cuda_bf16.h>

#include "bp.cuh"
#include "common.cuh"
#include "tc.cuh"

namespace jmd {

__device__ __forceinline__ float sgm(float x) { return 1.0f / (1.0f + __expf(-x)); }

// shared-memory plan (bytes): weights then the four A operands
constexpr int TC_M = 128;
constexpr uint32_t SM_W1 = 0;                     // [64 x 16]  B of MMA1 (W1, rows = out units)
constexpr uint32_t SM_W2 = SM_W1 + 64 * 16 * 2;   // [64 x 64]  B of MMA2 (W2)
constexpr uint32_t SM_W2T = SM_W2 + 64 * 64 * 2;  // [64 x 64]  B of MMA3 (W2^T)
constexpr uint32_t SM_W1T = SM_W2T + 64 * 64 * 2; // [16 x 64]  B of MMA4 (W1^T)
constexpr uint32_t SM_X = SM_W1T + 16 * 64 * 2;   // [128 x 16]
constexpr uint32_t SM_H1 = SM_X + TC_M * 16 * 2;  // [128 x 64]
constexpr uint32_t SM_G2 = SM_H1 + TC_M * 64 * 2; // [128 x 64]
constexpr uint32_t SM_G1 = SM_G2 + TC_M * 64 * 2; // [128 x 64]
constexpr uint32_t SM_TOTAL = SM_G1 + TC_M * 64 * 2;
constexpr uint32_t SM_LAUNCH = 100 * 1024;          // >= SM_TOTAL; at most 2 CTAs per SM
static_assert(SM_LAUNCH >= SM_TOTAL, "the launch must cover the layout");
constexpr uint32_t TMEM_COLS = 256;               // D1 [0,64) D2 [64,128) D3 [128,192) D4 [192,208)

struct TcSmallSmem {
    uint64_t bar;
    uint32_t tmem_base;
    uint32_t timeout;
    float b1[64], b2[64], w3[64], mu[16], isd[16];
    float b3;
};

__global__ void __launch_bounds__(128, 1) k_mlp_infer_tc(const float *P, const float *norm, const float *G, int N,
                                                         float *Ei, float *dEdG, uint32_t *status)
{
    count_launch();
    extern __shared__ __align__(1024) unsigned char tc_smem[];
    __shared__ TcSmallSmem S;
    const int tid = threadIdx.x, warp = tid >> 5;
    unsigned char *sm = tc_smem;
    const uint32_t sbase = smem_u32(sm);

    // stage weights (BF16, canonical layouts) and small vectors
    for (int e = tid; e < 64 * 16; e += blockDim.x) {
        int h = e / 16, q = e % 16;
        __nv_bfloat16 v = __float2bfloat16_rn(P[P_W1 + e]);
        *reinterpret_cast<__nv_bfloat16 *>(sm + SM_W1 + kmajor_off(h, q, 16)) = v;   // W1 [h][q]
        *reinterpret_cast<__nv_bfloat16 *>(sm + SM_W1T + kmajor_off(q, h, 64)) = v;  // W1^T [q][h]
    }
    for (int e = tid; e < 64 * 64; e += blockDim.x) {
        int h = e / 64, c = e % 64;
        __nv_bfloat16 v = __float2bfloat16_rn(P[P_W2 + e]);
        *reinterpret_cast<__nv_bfloat16 *>(sm + SM_W2 + kmajor_off(h, c, 64)) = v;   // W2 [h][c]
        *reinterpret_cast<__nv_bfloat16 *>(sm + SM_W2T + kmajor_off(c, h, 64)) = v;  // W2^T [c][h]
    }
    if (tid < 64) {
        S.b1[tid] = P[P_B1 + tid];
        S.b2[tid] = P[P_B2 + tid];
        S.w3[tid] = P[P_W3 + tid];
    }
    if (tid < 16) {
        S.mu[tid] = norm[tid];
        S.isd[tid] = 1.0f / norm[16 + tid];
    }
    if (tid == 0) {
        S.b3 = P[P_B3];
        S.timeout = 0u;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&S.bar)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&S.tmem_base)),
                     "r"(TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    fence_async_smem();
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    const uint32_t tmem = S.tmem_base;
    const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
    const uint32_t row_addr = tmem + lane_base;
    uint32_t phase = 0;

    const uint32_t id64 = idesc_bf16(TC_M, 64), id16 = idesc_bf16(TC_M, 16);
    // B operands: rows = N (out units), K contiguous: LBO = 128, SBO = K/8*128
    const uint64_t dW1 = sdesc(sbase + SM_W1, 128, 2 * 128);
    const uint64_t dX = sdesc(sbase + SM_X, 128, 2 * 128);

    auto wait_mma = [&]() {
        uint32_t it = 0;
        while (!mbar_try_wait(&S.bar, phase)) {
            if (++it > (1u << 26)) {
                S.timeout = 1u;
                break;
            }
        }
        phase ^= 1u;
        tc_after_sync();
    };
    auto issue = [&](int which) {
        if (tid == 0) {
            tc_after_sync();
            if (which == 1) {
                mma_bf16(tmem + 0, dX, dW1, id64, 0u);
            } else {
                uint32_t a = which == 2 ? SM_H1 : (which == 3 ? SM_G2 : SM_G1);
                uint32_t b = which == 2 ? SM_W2 : (which == 3 ? SM_W2T : SM_W1T);
                uint32_t d = which == 2 ? 64u : (which == 3 ? 128u : 192u);
                uint32_t id = which == 4 ? id16 : id64;
                for (int kk = 0; kk < 4; ++kk) {   // K = 64 in four K = 16 steps (2 core matrices each)
                    uint64_t da = sdesc(sbase + a + kk * 2 * 128, 128, 8 * 128);
                    uint64_t db = sdesc(sbase + b + kk * 2 * 128, 128, 8 * 128);
                    mma_bf16(tmem + d, da, db, id, kk > 0 ? 1u : 0u);
                }
            }
            mma_commit(&S.bar);
        }
    };

    const int ntiles = (N + TC_M - 1) / TC_M;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int i = tile * TC_M + tid;
        const bool valid = i < N;
        // X = (G - mu) / sd  (BF16), zeros past the end
        {
            float g[16];
            if (valid) {
                const float4 *gp = reinterpret_cast<const float4 *>(G + (size_t)i * 16);
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    float4 v = __ldg(gp + k);
                    g[4 * k] = v.x;
                    g[4 * k + 1] = v.y;
                    g[4 * k + 2] = v.z;
                    g[4 * k + 3] = v.w;
                }
            }
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                float x = valid ? (g[q] - S.mu[q]) * S.isd[q] : 0.0f;
                *reinterpret_cast<__nv_bfloat16 *>(sm + SM_X + kmajor_off(tid, q, 16)) = __float2bfloat16_rn(x);
            }
        }
        fence_async_smem();
        tc_before_sync();
        __syncthreads();
        issue(1);
        wait_mma();
        // h1 = silu(D1 + b1) -> H1
#pragma unroll
        for (int c0 = 0; c0 < 64; c0 += 16) {
            float d[16];
            tmem_ld16(row_addr + c0, d);
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                float a = d[k] + S.b1[c0 + k];
                float h = a * sgm(a);
                *reinterpret_cast<__nv_bfloat16 *>(sm + SM_H1 + kmajor_off(tid, c0 + k, 64)) = __float2bfloat16_rn(h);
            }
        }
        fence_async_smem();
        tc_before_sync();
        __syncthreads();
        issue(2);
        wait_mma();
        // a2 = D2 + b2; E = w3 . silu(a2) + b3; G2 = w3 * silu'(a2)
        float E = S.b3;
#pragma unroll
        for (int c0 = 0; c0 < 64; c0 += 16) {
            float d[16];
            tmem_ld16(row_addr + 64 + c0, d);
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                float a = d[k] + S.b2[c0 + k];
                float s = sgm(a);
                E += S.w3[c0 + k] * a * s;
                float g2 = S.w3[c0 + k] * s * (1.0f + a * (1.0f - s));
                *reinterpret_cast<__nv_bfloat16 *>(sm + SM_G2 + kmajor_off(tid, c0 + k, 64)) =
                    __float2bfloat16_rn(g2);
            }
        }
        if (valid) Ei[i] = E;
        fence_async_smem();
        tc_before_sync();
        __syncthreads();
        issue(3);
        wait_mma();
        // G1 = D3 * silu'(D1 + b1)
#pragma unroll
        for (int c0 = 0; c0 < 64; c0 += 16) {
            float d3[16], d1[16];
            tmem_ld16(row_addr + 128 + c0, d3);
            tmem_ld16(row_addr + c0, d1);
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                float a = d1[k] + S.b1[c0 + k];
                float s = sgm(a);
                float g1 = d3[k] * s * (1.0f + a * (1.0f - s));
                *reinterpret_cast<__nv_bfloat16 *>(sm + SM_G1 + kmajor_off(tid, c0 + k, 64)) =
                    __float2bfloat16_rn(g1);
            }
        }
        fence_async_smem();
        tc_before_sync();
        __syncthreads();
        issue(4);
        wait_mma();
        // dE/dG = D4 / sd
        {
            float d[16];
            tmem_ld16(row_addr + 192, d);
            if (valid) {
                float4 *o = reinterpret_cast<float4 *>(dEdG + (size_t)i * 16);
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    o[k] = make_float4(d[4 * k] * S.isd[4 * k], d[4 * k + 1] * S.isd[4 * k + 1],
                                       d[4 * k + 2] * S.isd[4 * k + 2], d[4 * k + 3] * S.isd[4 * k + 3]);
            }
        }
        tc_before_sync();
        __syncthreads();   // every lane's TMEM reads done before the next tile's MMAs
    }
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
    if (tid == 0 && S.timeout) raise_status(status, MD_ERR_TIMEOUT);
}

void enqueue_mlp_infer_tc(const float *P, const float *norm, const float *G, int N, float *Ei, float *dEdG,
                          uint32_t *status, cudaStream_t st)
{
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms < 1) sms = 1;
        cudaFuncSetAttribute(k_mlp_infer_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM_LAUNCH);
    }
    // two CTAs per SM: each holds 256 of the SM's 512 tensor-memory columns,
    // and the shared memory requested per CTA (SM_LAUNCH) keeps a third off
    // the SM, where its allocation would wait for one of the two to finish
    int tiles = (N + TC_M - 1) / TC_M;
    int g = tiles < 2 * sms ? tiles : 2 * sms;
    k_mlp_infer_tc<<<g, 128, SM_LAUNCH, st>>>(P, norm, G, N, Ei, dEdG, status);
}

}  // namespace jmd

using namespace jmd;

extern "C" md_status md_bp_mlp_infer_tc(const float *d_params, const float *d_norm, const float *d_G, int N,
                                        float *d_Ei, float *d_dEdG, uint32_t *d_status, md_stream_t stream)
{
    if (!d_params || !d_norm || !d_G || !d_Ei || !d_dEdG || N < 1) return MD_ERR_INVALID;
    enqueue_mlp_infer_tc(d_params, d_norm, d_G, N, d_Ei, d_dEdG, d_status, (cudaStream_t)stream);
    JMD_CUDA_TRY(cudaGetLastError());
    return MD_OK;
}
