// mlp_tc.cu -- the per-atom network of the learned potential on the 5th-
// generation tensor cores (tcgen05, BF16 operands, FP32 accumulation in
// tensor memory): energy E_i and input gradient dE_i/dG_i for tiles of 128
// atoms (Sec. 4.1 deployment; same network as mlp.cu).
//
// Per tile (one CTA of 8 warps; two threads per row/atom: thread t owns row
// t % 128, which is TMEM lane t % 128, and the column half t / 128 of every
// 64-column accumulator, so that each thread runs half of the element-wise
// work between the MMA rounds):
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
#include <cstring>

#include <cuda_bf16.h>

#include "bp.cuh"
#include "bp_terms.cuh"
#include "common.cuh"
#include "tc.cuh"

namespace jmd {

// Logistic sigmoid as 1/2 + tanh(x/2)/2 with the PTX approximate tanh (one
// special-function instruction; its error, about 2^-11 relative, is below
// the BF16 rounding the network's operands get anyway).
__device__ __forceinline__ float sgm(float x)
{
    float t;
    asm("tanh.approx.f32 %0, %1;" : "=f"(t) : "f"(0.5f * x));
    return fmaf(0.5f, t, 0.5f);
}

// shared-memory plan (bytes): weights, then the A operands.  One buffer
// holds H1, then G2, then G1: each is written only after the MMA that read
// the previous one has completed.
constexpr int TC_M = 128;
constexpr uint32_t SM_X = 0;                      // [128 x 16]  A of MMA1
constexpr uint32_t SM_W1 = SM_X + TC_M * 16 * 2;  // [64 x 16]  B of MMA1 (W1, rows = out units)
constexpr uint32_t SM_W2 = SM_W1 + 64 * 16 * 2;   // [64 x 64]  B of MMA2 (W2)
constexpr uint32_t SM_W2T = SM_W2 + 64 * 64 * 2;  // [64 x 64]  B of MMA3 (W2^T)
constexpr uint32_t SM_W1T = SM_W2T + 64 * 64 * 2; // [16 x 64]  B of MMA4 (W1^T)
constexpr uint32_t SM_A = SM_W1T + 16 * 64 * 2;   // [128 x 64] H1, G2, G1 in turn
constexpr uint32_t SM_TOTAL = SM_A + TC_M * 64 * 2;
// the descriptor phase of the fused kernel keeps its partner lists (eight
// warps x four atoms x BP_MAXN float4) over the weights and A, which it
// stages afterwards
constexpr uint32_t SM_ND = SM_W1;
static_assert(SM_ND + 8 * 4 * BP_MAXN * 16 <= SM_TOTAL, "the partner lists must fit over the weights");
// requested per CTA: at least the layout, and enough that a fifth CTA
// never fits on an SM (its tensor-memory allocation would have to wait)
constexpr uint32_t SM_LAUNCH = 52 * 1024;
static_assert(SM_LAUNCH >= SM_TOTAL, "the launch must cover the layout");
// tensor-memory columns: D1 [0,64) (kept for silu'(a1) of the backward
// pass); D2, then D3, then D4 in [64,128), each written after the previous
// one has been read.  128 columns: four CTAs per SM.
constexpr uint32_t TMEM_COLS = 128;
constexpr uint32_t TC_D1 = 0, TC_D2 = 64, TC_D3 = 64, TC_D4 = 64;

__device__ __forceinline__ uint32_t tc_pack(float a, float b)
{
    return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(a)) |
           ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(b)) << 16);
}
// 8 consecutive K elements (k0 a multiple of 8) of row `row`, one 16-byte store
__device__ __forceinline__ void tc_row8(unsigned char *sm, uint32_t buf, int row, int k0, int K, const float *v)
{
    *reinterpret_cast<uint4 *>(sm + buf + kmajor_off(row, k0, K)) =
        make_uint4(tc_pack(v[0], v[1]), tc_pack(v[2], v[3]), tc_pack(v[4], v[5]), tc_pack(v[6], v[7]));
}

constexpr int TC_THREADS = 2 * TC_M;

struct TcSmallSmem {
    uint64_t bar;
    uint32_t tmem_base;
    uint32_t timeout;
    float b1[64], b2[64], w3[64], mu[16], isd[16];
    float b3;
    float Eh[TC_M];   // the second column half's part of E
};

// DESC 0: X from the descriptors G in global memory.  DESC 1 (the fused
// chain of a learned-potential evaluation): each tile first computes its 128
// atoms' descriptors itself (desc_group, eight lanes per atom, four passes of
// 32 atoms; the partner lists go to ba's lists when it carries them), writes
// X straight into shared memory and then stages the weights over the space
// the descriptor phase used.  G is not written; X has the bits the unfused
// path gives it.
template <bool DESC>
__global__ void __launch_bounds__(TC_THREADS, 4) k_mlp_infer_tc(const float *P, const float *norm, const float *G, int N,
                                                         float *Ei, float *dEdG, uint32_t *status, BpArgs ba)
{
    count_launch();
    extern __shared__ __align__(1024) unsigned char tc_smem[];
    __shared__ TcSmallSmem S;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int row = tid & (TC_M - 1), ch = tid >> 7;   // TMEM lane and column half
    unsigned char *sm = tc_smem;
    const uint32_t sbase = smem_u32(sm);

    // stage weights (BF16, canonical layouts): each thread packs blocks of 8
    // consecutive K elements of a row into one 16-byte store; W1 [h][q] and
    // W2 [h][c] rows are contiguous in P, the transposes read a column
    auto stage_weights = [&]() {
    for (int b = tid; b < 64 * 2 + 16 * 8 + 64 * 8 * 2; b += blockDim.x) {
        float v[8];
        uint32_t buf;
        int row, k0, K;
        if (b < 128) {                       // W1 [64 x 16]
            row = b >> 1, k0 = (b & 1) * 8, K = 16, buf = SM_W1;
#pragma unroll
            for (int k = 0; k < 8; ++k) v[k] = __ldg(P + P_W1 + row * 16 + k0 + k);
        } else if (b < 256) {                // W1^T [16 x 64]
            const int e = b - 128;
            row = e >> 3, k0 = (e & 7) * 8, K = 64, buf = SM_W1T;
#pragma unroll
            for (int k = 0; k < 8; ++k) v[k] = __ldg(P + P_W1 + (k0 + k) * 16 + row);
        } else if (b < 768) {                // W2 [64 x 64]
            const int e = b - 256;
            row = e >> 3, k0 = (e & 7) * 8, K = 64, buf = SM_W2;
#pragma unroll
            for (int k = 0; k < 8; ++k) v[k] = __ldg(P + P_W2 + row * 64 + k0 + k);
        } else {                             // W2^T [64 x 64]
            const int e = b - 768;
            row = e >> 3, k0 = (e & 7) * 8, K = 64, buf = SM_W2T;
#pragma unroll
            for (int k = 0; k < 8; ++k) v[k] = __ldg(P + P_W2 + (k0 + k) * 64 + row);
        }
        tc_row8(sm, buf, row, k0, K, v);
    }
    };
    if (!DESC) stage_weights();
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
    const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;   // a warp reads lanes 32 (warp % 4) + [0, 32)
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
                mma_bf16(tmem + TC_D1, dX, dW1, id64, 0u);
            } else {
                const uint32_t a = SM_A;
                uint32_t b = which == 2 ? SM_W2 : (which == 3 ? SM_W2T : SM_W1T);
                uint32_t d = which == 2 ? TC_D2 : (which == 3 ? TC_D3 : TC_D4);
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
    const int c0h = 32 * ch;   // this thread's first column of a 64-column accumulator
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int i = tile * TC_M + row;
        const bool valid = i < N;
        if (DESC) {
            // descriptors of the tile's atoms, eight lanes each: pass p
            // takes local atoms 32 p + 4 warp + group
            const BpConst c = bp_const();
            const int lane = tid & 31, grp = lane >> 3, gl = lane & 7;
            const unsigned gmask = 0xffu << (grp * 8);
            const unsigned below = (1u << lane) - 1u;
            float4 *ndg = reinterpret_cast<float4 *>(sm + SM_ND) + (warp * 4 + grp) * BP_MAXN;
#pragma unroll 1
            for (int pass = 0; pass < TC_M / 32; ++pass) {
                const int loc = pass * 32 + warp * 4 + grp;
                const int ia = tile * TC_M + loc;
                const bool va = ia < N;
                float Gd[16];
                desc_group<8>(ba, c, ia, va, ndg, gl, gmask, below, Gd);
                if (gl < 2) {   // lanes 0 and 1 of the group: features 8 gl + [0, 8) of X
                    float x[8];
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const float g = gl ? Gd[8 + q] : Gd[q];
                        x[q] = va ? (g - S.mu[8 * gl + q]) * S.isd[8 * gl + q] : 0.0f;
                    }
                    tc_row8(sm, SM_X, loc, 8 * gl, 16, x);
                }
                __syncwarp();
            }
            __syncthreads();   // the partner lists are done with: the weights go over them
            stage_weights();
        } else {
            // X = (G - mu) / sd  (BF16), zeros past the end: features 8 ch + [0, 8)
            float x[8];
            if (valid) {
                const float4 *gp = reinterpret_cast<const float4 *>(G + (size_t)i * 16 + 8 * ch);
                const float4 u = __ldg(gp), v = __ldg(gp + 1);
                const float g[8] = {u.x, u.y, u.z, u.w, v.x, v.y, v.z, v.w};
#pragma unroll
                for (int q = 0; q < 8; ++q) x[q] = (g[q] - S.mu[8 * ch + q]) * S.isd[8 * ch + q];
            } else {
#pragma unroll
                for (int q = 0; q < 8; ++q) x[q] = 0.0f;
            }
            tc_row8(sm, SM_X, row, 8 * ch, 16, x);
        }
        fence_async_smem();
        tc_before_sync();
        __syncthreads();
        issue(1);
        wait_mma();
        // h1 = silu(D1 + b1) -> H1
#pragma unroll
        for (int c0 = c0h; c0 < c0h + 32; c0 += 16) {
            float d[16], h[16];
            tmem_ld16(row_addr + TC_D1 + c0, d);
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                float a = d[k] + S.b1[c0 + k];
                h[k] = a * sgm(a);
            }
            tc_row8(sm, SM_A, row, c0, 64, h);
            tc_row8(sm, SM_A, row, c0 + 8, 64, h + 8);
        }
        fence_async_smem();
        tc_before_sync();
        __syncthreads();
        issue(2);
        wait_mma();
        // a2 = D2 + b2; E = w3 . silu(a2) + b3; G2 = w3 * silu'(a2)
        float E = 0.0f;
#pragma unroll
        for (int c0 = c0h; c0 < c0h + 32; c0 += 16) {
            float d[16], g2[16];
            tmem_ld16(row_addr + TC_D2 + c0, d);
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                float a = d[k] + S.b2[c0 + k];
                float s = sgm(a);
                E += S.w3[c0 + k] * a * s;
                g2[k] = S.w3[c0 + k] * s * (1.0f + a * (1.0f - s));
            }
            tc_row8(sm, SM_A, row, c0, 64, g2);
            tc_row8(sm, SM_A, row, c0 + 8, 64, g2 + 8);
        }
        if (ch) S.Eh[row] = E;
        fence_async_smem();
        tc_before_sync();
        __syncthreads();
        issue(3);
        if (!ch && valid) Ei[i] = S.b3 + E + S.Eh[row];
        wait_mma();
        // G1 = D3 * silu'(D1 + b1)
#pragma unroll
        for (int c0 = c0h; c0 < c0h + 32; c0 += 16) {
            float d3[16], d1[16], g1[16];
            tmem_ld16(row_addr + TC_D3 + c0, d3);
            tmem_ld16(row_addr + TC_D1 + c0, d1);
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                float a = d1[k] + S.b1[c0 + k];
                float s = sgm(a);
                g1[k] = d3[k] * s * (1.0f + a * (1.0f - s));
            }
            tc_row8(sm, SM_A, row, c0, 64, g1);
            tc_row8(sm, SM_A, row, c0 + 8, 64, g1 + 8);
        }
        fence_async_smem();
        tc_before_sync();
        __syncthreads();
        issue(4);
        wait_mma();
        // dE/dG = D4 / sd: features 8 ch + [0, 8) (both halves load the 16
        // columns: tcgen05.ld is warp-wide)
        {
            float d[16];
            tmem_ld16(row_addr + TC_D4, d);
            if (valid) {
                float4 *o = reinterpret_cast<float4 *>(dEdG + (size_t)i * 16 + 8 * ch);
                const float *dh = d + 8 * ch;
                const float *sh = S.isd + 8 * ch;
                o[0] = make_float4(dh[0] * sh[0], dh[1] * sh[1], dh[2] * sh[2], dh[3] * sh[3]);
                o[1] = make_float4(dh[4] * sh[4], dh[5] * sh[5], dh[6] * sh[6], dh[7] * sh[7]);
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

static int tc_grid(int N)
{
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms < 1) sms = 1;
        cudaFuncSetAttribute(k_mlp_infer_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM_LAUNCH);
        cudaFuncSetAttribute(k_mlp_infer_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM_LAUNCH);
    }
    // four CTAs per SM: each holds 128 of the SM's 512 tensor-memory
    // columns; the grid never exceeds four per SM, so no allocation waits
    int tiles = (N + TC_M - 1) / TC_M;
    return tiles < 4 * sms ? tiles : 4 * sms;
}

void enqueue_mlp_infer_tc(const float *P, const float *norm, const float *G, int N, float *Ei, float *dEdG,
                          uint32_t *status, cudaStream_t st)
{
    BpArgs none;
    memset(&none, 0, sizeof(none));
    k_mlp_infer_tc<false><<<tc_grid(N), TC_THREADS, SM_LAUNCH, st>>>(P, norm, G, N, Ei, dEdG, status, none);
}

void enqueue_bp_desc_mlp_tc(const BpArgs &b, const float *P, const float *norm, float *Ei, float *dEdG,
                            uint32_t *status, cudaStream_t st)
{
    k_mlp_infer_tc<true><<<tc_grid(b.N), TC_THREADS, SM_LAUNCH, st>>>(P, norm, nullptr, b.N, Ei, dEdG, status, b);
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
