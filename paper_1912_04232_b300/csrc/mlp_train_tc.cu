// mlp_train_tc.cu -- the training gradient of the learned potential's
// per-atom network (Sec. 4.1: energy + force loss) on the 5th-generation
// tensor cores (tcgen05, BF16 operands, FP32 accumulation in tensor
// memory).  Same objective as k_mlp_train / k_mlp_grads in mlp.cu:
//   J = sum_i c_E,i E_i - c_F dE_i/dG_i . V_i
// whose gradient needs, per atom, the forward pass, its tangent along
// v = V / sd, and the reverse pass through both ("double backward").
//
// One CTA of 4 warps per SM; thread t owns atom t of a 128-atom tile (TMEM
// lane t).  Per tile:
//   MMA1  D1 = X W1^T, DT1 = VT W1^T                  a1, tangent of a1
//         h1 = silu(a1), h1' = silu'(a1) DT1
//   MMA2  D2 = H1 W2^T, DT2 = H1' W2^T                a2, tangent of a2
//         d2 = dJ/da2 = c_E w3 silu'(a2) - c_F w3 silu''(a2) DT2
//         e2 = dJ/d(tangent of a2) = -c_F w3 silu'(a2)
//         c3 = dJ/dw3 per atom = c_E h2 - c_F h2'
//   MMA3  U = d2 W2, UE = e2 W2                       (back to layer 1)
//         d1 = U silu'(a1) + UE silu''(a1) DT1,  e1 = UE silu'(a1)
// and the sums over atoms, as MMAs with the atoms as the K dimension,
// accumulated in tensor memory across all tiles of the CTA:
//   dW2 += d2^T h1 + e2^T h1'      dW1 += d1^T x + e1^T v
//   db2 += d2^T 1, dw3 += c3^T 1   db1 += d1^T 1, db3 += c_E^T 1
// The transposed factors are written by the threads into K-major (atoms
// contiguous) operand buffers.  M is 128 for every MMA: a factor of 64
// units fills half the rows, the other half holds the next factor or
// whatever lies after it in shared memory, and those rows of the result
// are not read.  Each CTA writes its partial gradient; k_mlp_grads_sum adds
// the partials of all CTAs in a fixed order in FP64, so the result is
// deterministic.  Every wait is bounded and reports MD_ERR_TIMEOUT.
#include <cuda_bf16.h>

#include "bp.cuh"
#include "common.cuh"
#include "tc.cuh"

namespace jmd {

constexpr int TR_M = 128;   // atoms per tile
// shared-memory plan (bytes); every buffer is a BF16 operand in the
// canonical K-major no-swizzle layout ([rows x K])
constexpr uint32_t TS_W1 = 0;                          // [64 x 16]   W1 (B of the first layer)
constexpr uint32_t TS_W2 = TS_W1 + 64 * 16 * 2;        // [64 x 64]   W2 (B of the second layer)
constexpr uint32_t TS_W2T = TS_W2 + 64 * 64 * 2;       // [64 x 64]   W2^T (B of the backward product)
constexpr uint32_t TS_ONE = TS_W2T + 64 * 64 * 2;      // [16 x 128]  ones (B of the column sums)
constexpr uint32_t TS_X = TS_ONE + 16 * 128 * 2;       // [128 x 16]  x
constexpr uint32_t TS_VT = TS_X + 128 * 16 * 2;        // [128 x 16]  v = V / sd
constexpr uint32_t TS_XT = TS_VT + 128 * 16 * 2;       // [16 x 128]  x^T
constexpr uint32_t TS_VTT = TS_XT + 16 * 128 * 2;      // [16 x 128]  v^T
constexpr uint32_t TS_H1 = TS_VTT + 16 * 128 * 2;      // [128 x 64]  h1, then d2
constexpr uint32_t TS_HD1 = TS_H1 + 128 * 64 * 2;      // [128 x 64]  h1', then e2
constexpr uint32_t TS_T1 = TS_HD1 + 128 * 64 * 2;      // [200 x 128] d2^T 0-63, c3^T 64-127, d1^T 128-191, c_E 192
constexpr uint32_t TS_T2 = TS_T1 + 200 * 128 * 2;      // [128 x 128] e2^T 0-63, e1^T 64-127
constexpr uint32_t TS_H1T = TS_T2 + 128 * 128 * 2;     // [64 x 128]  h1^T
constexpr uint32_t TS_HD1T = TS_H1T + 64 * 128 * 2;    // [64 x 128]  h1'^T
constexpr uint32_t TS_TOTAL = TS_HD1T + 64 * 128 * 2;  // 188,416 bytes: one CTA per SM
// The MMAs that take rows 128-255 of T1 and rows 64-191 of T2 read past
// their buffers into the ones after them (rows whose results are unused);
// those reads stay inside the layout.
static_assert(TS_T1 + 256 * 128 * 2 <= TS_TOTAL && TS_T2 + 192 * 128 * 2 <= TS_TOTAL, "reads past T1, T2");

// tensor-memory columns (512 allocated)
constexpr uint32_t C_D1 = 0, C_DT1 = 64, C_D2 = 128, C_DT2 = 192, C_U = 256, C_UE = 320;
constexpr uint32_t C_GW2 = 384, C_GS1 = 448, C_GW1 = 464, C_GS2 = 480;
constexpr uint32_t TR_TMEM_COLS = 512;

struct TrSmall {
    uint64_t bar;
    uint32_t tmem_base;
    uint32_t timeout;
    float b1[64], b2[64], w3[64], mu[16], isd[16];
};

// Logistic sigmoid as 1/2 + tanh(x/2)/2 with the PTX approximate tanh (its
// error, about 2^-11 relative, is below the BF16 rounding of the operands).
__device__ __forceinline__ float tr_sigm(float x)
{
    float t;
    asm("tanh.approx.f32 %0, %1;" : "=f"(t) : "f"(0.5f * x));
    return fmaf(0.5f, t, 0.5f);
}

__device__ __forceinline__ uint32_t bf16_bits(float v) { return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(v)); }
__device__ __forceinline__ uint32_t bf16_pack(float a, float b) { return bf16_bits(a) | (bf16_bits(b) << 16); }

// Row `tid` of a K-major operand, 8 consecutive K elements from k0 (a
// multiple of 8) as one 16-byte store.
__device__ __forceinline__ void st_row8(unsigned char *sm, uint32_t buf, int tid, int k0, int K, const float *v)
{
    *reinterpret_cast<uint4 *>(sm + buf + kmajor_off(tid, k0, K)) =
        make_uint4(bf16_pack(v[0], v[1]), bf16_pack(v[2], v[3]), bf16_pack(v[4], v[5]), bf16_pack(v[6], v[7]));
}

// Element (row r, K index = atom tid) of a transposed operand with K = 128:
// neighbouring atoms share 4 bytes, so even lanes store their own and the
// odd neighbour's value together.  Warp-collective.
__device__ __forceinline__ void st_t(unsigned char *sm, uint32_t buf, int r, int tid, float v)
{
    const uint32_t b = bf16_bits(v);
    const uint32_t o = __shfl_xor_sync(0xffffffffu, b, 1);
    if (!(tid & 1)) *reinterpret_cast<uint32_t *>(sm + buf + kmajor_off(r, tid, TR_M)) = b | (o << 16);
}

__global__ void __launch_bounds__(128, 1) k_mlp_train_tc(const float *P, const float *norm, const float *G,
                                                         const float *V, const float *cE, float cF, int N,
                                                         float *part, uint32_t *status)
{
    count_launch();
    extern __shared__ __align__(1024) unsigned char tsm[];
    __shared__ TrSmall S;
    const int tid = threadIdx.x, warp = tid >> 5;
    unsigned char *sm = tsm;
    const uint32_t sb = smem_u32(sm);

    // weights in BF16: W1 [h][q], W2 [h][c], W2^T [c][h]; the ones operand
    for (int e = tid; e < 64 * 16; e += blockDim.x) {
        const int h = e / 16, q = e % 16;
        *reinterpret_cast<__nv_bfloat16 *>(sm + TS_W1 + kmajor_off(h, q, 16)) = __float2bfloat16_rn(P[P_W1 + e]);
    }
    for (int e = tid; e < 64 * 64; e += blockDim.x) {
        const int h = e / 64, c = e % 64;
        const __nv_bfloat16 v = __float2bfloat16_rn(P[P_W2 + e]);
        *reinterpret_cast<__nv_bfloat16 *>(sm + TS_W2 + kmajor_off(h, c, 64)) = v;
        *reinterpret_cast<__nv_bfloat16 *>(sm + TS_W2T + kmajor_off(c, h, 64)) = v;
    }
    for (int e = tid; e < 16 * TR_M; e += blockDim.x)
        *reinterpret_cast<__nv_bfloat16 *>(sm + TS_ONE + kmajor_off(e / TR_M, e % TR_M, TR_M)) =
            __float2bfloat16_rn(1.0f);
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
        S.timeout = 0u;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&S.bar)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&S.tmem_base)),
                     "r"(TR_TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    fence_async_smem();
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    const uint32_t tmem = S.tmem_base;
    const uint32_t lrow = tmem + ((uint32_t)(warp * 32) << 16);
    uint32_t phase = 0;
    const uint32_t id64 = idesc_bf16(TR_M, 64), id16 = idesc_bf16(TR_M, 16);

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
    // D[col] (+)= A B^T over `ks` K-steps of 16: A at byte offset a, B at b,
    // both K-major with stride-dimension offsets sa, sb_ (bytes per 8 rows)
    auto mma = [&](uint32_t col, uint32_t a, uint32_t sa, uint32_t b, uint32_t sbo, uint32_t id, int ks, bool acc) {
        for (int kk = 0; kk < ks; ++kk) {
            const uint64_t da = sdesc(sb + a + (uint32_t)kk * 256u, 128, sa);
            const uint64_t db = sdesc(sb + b + (uint32_t)kk * 256u, 128, sbo);
            mma_bf16(tmem + col, da, db, id, (acc || kk > 0) ? 1u : 0u);
        }
    };
    // operands written by the threads, visible to the tensor cores
    auto publish = [&]() {
        fence_async_smem();
        tc_before_sync();
        __syncthreads();
    };

    constexpr uint32_t S16 = 2 * 128, S64 = 8 * 128, S128 = 16 * 128;   // bytes per 8 rows for K = 16, 64, 128
    const int ntiles = (N + TR_M - 1) / TR_M;
    bool first = true;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int i = tile * TR_M + tid;
        const bool valid = i < N;
        // x = (G - mu) / sd, v = V / sd, c_E; zeros past the end
        float x[16], vt[16];
        float ce = 0.0f;
        {
            float g[16], w[16];
#pragma unroll
            for (int q = 0; q < 16; ++q) g[q] = w[q] = 0.0f;
            if (valid) {
                const float4 *gp = reinterpret_cast<const float4 *>(G + (size_t)i * 16);
                const float4 *vp = reinterpret_cast<const float4 *>(V + (size_t)i * 16);
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const float4 a = __ldg(gp + k), b = __ldg(vp + k);
                    g[4 * k] = a.x;
                    g[4 * k + 1] = a.y;
                    g[4 * k + 2] = a.z;
                    g[4 * k + 3] = a.w;
                    w[4 * k] = b.x;
                    w[4 * k + 1] = b.y;
                    w[4 * k + 2] = b.z;
                    w[4 * k + 3] = b.w;
                }
                ce = cE[i];
            }
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                x[q] = valid ? (g[q] - S.mu[q]) * S.isd[q] : 0.0f;
                vt[q] = w[q] * S.isd[q];
            }
        }
        st_row8(sm, TS_X, tid, 0, 16, x);
        st_row8(sm, TS_X, tid, 8, 16, x + 8);
        st_row8(sm, TS_VT, tid, 0, 16, vt);
        st_row8(sm, TS_VT, tid, 8, 16, vt + 8);
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            st_t(sm, TS_XT, q, tid, x[q]);
            st_t(sm, TS_VTT, q, tid, vt[q]);
        }
        st_t(sm, TS_T1, 192, tid, ce);
        publish();
        if (tid == 0) {
            tc_after_sync();
            mma(C_D1, TS_X, S16, TS_W1, S16, id64, 1, false);
            mma(C_DT1, TS_VT, S16, TS_W1, S16, id64, 1, false);
            mma_commit(&S.bar);
        }
        wait_mma();
        // layer 1: h1 = silu(a1), h1' = silu'(a1) DT1
#pragma unroll
        for (int c0 = 0; c0 < 64; c0 += 16) {
            float d[16], t[16], h[16], hd[16];
            tmem_ld16(lrow + C_D1 + c0, d);
            tmem_ld16(lrow + C_DT1 + c0, t);
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                const float a = d[k] + S.b1[c0 + k];
                const float s = tr_sigm(a);
                h[k] = a * s;
                hd[k] = s * (1.0f + a * (1.0f - s)) * t[k];
                st_t(sm, TS_H1T, c0 + k, tid, h[k]);
                st_t(sm, TS_HD1T, c0 + k, tid, hd[k]);
            }
            st_row8(sm, TS_H1, tid, c0, 64, h);
            st_row8(sm, TS_H1, tid, c0 + 8, 64, h + 8);
            st_row8(sm, TS_HD1, tid, c0, 64, hd);
            st_row8(sm, TS_HD1, tid, c0 + 8, 64, hd + 8);
        }
        publish();
        if (tid == 0) {
            tc_after_sync();
            mma(C_D2, TS_H1, S64, TS_W2, S64, id64, 4, false);
            mma(C_DT2, TS_HD1, S64, TS_W2, S64, id64, 4, false);
            mma_commit(&S.bar);
        }
        wait_mma();
        // layer 2 and its reverse: d2, e2 (into the H1, H1' buffers, which
        // the finished MMA2 no longer reads) and c3
#pragma unroll
        for (int c0 = 0; c0 < 64; c0 += 16) {
            float d[16], t[16], dv[16], ev[16];
            tmem_ld16(lrow + C_D2 + c0, d);
            tmem_ld16(lrow + C_DT2 + c0, t);
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                const float a = d[k] + S.b2[c0 + k];
                const float s = tr_sigm(a);
                const float s1 = s * (1.0f + a * (1.0f - s));
                const float s2 = s * (1.0f - s) * (2.0f + a * (1.0f - 2.0f * s));
                const float w = S.w3[c0 + k];
                dv[k] = ce * w * s1 - cF * w * s2 * t[k];
                ev[k] = -cF * w * s1;
                const float c3 = ce * a * s - cF * s1 * t[k];
                st_t(sm, TS_T1, c0 + k, tid, dv[k]);
                st_t(sm, TS_T1, 64 + c0 + k, tid, c3);
                st_t(sm, TS_T2, c0 + k, tid, ev[k]);
            }
            st_row8(sm, TS_H1, tid, c0, 64, dv);
            st_row8(sm, TS_H1, tid, c0 + 8, 64, dv + 8);
            st_row8(sm, TS_HD1, tid, c0, 64, ev);
            st_row8(sm, TS_HD1, tid, c0 + 8, 64, ev + 8);
        }
        publish();
        if (tid == 0) {
            tc_after_sync();
            mma(C_U, TS_H1, S64, TS_W2T, S64, id64, 4, false);
            mma(C_UE, TS_HD1, S64, TS_W2T, S64, id64, 4, false);
            mma(C_GW2, TS_T1, S128, TS_H1T, S128, id64, 8, !first);   // d2^T h1 (rows 0-63)
            mma(C_GW2, TS_T2, S128, TS_HD1T, S128, id64, 8, true);    // + e2^T h1'
            mma(C_GS1, TS_T1, S128, TS_ONE, S128, id16, 8, !first);   // db2 (rows 0-63), dw3 (64-127)
            mma_commit(&S.bar);
        }
        wait_mma();
        // back to layer 1: d1, e1
#pragma unroll
        for (int c0 = 0; c0 < 64; c0 += 16) {
            float u[16], ue[16], d[16], t[16];
            tmem_ld16(lrow + C_U + c0, u);
            tmem_ld16(lrow + C_UE + c0, ue);
            tmem_ld16(lrow + C_D1 + c0, d);
            tmem_ld16(lrow + C_DT1 + c0, t);
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                const float a = d[k] + S.b1[c0 + k];
                const float s = tr_sigm(a);
                const float s1 = s * (1.0f + a * (1.0f - s));
                const float s2 = s * (1.0f - s) * (2.0f + a * (1.0f - 2.0f * s));
                st_t(sm, TS_T1, 128 + c0 + k, tid, u[k] * s1 + ue[k] * s2 * t[k]);
                st_t(sm, TS_T2, 64 + c0 + k, tid, ue[k] * s1);
            }
        }
        publish();
        if (tid == 0) {
            tc_after_sync();
            mma(C_GW1, TS_T1 + 16 * S128, S128, TS_XT, S128, id16, 8, !first);   // d1^T x (rows 0-63)
            mma(C_GW1, TS_T2 + 8 * S128, S128, TS_VTT, S128, id16, 8, true);     // + e1^T v
            mma(C_GS2, TS_T1 + 16 * S128, S128, TS_ONE, S128, id16, 8, !first);  // db1 (rows 0-63), db3 (64)
            mma_commit(&S.bar);
        }
        wait_mma();
        first = false;
    }
    // this CTA's partial gradient (every CTA of the grid has a tile)
    float *pp = part + (size_t)blockIdx.x * P_TOTAL;
    if (!first) {
        float v[16];
        if (warp < 2) {   // rows 0-63: unit h = tid
#pragma unroll
            for (int c0 = 0; c0 < 64; c0 += 16) {
                tmem_ld16(lrow + C_GW2 + c0, v);
#pragma unroll
                for (int k = 0; k < 16; ++k) pp[P_W2 + tid * 64 + c0 + k] = v[k];
            }
            tmem_ld16(lrow + C_GW1, v);
#pragma unroll
            for (int k = 0; k < 16; ++k) pp[P_W1 + tid * 16 + k] = v[k];
            tmem_ld16(lrow + C_GS1, v);
            pp[P_B2 + tid] = v[0];
            tmem_ld16(lrow + C_GS2, v);
            pp[P_B1 + tid] = v[0];
        } else {          // rows 64-127
            tmem_ld16(lrow + C_GS1, v);
            pp[P_W3 + tid - 64] = v[0];
            tmem_ld16(lrow + C_GS2, v);
            if (tid == 64) pp[P_B3] = v[0];
        }
    }
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TR_TMEM_COLS));
    if (tid == 0 && S.timeout) raise_status(status, MD_ERR_TIMEOUT);
}

// grad[k] = sum over the CTAs' partials in CTA order (FP64).
__global__ void __launch_bounds__(256) k_mlp_grads_sum(const float *part, int nb, float *grad)
{
    count_launch();
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= P_TOTAL) return;
    double s = 0.0;
    for (int b = 0; b < nb; ++b) s += (double)part[(size_t)b * P_TOTAL + k];
    grad[k] = (float)s;
}

static int train_tc_grid(int N)
{
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms < 1) sms = 1;
        cudaFuncSetAttribute(k_mlp_train_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TS_TOTAL);
    }
    const int tiles = (N + TR_M - 1) / TR_M;
    return tiles < sms ? tiles : sms;
}

size_t mlp_train_tc_scratch(int N) { return sizeof(float) * (size_t)P_TOTAL * (size_t)((N + TR_M - 1) / TR_M); }

}  // namespace jmd

using namespace jmd;

extern "C" md_status md_bp_mlp_train_tc(const float *d_params, const float *d_norm, const float *d_G, const float *d_V,
                                        const float *d_cE, float cF, int N, void *d_scratch, float *d_grad,
                                        uint32_t *d_status, md_stream_t stream)
{
    if (!d_params || !d_norm || !d_G || !d_V || !d_cE || !d_scratch || !d_grad || N < 1) return MD_ERR_INVALID;
    if (((uintptr_t)d_scratch & 15u) || ((uintptr_t)d_G & 15u) || ((uintptr_t)d_V & 15u)) return MD_ERR_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    const int g = train_tc_grid(N);
    float *part = (float *)d_scratch;
    k_mlp_train_tc<<<g, 128, TS_TOTAL, st>>>(d_params, d_norm, d_G, d_V, d_cE, cF, N, part, d_status);
    k_mlp_grads_sum<<<(P_TOTAL + 255) / 256, 256, 0, st>>>(part, g, d_grad);
    JMD_CUDA_TRY(cudaGetLastError());
    return MD_OK;
}
