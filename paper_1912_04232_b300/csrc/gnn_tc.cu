// gnn_tc.cu -- the graph-network potential (same model as gnn.cu) with its
// products on the 5th-generation tensor cores: BF16 operands, FP32
// accumulation in tensor memory, H = 64.
//
// The edges with r < r_c are compacted in receiver order (CSR: the edges of
// atom i are eoff[i] .. eoff[i+1]), so every tile is 128 real rows:
//   k_gnnt_prep     per row slot: reverse slot, displacement, cutoff; count
//   k_gnnt_scan1/2  exclusive scan of the counts (chunks of 1024, then totals)
//   k_gnnt_compact  compact arrays (receiver, sender, slot, d, s)
//   k_gnnt_erev     compact index of every edge's reverse edge
// then, per message-passing step t (tiles of 128 rows, thread = row = TMEM
// lane, one elected thread issues the MMAs, completion on an mbarrier with
// a bounded wait):
//   k_gnnt_fe(t)    edges:  z = A_e e + (A_r v_i + a) + A_s v_j   [128x64]x[64x64]
//   k_gnnt_fn(t)    atoms:  m_i = sum s silu(z) (CSR row), zv = B [v; m] + b  [128x128]x[128x64],
//                   then [A_r; A_s] v of the next step [128x64]x[64x128], or the
//                   decoder D v and its transpose D^T g for the reverse pass
// and in reverse:
//   k_gnnt_bn(t)    atoms:  g_v = g_v(direct) + [A_r^T | A_s^T] [sum own gz; sum reverse gz],
//                   then [B_v^T; B_m^T] (g_v silu'(zv))           (step t + 1's products)
//   k_gnnt_be(t)    edges:  gz = (s g_m(i) + A_e^T gz(t + 1)) silu'(z); step 0 goes on
//                   through A_e^T into the encoder to dE/d(R_j - R_i)
//   k_gnnt_force    F_i = sum over its edges of g(i <- j) - g(j <- i)
#include <cuda_bf16.h>

#include <algorithm>

#include "common.cuh"
#include "gnn.cuh"
#include "kernels.cuh"
#include "reduce.cuh"
#include "tc.cuh"

namespace jmd {

constexpr int TH = 64;                    // hidden width of this path
constexpr int TM = 128;                   // rows per tile
constexpr int TT = 256;                   // threads per tile CTA: two per row
constexpr uint32_t TCOLS = 256;           // tensor-memory columns per CTA
constexpr uint32_t SMEM_TC = 108 * 1024;  // dynamic shared memory (also caps residency at 2 CTAs per SM)

struct TcBar {
    uint64_t bar;
    uint32_t tmem;
    uint32_t timeout;
};

__device__ __forceinline__ uint32_t bf2(float a, float b)
{
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t *>(&h);
}

// Eight consecutive K values (k0 a multiple of 8) of operand row `row`,
// split as v = hi + lo with hi and lo both BF16 (the pair carries 16
// significant bits, so the two MMAs below reproduce an FP32 activation to
// about 2^-17 relative).  hi goes to off, lo to off + lo_off.
__device__ __forceinline__ void put8(unsigned char *sm, uint32_t off, uint32_t lo_off, int row, int k0, int K,
                                     const float *v)
{
    float hi[8], lo[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        hi[q] = __bfloat162float(__float2bfloat16_rn(v[q]));
        lo[q] = v[q] - hi[q];
    }
    const uint32_t o = off + kmajor_off(row, k0, K);
    *reinterpret_cast<uint4 *>(sm + o) =
        make_uint4(bf2(hi[0], hi[1]), bf2(hi[2], hi[3]), bf2(hi[4], hi[5]), bf2(hi[6], hi[7]));
    *reinterpret_cast<uint4 *>(sm + o + lo_off) =
        make_uint4(bf2(lo[0], lo[1]), bf2(lo[2], lo[3]), bf2(lo[4], lo[5]), bf2(lo[6], lo[7]));
}

// B operand [n_out][K] (K-major) from a function of (out, k).
template <class F>
__device__ void stage_b(unsigned char *sm, uint32_t off, int n_out, int K, F f)
{
    for (int x = threadIdx.x; x < n_out * K; x += blockDim.x) {
        const int n = x / K, k = x - n * K;
        *reinterpret_cast<__nv_bfloat16 *>(sm + off + kmajor_off(n, k, K)) = __float2bfloat16_rn(f(n, k));
    }
}

__device__ __forceinline__ void tc_setup(TcBar &B)
{
    if (threadIdx.x == 0) {
        B.timeout = 0u;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&B.bar)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if ((threadIdx.x >> 5) == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&B.tmem)),
                     "r"(TCOLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    fence_async_smem();
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
}

__device__ __forceinline__ void tc_teardown(TcBar &B, uint32_t *status)
{
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    if ((threadIdx.x >> 5) == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(B.tmem), "r"(TCOLS));
    if (threadIdx.x == 0 && B.timeout) raise_status(status, MD_ERR_TIMEOUT);
}

// D[128 x N] (tensor-memory column d_col) = (A_hi + A_lo)[128 x K] B[N x K]^T
// (A_lo at a_off + lo_off); the operands written by all threads are made
// visible first; one thread issues both passes into the same accumulator.
__device__ __forceinline__ void tc_mma(TcBar &B, uint32_t &phase, uint32_t sbase, uint32_t a_off, uint32_t lo_off,
                                       uint32_t b_off, int K, int N, uint32_t d_col)
{
    fence_async_smem();
    tc_before_sync();
    __syncthreads();
    if (threadIdx.x == 0) {
        tc_after_sync();
        const uint32_t id = idesc_bf16(TM, N);
        for (int part = 0; part < 2; ++part) {
            const uint32_t a = a_off + (part ? lo_off : 0u);
            for (int kk = 0; kk < K / 16; ++kk) {
                const uint64_t da = sdesc(sbase + a + kk * 256, 128, (uint32_t)(K / 8) * 128);
                const uint64_t db = sdesc(sbase + b_off + kk * 256, 128, (uint32_t)(K / 8) * 128);
                mma_bf16(B.tmem + d_col, da, db, id, (part > 0 || kk > 0) ? 1u : 0u);
            }
        }
        mma_commit(&B.bar);
    }
    uint32_t it = 0;
    while (!mbar_try_wait(&B.bar, phase)) {
        if (++it > (1u << 26)) {
            B.timeout = 1u;
            break;
        }
    }
    phase ^= 1u;
    tc_after_sync();
}

// All tensor-memory reads of a tile done before the next tile's MMAs.
__device__ __forceinline__ void tc_tile_end()
{
    tc_before_sync();
    __syncthreads();
}

// This thread's tensor-memory lane quarter (warp w reads lanes 32 (w % 4) ..).
__device__ __forceinline__ uint32_t tc_row(const TcBar &B) { return B.tmem + ((uint32_t)(threadIdx.x & 96) << 16); }

__device__ __forceinline__ void ld4(const float *p, float *v)
{
    const float4 x = *reinterpret_cast<const float4 *>(p);
    v[0] = x.x;
    v[1] = x.y;
    v[2] = x.z;
    v[3] = x.w;
}
__device__ __forceinline__ void st4(float *p, const float *v)
{
    *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
}

// ---------------------------------------------------------------------------
// edge compaction
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_gnnt_prep(GnnArgs a)
{
    count_launch();
    const int lane = threadIdx.x & 31;
    for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < a.N; i += (gridDim.x * blockDim.x) >> 5) {
        int n = a.cnt[i];
        n = n < a.cap ? n : a.cap;
        const float4 ri = a.r[i];
        int nvalid = 0;
        for (int k0 = 0; k0 < n; k0 += 32) {
            const int k = k0 + lane;
            bool ok = false;
            if (k < n) {
                const size_t E = (size_t)i * a.cap + k;
                const int base = a.sys_n ? (i / a.sys_n) * a.sys_n : 0;
                const int j = a.nbr[E] + base;
                int rv = -1;
                float4 d4 = make_float4(0.f, 0.f, 0.f, -1.0f);
                if (j >= base && j < (a.sys_n ? base + a.sys_n : a.N) && j < a.N && j != i) {
                    float dx, dy, dz;
                    const float r2 = dist2_rn<3>(a.r[j], ri, a.box, dx, dy, dz);
                    if (r2 < a.rc2) {
                        int nj = a.cnt[j];
                        nj = nj < a.cap ? nj : a.cap;
                        const int32_t *rowj = a.nbr + (size_t)j * a.cap;
                        for (int p = 0; p < nj; ++p)
                            if (rowj[p] + base == i) {
                                rv = j * a.cap + p;
                                break;
                            }
                        if (rv < 0) raise_status(a.status, MD_ERR_NBR_OVERFLOW);
                        d4 = make_float4(dx, dy, dz, sqrtf(r2));
                        float sc, dsr;
                        gnn_cut(d4.w, a.rc, sc, dsr);
                        a.cut[E] = make_float2(sc, dsr);
                    }
                } else {
                    raise_status(a.status, MD_ERR_BOUNDS);
                }
                a.rev[E] = rv;
                a.dr[E] = d4;
                a.cidx[E] = -1;
                ok = rv >= 0;
            }
            nvalid += __popc(__ballot_sync(0xffffffffu, ok));
        }
        if (lane == 0) a.nv[i] = nvalid;
    }
}

// Block-wide exclusive scan of one int per thread (1024 threads); returns
// the thread's exclusive prefix, total in *tot.
__device__ __forceinline__ int block_scan_1024(int v, int *ws, int *tot)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) ws[w] = x;
    __syncthreads();
    if (w == 0) {
        int s = ws[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        ws[lane] = s;
    }
    __syncthreads();
    *tot = ws[31];
    return x - v + (w > 0 ? ws[w - 1] : 0);
}

// Exclusive scan of nv into eoff, in two levels: chunks of 1024 atoms
// (coalesced, one block each), then the chunk totals (one block).
__global__ void __launch_bounds__(1024) k_gnnt_scan1(GnnArgs a)
{
    count_launch();
    __shared__ int ws[32];
    const int i = blockIdx.x * 1024 + threadIdx.x;
    int tot;
    const int ex = block_scan_1024(i < a.N ? a.nv[i] : 0, ws, &tot);
    if (i < a.N) a.eoff[i] = ex;
    if (threadIdx.x == 0) a.ctot[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(1024) k_gnnt_scan2(GnnArgs a, int nchunk)
{
    count_launch();
    __shared__ int ws[32];
    __shared__ int base;
    // chunk totals to offsets, 1024 at a time
    if (threadIdx.x == 0) base = 0;
    __syncthreads();
    for (int c0 = 0; c0 < nchunk; c0 += 1024) {
        const int c = c0 + threadIdx.x;
        int tot;
        const int ex = block_scan_1024(c < nchunk ? a.ctot[c] : 0, ws, &tot);
        const int b0 = base;
        __syncthreads();
        if (c < nchunk) a.ctot[c] = b0 + ex;
        if (threadIdx.x == 0) base = b0 + tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) a.eoff[a.N] = base;   // k_gnnt_compact adds the chunk offsets
}

__global__ void __launch_bounds__(256) k_gnnt_compact(GnnArgs a)
{
    count_launch();
    const int lane = threadIdx.x & 31;
    for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < a.N; i += (gridDim.x * blockDim.x) >> 5) {
        int n = a.cnt[i];
        n = n < a.cap ? n : a.cap;
        int x = a.eoff[i] + a.ctot[i >> 10];
        __syncwarp();
        if (lane == 0) a.eoff[i] = x;
        for (int k0 = 0; k0 < n; k0 += 32) {
            const int k = k0 + lane;
            const size_t E = (size_t)i * a.cap + k;
            const int rv = k < n ? a.rev[E] : -1;
            const unsigned b = __ballot_sync(0xffffffffu, rv >= 0);
            if (rv >= 0) {
                const int e = x + __popc(b & ((1u << lane) - 1u));
                a.erecv[e] = i;
                a.esend[e] = rv / a.cap;
                a.eslot[e] = (int)E;
                a.cidx[E] = e;
                a.edr[e] = a.dr[E];
                a.ecut[e] = a.cut[E];
            }
            x += __popc(b);
        }
    }
}

__global__ void __launch_bounds__(256) k_gnnt_erev(GnnArgs a)
{
    count_launch();
    const int E = a.eoff[a.N];
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < E; e += gridDim.x * blockDim.x) {
        const int er = a.cidx[a.rev[a.eslot[e]]];
        if (er < 0 || er >= E) {
            raise_status(a.status, MD_ERR_BOUNDS);
            a.erev[e] = e;
        } else {
            a.erev[e] = er;
        }
    }
}

// ---------------------------------------------------------------------------
// forward
// ---------------------------------------------------------------------------
// Two threads per row (TT = 256): thread x owns row x & 127 (tensor-memory
// lane) and the column half cb = 32 (x >> 7) of every 64-wide block, so each
// row's loads are split over two threads and more of them are in flight.
__global__ void __launch_bounds__(TT, 2) k_gnnt_fe(GnnArgs a, int t)
{
    count_launch();
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ TcBar B;
    __shared__ float cv[2 * TH], wenc[3 * TH], benc[TH];
    constexpr uint32_t SW = 0, SX = SW + TH * TH * 2, LO = TM * TH * 2;   // X_lo at SX + LO
    const uint32_t sbase = smem_u32(sm);
    const GnnOff &o = a.off;
    const float *P = a.P;
    stage_b(sm, SW, TH, TH, [&](int n, int k) { return __ldg(P + o.A[t] + n * 3 * TH + k); });
    for (int h = threadIdx.x; h < TH; h += blockDim.x) {
        wenc[3 * h] = __ldg(P + o.Wenc + 3 * h);
        wenc[3 * h + 1] = __ldg(P + o.Wenc + 3 * h + 1);
        wenc[3 * h + 2] = __ldg(P + o.Wenc + 3 * h + 2);
        benc[h] = __ldg(P + o.benc + h);
        if (t == 0) {
            float sr = __ldg(P + o.a[0] + h), sp = 0.0f;
            for (int c = 0; c < TH; ++c) {
                const float uc = __ldg(P + o.u + c);
                sr += __ldg(P + o.A[0] + h * 3 * TH + TH + c) * uc;
                sp += __ldg(P + o.A[0] + h * 3 * TH + 2 * TH + c) * uc;
            }
            cv[h] = sr;
            cv[TH + h] = sp;
        }
    }
    tc_setup(B);
    uint32_t phase = 0;
    const int E = a.eoff[a.N];
    const size_t NE = (size_t)a.N * a.cap;
    float *ze_t = a.ze + (size_t)t * NE * TH;
    const float *ze_p = t > 0 ? a.ze + (size_t)(t - 1) * NE * TH : nullptr;
    const float inv_rc = 1.0f / a.rc;
    const int row = threadIdx.x & (TM - 1), cb = 32 * (threadIdx.x >> 7);
    for (int tile = blockIdx.x; tile * TM < E; tile += gridDim.x) {
        const int e = tile * TM + row;
        const bool valid = e < E;
        float v[32];
        if (!valid) {
#pragma unroll
            for (int q = 0; q < 32; ++q) v[q] = 0.0f;
        } else if (t == 0) {
            const float4 d4 = a.edr[e];
#pragma unroll
            for (int q = 0; q < 32; ++q) {
                const int c = cb + q;
                v[q] = gnn_silu(wenc[3 * c] * (d4.x * inv_rc) + wenc[3 * c + 1] * (d4.y * inv_rc) +
                                wenc[3 * c + 2] * (d4.z * inv_rc) + benc[c]);
            }
        } else {
#pragma unroll
            for (int q = 0; q < 32; q += 4) ld4(ze_p + (size_t)e * TH + cb + q, v + q);
#pragma unroll
            for (int q = 0; q < 32; ++q) v[q] = gnn_silu(v[q]);
        }
#pragma unroll
        for (int q = 0; q < 32; q += 8) put8(sm, SX, LO, row, cb + q, TH, v + q);
        tc_mma(B, phase, sbase, SX, LO, SW, TH, TH, 0);
        const int recv = valid ? a.erecv[e] : 0, send = valid ? a.esend[e] : 0;
        float x[32], y[32];
        if (valid) {
            if (t == 0) {
#pragma unroll
                for (int q = 0; q < 32; ++q) {
                    x[q] = cv[cb + q];
                    y[q] = cv[TH + cb + q];
                }
            } else {
#pragma unroll
                for (int q = 0; q < 32; q += 4) {
                    ld4(a.rr + (size_t)recv * TH + cb + q, x + q);
                    ld4(a.ps + (size_t)send * TH + cb + q, y + q);
                }
            }
        }
#pragma unroll
        for (int c0 = 0; c0 < 32; c0 += 16) {
            float d[16];
            tmem_ld16(tc_row(B) + cb + c0, d);
            if (valid) {
#pragma unroll
                for (int q = 0; q < 16; ++q) d[q] += x[c0 + q] + y[c0 + q];
#pragma unroll
                for (int q = 0; q < 16; q += 4) st4(ze_t + (size_t)e * TH + cb + c0 + q, d + q);
            }
        }
        tc_tile_end();
    }
    tc_teardown(B, a.status);
}

__global__ void __launch_bounds__(TT, 2) k_gnnt_fn(GnnArgs a, int t)
{
    count_launch();
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ TcBar B;
    __shared__ float bt[TH], an[TH], dd[TH], ww[TH], uu[TH];
    __shared__ float red[TM];
    constexpr uint32_t SWB = 0;                       // B_t: [64][128]
    constexpr uint32_t SWN = SWB + TH * 2 * TH * 2;   // [A_r; A_s] of t + 1: [128][64]; last: D [64][64]
    constexpr uint32_t SWD = SWN + 2 * TH * TH * 2;   // last: D^T [64][64]
    constexpr uint32_t SX = SWD + TH * TH * 2;        // [v; m]: [128][128], hi then lo
    constexpr uint32_t LO = TM * 2 * TH * 2;
    constexpr uint32_t SX2 = SX;                      // [128][64], hi then lo (after the first product)
    constexpr uint32_t LO2 = TM * TH * 2;
    const uint32_t sbase = smem_u32(sm);
    const GnnOff &o = a.off;
    const float *P = a.P;
    const bool last = t == a.T - 1;
    stage_b(sm, SWB, TH, 2 * TH, [&](int n, int k) { return __ldg(P + o.B[t] + n * 2 * TH + k); });
    if (!last) {
        stage_b(sm, SWN, 2 * TH, TH, [&](int n, int k) {
            return n < TH ? __ldg(P + o.A[t + 1] + n * 3 * TH + TH + k)
                          : __ldg(P + o.A[t + 1] + (n - TH) * 3 * TH + 2 * TH + k);
        });
    } else {
        stage_b(sm, SWN, TH, TH, [&](int n, int k) { return __ldg(P + o.D + n * TH + k); });
        stage_b(sm, SWD, TH, TH, [&](int n, int k) { return __ldg(P + o.D + k * TH + n); });
    }
    for (int h = threadIdx.x; h < TH; h += blockDim.x) {
        bt[h] = __ldg(P + o.b[t] + h);
        an[h] = last ? 0.0f : __ldg(P + o.a[t + 1] + h);
        dd[h] = __ldg(P + o.d + h);
        ww[h] = __ldg(P + o.w + h);
        uu[h] = __ldg(P + o.u + h);
    }
    tc_setup(B);
    uint32_t phase = 0;
    const size_t NE = (size_t)a.N * a.cap;
    const float *ze_t = a.ze + (size_t)t * NE * TH;
    const float cdec = __ldg(P + o.c);
    const int row = threadIdx.x & (TM - 1), hf = threadIdx.x >> 7, cb = 32 * hf;
    for (int tile = blockIdx.x; tile * TM < a.N; tile += gridDim.x) {
        const int i = tile * TM + row;
        const bool valid = i < a.N;
        const int e0 = valid ? a.eoff[i] : 0, e1 = valid ? a.eoff[i + 1] : 0;
        // A row: [v of step t - 1 | m], columns cb .. cb + 32 of each half
        {
            float v[32], m[32];
            if (!valid) {
#pragma unroll
                for (int q = 0; q < 32; ++q) v[q] = 0.0f;
            } else if (t == 0) {
#pragma unroll
                for (int q = 0; q < 32; ++q) v[q] = uu[cb + q];
            } else {
                const float *zp = a.zv + ((size_t)(t - 1) * a.N + i) * TH + cb;
#pragma unroll
                for (int q = 0; q < 32; q += 4) ld4(zp + q, v + q);
#pragma unroll
                for (int q = 0; q < 32; ++q) v[q] = gnn_silu(v[q]);
            }
#pragma unroll
            for (int q = 0; q < 32; ++q) m[q] = 0.0f;
            for (int e = e0; e < e1; ++e) {
                const float s = a.ecut[e].x;
                float z[32];
#pragma unroll
                for (int q = 0; q < 32; q += 4) ld4(ze_t + (size_t)e * TH + cb + q, z + q);
#pragma unroll
                for (int q = 0; q < 32; ++q) m[q] += s * gnn_silu(z[q]);
            }
#pragma unroll
            for (int q = 0; q < 32; q += 8) {
                put8(sm, SX, LO, row, cb + q, 2 * TH, v + q);
                put8(sm, SX, LO, row, TH + cb + q, 2 * TH, m + q);
            }
        }
        tc_mma(B, phase, sbase, SX, LO, SWB, 2 * TH, TH, 0);
        // zv = D + b; v = silu(zv)
#pragma unroll
        for (int c0 = 0; c0 < 32; c0 += 16) {
            float d[16];
            tmem_ld16(tc_row(B) + cb + c0, d);
#pragma unroll
            for (int q = 0; q < 16; ++q) d[q] += bt[cb + c0 + q];
            if (valid) {
#pragma unroll
                for (int q = 0; q < 16; q += 4) st4(a.zv + ((size_t)t * a.N + i) * TH + cb + c0 + q, d + q);
            }
#pragma unroll
            for (int q = 0; q < 16; ++q) d[q] = valid ? gnn_silu(d[q]) : 0.0f;
            put8(sm, SX2, LO2, row, cb + c0, TH, d);
            put8(sm, SX2, LO2, row, cb + c0 + 8, TH, d + 8);
        }
        if (!last) {
            // receiver term (first half of the threads) and sender term (second)
            tc_mma(B, phase, sbase, SX2, LO2, SWN, TH, 2 * TH, TH);
            float *dst = (hf ? a.ps : a.rr) + (size_t)i * TH;
#pragma unroll
            for (int c0 = 0; c0 < TH; c0 += 16) {
                float d[16];
                tmem_ld16(tc_row(B) + TH + hf * TH + c0, d);
                if (valid) {
                    if (!hf) {
#pragma unroll
                        for (int q = 0; q < 16; ++q) d[q] += an[c0 + q];
                    }
#pragma unroll
                    for (int q = 0; q < 16; q += 4) st4(dst + c0 + q, d + q);
                }
            }
        } else {
            // decoder: E_i = w . silu(D v + d) + c, and g = w silu'(D v + d) for D^T g
            tc_mma(B, phase, sbase, SX2, LO2, SWN, TH, TH, TH);
            float part = 0.0f;
#pragma unroll
            for (int c0 = 0; c0 < 32; c0 += 16) {
                float d[16];
                tmem_ld16(tc_row(B) + TH + cb + c0, d);
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const int c = cb + c0 + q;
                    const float z = d[q] + dd[c], sg = gnn_sig(z);
                    part += ww[c] * z * sg;
                    d[q] = valid ? ww[c] * sg * (1.0f + z * (1.0f - sg)) : 0.0f;
                }
                put8(sm, SX2, LO2, row, cb + c0, TH, d);
                put8(sm, SX2, LO2, row, cb + c0 + 8, TH, d + 8);
            }
            if (hf) red[row] = part;
            __syncthreads();
            if (!hf && valid) a.Ei[i] = part + red[row] + cdec;
            tc_mma(B, phase, sbase, SX2, LO2, SWD, TH, TH, 2 * TH);
#pragma unroll
            for (int c0 = 0; c0 < 32; c0 += 16) {
                float d[16];
                tmem_ld16(tc_row(B) + 2 * TH + cb + c0, d);
                if (valid) {
#pragma unroll
                    for (int q = 0; q < 16; q += 4) st4(a.gvd + (size_t)i * TH + cb + c0 + q, d + q);
                }
            }
        }
        tc_tile_end();
    }
    tc_teardown(B, a.status);
}

// ---------------------------------------------------------------------------
// reverse
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(TT, 2) k_gnnt_bn(GnnArgs a, int t)
{
    count_launch();
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ TcBar B;
    constexpr uint32_t SWS = 0;                       // [A_r^T | A_s^T] of t + 1: [64][128]
    constexpr uint32_t SWB = SWS + TH * 2 * TH * 2;   // [B_v^T; B_m^T] of t: [128][64]
    constexpr uint32_t SX = SWB + 2 * TH * TH * 2;    // [sum own; sum reverse]: [128][128], hi then lo
    constexpr uint32_t LO = TM * 2 * TH * 2;
    constexpr uint32_t SX2 = SX;                      // [128][64], hi then lo (after the first product)
    constexpr uint32_t LO2 = TM * TH * 2;
    const uint32_t sbase = smem_u32(sm);
    const GnnOff &o = a.off;
    const float *P = a.P;
    const bool last = t == a.T - 1;
    if (!last) {
        stage_b(sm, SWS, TH, 2 * TH, [&](int n, int k) {
            return k < TH ? __ldg(P + o.A[t + 1] + k * 3 * TH + TH + n)
                          : __ldg(P + o.A[t + 1] + (k - TH) * 3 * TH + 2 * TH + n);
        });
    }
    stage_b(sm, SWB, 2 * TH, TH, [&](int n, int k) { return __ldg(P + o.B[t] + k * 2 * TH + n); });
    tc_setup(B);
    uint32_t phase = 0;
    const size_t NE = (size_t)a.N * a.cap;
    const float *gz_n = last ? nullptr : a.ze + (size_t)(t + 1) * NE * TH;
    const int row = threadIdx.x & (TM - 1), hf = threadIdx.x >> 7, cb = 32 * hf;
    for (int tile = blockIdx.x; tile * TM < a.N; tile += gridDim.x) {
        const int i = tile * TM + row;
        const bool valid = i < a.N;
        if (!last) {
            const int e0 = valid ? a.eoff[i] : 0, e1 = valid ? a.eoff[i + 1] : 0;
            float sr[32], ss[32];
#pragma unroll
            for (int q = 0; q < 32; ++q) sr[q] = ss[q] = 0.0f;
            for (int e = e0; e < e1; ++e) {
                const int er = a.erev[e];
                float x[32], y[32];
#pragma unroll
                for (int q = 0; q < 32; q += 4) {
                    ld4(gz_n + (size_t)e * TH + cb + q, x + q);
                    ld4(gz_n + (size_t)er * TH + cb + q, y + q);
                }
#pragma unroll
                for (int q = 0; q < 32; ++q) {
                    sr[q] += x[q];
                    ss[q] += y[q];
                }
            }
#pragma unroll
            for (int q = 0; q < 32; q += 8) {
                put8(sm, SX, LO, row, cb + q, 2 * TH, sr + q);
                put8(sm, SX, LO, row, TH + cb + q, 2 * TH, ss + q);
            }
            tc_mma(B, phase, sbase, SX, LO, SWS, 2 * TH, TH, 0);
        }
        // g_v silu'(zv) -> A operand of the node-update transpose
#pragma unroll
        for (int c0 = 0; c0 < 32; c0 += 16) {
            float g[16];
            if (!last) tmem_ld16(tc_row(B) + cb + c0, g);
            else {
#pragma unroll
                for (int q = 0; q < 16; ++q) g[q] = 0.0f;
            }
            if (valid) {
                float gd[16], z[16];
#pragma unroll
                for (int q = 0; q < 16; q += 4) {
                    ld4(a.gvd + (size_t)i * TH + cb + c0 + q, gd + q);
                    ld4(a.zv + ((size_t)t * a.N + i) * TH + cb + c0 + q, z + q);
                }
#pragma unroll
                for (int q = 0; q < 16; ++q) g[q] = (g[q] + gd[q]) * gnn_dsilu(z[q]);
            } else {
#pragma unroll
                for (int q = 0; q < 16; ++q) g[q] = 0.0f;
            }
            put8(sm, SX2, LO2, row, cb + c0, TH, g);
            put8(sm, SX2, LO2, row, cb + c0 + 8, TH, g + 8);
        }
        tc_mma(B, phase, sbase, SX2, LO2, SWB, TH, 2 * TH, TH);
        // direct gradient of step t - 1 (first half) and message gradient (second)
        if (hf == 1 || t > 0) {
            float *dst = (hf ? a.gm : a.gvd) + (size_t)i * TH;
#pragma unroll
            for (int c0 = 0; c0 < TH; c0 += 16) {
                float d[16];
                tmem_ld16(tc_row(B) + TH + hf * TH + c0, d);
                if (valid) {
#pragma unroll
                    for (int q = 0; q < 16; q += 4) st4(dst + c0 + q, d + q);
                }
            }
        }
        tc_tile_end();
    }
    tc_teardown(B, a.status);
}

__global__ void __launch_bounds__(TT, 2) k_gnnt_be(GnnArgs a, int t)
{
    count_launch();
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ TcBar B;
    __shared__ float wenc[3 * TH], benc[TH];
    __shared__ float4 red[TM];
    constexpr uint32_t SWA = 0;                  // A_e^T of step t + 1: [64][64]
    constexpr uint32_t SW0 = SWA + TH * TH * 2;  // A_e^T of step 0: [64][64]
    constexpr uint32_t SX = SW0 + TH * TH * 2;   // gz of step t + 1: [128][64], hi then lo
    constexpr uint32_t LO = TM * TH * 2;
    constexpr uint32_t SX2 = SX + 2 * LO;        // gz of step 0: [128][64], hi then lo
    const uint32_t sbase = smem_u32(sm);
    const GnnOff &o = a.off;
    const float *P = a.P;
    const bool last = t == a.T - 1;
    if (!last) stage_b(sm, SWA, TH, TH, [&](int n, int k) { return __ldg(P + o.A[t + 1] + k * 3 * TH + n); });
    if (t == 0) stage_b(sm, SW0, TH, TH, [&](int n, int k) { return __ldg(P + o.A[0] + k * 3 * TH + n); });
    for (int h = threadIdx.x; h < TH; h += blockDim.x) {
        wenc[3 * h] = __ldg(P + o.Wenc + 3 * h);
        wenc[3 * h + 1] = __ldg(P + o.Wenc + 3 * h + 1);
        wenc[3 * h + 2] = __ldg(P + o.Wenc + 3 * h + 2);
        benc[h] = __ldg(P + o.benc + h);
    }
    tc_setup(B);
    uint32_t phase = 0;
    const int E = a.eoff[a.N];
    const size_t NE = (size_t)a.N * a.cap;
    float *ze_t = a.ze + (size_t)t * NE * TH;
    const float *gz_n = last ? nullptr : a.ze + (size_t)(t + 1) * NE * TH;
    const float inv_rc = 1.0f / a.rc;
    const int row = threadIdx.x & (TM - 1), hf = threadIdx.x >> 7, cb = 32 * hf;
    for (int tile = blockIdx.x; tile * TM < E; tile += gridDim.x) {
        const int e = tile * TM + row;
        const bool valid = e < E;
        if (!last) {
            float v[32];
            if (valid) {
#pragma unroll
                for (int q = 0; q < 32; q += 4) ld4(gz_n + (size_t)e * TH + cb + q, v + q);
            } else {
#pragma unroll
                for (int q = 0; q < 32; ++q) v[q] = 0.0f;
            }
#pragma unroll
            for (int q = 0; q < 32; q += 8) put8(sm, SX, LO, row, cb + q, TH, v + q);
            tc_mma(B, phase, sbase, SX, LO, SWA, TH, TH, 0);
        }
        const int recv = valid ? a.erecv[e] : 0;
        const float s = valid ? a.ecut[e].x : 0.0f;
        float z[32], gm[32];
        if (valid) {
#pragma unroll
            for (int q = 0; q < 32; q += 4) {
                ld4(ze_t + (size_t)e * TH + cb + q, z + q);
                ld4(a.gm + (size_t)recv * TH + cb + q, gm + q);
            }
        }
        float gsv = 0.0f;
#pragma unroll
        for (int c0 = 0; c0 < 32; c0 += 16) {
            float d[16];
            if (!last) tmem_ld16(tc_row(B) + cb + c0, d);
            else {
#pragma unroll
                for (int q = 0; q < 16; ++q) d[q] = 0.0f;
            }
            if (valid) {
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const float zz = z[c0 + q], sg = gnn_sig(zz);
                    gsv += gm[c0 + q] * (zz * sg);
                    d[q] = (s * gm[c0 + q] + d[q]) * (sg * (1.0f + zz * (1.0f - sg)));
                }
                if (t > 0) {
#pragma unroll
                    for (int q = 0; q < 16; q += 4) st4(ze_t + (size_t)e * TH + cb + c0 + q, d + q);
                }
            } else {
#pragma unroll
                for (int q = 0; q < 16; ++q) d[q] = 0.0f;
            }
            if (t == 0) {
                put8(sm, SX2, LO, row, cb + c0, TH, d);
                put8(sm, SX2, LO, row, cb + c0 + 8, TH, d + 8);
            }
        }
        // dE/ds of the edge: the two halves' parts
        if (hf) red[row].x = gsv;
        __syncthreads();
        float gs_tot = 0.0f;
        if (!hf && valid) {
            gs_tot = (last ? 0.0f : a.gs[e]) + gsv + red[row].x;
            a.gs[e] = gs_tot;
        }
        if (t == 0) {
            // through step 0's A_e into the encoder, then to the displacement
            tc_mma(B, phase, sbase, SX2, LO, SW0, TH, TH, TH);
            const float4 d4 = valid ? a.edr[e] : make_float4(0.f, 0.f, 0.f, 1.f);
            float gx = 0.f, gy = 0.f, gz = 0.f;
#pragma unroll
            for (int c0 = 0; c0 < 32; c0 += 16) {
                float g0[16];
                tmem_ld16(tc_row(B) + TH + cb + c0, g0);
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const int c = cb + c0 + q;
                    const float z0 = wenc[3 * c] * (d4.x * inv_rc) + wenc[3 * c + 1] * (d4.y * inv_rc) +
                                     wenc[3 * c + 2] * (d4.z * inv_rc) + benc[c];
                    const float g = g0[q] * gnn_dsilu(z0);
                    gx += wenc[3 * c] * g;
                    gy += wenc[3 * c + 1] * g;
                    gz += wenc[3 * c + 2] * g;
                }
            }
            if (hf) red[row] = make_float4(gx, gy, gz, 0.0f);
            __syncthreads();
            if (!hf && valid) {
                const float4 o2 = red[row];
                const float cc = gs_tot * a.ecut[e].y;
                a.gpos[e] = make_float4((gx + o2.x) * inv_rc + cc * d4.x, (gy + o2.y) * inv_rc + cc * d4.y,
                                        (gz + o2.z) * inv_rc + cc * d4.z, 0.0f);
            }
        }
        tc_tile_end();
    }
    tc_teardown(B, a.status);
}

template <int KICK>
__global__ void __launch_bounds__(256) k_gnnt_force(GnnArgs g, PairArgs pa)
{
    count_launch();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float pe_acc = 0.0f, ke_acc = 0.0f;
    for (int i = blockIdx.x * 8 + w; i < g.N; i += gridDim.x * 8) {
        const int e0 = g.eoff[i], e1 = g.eoff[i + 1];
        float fx = 0.f, fy = 0.f, fz = 0.f;
        for (int e = e0 + lane; e < e1; e += 32) {
            const float4 a4 = g.gpos[e], b4 = g.gpos[g.erev[e]];
            fx += a4.x - b4.x;
            fy += a4.y - b4.y;
            fz += a4.z - b4.z;
        }
        fx = gnn_wsum(fx);
        fy = gnn_wsum(fy);
        fz = gnn_wsum(fz);
        if (lane == 0) {
            const float ei = g.Ei[i];
            pa.f[i] = make_float4(fx, fy, fz, ei);
            pe_acc += ei;
            if (KICK) ke_acc += half_kick<3>(pa, i, fx, fy, fz);
        }
        __syncwarp();
    }
    if (!pa.E_out && !KICK && !pa.nhc) return;
    energy_epilogue(pe_acc, ke_acc, pa);
}

// The edges with r < r_c compacted in receiver order (also used by the
// training kernels of gnn_train.cu).
void enqueue_gnn_compact(const GnnArgs &g, cudaStream_t st)
{
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms < 1) sms = 1;
    }
    const int wgrid = std::max(1, std::min((g.N * 32 + 255) / 256, sms * 8));
    k_gnnt_prep<<<wgrid, 256, 0, st>>>(g);
    const int nchunk = (g.N + 1023) / 1024;
    k_gnnt_scan1<<<nchunk, 1024, 0, st>>>(g);
    k_gnnt_scan2<<<1, 1024, 0, st>>>(g, nchunk);
    k_gnnt_compact<<<wgrid, 256, 0, st>>>(g);
    k_gnnt_erev<<<sms * 4, 256, 0, st>>>(g);
}

void enqueue_gnn_tc(const GnnArgs &g, const PairArgs &pa, int kick, cudaStream_t st)
{
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms < 1) sms = 1;
        cudaFuncSetAttribute(k_gnnt_fe, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_TC);
        cudaFuncSetAttribute(k_gnnt_fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_TC);
        cudaFuncSetAttribute(k_gnnt_bn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_TC);
        cudaFuncSetAttribute(k_gnnt_be, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_TC);
    }
    enqueue_gnn_compact(g, st);
    const int tgrid = 2 * sms;
    for (int t = 0; t < g.T; ++t) {
        k_gnnt_fe<<<tgrid, TT, SMEM_TC, st>>>(g, t);
        k_gnnt_fn<<<tgrid, TT, SMEM_TC, st>>>(g, t);
    }
    for (int t = g.T - 1; t >= 0; --t) {
        k_gnnt_bn<<<tgrid, TT, SMEM_TC, st>>>(g, t);
        k_gnnt_be<<<tgrid, TT, SMEM_TC, st>>>(g, t);
    }
    const int fgrid = std::max(1, std::min((g.N + 7) / 8, pa.max_blocks));
    if (kick) k_gnnt_force<1><<<fgrid, 256, 0, st>>>(g, pa);
    else k_gnnt_force<0><<<fgrid, 256, 0, st>>>(g, pa);
}

}  // namespace jmd
