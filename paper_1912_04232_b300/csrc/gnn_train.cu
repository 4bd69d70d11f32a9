// gnn_train.cu -- gradient of the graph network's energy + force loss with
// respect to its parameters (Sec. 4.1: the GNN is fitted to energies and
// forces), FP32 CUDA cores, H = 64.
//
// With c_E,i = dL/dE_i and u_k = dL/dF_k (md_bp_loss_prep), the loss
// gradient is that of
//     J = sum_i c_E,i E_i - psi,   psi = sum_k u_k . dE/dR_k
// (F = -dE/dR).  psi is the derivative of E along the position tangent u:
// it is computed forward, every activation carrying its tangent (x' =
// (u_j - u_i)/r_c on the edge inputs, s' = s'(r) d.(u_j - u_i)/r on the
// cutoff), and dJ/dtheta by one reverse sweep through both the values and
// the tangents -- second derivatives of silu appear where a tangent meets
// its value.  Seeds: c_E on E_i, -1 on the tangent of E_i.
//
//   k_gt_tan   per compact edge: (u_j - u_i, s')
//   k_gt_fe(t) per edge (one warp): z = A_e e + A_r v_i + A_s v_j + a and z'
//   k_gt_fn(t) per atom (one warp): m, m', zv = B [v; m] + b and zv', the next
//              step's node terms, or (last step) the decoder with its
//              reverse: zd, zd', their adjoints and D^T of them
//   k_gt_bn(t) per atom: adjoints of v and v' -> zv, zv' -> m, m' and the
//              direct part of the step below
//   k_gt_be(t) per edge: adjoints of e, e' -> z, z' (stored over z, z');
//              step 0 continues into the encoder
//   k_gt_outer outer-product sums over rows (edges or atoms), one 64 x 16
//              output tile per block and one chunk of rows per grid row,
//              FP32 within a staged batch of rows, FP64 across batches;
//   k_gt_reduce the chunks in fixed order into the gradient
// Every sum has a fixed order; no atomics.
#include <algorithm>

#include "common.cuh"
#include "gnn.cuh"
#include "kernels.cuh"

namespace jmd {

constexpr int GT_H = 64;
constexpr int GT_WARPS = 8;
constexpr int GT_CHUNKS = 64;    // row chunks of the outer-product sums

struct GtArgs {
    GnnArgs g;
    const float4 *u;     // [N] dL/dF
    const float *cE;     // [N] dL/dE_i
    float *zt;           // [T][Ecap][64] edge tangents z'
    float *zvt;          // [T][N][64]  node tangents zv'
    float *m, *mt;       // [T][N][64]  messages and their tangents
    float *rrt, *pst;    // [N][64]     tangents of the next step's node terms
    float *zd, *zdt;     // [N][64]     decoder pre-activation and tangent
    float *zdb, *zdbt;   // [N][64]     their adjoints
    float *vb, *vbt;     // [N][64]     node adjoints carried down
    float *zvb, *zvbt;   // [N][64]     adjoints of zv, zv' of the current step
    float *mb, *mbt;     // [N][64]     adjoints of m, m'
    float4 *etan;        // [Ecap]      u_j - u_i, s'
    float *encb, *encbt; // [Ecap][64]  encoder adjoints
    double *part;        // [GT_CHUNKS][64][193] outer-sum chunks
    double *cbar;        // [1]
    float *grad;         // [param count]
};

__device__ __forceinline__ void gt_sl3(float x, float &v, float &d1, float &d2)
{
    const float s = gnn_sig(x);
    v = x * s;
    d1 = s * (1.0f + x * (1.0f - s));
    d2 = s * (1.0f - s) * (2.0f + x * (1.0f - 2.0f * s));
}

// W block (rows h, columns c0 .. c0 + K of a row-major matrix with ld
// columns) in shared memory as M[k][h]: lane h of a product W x reads
// consecutive words.
__device__ void gt_stage_fwd(float *M, const float *P, int base, int ld, int c0, int K)
{
    for (int x = threadIdx.x; x < K * GT_H; x += blockDim.x) {
        const int k = x / GT_H, h = x - k * GT_H;
        M[x] = __ldg(P + base + (size_t)h * ld + c0 + k);
    }
}

// The same block as M[h][c]: lane c of a product W^T g reads consecutive
// words.
__device__ void gt_stage_bwd(float *M, const float *P, int base, int ld, int c0)
{
    for (int x = threadIdx.x; x < GT_H * GT_H; x += blockDim.x) {
        const int h = x / GT_H, c = x - h * GT_H;
        M[x] = __ldg(P + base + (size_t)h * ld + c0 + c);
    }
}

// y0, y1 += sum_k M[k][lane (+32)] x[k]
__device__ __forceinline__ void gt_mv(const float *M, int K, const float *x, float &y0, float &y1)
{
    const int lane = threadIdx.x & 31;
#pragma unroll 8
    for (int k = 0; k < K; ++k) {
        const float xk = x[k];
        y0 += M[k * GT_H + lane] * xk;
        y1 += M[k * GT_H + lane + 32] * xk;
    }
}

__global__ void __launch_bounds__(256) k_gt_tan(GtArgs a)
{
    count_launch();
    const GnnArgs &g = a.g;
    const int E = g.eoff[g.N];
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < E; e += gridDim.x * blockDim.x) {
        const float4 ui = a.u[g.erecv[e]], uj = a.u[g.esend[e]], d4 = g.edr[e];
        const float tx = uj.x - ui.x, ty = uj.y - ui.y, tz = uj.z - ui.z;
        a.etan[e] = make_float4(tx, ty, tz, g.ecut[e].y * (d4.x * tx + d4.y * ty + d4.z * tz));
    }
}

// Step t, edges: the input e (and e') of the step below or of the encoder,
// then z = A_e e + (A_r v_i + a) + A_s v_j and z' = A_e e' + A_r v_i' + A_s v_j'.
__global__ void __launch_bounds__(GT_WARPS * 32) k_gt_fe(GtArgs a, int t)
{
    count_launch();
    __shared__ float M[GT_H * GT_H];
    __shared__ float buf[GT_WARPS][2][GT_H];
    __shared__ float cst[2][GT_H];
    const GnnArgs &g = a.g;
    const GnnOff &o = g.off;
    gt_stage_fwd(M, g.P, o.A[t], 3 * GT_H, 0, GT_H);
    if (t == 0) {
        for (int h = threadIdx.x; h < GT_H; h += blockDim.x) {
            float sr = __ldg(g.P + o.a[0] + h), sp = 0.0f;
            for (int c = 0; c < GT_H; ++c) {
                const float uc = __ldg(g.P + o.u + c);
                sr += __ldg(g.P + o.A[0] + h * 3 * GT_H + GT_H + c) * uc;
                sp += __ldg(g.P + o.A[0] + h * 3 * GT_H + 2 * GT_H + c) * uc;
            }
            cst[0][h] = sr;
            cst[1][h] = sp;
        }
    }
    __syncthreads();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int E = g.eoff[g.N];
    const size_t EC = (size_t)g.N * g.cap;
    float *z_t = g.ze + (size_t)t * EC * GT_H, *zt_t = a.zt + (size_t)t * EC * GT_H;
    const float *z_p = t ? g.ze + (size_t)(t - 1) * EC * GT_H : nullptr;
    const float *zt_p = t ? a.zt + (size_t)(t - 1) * EC * GT_H : nullptr;
    const float irc = 1.0f / g.rc;
    for (int e = blockIdx.x * GT_WARPS + w; e < E; e += gridDim.x * GT_WARPS) {
        const float4 d4 = g.edr[e], tn = a.etan[e];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int h = lane + 32 * q;
            float z, zt;
            if (t == 0) {
                const float *W = g.P + o.Wenc + 3 * h;
                z = __ldg(W) * (d4.x * irc) + __ldg(W + 1) * (d4.y * irc) + __ldg(W + 2) * (d4.z * irc) +
                    __ldg(g.P + o.benc + h);
                zt = __ldg(W) * (tn.x * irc) + __ldg(W + 1) * (tn.y * irc) + __ldg(W + 2) * (tn.z * irc);
            } else {
                z = z_p[(size_t)e * GT_H + h];
                zt = zt_p[(size_t)e * GT_H + h];
            }
            float v, d1, d2;
            gt_sl3(z, v, d1, d2);
            buf[w][0][h] = v;
            buf[w][1][h] = d1 * zt;
        }
        __syncwarp();
        float y0 = 0.f, y1 = 0.f, t0 = 0.f, t1 = 0.f;
        gt_mv(M, GT_H, buf[w][0], y0, y1);
        gt_mv(M, GT_H, buf[w][1], t0, t1);
        const int i = g.erecv[e], j = g.esend[e];
        float y[2] = {y0, y1}, yt[2] = {t0, t1};
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int h = lane + 32 * q;
            if (t == 0) {
                y[q] += cst[0][h] + cst[1][h];
            } else {
                y[q] += g.rr[(size_t)i * GT_H + h] + g.ps[(size_t)j * GT_H + h];
                yt[q] += a.rrt[(size_t)i * GT_H + h] + a.pst[(size_t)j * GT_H + h];
            }
            z_t[(size_t)e * GT_H + h] = y[q];
            zt_t[(size_t)e * GT_H + h] = yt[q];
        }
        __syncwarp();
    }
}

// Step t, atoms: m = sum s silu(z), m' = sum (s' silu(z) + s silu'(z) z')
// over the CSR row; zv = B [v; m] + b, zv' = B [v'; m']; then the next
// step's A_r v + a, A_s v and tangents, or, after the last step, the
// decoder zd = D v + d, zd' = D v' with the adjoints
//   zd~ = c_E w silu'(zd) - w silu''(zd) zd',   zd'~ = -w silu'(zd)
// and v~ = D^T zd~, v'~ = D^T zd'~ for the reverse sweep.
// Dynamic shared memory: B [128][64], two [64][64] blocks, per-warp vectors.
__global__ void __launch_bounds__(GT_WARPS * 32) k_gt_fn(GtArgs a, int t)
{
    count_launch();
    extern __shared__ __align__(16) float sm[];
    float *MB = sm, *MN1 = MB + 2 * GT_H * GT_H, *MN2 = MN1 + GT_H * GT_H;
    float(*buf)[4][GT_H] = reinterpret_cast<float(*)[4][GT_H]>(MN2 + GT_H * GT_H);
    const GnnArgs &g = a.g;
    const GnnOff &o = g.off;
    const bool last = t == g.T - 1;
    gt_stage_fwd(MB, g.P, o.B[t], 2 * GT_H, 0, 2 * GT_H);
    if (!last) {
        gt_stage_fwd(MN1, g.P, o.A[t + 1], 3 * GT_H, GT_H, GT_H);
        gt_stage_fwd(MN2, g.P, o.A[t + 1], 3 * GT_H, 2 * GT_H, GT_H);
    } else {
        gt_stage_fwd(MN1, g.P, o.D, GT_H, 0, GT_H);
        gt_stage_bwd(MN2, g.P, o.D, GT_H, 0);
    }
    __syncthreads();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const size_t EC = (size_t)g.N * g.cap, NH = (size_t)g.N * GT_H;
    const float *z_t = g.ze + (size_t)t * EC * GT_H, *zt_t = a.zt + (size_t)t * EC * GT_H;
    for (int i = blockIdx.x * GT_WARPS + w; i < g.N; i += gridDim.x * GT_WARPS) {
        const int e0 = g.eoff[i], e1 = g.eoff[i + 1];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int h = lane + 32 * q;
            float m = 0.f, mt = 0.f;
            for (int e = e0; e < e1; ++e) {
                const float s = g.ecut[e].x, st = a.etan[e].w;
                float v, d1, d2;
                gt_sl3(z_t[(size_t)e * GT_H + h], v, d1, d2);
                m += s * v;
                mt += st * v + s * d1 * zt_t[(size_t)e * GT_H + h];
            }
            a.m[t * NH + (size_t)i * GT_H + h] = m;
            a.mt[t * NH + (size_t)i * GT_H + h] = mt;
            float vp, vtp;
            if (t == 0) {
                vp = __ldg(g.P + o.u + h);
                vtp = 0.0f;
            } else {
                float d1, d2;
                gt_sl3(g.zv[(t - 1) * NH + (size_t)i * GT_H + h], vp, d1, d2);
                vtp = d1 * a.zvt[(t - 1) * NH + (size_t)i * GT_H + h];
            }
            buf[w][0][h] = vp;
            buf[w][1][h] = m;
            buf[w][2][h] = vtp;
            buf[w][3][h] = mt;
        }
        __syncwarp();
        float z[2] = {0.f, 0.f}, zt[2] = {0.f, 0.f};
        gt_mv(MB, 2 * GT_H, buf[w][0], z[0], z[1]);
        gt_mv(MB, 2 * GT_H, buf[w][2], zt[0], zt[1]);
        __syncwarp();
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int h = lane + 32 * q;
            z[q] += __ldg(g.P + o.b[t] + h);
            g.zv[t * NH + (size_t)i * GT_H + h] = z[q];
            a.zvt[t * NH + (size_t)i * GT_H + h] = zt[q];
            float v, d1, d2;
            gt_sl3(z[q], v, d1, d2);
            buf[w][0][h] = v;
            buf[w][2][h] = d1 * zt[q];
        }
        __syncwarp();
        if (!last) {
            float r[2] = {0.f, 0.f}, p[2] = {0.f, 0.f}, rt[2] = {0.f, 0.f}, pt[2] = {0.f, 0.f};
            gt_mv(MN1, GT_H, buf[w][0], r[0], r[1]);
            gt_mv(MN2, GT_H, buf[w][0], p[0], p[1]);
            gt_mv(MN1, GT_H, buf[w][2], rt[0], rt[1]);
            gt_mv(MN2, GT_H, buf[w][2], pt[0], pt[1]);
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int h = lane + 32 * q;
                g.rr[(size_t)i * GT_H + h] = r[q] + __ldg(g.P + o.a[t + 1] + h);
                g.ps[(size_t)i * GT_H + h] = p[q];
                a.rrt[(size_t)i * GT_H + h] = rt[q];
                a.pst[(size_t)i * GT_H + h] = pt[q];
            }
        } else {
            float zd[2] = {0.f, 0.f}, zdt[2] = {0.f, 0.f};
            gt_mv(MN1, GT_H, buf[w][0], zd[0], zd[1]);
            gt_mv(MN1, GT_H, buf[w][2], zdt[0], zdt[1]);
            const float ce = a.cE[i];
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int h = lane + 32 * q;
                zd[q] += __ldg(g.P + o.d + h);
                a.zd[(size_t)i * GT_H + h] = zd[q];
                a.zdt[(size_t)i * GT_H + h] = zdt[q];
                float v, d1, d2;
                gt_sl3(zd[q], v, d1, d2);
                const float wh = __ldg(g.P + o.w + h);
                const float zb = ce * wh * d1 - wh * d2 * zdt[q], zbt = -wh * d1;
                a.zdb[(size_t)i * GT_H + h] = zb;
                a.zdbt[(size_t)i * GT_H + h] = zbt;
                buf[w][1][h] = zb;
                buf[w][3][h] = zbt;
            }
            __syncwarp();
            float vb[2] = {0.f, 0.f}, vbt[2] = {0.f, 0.f};
            gt_mv(MN2, GT_H, buf[w][1], vb[0], vb[1]);
            gt_mv(MN2, GT_H, buf[w][3], vbt[0], vbt[1]);
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int h = lane + 32 * q;
                a.vb[(size_t)i * GT_H + h] = vb[q];
                a.vbt[(size_t)i * GT_H + h] = vbt[q];
            }
        }
        __syncwarp();
    }
}

// Reverse of step t, atoms: v~ (and v'~) of the step's output: the
// decoder's (last step), else the direct part left by step t + 1 plus
// A_r^T and A_s^T of step t + 1 applied to its z~ summed over the atom's own
// and reverse edges; then
//   zv~ = v~ silu'(zv) + v'~ silu''(zv) zv',   zv'~ = v'~ silu'(zv)
//   m~ = B_m^T zv~, m'~ = B_m^T zv'~;   direct part of step t - 1: B_v^T zv~, B_v^T zv'~.
__global__ void __launch_bounds__(GT_WARPS * 32) k_gt_bn(GtArgs a, int t)
{
    count_launch();
    extern __shared__ __align__(16) float sm[];
    float *MAr = sm, *MAs = MAr + GT_H * GT_H, *MBv = MAs + GT_H * GT_H, *MBm = MBv + GT_H * GT_H;
    float(*buf)[4][GT_H] = reinterpret_cast<float(*)[4][GT_H]>(MBm + GT_H * GT_H);
    const GnnArgs &g = a.g;
    const GnnOff &o = g.off;
    const bool last = t == g.T - 1;
    if (!last) {
        gt_stage_bwd(MAr, g.P, o.A[t + 1], 3 * GT_H, GT_H);
        gt_stage_bwd(MAs, g.P, o.A[t + 1], 3 * GT_H, 2 * GT_H);
    }
    gt_stage_bwd(MBv, g.P, o.B[t], 2 * GT_H, 0);
    gt_stage_bwd(MBm, g.P, o.B[t], 2 * GT_H, GT_H);
    __syncthreads();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const size_t EC = (size_t)g.N * g.cap, NH = (size_t)g.N * GT_H;
    const float *zb_n = last ? nullptr : g.ze + (size_t)(t + 1) * EC * GT_H;
    const float *zbt_n = last ? nullptr : a.zt + (size_t)(t + 1) * EC * GT_H;
    for (int i = blockIdx.x * GT_WARPS + w; i < g.N; i += gridDim.x * GT_WARPS) {
        float vb[2], vbt[2];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            vb[q] = a.vb[(size_t)i * GT_H + lane + 32 * q];
            vbt[q] = a.vbt[(size_t)i * GT_H + lane + 32 * q];
        }
        if (!last) {
            const int e0 = g.eoff[i], e1 = g.eoff[i + 1];
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int h = lane + 32 * q;
                float sr = 0.f, ss = 0.f, srt = 0.f, sst = 0.f;
                for (int e = e0; e < e1; ++e) {
                    const size_t er = (size_t)g.erev[e];
                    sr += zb_n[(size_t)e * GT_H + h];
                    srt += zbt_n[(size_t)e * GT_H + h];
                    ss += zb_n[er * GT_H + h];
                    sst += zbt_n[er * GT_H + h];
                }
                buf[w][0][h] = sr;
                buf[w][1][h] = ss;
                buf[w][2][h] = srt;
                buf[w][3][h] = sst;
            }
            __syncwarp();
            gt_mv(MAr, GT_H, buf[w][0], vb[0], vb[1]);
            gt_mv(MAs, GT_H, buf[w][1], vb[0], vb[1]);
            gt_mv(MAr, GT_H, buf[w][2], vbt[0], vbt[1]);
            gt_mv(MAs, GT_H, buf[w][3], vbt[0], vbt[1]);
            __syncwarp();
        }
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int h = lane + 32 * q;
            const float zv = g.zv[t * NH + (size_t)i * GT_H + h], zvt = a.zvt[t * NH + (size_t)i * GT_H + h];
            float v, d1, d2;
            gt_sl3(zv, v, d1, d2);
            const float zb = vb[q] * d1 + vbt[q] * d2 * zvt, zbt = vbt[q] * d1;
            a.zvb[(size_t)i * GT_H + h] = zb;
            a.zvbt[(size_t)i * GT_H + h] = zbt;
            buf[w][0][h] = zb;
            buf[w][1][h] = zbt;
        }
        __syncwarp();
        float mb[2] = {0.f, 0.f}, mbt[2] = {0.f, 0.f}, nb[2] = {0.f, 0.f}, nbt[2] = {0.f, 0.f};
        gt_mv(MBm, GT_H, buf[w][0], mb[0], mb[1]);
        gt_mv(MBm, GT_H, buf[w][1], mbt[0], mbt[1]);
        gt_mv(MBv, GT_H, buf[w][0], nb[0], nb[1]);
        gt_mv(MBv, GT_H, buf[w][1], nbt[0], nbt[1]);
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const size_t x = (size_t)i * GT_H + lane + 32 * q;
            a.mb[x] = mb[q];
            a.mbt[x] = mbt[q];
            a.vb[x] = nb[q];
            a.vbt[x] = nbt[q];
        }
        __syncwarp();
    }
}

// Reverse of step t, edges:
//   e~ = s m~_i + s' m'~_i (+ A_e^T z~ of step t + 1),  e'~ = s m'~_i (+ A_e^T z'~ of step t + 1)
//   z~ = e~ silu'(z) + e'~ silu''(z) z',  z'~ = e'~ silu'(z)    (stored over z, z')
// step 0 goes on into the encoder (z0 = W_enc x + b_enc, z0' = W_enc x').
__global__ void __launch_bounds__(GT_WARPS * 32) k_gt_be(GtArgs a, int t)
{
    count_launch();
    __shared__ float MA[GT_H * GT_H], MA0[GT_H * GT_H];
    __shared__ float buf[GT_WARPS][2][GT_H];
    const GnnArgs &g = a.g;
    const GnnOff &o = g.off;
    const bool last = t == g.T - 1;
    if (!last) gt_stage_bwd(MA, g.P, o.A[t + 1], 3 * GT_H, 0);
    if (t == 0) gt_stage_bwd(MA0, g.P, o.A[0], 3 * GT_H, 0);
    __syncthreads();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int E = g.eoff[g.N];
    const size_t EC = (size_t)g.N * g.cap;
    float *z_t = g.ze + (size_t)t * EC * GT_H, *zt_t = a.zt + (size_t)t * EC * GT_H;
    const float *zb_n = last ? nullptr : g.ze + (size_t)(t + 1) * EC * GT_H;
    const float *zbt_n = last ? nullptr : a.zt + (size_t)(t + 1) * EC * GT_H;
    const float irc = 1.0f / g.rc;
    for (int e = blockIdx.x * GT_WARPS + w; e < E; e += gridDim.x * GT_WARPS) {
        const int i = g.erecv[e];
        const float s = g.ecut[e].x;
        const float4 tn = a.etan[e];
        float eb[2], ebt[2];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int h = lane + 32 * q;
            const float mb = a.mb[(size_t)i * GT_H + h], mbt = a.mbt[(size_t)i * GT_H + h];
            eb[q] = s * mb + tn.w * mbt;
            ebt[q] = s * mbt;
            if (!last) {
                buf[w][0][h] = zb_n[(size_t)e * GT_H + h];
                buf[w][1][h] = zbt_n[(size_t)e * GT_H + h];
            }
        }
        if (!last) {
            __syncwarp();
            gt_mv(MA, GT_H, buf[w][0], eb[0], eb[1]);
            gt_mv(MA, GT_H, buf[w][1], ebt[0], ebt[1]);
            __syncwarp();
        }
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int h = lane + 32 * q;
            const size_t x = (size_t)e * GT_H + h;
            const float z = z_t[x], zt = zt_t[x];
            float v, d1, d2;
            gt_sl3(z, v, d1, d2);
            const float zb = eb[q] * d1 + ebt[q] * d2 * zt, zbt = ebt[q] * d1;
            z_t[x] = zb;
            zt_t[x] = zbt;
            if (t == 0) {
                buf[w][0][h] = zb;
                buf[w][1][h] = zbt;
            }
        }
        if (t == 0) {
            __syncwarp();
            float e0[2] = {0.f, 0.f}, e0t[2] = {0.f, 0.f};
            gt_mv(MA0, GT_H, buf[w][0], e0[0], e0[1]);
            gt_mv(MA0, GT_H, buf[w][1], e0t[0], e0t[1]);
            const float4 d4 = g.edr[e];
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int h = lane + 32 * q;
                const float *W = g.P + o.Wenc + 3 * h;
                const float z0 = __ldg(W) * (d4.x * irc) + __ldg(W + 1) * (d4.y * irc) + __ldg(W + 2) * (d4.z * irc) +
                                 __ldg(g.P + o.benc + h);
                const float z0t = __ldg(W) * (tn.x * irc) + __ldg(W + 1) * (tn.y * irc) + __ldg(W + 2) * (tn.z * irc);
                float v, d1, d2;
                gt_sl3(z0, v, d1, d2);
                a.encb[(size_t)e * GT_H + h] = e0[q] * d1 + e0t[q] * d2 * z0t;
                a.encbt[(size_t)e * GT_H + h] = e0t[q] * d1;
            }
        }
        __syncwarp();
    }
}

// Outer-product sums G[h][c] = sum_rows (Xb[row][h] Y[row][c] + Xbt[row][h] Yt[row][c])
// for one parameter block; the last column (c = K) has Y = 1, Yt = 0 (the
// bias).  Row sources by mode:
enum { GT_A = 0, GT_B = 1, GT_D = 2, GT_ENC = 3, GT_W = 4, GT_U = 5 };

// v and v' of step t - 1 for atom i (t = 0: u, 0)
__device__ __forceinline__ void gt_node(const GtArgs &a, int t, int i, int c, float &v, float &vt)
{
    const GnnArgs &g = a.g;
    if (t == 0) {
        v = __ldg(g.P + g.off.u + c);
        vt = 0.0f;
        return;
    }
    const size_t x = (size_t)(t - 1) * g.N * GT_H + (size_t)i * GT_H + c;
    float d1, d2;
    gt_sl3(g.zv[x], v, d1, d2);
    vt = d1 * a.zvt[x];
}

__device__ __forceinline__ void gt_row_x(const GtArgs &a, int mode, int t, int r, int h, float &xb, float &xbt)
{
    const GnnArgs &g = a.g;
    const size_t EC = (size_t)g.N * g.cap;
    switch (mode) {
    case GT_A:
        xb = g.ze[(size_t)t * EC * GT_H + (size_t)r * GT_H + h];
        xbt = a.zt[(size_t)t * EC * GT_H + (size_t)r * GT_H + h];
        break;
    case GT_B:
        xb = a.zvb[(size_t)r * GT_H + h];
        xbt = a.zvbt[(size_t)r * GT_H + h];
        break;
    case GT_D:
        xb = a.zdb[(size_t)r * GT_H + h];
        xbt = a.zdbt[(size_t)r * GT_H + h];
        break;
    case GT_ENC:
        xb = a.encb[(size_t)r * GT_H + h];
        xbt = a.encbt[(size_t)r * GT_H + h];
        break;
    case GT_W: {   // dJ/dw_h per atom: c_E silu(zd) - silu'(zd) zd'
        float v, d1, d2;
        gt_sl3(a.zd[(size_t)r * GT_H + h], v, d1, d2);
        xb = a.cE[r] * v - d1 * a.zdt[(size_t)r * GT_H + h];
        xbt = 0.0f;
        break;
    }
    default:       // GT_U: the direct node adjoint left by step 0
        xb = a.vb[(size_t)r * GT_H + h];
        xbt = 0.0f;
        break;
    }
}

__device__ __forceinline__ void gt_row_y(const GtArgs &a, int mode, int t, int K, int r, int c, float &y, float &yt)
{
    const GnnArgs &g = a.g;
    y = yt = 0.0f;
    if (c == K) {
        y = 1.0f;
        return;
    }
    if (c > K) return;
    const size_t EC = (size_t)g.N * g.cap, NH = (size_t)g.N * GT_H;
    const float irc = 1.0f / g.rc;
    switch (mode) {
    case GT_A:
        if (c < GT_H) {   // e and e' of the step below (t = 0: the encoder)
            float z, zt;
            if (t == 0) {
                const float4 d4 = g.edr[r], tn = a.etan[r];
                const float *W = g.P + g.off.Wenc + 3 * c;
                z = __ldg(W) * (d4.x * irc) + __ldg(W + 1) * (d4.y * irc) + __ldg(W + 2) * (d4.z * irc) +
                    __ldg(g.P + g.off.benc + c);
                zt = __ldg(W) * (tn.x * irc) + __ldg(W + 1) * (tn.y * irc) + __ldg(W + 2) * (tn.z * irc);
            } else {
                z = g.ze[(size_t)(t - 1) * EC * GT_H + (size_t)r * GT_H + c];
                zt = a.zt[(size_t)(t - 1) * EC * GT_H + (size_t)r * GT_H + c];
            }
            float d1, d2;
            gt_sl3(z, y, d1, d2);
            yt = d1 * zt;
        } else if (c < 2 * GT_H) {
            gt_node(a, t, g.erecv[r], c - GT_H, y, yt);
        } else {
            gt_node(a, t, g.esend[r], c - 2 * GT_H, y, yt);
        }
        break;
    case GT_B:
        if (c < GT_H) {
            gt_node(a, t, r, c, y, yt);
        } else {
            y = a.m[t * NH + (size_t)r * GT_H + c - GT_H];
            yt = a.mt[t * NH + (size_t)r * GT_H + c - GT_H];
        }
        break;
    case GT_D:
        gt_node(a, g.T, r, c, y, yt);
        break;
    case GT_ENC: {
        const float4 d4 = g.edr[r], tn = a.etan[r];
        y = (c == 0 ? d4.x : c == 1 ? d4.y : d4.z) * irc;
        yt = (c == 0 ? tn.x : c == 1 ? tn.y : tn.z) * irc;
        break;
    }
    default:
        break;
    }
}

constexpr int GT_KP = 193;   // widest block: A (192 columns) + bias

__global__ void __launch_bounds__(256) k_gt_outer(GtArgs a, int mode, int t, int K, int R)
{
    count_launch();
    __shared__ float Xs[32][GT_H], Xts[32][GT_H], Ys[32][16], Yts[32][16];
    const int tid = threadIdx.x, h = tid & (GT_H - 1), cq = tid >> 6;
    const int cx = blockIdx.x, chunk = blockIdx.y;
    if (mode == GT_A || mode == GT_ENC) R = a.g.eoff[a.g.N];   // the compacted edges
    const int per = (R + GT_CHUNKS - 1) / GT_CHUNKS;
    const int r0 = chunk * per, r1 = min(R, r0 + per);
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int b0 = r0; b0 < r1; b0 += 32) {
        for (int x = tid; x < 32 * GT_H; x += blockDim.x) {
            const int row = x / GT_H, hh = x - row * GT_H, r = b0 + row;
            float xb = 0.f, xbt = 0.f;
            if (r < r1) gt_row_x(a, mode, t, r, hh, xb, xbt);
            Xs[row][hh] = xb;
            Xts[row][hh] = xbt;
        }
        for (int x = tid; x < 32 * 16; x += blockDim.x) {
            const int row = x / 16, cc = x - row * 16, r = b0 + row;
            float y = 0.f, yt = 0.f;
            if (r < r1) gt_row_y(a, mode, t, K, r, cx * 16 + cc, y, yt);
            Ys[row][cc] = y;
            Yts[row][cc] = yt;
        }
        __syncthreads();
        float s[4] = {0.f, 0.f, 0.f, 0.f};
        for (int row = 0; row < 32; ++row) {
            const float xb = Xs[row][h], xbt = Xts[row][h];
#pragma unroll
            for (int k = 0; k < 4; ++k) s[k] += xb * Ys[row][cq * 4 + k] + xbt * Yts[row][cq * 4 + k];
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) acc[k] += (double)s[k];
        __syncthreads();
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int c = cx * 16 + cq * 4 + k;
        if (c <= K) a.part[((size_t)chunk * GT_H + h) * GT_KP + c] = acc[k];
    }
}

// The chunks, in order, into the gradient of the block.
__global__ void k_gt_reduce(GtArgs a, int mode, int t, int K)
{
    count_launch();
    const GnnOff &o = a.g.off;
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < GT_H * (K + 1); x += gridDim.x * blockDim.x) {
        const int h = x / (K + 1), c = x - h * (K + 1);
        double s = 0.0;
        for (int ch = 0; ch < GT_CHUNKS; ++ch) s += a.part[((size_t)ch * GT_H + h) * GT_KP + c];
        const float v = (float)s;
        switch (mode) {
        case GT_A: a.grad[c < K ? o.A[t] + h * 3 * GT_H + c : o.a[t] + h] = v; break;
        case GT_B: a.grad[c < K ? o.B[t] + h * 2 * GT_H + c : o.b[t] + h] = v; break;
        case GT_D: a.grad[c < K ? o.D + h * GT_H + c : o.d + h] = v; break;
        case GT_ENC: a.grad[c < K ? o.Wenc + h * 3 + c : o.benc + h] = v; break;
        case GT_W: a.grad[o.w + h] = v; break;
        default: a.grad[o.u + h] = v; break;
        }
    }
}

// u~ = (direct part) + (A_r + A_s)^T of step 0 applied to sum_e z~ (= a~ of
// step 0); c~ = sum_i c_E,i (one block, fixed order).
__global__ void __launch_bounds__(256) k_gt_final(GtArgs a)
{
    count_launch();
    __shared__ double sh[32];
    const GnnArgs &g = a.g;
    const GnnOff &o = g.off;
    double s = 0.0;
    for (int i = threadIdx.x; i < g.N; i += blockDim.x) s += (double)a.cE[i];
    s = block_sum_f64(s, sh);
    if (threadIdx.x == 0) a.grad[o.c] = (float)s;
    for (int h = threadIdx.x; h < GT_H; h += blockDim.x) {
        float acc = a.grad[o.u + h];
        for (int c = 0; c < GT_H; ++c) {
            const float ab = a.grad[o.a[0] + c];
            acc += (__ldg(g.P + o.A[0] + c * 3 * GT_H + GT_H + h) + __ldg(g.P + o.A[0] + c * 3 * GT_H + 2 * GT_H + h)) *
                   ab;
        }
        a.grad[o.u + h] = acc;
    }
}

struct GtWs {
    size_t zt, zvt, m, mt, rrt, pst, zd, zdt, zdb, zdbt, vb, vbt, zvb, zvbt, mb, mbt, etan, encb, encbt, part, cbar,
        total;
};

static GtWs gt_ws_layout(int N, int cap, int T)
{
    GtWs w;
    const size_t EC = (size_t)N * cap, NH = (size_t)N * GT_H, f = sizeof(float);
    size_t o = 0;
    w.zt = o;    o = align256(o + f * (size_t)T * EC * GT_H);
    w.zvt = o;   o = align256(o + f * (size_t)T * NH);
    w.m = o;     o = align256(o + f * (size_t)T * NH);
    w.mt = o;    o = align256(o + f * (size_t)T * NH);
    size_t *one[] = {&w.rrt, &w.pst, &w.zd, &w.zdt, &w.zdb, &w.zdbt, &w.vb, &w.vbt, &w.zvb, &w.zvbt, &w.mb, &w.mbt};
    for (size_t *p : one) {
        *p = o;
        o = align256(o + f * NH);
    }
    w.etan = o;  o = align256(o + sizeof(float4) * EC);
    w.encb = o;  o = align256(o + f * EC * GT_H);
    w.encbt = o; o = align256(o + f * EC * GT_H);
    w.part = o;  o = align256(o + sizeof(double) * (size_t)GT_CHUNKS * GT_H * GT_KP);
    w.cbar = o;  o = align256(o + sizeof(double));
    w.total = o;
    return w;
}

}  // namespace jmd

using namespace jmd;

extern "C" size_t md_gnn_train_scratch_bytes(int N, int cap, int H, int T)
{
    if (N < 1 || cap < 1 || cap > GNN_MAXCAP || H != GT_H || T < 1 || T > GNN_MAXT) return 0;
    return gt_ws_layout(N, cap, T).total;
}

extern "C" md_status md_gnn_train_grad(const md_space *s, const float *d_r, const md_nbr *nb, const md_gnn_model *m,
                                       const float *d_cE, const float *d_dF, void *d_scratch, size_t scratch_bytes,
                                       float *d_grad, uint32_t *d_status, md_stream_t stream)
{
    if (!s || !d_r || !nb || !m || !d_cE || !d_dF || !d_scratch || !d_grad) return MD_ERR_INVALID;
    if (s->dim != 3 || nb->dim != 3 || !nb->nbr || !nb->cnt || m->H != GT_H) return MD_ERR_INVALID;
    if (!gnn_model_ok(m, nb) || (size_t)nb->N * nb->cap >= (size_t)INT32_MAX) return MD_ERR_INVALID;
    const GtWs L = gt_ws_layout(nb->N, nb->cap, m->T);
    if (scratch_bytes < L.total || ((uintptr_t)d_scratch & 255u)) return MD_ERR_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    GtArgs a;
    memset(&a, 0, sizeof(a));
    GnnArgs &g = a.g;
    g.box = make_box(s);
    g.N = nb->N;
    g.cap = nb->cap;
    g.T = m->T;
    g.sys_n = m->sys_n;
    g.rc = m->r_cut;
    g.rc2 = m->r_cut * m->r_cut;
    g.r = (const float4 *)d_r;
    g.nbr = nb->nbr;
    g.cnt = nb->cnt;
    g.P = m->params;
    g.off = gnn_offsets(m->H, m->T);
    g.status = d_status;
    gnn_bind_workspace(g, m);
    unsigned char *b = (unsigned char *)d_scratch;
    a.u = (const float4 *)d_dF;
    a.cE = d_cE;
    a.zt = (float *)(b + L.zt);
    a.zvt = (float *)(b + L.zvt);
    a.m = (float *)(b + L.m);
    a.mt = (float *)(b + L.mt);
    a.rrt = (float *)(b + L.rrt);
    a.pst = (float *)(b + L.pst);
    a.zd = (float *)(b + L.zd);
    a.zdt = (float *)(b + L.zdt);
    a.zdb = (float *)(b + L.zdb);
    a.zdbt = (float *)(b + L.zdbt);
    a.vb = (float *)(b + L.vb);
    a.vbt = (float *)(b + L.vbt);
    a.zvb = (float *)(b + L.zvb);
    a.zvbt = (float *)(b + L.zvbt);
    a.mb = (float *)(b + L.mb);
    a.mbt = (float *)(b + L.mbt);
    a.etan = (float4 *)(b + L.etan);
    a.encb = (float *)(b + L.encb);
    a.encbt = (float *)(b + L.encbt);
    a.part = (double *)(b + L.part);
    a.cbar = (double *)(b + L.cbar);
    a.grad = d_grad;

    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms < 1) sms = 1;
        const int dyn = (int)(sizeof(float) * (4 * GT_H * GT_H + GT_WARPS * 4 * GT_H));
        cudaFuncSetAttribute(k_gt_fn, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
        cudaFuncSetAttribute(k_gt_bn, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
    }
    const size_t dyn = sizeof(float) * (4 * GT_H * GT_H + GT_WARPS * 4 * GT_H);
    const int wg = sms * 4;   // warp-per-row kernels, grid-stride
    const int N = g.N, T = g.T;
    const int Ecap = N * g.cap;   // edge sums: k_gt_outer takes the compacted count from the device
    enqueue_gnn_compact(g, st);
    k_gt_tan<<<sms * 4, 256, 0, st>>>(a);
    for (int t = 0; t < T; ++t) {
        k_gt_fe<<<wg, GT_WARPS * 32, 0, st>>>(a, t);
        k_gt_fn<<<wg, GT_WARPS * 32, dyn, st>>>(a, t);
    }
    auto outer = [&](int mode, int t, int K, int R) {
        dim3 grid((K + 1 + 15) / 16, GT_CHUNKS);
        k_gt_outer<<<grid, 256, 0, st>>>(a, mode, t, K, R);
        k_gt_reduce<<<(GT_H * (K + 1) + 255) / 256, 256, 0, st>>>(a, mode, t, K);
    };
    outer(GT_D, 0, GT_H, N);
    outer(GT_W, 0, 0, N);
    for (int t = T - 1; t >= 0; --t) {
        k_gt_bn<<<wg, GT_WARPS * 32, dyn, st>>>(a, t);
        outer(GT_B, t, 2 * GT_H, N);
        k_gt_be<<<wg, GT_WARPS * 32, 0, st>>>(a, t);
        outer(GT_A, t, 3 * GT_H, Ecap);
    }
    outer(GT_ENC, 0, 3, Ecap);
    outer(GT_U, 0, 0, N);
    k_gt_final<<<1, 256, 0, st>>>(a);
    JMD_CUDA_TRY(cudaGetLastError());
    return MD_OK;
}
