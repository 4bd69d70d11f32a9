// gnn.cu -- graph-network potential (Sec. 3.2.4: GraphNet blocks, the
// network Bapst et al. used for glasses; Sec. 4.1: energy model whose forces
// are the negative gradient), energy and forces on the neighbor list:
//
//   edges      (i <- j) for the list pairs with r_ij < r_c (i receives)
//   encode     e_ij = silu(W_enc x_ij + b_enc), x_ij = (R_j - R_i) / r_c;  v_i = u
//   step t     e_ij = silu(A_e e_ij + A_r v_i + A_s v_j + a)
//              m_i  = sum_j s(r_ij) e_ij,  s(r) = (cos(pi r / r_c) + 1) / 2
//              v_i  = silu(B_v v_i + B_m m_i + b)
//   decode     E_i = w . silu(D v_i + d) + c,  F = -dE/dR
//
// Kernels (one warp per group of 8 atoms, lane l owns hidden units l and
// l + 32; weights staged in shared memory in the orientation each product
// needs, so a lane reads consecutive words and the vectors are broadcasts;
// every weight word read feeds 8 FMAs, one per atom or edge of a batch):
//   k_gnn_fwd<H>(t)  step t for every edge of the group (batches of 8
//                    edges), the message sums and the node updates; stores the pre-activations (edges and nodes),
//                    the next step's receiver and sender terms A_r v + a and
//                    A_s v, or, after the last step, E_i and the decoder's
//                    gradient.  Step 0 also records each edge's
//                    displacement and the slot of its reverse edge (j <- i)
//                    in j's row.
//   k_gnn_bwd<H>(t)  reverse of step t: node gradient (the decoder's, or the
//                    direct part plus the receiver and sender parts of step
//                    t + 1 summed over the atom's own and reverse edges),
//                    message and edge gradients; step 0 continues through
//                    the encoder to dE/d(R_j - R_i) per edge.
//   k_gnn_force      F_i = sum_k [g(i <- j_k) - g(j_k <- i)], the energy
//                    epilogue and, for velocity Verlet, the closing half-kick.
// Reverse edges are found in the partner's row, so no atomics are used and
// every sum has a fixed order.
#include <algorithm>

#include "common.cuh"
#include "gnn.cuh"
#include "kernels.cuh"
#include "reduce.cuh"

namespace jmd {

// Stage an H x K block of a row-major matrix (rows h, ld columns, first
// column c0) in shared memory as M[c][h] (forward product W v: lane h reads
// M[c][h], the vector element c is a broadcast).
template <int H>
__device__ void stage_fwd(float *M, const float *P, int base, int ld, int c0, int K)
{
    for (int k = threadIdx.x; k < K * H; k += blockDim.x) {
        const int c = k / H, h = k - c * H;
        M[k] = __ldg(P + base + (size_t)h * ld + c0 + c);
    }
}

// Stage the H x H block as M[h][c] (transposed product W^T g: lane c reads
// M[h][c], g_h is a broadcast).
template <int H>
__device__ void stage_bwd(float *M, const float *P, int base, int ld, int c0)
{
    for (int k = threadIdx.x; k < H * H; k += blockDim.x) {
        const int h = k / H, c = k - h * H;
        M[k] = __ldg(P + base + (size_t)h * ld + c0 + c);
    }
}

// acc[e][q] += sum_{c < K} M[c][lane + 32 q] X[e][c] for e < ne (X rows of
// stride XS floats, 16-byte aligned; K a multiple of 4).
template <int H, int NE>
__device__ __forceinline__ void wmv(const float *M, int K, const float *X, int XS, float (&acc)[NE][H / 32], int ne)
{
    constexpr int HL = H / 32;
    const int lane = threadIdx.x & 31;
    for (int c = 0; c < K; c += 4) {
        float w[4][HL];
#pragma unroll
        for (int cc = 0; cc < 4; ++cc)
#pragma unroll
            for (int q = 0; q < HL; ++q) w[cc][q] = M[(c + cc) * H + lane + 32 * q];
#pragma unroll
        for (int e = 0; e < NE; ++e) {
            if (e < ne) {
                const float4 x = *reinterpret_cast<const float4 *>(X + e * XS + c);
#pragma unroll
                for (int q = 0; q < HL; ++q)
                    acc[e][q] += w[0][q] * x.x + w[1][q] * x.y + w[2][q] * x.z + w[3][q] * x.w;
            }
        }
    }
}

// Each warp takes a group of G consecutive atoms (1, 2, 4 or 8), so that
// every node product runs over G vectors and every weight word read from
// shared memory feeds G FMAs; the group's edges with r < r_c are listed in
// atom then row order (el: atom * 64 + slot) and processed in batches of
// GNN_EB.
template <int H, int G>
struct __align__(16) GnnWarpSmem {
    float XN[G][2 * H];       // node vectors per atom: [v; m] or gradients
    float X[GNN_EB][H];       // edge vectors of a batch
    float GM[G][H];           // message gradient per atom (reverse)
    uint16_t el[G * GNN_MAXCAP];
    int es[G + 1];            // start of each atom's edges in el
};

// Row lengths of the group's atoms: lane g holds atom g's.
__device__ __forceinline__ int gnn_group_counts(const GnnArgs &a, int i0, int na)
{
    const int lane = threadIdx.x & 31;
    int n = lane < na ? a.cnt[i0 + lane] : 0;
    return n < a.cap ? n : a.cap;
}

// List the group's edges (rev >= 0) in atom then row order; the group's rows
// are contiguous, so the scan reads them coalesced.  Returns their number.
template <int H, int G>
__device__ __forceinline__ int gnn_group_edges(const GnnArgs &a, int i0, int na, int n_l, GnnWarpSmem<H, G> &W)
{
    const int lane = threadIdx.x & 31;
    const int tot = na * a.cap;
    const int32_t *rev = a.rev + (size_t)i0 * a.cap;
    int nv = 0;
#pragma unroll 4
    for (int x0 = 0; x0 < tot; x0 += 32) {
        const int x = x0 + lane;
        const int g = x / a.cap, k = x - g * a.cap;
        const int ng = __shfl_sync(0xffffffffu, n_l, g < G ? g : 0);
        const bool ok = x < tot && k < ng && rev[x] >= 0;
        const unsigned b = __ballot_sync(0xffffffffu, ok);
        const int before = nv + __popc(b & ((1u << lane) - 1u));
        if (ok) W.el[before] = (uint16_t)(g * GNN_MAXCAP + k);
        if (x < tot && k == 0) W.es[g] = before;
        nv += __popc(b);
    }
    if (lane == 0) W.es[na] = nv;
    __syncwarp();
    return nv;
}

template <int H, int G>
__global__ void __launch_bounds__(gnn_warps(G) * 32) k_gnn_fwd(GnnArgs a, int t)
{
    count_launch();
    constexpr int HL = H / 32;
    extern __shared__ __align__(16) float sm[];
    const bool last = t == a.T - 1;
    float *MAe = sm;                  // [H][H]
    float *MB = MAe + H * H;          // [2H][H]: B_v then B_m
    float *MN = MB + 2 * H * H;       // next step: A_r, A_s ([H][H] each); or D
    float *cvec = MN + 2 * H * H;     // step 0: A_r u + a, A_s u, u
    GnnWarpSmem<H, G> *ws = reinterpret_cast<GnnWarpSmem<H, G> *>(cvec + 3 * H);
    const GnnOff &o = a.off;
    stage_fwd<H>(MAe, a.P, o.A[t], 3 * H, 0, H);
    stage_fwd<H>(MB, a.P, o.B[t], 2 * H, 0, 2 * H);
    if (!last) {
        stage_fwd<H>(MN, a.P, o.A[t + 1], 3 * H, H, H);
        stage_fwd<H>(MN + H * H, a.P, o.A[t + 1], 3 * H, 2 * H, H);
    } else {
        stage_fwd<H>(MN, a.P, o.D, H, 0, H);
    }
    if (t == 0) {
        for (int h = threadIdx.x; h < H; h += blockDim.x) {
            float sr = __ldg(a.P + o.a[0] + h), sp = 0.0f;
            for (int c = 0; c < H; ++c) {
                const float uc = __ldg(a.P + o.u + c);
                sr += __ldg(a.P + o.A[0] + (size_t)h * 3 * H + H + c) * uc;
                sp += __ldg(a.P + o.A[0] + (size_t)h * 3 * H + 2 * H + c) * uc;
            }
            cvec[h] = sr;
            cvec[H + h] = sp;
            cvec[2 * H + h] = __ldg(a.P + o.u + h);
        }
    }
    __syncthreads();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    GnnWarpSmem<H, G> &W = ws[w];
    float wenc[HL][3], benc[HL], bt[HL], an[HL], dd[HL], ww[HL];
#pragma unroll
    for (int q = 0; q < HL; ++q) {
        const int h = lane + 32 * q;
        for (int c = 0; c < 3; ++c) wenc[q][c] = __ldg(a.P + o.Wenc + 3 * h + c);
        benc[q] = __ldg(a.P + o.benc + h);
        bt[q] = __ldg(a.P + o.b[t] + h);
        an[q] = last ? 0.0f : __ldg(a.P + o.a[t + 1] + h);
        dd[q] = __ldg(a.P + o.d + h);
        ww[q] = __ldg(a.P + o.w + h);
    }
    const float cdec = __ldg(a.P + o.c);
    const float inv_rc = 1.0f / a.rc;
    const size_t NE = (size_t)a.N * a.cap;
    float *ze_t = a.ze + (size_t)t * NE * H;
    const float *ze_p = t > 0 ? a.ze + (size_t)(t - 1) * NE * H : nullptr;
    const float *rr_t = a.rr + (size_t)(t & 1) * a.N * H;
    const float *ps_t = a.ps + (size_t)(t & 1) * a.N * H;
    const int ngroups = (a.N + G - 1) / G;
    for (int grp = blockIdx.x * gnn_warps(G) + w; grp < ngroups; grp += gridDim.x * gnn_warps(G)) {
        const int i0 = grp * G, na = min(G, a.N - i0);
        const int n_l = gnn_group_counts(a, i0, na);
        if (t == 0) {
            // displacements and reverse slots of the group's rows
            const int tot = na * a.cap;
            for (int x = lane; x < tot; x += 32) {
                const int g = x / a.cap, k = x - g * a.cap;
                const int i = i0 + g;
                int n = a.cnt[i];
                n = n < a.cap ? n : a.cap;
                if (k >= n) continue;
                const size_t E = (size_t)i * a.cap + k;
                const int base = a.sys_n ? (i / a.sys_n) * a.sys_n : 0;
                const int j = a.nbr[E] + base;
                int rv = -1;
                float4 d4 = make_float4(0.f, 0.f, 0.f, -1.0f);
                if (j >= base && j < (a.sys_n ? base + a.sys_n : a.N) && j < a.N && j != i) {
                    float dx, dy, dz;
                    const float r2 = dist2_rn<3>(a.r[j], a.r[i], a.box, dx, dy, dz);
                    if (r2 < a.rc2) {
                        int nj = a.cnt[j];
                        nj = nj < a.cap ? nj : a.cap;
                        const int32_t *rowj = a.nbr + (size_t)j * a.cap;
                        for (int p = 0; p < nj && rv < 0; p += 4) {
                            int q4[4];
#pragma unroll
                            for (int u = 0; u < 4; ++u) q4[u] = p + u < nj ? rowj[p + u] + base : -1;
#pragma unroll
                            for (int u = 0; u < 4; ++u)
                                if (rv < 0 && q4[u] == i) rv = j * a.cap + p + u;
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
            }
            __syncwarp();
        }
        const int nv = gnn_group_edges<H, G>(a, i0, na, n_l, W);
        // node inputs v and zeroed message sums
#pragma unroll
        for (int g = 0; g < G; ++g) {
            if (g < na) {
#pragma unroll
                for (int q = 0; q < HL; ++q) {
                    const int h = lane + 32 * q;
                    W.XN[g][h] = t == 0 ? cvec[2 * H + h] : gnn_silu(a.zv[((size_t)(t - 1) * a.N + i0 + g) * H + h]);
                    W.XN[g][H + h] = 0.0f;
                }
            }
        }
        __syncwarp();
        for (int b0 = 0; b0 < nv; b0 += GNN_EB) {
            const int ne = min(GNN_EB, nv - b0);
            float acc[GNN_EB][HL];
#pragma unroll
            for (int e = 0; e < GNN_EB; ++e) {
                if (e < ne) {
                    const int code = W.el[b0 + e], g = code / GNN_MAXCAP, k = code - g * GNN_MAXCAP;
                    const int i = i0 + g;
                    const size_t E = (size_t)i * a.cap + k;
                    const int j = a.rev[E] / a.cap;
                    const float4 d4 = a.dr[E];
#pragma unroll
                    for (int q = 0; q < HL; ++q) {
                        const int h = lane + 32 * q;
                        float x;
                        if (t == 0) {
                            const float z0 = wenc[q][0] * (d4.x * inv_rc) + wenc[q][1] * (d4.y * inv_rc) +
                                             wenc[q][2] * (d4.z * inv_rc) + benc[q];
                            x = gnn_silu(z0);
                        } else {
                            x = gnn_silu(ze_p[E * H + h]);
                        }
                        W.X[e][h] = x;
                        acc[e][q] = (t == 0 ? cvec[h] + cvec[H + h] : rr_t[(size_t)i * H + h] + ps_t[(size_t)j * H + h]);
                    }
                }
            }
            __syncwarp();
            wmv<H, GNN_EB>(MAe, H, &W.X[0][0], H, acc, ne);
#pragma unroll
            for (int e = 0; e < GNN_EB; ++e) {
                if (e < ne) {
                    const int code = W.el[b0 + e], g = code / GNN_MAXCAP, k = code - g * GNN_MAXCAP;
                    const size_t E = (size_t)(i0 + g) * a.cap + k;
                    const float s = a.cut[E].x;
#pragma unroll
                    for (int q = 0; q < HL; ++q) {
                        ze_t[E * H + lane + 32 * q] = acc[e][q];
                        W.XN[g][H + lane + 32 * q] += s * gnn_silu(acc[e][q]);
                    }
                }
            }
            __syncwarp();
        }
        // node update for the group: zv = B_v v + B_m m + b
        float zv[G][HL];
#pragma unroll
        for (int g = 0; g < G; ++g)
#pragma unroll
            for (int q = 0; q < HL; ++q) zv[g][q] = bt[q];
        wmv<H, G>(MB, 2 * H, &W.XN[0][0], 2 * H, zv, na);
        __syncwarp();
#pragma unroll
        for (int g = 0; g < G; ++g) {
            if (g < na) {
#pragma unroll
                for (int q = 0; q < HL; ++q) {
                    const int h = lane + 32 * q;
                    a.zv[((size_t)t * a.N + i0 + g) * H + h] = zv[g][q];
                    W.XN[g][h] = gnn_silu(zv[g][q]);
                }
            }
        }
        __syncwarp();
        if (!last) {
            float nr[G][HL];
#pragma unroll
            for (int g = 0; g < G; ++g)
#pragma unroll
                for (int q = 0; q < HL; ++q) nr[g][q] = an[q];
            wmv<H, G>(MN, H, &W.XN[0][0], 2 * H, nr, na);
            float *rr_n = a.rr + (size_t)((t + 1) & 1) * a.N * H;
            float *ps_n = a.ps + (size_t)((t + 1) & 1) * a.N * H;
#pragma unroll
            for (int g = 0; g < G; ++g) {
                if (g < na) {
#pragma unroll
                    for (int q = 0; q < HL; ++q) rr_n[(size_t)(i0 + g) * H + lane + 32 * q] = nr[g][q];
                }
            }
#pragma unroll
            for (int g = 0; g < G; ++g)
#pragma unroll
                for (int q = 0; q < HL; ++q) nr[g][q] = 0.0f;
            wmv<H, G>(MN + H * H, H, &W.XN[0][0], 2 * H, nr, na);
#pragma unroll
            for (int g = 0; g < G; ++g) {
                if (g < na) {
#pragma unroll
                    for (int q = 0; q < HL; ++q) ps_n[(size_t)(i0 + g) * H + lane + 32 * q] = nr[g][q];
                }
            }
        } else {
            float zd[G][HL];
#pragma unroll
            for (int g = 0; g < G; ++g)
#pragma unroll
                for (int q = 0; q < HL; ++q) zd[g][q] = dd[q];
            wmv<H, G>(MN, H, &W.XN[0][0], 2 * H, zd, na);
#pragma unroll
            for (int g = 0; g < G; ++g) {
                if (g < na) {
                    float e = 0.0f;
#pragma unroll
                    for (int q = 0; q < HL; ++q) {
                        e += ww[q] * gnn_silu(zd[g][q]);
                        // decoder gradient dE_i/d(D v + d), for the reverse pass
                        a.gvd[(size_t)(i0 + g) * H + lane + 32 * q] = ww[q] * gnn_dsilu(zd[g][q]);
                    }
                    e = gnn_wsum(e);
                    if (lane == 0) a.Ei[i0 + g] = e + cdec;
                }
            }
        }
        __syncwarp();
    }
}

template <int H, int G>
__global__ void __launch_bounds__(gnn_warps(G) * 32) k_gnn_bwd(GnnArgs a, int t)
{
    count_launch();
    constexpr int HL = H / 32;
    extern __shared__ __align__(16) float sm[];
    const bool last = t == a.T - 1;
    float *MBv = sm;              // [H][H] B_v^T form
    float *MBm = MBv + H * H;     // B_m^T
    float *MN = MBm + H * H;      // last: D^T; else A_r^T, A_s^T, A_e^T of step t + 1
    float *MA0 = MN + 3 * H * H;  // step 0: A_e^T of step 0
    GnnWarpSmem<H, G> *ws = reinterpret_cast<GnnWarpSmem<H, G> *>(MA0 + (t == 0 ? H * H : 0));
    const GnnOff &o = a.off;
    stage_bwd<H>(MBv, a.P, o.B[t], 2 * H, 0);
    stage_bwd<H>(MBm, a.P, o.B[t], 2 * H, H);
    if (last) {
        stage_bwd<H>(MN, a.P, o.D, H, 0);
    } else {
        stage_bwd<H>(MN, a.P, o.A[t + 1], 3 * H, H);
        stage_bwd<H>(MN + H * H, a.P, o.A[t + 1], 3 * H, 2 * H);
        stage_bwd<H>(MN + 2 * H * H, a.P, o.A[t + 1], 3 * H, 0);
    }
    if (t == 0) stage_bwd<H>(MA0, a.P, o.A[0], 3 * H, 0);
    __syncthreads();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    GnnWarpSmem<H, G> &W = ws[w];
    float wenc[HL][3], benc[HL];
#pragma unroll
    for (int q = 0; q < HL; ++q) {
        const int h = lane + 32 * q;
        for (int c = 0; c < 3; ++c) wenc[q][c] = __ldg(a.P + o.Wenc + 3 * h + c);
        benc[q] = __ldg(a.P + o.benc + h);
    }
    const float inv_rc = 1.0f / a.rc;
    const size_t NE = (size_t)a.N * a.cap;
    float *ze_t = a.ze + (size_t)t * NE * H;
    const float *gz_n = last ? nullptr : a.ze + (size_t)(t + 1) * NE * H;   // gradients of step t + 1
    const int ngroups = (a.N + G - 1) / G;
    for (int grp = blockIdx.x * gnn_warps(G) + w; grp < ngroups; grp += gridDim.x * gnn_warps(G)) {
        const int i0 = grp * G, na = min(G, a.N - i0);
        const int nv = gnn_group_edges<H, G>(a, i0, na, gnn_group_counts(a, i0, na), W);
        // node gradients dE/dv of step t's output, for the group
        float gv[G][HL];
        if (last) {
#pragma unroll
            for (int g = 0; g < G; ++g) {
                if (g < na) {
#pragma unroll
                    for (int q = 0; q < HL; ++q)
                        W.XN[g][lane + 32 * q] = a.gvd[(size_t)(i0 + g) * H + lane + 32 * q];
                }
            }
#pragma unroll
            for (int g = 0; g < G; ++g)
#pragma unroll
                for (int q = 0; q < HL; ++q) gv[g][q] = 0.0f;
            __syncwarp();
            wmv<H, G>(MN, H, &W.XN[0][0], 2 * H, gv, na);
        } else {
            // receiver sums over the atom's edges, sender sums over its
            // reverse edges (batches of GNN_EB edges, loads in flight together)
#pragma unroll
            for (int g = 0; g < G; ++g)
#pragma unroll
                for (int q = 0; q < HL; ++q) {
                    W.XN[g][lane + 32 * q] = 0.0f;
                    W.XN[g][H + lane + 32 * q] = 0.0f;
                }
            __syncwarp();
            for (int b0 = 0; b0 < nv; b0 += GNN_EB) {
                float vr[GNN_EB][HL], vs[GNN_EB][HL];
                int ge[GNN_EB];
#pragma unroll
                for (int e = 0; e < GNN_EB; ++e) {
                    ge[e] = -1;
                    if (b0 + e < nv) {
                        const int code = W.el[b0 + e], g = code / GNN_MAXCAP, k = code - g * GNN_MAXCAP;
                        const size_t E = (size_t)(i0 + g) * a.cap + k;
                        const size_t Er = (size_t)a.rev[E];
                        ge[e] = g;
#pragma unroll
                        for (int q = 0; q < HL; ++q) {
                            vr[e][q] = gz_n[E * H + lane + 32 * q];
                            vs[e][q] = gz_n[Er * H + lane + 32 * q];
                        }
                    }
                }
#pragma unroll
                for (int e = 0; e < GNN_EB; ++e) {
                    if (ge[e] >= 0) {
#pragma unroll
                        for (int q = 0; q < HL; ++q) {
                            W.XN[ge[e]][lane + 32 * q] += vr[e][q];
                            W.XN[ge[e]][H + lane + 32 * q] += vs[e][q];
                        }
                    }
                }
            }
#pragma unroll
            for (int g = 0; g < G; ++g) {
#pragma unroll
                for (int q = 0; q < HL; ++q) gv[g][q] = g < na ? a.gvd[(size_t)(i0 + g) * H + lane + 32 * q] : 0.0f;
            }
            __syncwarp();
            wmv<H, G>(MN, H, &W.XN[0][0], 2 * H, gv, na);
            wmv<H, G>(MN + H * H, H, &W.XN[0][H], 2 * H, gv, na);
        }
        __syncwarp();
        // through the node update: gz_v = gv silu'(zv)
#pragma unroll
        for (int g = 0; g < G; ++g) {
            if (g < na) {
#pragma unroll
                for (int q = 0; q < HL; ++q) {
                    const int h = lane + 32 * q;
                    W.XN[g][h] = gv[g][q] * gnn_dsilu(a.zv[((size_t)t * a.N + i0 + g) * H + h]);
                }
            }
        }
        __syncwarp();
        {
            float gm[G][HL];
#pragma unroll
            for (int g = 0; g < G; ++g)
#pragma unroll
                for (int q = 0; q < HL; ++q) gm[g][q] = 0.0f;
            wmv<H, G>(MBm, H, &W.XN[0][0], 2 * H, gm, na);
#pragma unroll
            for (int g = 0; g < G; ++g)
#pragma unroll
                for (int q = 0; q < HL; ++q) W.GM[g][lane + 32 * q] = gm[g][q];
        }
        if (t > 0) {
            float gd[G][HL];
#pragma unroll
            for (int g = 0; g < G; ++g)
#pragma unroll
                for (int q = 0; q < HL; ++q) gd[g][q] = 0.0f;
            wmv<H, G>(MBv, H, &W.XN[0][0], 2 * H, gd, na);
#pragma unroll
            for (int g = 0; g < G; ++g) {
                if (g < na) {
#pragma unroll
                    for (int q = 0; q < HL; ++q) a.gvd[(size_t)(i0 + g) * H + lane + 32 * q] = gd[g][q];
                }
            }
        }
        __syncwarp();
        // edges: ge = s gm (+ A_e^T gz of step t + 1); gz = ge silu'(z)
        for (int b0 = 0; b0 < nv; b0 += GNN_EB) {
            const int ne = min(GNN_EB, nv - b0);
            float acc[GNN_EB][HL];
#pragma unroll
            for (int e = 0; e < GNN_EB; ++e) {
                if (e < ne) {
                    const int code = W.el[b0 + e], g = code / GNN_MAXCAP, k = code - g * GNN_MAXCAP;
                    const size_t E = (size_t)(i0 + g) * a.cap + k;
                    const float s = a.cut[E].x;
#pragma unroll
                    for (int q = 0; q < HL; ++q) {
                        acc[e][q] = s * W.GM[g][lane + 32 * q];
                        if (!last) W.X[e][lane + 32 * q] = gz_n[E * H + lane + 32 * q];
                    }
                }
            }
            __syncwarp();
            if (!last) wmv<H, GNN_EB>(MN + 2 * H * H, H, &W.X[0][0], H, acc, ne);
            __syncwarp();
#pragma unroll
            for (int e = 0; e < GNN_EB; ++e) {
                if (e < ne) {
                    const int code = W.el[b0 + e], g = code / GNN_MAXCAP, k = code - g * GNN_MAXCAP;
                    const size_t E = (size_t)(i0 + g) * a.cap + k;
                    float gsv = 0.0f;
#pragma unroll
                    for (int q = 0; q < HL; ++q) {
                        const int h = lane + 32 * q;
                        const float z = ze_t[E * H + h];
                        const float sg = gnn_sig(z);
                        gsv += W.GM[g][h] * (z * sg);
                        const float gz = acc[e][q] * (sg * (1.0f + z * (1.0f - sg)));
                        if (t > 0) ze_t[E * H + h] = gz;
                        else W.X[e][h] = gz;
                    }
                    gsv = gnn_wsum(gsv);
                    if (lane == 0) a.gs[E] = last ? gsv : a.gs[E] + gsv;
                }
            }
            __syncwarp();
            if (t == 0) {
                // through step 0's A_e into the encoder, then to the displacement
                float g0[GNN_EB][HL];
#pragma unroll
                for (int e = 0; e < GNN_EB; ++e)
#pragma unroll
                    for (int q = 0; q < HL; ++q) g0[e][q] = 0.0f;
                wmv<H, GNN_EB>(MA0, H, &W.X[0][0], H, g0, ne);
#pragma unroll
                for (int e = 0; e < GNN_EB; ++e) {
                    if (e < ne) {
                        const int code = W.el[b0 + e], g = code / GNN_MAXCAP, k = code - g * GNN_MAXCAP;
                        const size_t E = (size_t)(i0 + g) * a.cap + k;
                        const float4 d4 = a.dr[E];
                        float gx = 0.f, gy = 0.f, gz = 0.f;
#pragma unroll
                        for (int q = 0; q < HL; ++q) {
                            const float z0 = wenc[q][0] * (d4.x * inv_rc) + wenc[q][1] * (d4.y * inv_rc) +
                                             wenc[q][2] * (d4.z * inv_rc) + benc[q];
                            const float gg = g0[e][q] * gnn_dsilu(z0);
                            gx += wenc[q][0] * gg;
                            gy += wenc[q][1] * gg;
                            gz += wenc[q][2] * gg;
                        }
                        gx = gnn_wsum(gx);
                        gy = gnn_wsum(gy);
                        gz = gnn_wsum(gz);
                        if (lane == 0) {
                            const float c = a.gs[E] * a.cut[E].y;
                            a.gpos[E] = make_float4(gx * inv_rc + c * d4.x, gy * inv_rc + c * d4.y,
                                                    gz * inv_rc + c * d4.z, 0.0f);
                        }
                    }
                }
                __syncwarp();
            }
        }
    }
}

// F_i = sum over the atom's edges of g(i <- j) - g(j <- i); KICK: closing
// half-kick of velocity Verlet.
template <int KICK>
__global__ void __launch_bounds__(256) k_gnn_force(GnnArgs g, PairArgs pa)
{
    count_launch();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float pe_acc = 0.0f, ke_acc = 0.0f;
    for (int i = blockIdx.x * 8 + w; i < g.N; i += gridDim.x * 8) {
        int n = g.cnt[i];
        n = n < g.cap ? n : g.cap;
        float fx = 0.f, fy = 0.f, fz = 0.f;
        for (int k = lane; k < n; k += 32) {
            const size_t E = (size_t)i * g.cap + k;
            const int rv = g.rev[E];
            if (rv < 0) continue;
            const float4 a4 = g.gpos[E], b4 = g.gpos[rv];
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

template <int H, int G>
static size_t gnn_smem_fwd()
{
    return sizeof(float) * (5 * H * H + 3 * H) + sizeof(GnnWarpSmem<H, G>) * gnn_warps(G);
}
template <int H, int G>
static size_t gnn_smem_bwd(int t)
{
    return sizeof(float) * ((t == 0 ? 6 : 5) * H * H) + sizeof(GnnWarpSmem<H, G>) * gnn_warps(G);
}


static int g_gnn_group = 4;   // atoms per warp (md_gnn_set_group)
static int g_gnn_tc = 0;      // 1: the tensor-core kernels (gnn_tc.cu; H = 64)
int gnn_variant() { return g_gnn_tc | (g_gnn_group << 1); }

static int gnn_sms()
{
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms < 1) sms = 1;
    }
    return sms;
}

template <int H, int G>
static void gnn_launch_all(const GnnArgs &g, cudaStream_t st)
{
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_gnn_fwd<H, G>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gnn_smem_fwd<H, G>());
        cudaFuncSetAttribute(k_gnn_bwd<H, G>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gnn_smem_bwd<H, G>(0));
        attr = true;
    }
    const int per_block = G * gnn_warps(G);
    const int grid = std::max(1, std::min((g.N + per_block - 1) / per_block, gnn_sms()));
    for (int t = 0; t < g.T; ++t) k_gnn_fwd<H, G><<<grid, gnn_warps(G) * 32, gnn_smem_fwd<H, G>(), st>>>(g, t);
    for (int t = g.T - 1; t >= 0; --t)
        k_gnn_bwd<H, G><<<grid, gnn_warps(G) * 32, gnn_smem_bwd<H, G>(t), st>>>(g, t);
}

template <int H>
static void gnn_launch_h(const GnnArgs &g, cudaStream_t st)
{
    switch (g_gnn_group) {
    case 8: gnn_launch_all<H, 8>(g, st); break;
    case 4: gnn_launch_all<H, 4>(g, st); break;
    case 2: gnn_launch_all<H, 2>(g, st); break;
    default: gnn_launch_all<H, 1>(g, st); break;
    }
}

bool gnn_model_ok(const md_gnn_model *m, const md_nbr *nb)
{
    if (!m || !m->params || !m->ws || !nb) return false;
    if (m->H != 32 && m->H != 64) return false;
    if (m->T < 1 || m->T > GNN_MAXT) return false;
    if (!(m->r_cut > 0.0f) || m->r_cut > nb->r_list) return false;
    if (nb->cap > GNN_MAXCAP || nb->dim != 3) return false;
    if (m->sys_n < 0 || (m->sys_n > 0 && nb->N % m->sys_n != 0)) return false;
    return m->ws_bytes >= gnn_ws_layout(nb->N, nb->cap, m->H, m->T).total;
}

void gnn_bind_workspace(GnnArgs &g, const md_gnn_model *m)
{
    const GnnWs L = gnn_ws_layout(g.N, g.cap, m->H, m->T);
    unsigned char *b = (unsigned char *)m->ws;
    g.rev = (int32_t *)(b + L.rev);
    g.dr = (float4 *)(b + L.dr);
    g.cut = (float2 *)(b + L.cut);
    g.gs = (float *)(b + L.gs);
    g.gpos = (float4 *)(b + L.gpos);
    g.ze = (float *)(b + L.ze);
    g.zv = (float *)(b + L.zv);
    g.rr = (float *)(b + L.rr);
    g.ps = (float *)(b + L.ps);
    g.gvd = (float *)(b + L.gvd);
    g.Ei = (float *)(b + L.Ei);
    g.H = m->H;
    g.nv = (int *)(b + L.nv);
    g.eoff = (int *)(b + L.off);
    g.ctot = (int *)(b + L.ctot);
    g.erecv = (int *)(b + L.erecv);
    g.esend = (int *)(b + L.esend);
    g.erev = (int *)(b + L.erev);
    g.eslot = (int *)(b + L.eslot);
    g.cidx = (int *)(b + L.cidx);
    g.edr = (float4 *)(b + L.edr);
    g.ecut = (float2 *)(b + L.ecut);
    g.gm = (float *)(b + L.gm);
}

void enqueue_gnn_step(const PairArgs &pa, int kick, cudaStream_t st)
{
    const md_gnn_model *m = &pa.gnn;
    GnnArgs g;
    memset(&g, 0, sizeof(g));
    g.box = pa.box;
    g.N = pa.N;
    g.cap = pa.cap;
    g.T = m->T;
    g.rc = m->r_cut;
    g.rc2 = m->r_cut * m->r_cut;
    g.r = pa.r;
    g.nbr = pa.nbr;
    g.cnt = pa.cnt;
    g.P = m->params;
    g.off = gnn_offsets(m->H, m->T);
    g.sys_n = m->sys_n;
    gnn_bind_workspace(g, m);
    g.status = pa.status;
    if (g_gnn_tc && m->H == 64) {
        enqueue_gnn_tc(g, pa, kick, st);
        return;
    }
    if (m->H == 64) gnn_launch_h<64>(g, st);
    else gnn_launch_h<32>(g, st);
    const int fgrid = std::max(1, std::min((pa.N + 7) / 8, pa.max_blocks));
    if (kick) k_gnn_force<1><<<fgrid, 256, 0, st>>>(g, pa);
    else k_gnn_force<0><<<fgrid, 256, 0, st>>>(g, pa);
}

}  // namespace jmd

using namespace jmd;

extern "C" size_t md_gnn_param_count(int H, int T)
{
    if ((H != 32 && H != 64) || T < 1 || T > GNN_MAXT) return 0;
    return (size_t)gnn_offsets(H, T).count;
}

extern "C" md_status md_gnn_set_tensor_cores(int on)
{
    if (on != 0 && on != 1) return MD_ERR_INVALID;
    g_gnn_tc = on;
    return MD_OK;
}

extern "C" md_status md_gnn_set_group(int G)
{
    if (G != 1 && G != 2 && G != 4 && G != 8) return MD_ERR_INVALID;
    g_gnn_group = G;
    return MD_OK;
}

extern "C" size_t md_gnn_workspace_bytes(int N, int cap, int H, int T)
{
    if (N < 1 || cap < 1 || cap > GNN_MAXCAP || (H != 32 && H != 64) || T < 1 || T > GNN_MAXT) return 0;
    return gnn_ws_layout(N, cap, H, T).total;
}
