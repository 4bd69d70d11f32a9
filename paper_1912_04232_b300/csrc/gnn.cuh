// gnn.cuh -- shared parts of the graph-network potential (gnn.cu: FP32
// CUDA-core kernels; gnn_tc.cu: tensor-core kernels): parameter offsets,
// kernel arguments, workspace layout and the element-wise functions.
#pragma once

#include "common.cuh"

namespace jmd {

// warps per block for a group size (shared memory: weights + per-warp buffers)
__host__ __device__ constexpr int gnn_warps(int G) { return G >= 8 ? 12 : 16; }
constexpr int GNN_EB = 8;    // edges per batch
constexpr int GNN_MAXT = 4;
constexpr int GNN_MAXCAP = 64;

struct GnnOff {
    int Wenc, benc, u, A[GNN_MAXT], a[GNN_MAXT], B[GNN_MAXT], b[GNN_MAXT], D, d, w, c, count;
};

inline GnnOff gnn_offsets(int H, int T)
{
    GnnOff o;
    memset(&o, 0, sizeof(o));
    int p = 0;
    o.Wenc = p; p += 3 * H;
    o.benc = p; p += H;
    o.u = p;    p += H;
    for (int t = 0; t < T; ++t) {
        o.A[t] = p; p += 3 * H * H;
        o.a[t] = p; p += H;
        o.B[t] = p; p += 2 * H * H;
        o.b[t] = p; p += H;
    }
    o.D = p; p += H * H;
    o.d = p; p += H;
    o.w = p; p += H;
    o.c = p; p += 1;
    o.count = p;
    return o;
}

struct GnnArgs {
    Box box;
    int N, cap, T;
    int sys_n;        // 0: rows hold global indices; else atoms per system, rows local to each system
    float rc, rc2;
    const float4 *r;
    const int32_t *nbr, *cnt;
    const float *P;
    GnnOff off;
    int32_t *rev;     // [N*cap] slot of the reverse edge (j*cap + p), -1: no edge
    float4 *dr;       // [N*cap] R_j - R_i (minimum image), r
    float2 *cut;      // [N*cap] s(r), s'(r) / r
    float *gs;        // [N*cap] dE/ds summed over the steps
    float4 *gpos;     // [N*cap] dE/d(R_j - R_i)
    float *ze;        // [T][N*cap][H] edge pre-activations; reverse: their gradients
    float *zv;        // [T][N][H] node pre-activations
    float *rr, *ps;   // [2][N][H] receiver term A_r v + a and sender term A_s v of the next step
    float *gvd;       // [N][H] node gradient carried to the step below
    float *Ei;        // [N]
    uint32_t *status;
    // tensor-core path: the edges with r < r_c compacted in receiver order
    // (per-edge arrays above are then indexed by the compact edge e)
    int H;
    int *nv, *eoff;                  // [N] valid edges per atom, [N+1] their offsets
    int *ctot;                       // [N/1024 + 1] scan scratch
    int *erecv, *esend, *erev, *eslot;   // [N*cap] receiver, sender, reverse edge, row slot
    int *cidx;                       // [N*cap] compact index of a row slot
    float4 *edr;                     // [N*cap] R_j - R_i, r of edge e
    float2 *ecut;                    // [N*cap] s, s'/r of edge e
    float *gm;                       // [N][H] message gradient (reverse)
};

__device__ __forceinline__ float gnn_sig(float x) { return __fdividef(1.0f, 1.0f + __expf(-x)); }
__device__ __forceinline__ float gnn_silu(float x) { return x * gnn_sig(x); }
__device__ __forceinline__ float gnn_dsilu(float x)
{
    const float s = gnn_sig(x);
    return s * (1.0f + x * (1.0f - s));
}

__device__ __forceinline__ float gnn_wsum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// s(r) and s'(r)/r
__device__ __forceinline__ void gnn_cut(float r, float rc, float &s, float &dsr)
{
    float sn, cs;
    sincospif(r / rc, &sn, &cs);
    s = 0.5f * (cs + 1.0f);
    // s'(r) / r = -pi sin(pi r / r_c) / (2 r_c r); its limit at r = 0 is -pi^2 / (2 r_c^2)
    dsr = r > 0.0f ? -0.5f * 3.14159265358979f * sn / (rc * r) : -0.5f * 9.8696044010894f / (rc * rc);
}

struct GnnWs {
    size_t rev, dr, cut, gs, gpos, ze, zv, rr, ps, gvd, Ei, nv, off, ctot, erecv, esend, erev, eslot, cidx, edr, ecut, gm,
        total;
};

inline GnnWs gnn_ws_layout(int N, int cap, int H, int T)
{
    GnnWs w;
    const size_t NE = (size_t)N * cap;
    size_t o = 0;
    w.rev = o;  o = align256(o + sizeof(int32_t) * NE);
    w.dr = o;   o = align256(o + sizeof(float4) * NE);
    w.cut = o;  o = align256(o + sizeof(float2) * NE);
    w.gs = o;   o = align256(o + sizeof(float) * NE);
    w.gpos = o; o = align256(o + sizeof(float4) * NE);
    w.ze = o;   o = align256(o + sizeof(float) * (size_t)T * NE * H);
    w.zv = o;   o = align256(o + sizeof(float) * (size_t)T * N * H);
    w.rr = o;   o = align256(o + sizeof(float) * 2 * (size_t)N * H);
    w.ps = o;   o = align256(o + sizeof(float) * 2 * (size_t)N * H);
    w.gvd = o;  o = align256(o + sizeof(float) * (size_t)N * H);
    w.Ei = o;   o = align256(o + sizeof(float) * (size_t)N);
    w.nv = o;    o = align256(o + sizeof(int) * (size_t)N);
    w.off = o;   o = align256(o + sizeof(int) * ((size_t)N + 1));
    w.ctot = o;  o = align256(o + sizeof(int) * ((size_t)N / 1024 + 2));
    w.erecv = o; o = align256(o + sizeof(int) * NE);
    w.esend = o; o = align256(o + sizeof(int) * NE);
    w.erev = o;  o = align256(o + sizeof(int) * NE);
    w.eslot = o; o = align256(o + sizeof(int) * NE);
    w.cidx = o;  o = align256(o + sizeof(int) * NE);
    w.edr = o;   o = align256(o + sizeof(float4) * NE);
    w.ecut = o;  o = align256(o + sizeof(float2) * NE);
    w.gm = o;    o = align256(o + sizeof(float) * (size_t)N * H);
    w.total = o;
    return w;
}

struct PairArgs;
void enqueue_gnn_tc(const GnnArgs &g, const PairArgs &pa, int kick, cudaStream_t st);
void enqueue_gnn_compact(const GnnArgs &g, cudaStream_t st);
// Points g's arrays into the model's workspace (g.N, g.cap, g.T set).
void gnn_bind_workspace(GnnArgs &g, const md_gnn_model *m);

}  // namespace jmd
