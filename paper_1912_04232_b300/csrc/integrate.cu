// integrate.cu -- dynamics and minimisation (Sec. 3.3.1).
//
// Velocity-Verlet NVE step as three stages:
//   k_kick_drift   v += dt/2 F/m; r = wrap(r + dt v); displacement check
//   rebuild chain  (only when some particle moved > skin/2; see nbr.cu)
//   k_pair<KICK>   F(r), then v += dt/2 F/m, FP64 PE/KE of the step
// Gradient-descent step:
//   k_pair         F(r_t), U(r_t)
//   k_gd_step      r += eta F (unwrapped), displacement check
//   rebuild chain
#include <cmath>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"
#include "nhc.cuh"

namespace jmd {

template <int DIM, int COND>
__global__ void __launch_bounds__(256) k_kick_drift(float4 *r, float4 *v, const float4 *f, const float4 *rref, int N,
                                                    float hdm, float dt, Box box, float half_skin2, uint32_t *ctl,
                                                    unsigned long long cond_if)
{
    count_launch();
    __shared__ bool last;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    bool mv = false;
    if (i < N) {
        float4 fi = f[i], vi = v[i], ri = r[i];
        vi.x += hdm * fi.x;
        vi.y += hdm * fi.y;
        ri.x = wrap_coord(ri.x + dt * vi.x, box.L[0], box.Linv[0]);
        ri.y = wrap_coord(ri.y + dt * vi.y, box.L[1], box.Linv[1]);
        if (DIM == 3) {
            vi.z += hdm * fi.z;
            ri.z = wrap_coord(ri.z + dt * vi.z, box.L[2], box.Linv[2]);
        }
        v[i] = vi;
        r[i] = ri;
        float dx, dy, dz;
        mv = dist2_rn<DIM>(ri, rref[i], box, dx, dy, dz) > half_skin2;
    }
    if (__any_sync(0xffffffffu, mv) && (threadIdx.x & 31) == 0) {
        ctl[CTL_REBUILD] = 1u;
        if (COND) __threadfence();
    }
    if (COND) {
        // the last block to finish hands the rebuild decision to the graph's
        // IF node (a single caller of cudaGraphSetConditional per launch)
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            unsigned t = atomicAdd(&ctl[CTL_TICKET2], 1u);
            last = (t == gridDim.x - 1);
        }
        __syncthreads();
        if (last && threadIdx.x == 0) {
            __threadfence();
            unsigned flag = *(volatile uint32_t *)&ctl[CTL_REBUILD];
            ctl[CTL_TICKET2] = 0u;
            cudaGraphSetConditional((cudaGraphConditionalHandle)cond_if, flag ? 1u : 0u);
        }
    }
}

// Nose-Hoover chain step, first part: the velocity factor left by the
// thermostat half-steps (previous step's closing and this step's opening
// one), then the kick and the drift, as k_kick_drift.
template <int DIM, int COND>
__global__ void __launch_bounds__(256) k_nhc_kick_drift(float4 *r, float4 *v, const float4 *f, const float4 *rref,
                                                        int N, float hdm, float dt, Box box, float half_skin2,
                                                        uint32_t *ctl, unsigned long long cond_if, const double *nhc,
                                                        int M)
{
    count_launch();
    __shared__ bool last;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    bool mv = false;
    if (i < N) {
        const float sc = (float)nhc[3 * M + NHC_SCLOSE], so = (float)nhc[3 * M + NHC_SOPEN];
        float4 fi = f[i], vi = v[i], ri = r[i];
        vi.x *= sc;
        vi.y *= sc;
        vi.z *= sc;
        vi.x = vi.x * so + hdm * fi.x;
        vi.y = vi.y * so + hdm * fi.y;
        ri.x = wrap_coord(ri.x + dt * vi.x, box.L[0], box.Linv[0]);
        ri.y = wrap_coord(ri.y + dt * vi.y, box.L[1], box.Linv[1]);
        if (DIM == 3) {
            vi.z = vi.z * so + hdm * fi.z;
            ri.z = wrap_coord(ri.z + dt * vi.z, box.L[2], box.Linv[2]);
        }
        v[i] = vi;
        r[i] = ri;
        float dx, dy, dz;
        mv = dist2_rn<DIM>(ri, rref[i], box, dx, dy, dz) > half_skin2;
    }
    if (__any_sync(0xffffffffu, mv) && (threadIdx.x & 31) == 0) {
        ctl[CTL_REBUILD] = 1u;
        if (COND) __threadfence();
    }
    if (COND) {
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            unsigned t = atomicAdd(&ctl[CTL_TICKET2], 1u);
            last = (t == gridDim.x - 1);
        }
        __syncthreads();
        if (last && threadIdx.x == 0) {
            __threadfence();
            unsigned flag = *(volatile uint32_t *)&ctl[CTL_REBUILD];
            ctl[CTL_TICKET2] = 0u;
            cudaGraphSetConditional((cudaGraphConditionalHandle)cond_if, flag ? 1u : 0u);
        }
    }
}

// Before the loop (one block): the first step's opening thermostat
// half-step, from the kinetic energy of the initial velocities (reset) or
// the one the previous call's last step left (continuation, whose closing
// factor the velocities already carry).
__global__ void __launch_bounds__(1024) k_nhc_begin(const float4 *v, int N, float mass, double *nhc, int M,
                                                    int reset)
{
    count_launch();
    __shared__ double sh[32];
    double *c = nhc + 3 * M;
    double K = 0.0;
    if (reset) {
        float k = 0.0f;
        for (int i = threadIdx.x; i < N; i += blockDim.x) {
            const float4 vi = v[i];
            k += 0.5f * mass * (vi.x * vi.x + vi.y * vi.y + vi.z * vi.z);
        }
        K = block_sum_f64((double)k, sh);
    }
    if (threadIdx.x == 0) {
        if (!reset) K = c[NHC_K];
        c[NHC_SCLOSE] = 1.0;
        c[NHC_SOPEN] = nhc_half_step(nhc, M, K);
    }
}

// After each force kernel (one thread): the closing thermostat half-step of
// the step from the kinetic energy the force kernel left, the extended
// energy, and, if another step follows, the next step's opening half-step.
// The next kick-drift applies both velocity factors (the closing one alone
// at the end of the loop); the series get the thermostatted state.  The
// force kernel has already advanced the step counter.
// The chain's scalars are held in registers (the chain length is a
// compile-time constant of the unrolled code) and the reciprocal masses are
// taken once for both half-steps.
__global__ void k_nhc_update(double *nhc_g, int M, const uint32_t *ctl, double *KE_out, double *H_out)
{
    count_launch();
    double *c = nhc_g + 3 * M;
    const unsigned step = ctl[CTL_STEP] - 1u;
    const double gkT = c[NHC_GKT], kT = c[NHC_KT], dt = c[NHC_DT], pe = c[NHC_PE];
    const bool more = step + 1u < ctl[CTL_NSTEPS];
    double K = c[NHC_KRAW], sclose = 1.0, sopen = 1.0, H = 0.0;
    nhc_dispatch(M, [&](auto m) {
        constexpr int MM = decltype(m)::value;
        nhc_with_state<MM>(nhc_g, [&](double *xi, double *w, const double *Q, const double *iQ) {
            sclose = nhc_half_step_m<MM>(xi, w, Q, iQ, gkT, kT, dt, K);
            // the extended energy after the closing half-step
            double e = gkT * xi[0];
#pragma unroll
            for (int k = 0; k < MM; ++k) e += 0.5 * Q[k] * w[k] * w[k];
#pragma unroll
            for (int k = 1; k < MM; ++k) e += kT * xi[k];
            H = pe + K + e;
            if (KE_out) KE_out[step] = K;
            if (H_out) H_out[step] = H;
            c[NHC_K] = K;
            if (more) sopen = nhc_half_step_m<MM>(xi, w, Q, iQ, gkT, kT, dt, K);
        });
    });
    c[NHC_SCLOSE] = sclose;
    c[NHC_SOPEN] = sopen;
}

// After the loop: the last step's closing velocity factor.
__global__ void __launch_bounds__(256) k_nhc_end(float4 *v, int N, const double *nhc, int M)
{
    count_launch();
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const float sc = (float)nhc[3 * M + NHC_SCLOSE];
    float4 vi = v[i];
    vi.x *= sc;
    vi.y *= sc;
    vi.z *= sc;
    v[i] = vi;
}

// BAOAB Langevin (Sec. 3.3.1), first part B-A-O-A:
//   v += dt/2 F/m;  r += dt/2 v;  v = c1 v + c2 z;  r += dt/2 v;  wrap
// with c1 = exp(-gamma dt), c2 = sqrt((1 - c1^2) kT / m) and z from Philox
// counter (i, step0 + step).  The closing B is the force kernel's kick.
template <int COND>
__global__ void __launch_bounds__(256) k_baoa(float4 *r, float4 *v, const float4 *f, const float4 *rref, int N,
                                              float hdm, float dt, float c1, float c2, Box box, float half_skin2,
                                              uint32_t *ctl, unsigned long long cond_if)
{
    count_launch();
    __shared__ bool last;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    bool mv = false;
    if (i < N) {
        const unsigned s = ctl[CTL_STEP0] + ctl[CTL_STEP];
        const uint2 key = make_uint2(ctl[CTL_SEED_LO], ctl[CTL_SEED_HI]);
        float3 z = normal3((unsigned)i, s, key);
        float4 fi = f[i], vi = v[i], ri = r[i];
        const float h = 0.5f * dt;
        vi.x += hdm * fi.x;
        vi.y += hdm * fi.y;
        vi.z += hdm * fi.z;
        ri.x += h * vi.x;
        ri.y += h * vi.y;
        ri.z += h * vi.z;
        vi.x = c1 * vi.x + c2 * z.x;
        vi.y = c1 * vi.y + c2 * z.y;
        vi.z = c1 * vi.z + c2 * z.z;
        ri.x = wrap_coord(ri.x + h * vi.x, box.L[0], box.Linv[0]);
        ri.y = wrap_coord(ri.y + h * vi.y, box.L[1], box.Linv[1]);
        ri.z = wrap_coord(ri.z + h * vi.z, box.L[2], box.Linv[2]);
        v[i] = vi;
        r[i] = ri;
        float dx, dy, dz;
        mv = dist2_rn<3>(ri, rref[i], box, dx, dy, dz) > half_skin2;
    }
    if (__any_sync(0xffffffffu, mv) && (threadIdx.x & 31) == 0) {
        ctl[CTL_REBUILD] = 1u;
        if (COND) __threadfence();
    }
    if (COND) {
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            unsigned t = atomicAdd(&ctl[CTL_TICKET2], 1u);
            last = (t == gridDim.x - 1);
        }
        __syncthreads();
        if (last && threadIdx.x == 0) {
            __threadfence();
            unsigned flag = *(volatile uint32_t *)&ctl[CTL_REBUILD];
            ctl[CTL_TICKET2] = 0u;
            cudaGraphSetConditional((cudaGraphConditionalHandle)cond_if, flag ? 1u : 0u);
        }
    }
}

template <int DIM>
__global__ void __launch_bounds__(256) k_gd_step(float4 *r, const float4 *f, const float4 *rref, int N, float eta,
                                                 Box box, float half_skin2, uint32_t *ctl)
{
    count_launch();
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    bool mv = false;
    if (i < N) {
        float4 fi = f[i], ri = r[i];
        ri.x += eta * fi.x;
        ri.y += eta * fi.y;
        if (DIM == 3) ri.z += eta * fi.z;
        r[i] = ri;
        float dx, dy, dz;
        mv = dist2_rn<DIM>(ri, rref[i], box, dx, dy, dz) > half_skin2;
    }
    if (__any_sync(0xffffffffu, mv) && (threadIdx.x & 31) == 0) ctl[CTL_REBUILD] = 1u;
}

// Fused NVE loop: positions alternate between r and r_alt, so after an even
// number of steps the final positions are in r_alt.
__global__ void __launch_bounds__(256) k_final_positions(float4 *r, const float4 *r_alt, int N, const uint32_t *ctl)
{
    count_launch();
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N && (ctl[CTL_NSTEPS] & 1u) == 0u) r[i] = r_alt[i];
}

__global__ void k_loop_init(uint32_t *ctl, uint32_t nsteps, uint32_t step0, unsigned long long seed)
{
    count_launch();
    ctl[CTL_STEP] = 0u;
    ctl[CTL_NSTEPS] = nsteps;
    ctl[CTL_STEP0] = step0;
    ctl[CTL_SEED_LO] = (uint32_t)seed;
    ctl[CTL_SEED_HI] = (uint32_t)(seed >> 32);
}

void enqueue_loop_init(uint32_t *ctl, uint32_t nsteps, cudaStream_t st)
{
    k_loop_init<<<1, 1, 0, st>>>(ctl, nsteps, 0u, 0ull);
}

struct NveCtx {
    Box box;
    int dim, N;
    float4 *r, *v, *f, *rref;
    float hdm, dt, half_skin2;
    uint32_t *ctl;
    NbrArgs na;
    int ncell_total;
    PairArgs pa;
    int pot;
    int langevin;                 // 0: NVE kick-drift, 1: BAOAB first part
    int fused;                    // 1: kick-drift fused into the force kernel (pair potentials, NVE)
    int nhc;                      // 1: Nose-Hoover chain (thermostat state in pa.nhc)
    int nhc_reset;                // 1: the chain starts at rest, K from the initial velocities
    float c1, c2;                 // Langevin O-step coefficients
    unsigned long long cond_if;   // graph IF handle (0 outside graphs)
};

static void enqueue_kick_drift(const NveCtx &c, int cond, cudaStream_t st)
{
    int g = (c.N + 255) / 256;
    if (c.nhc) {
        const unsigned long long ci = cond ? c.cond_if : 0ull;
        if (c.dim == 3) {
            if (cond)
                k_nhc_kick_drift<3, 1><<<g, 256, 0, st>>>(c.r, c.v, c.f, c.rref, c.N, c.hdm, c.dt, c.box, c.half_skin2,
                                                          c.ctl, ci, c.pa.nhc, c.pa.nhc_M);
            else
                k_nhc_kick_drift<3, 0><<<g, 256, 0, st>>>(c.r, c.v, c.f, c.rref, c.N, c.hdm, c.dt, c.box, c.half_skin2,
                                                          c.ctl, ci, c.pa.nhc, c.pa.nhc_M);
        } else {
            if (cond)
                k_nhc_kick_drift<2, 1><<<g, 256, 0, st>>>(c.r, c.v, c.f, c.rref, c.N, c.hdm, c.dt, c.box, c.half_skin2,
                                                          c.ctl, ci, c.pa.nhc, c.pa.nhc_M);
            else
                k_nhc_kick_drift<2, 0><<<g, 256, 0, st>>>(c.r, c.v, c.f, c.rref, c.N, c.hdm, c.dt, c.box, c.half_skin2,
                                                          c.ctl, ci, c.pa.nhc, c.pa.nhc_M);
        }
        return;
    }
    if (c.langevin) {
        if (cond)
            k_baoa<1><<<g, 256, 0, st>>>(c.r, c.v, c.f, c.rref, c.N, c.hdm, c.dt, c.c1, c.c2, c.box, c.half_skin2,
                                         c.ctl, c.cond_if);
        else
            k_baoa<0><<<g, 256, 0, st>>>(c.r, c.v, c.f, c.rref, c.N, c.hdm, c.dt, c.c1, c.c2, c.box, c.half_skin2,
                                         c.ctl, 0ull);
        return;
    }
    if (c.dim == 3) {
        if (cond)
            k_kick_drift<3, 1><<<g, 256, 0, st>>>(c.r, c.v, c.f, c.rref, c.N, c.hdm, c.dt, c.box, c.half_skin2, c.ctl,
                                                  c.cond_if);
        else
            k_kick_drift<3, 0><<<g, 256, 0, st>>>(c.r, c.v, c.f, c.rref, c.N, c.hdm, c.dt, c.box, c.half_skin2, c.ctl,
                                                  0ull);
    } else {
        if (cond)
            k_kick_drift<2, 1><<<g, 256, 0, st>>>(c.r, c.v, c.f, c.rref, c.N, c.hdm, c.dt, c.box, c.half_skin2, c.ctl,
                                                  c.cond_if);
        else
            k_kick_drift<2, 0><<<g, 256, 0, st>>>(c.r, c.v, c.f, c.rref, c.N, c.hdm, c.dt, c.box, c.half_skin2, c.ctl,
                                                  0ull);
    }
}

static void enqueue_nhc_update(const NveCtx &c, cudaStream_t st)
{
    k_nhc_update<<<1, 1, 0, st>>>(c.pa.nhc, c.pa.nhc_M, c.ctl, c.pa.KE_out, c.pa.H_out);
}

static void enqueue_nve_step(const NveCtx &c, cudaStream_t st)
{
    if (!c.fused) enqueue_kick_drift(c, 0, st);
    enqueue_rebuild_chain(c.na, c.ncell_total, st);
    enqueue_forces(c.pa, c.dim, c.pot, c.fused ? 2 : 1, st);
    if (c.nhc) enqueue_nhc_update(c, st);
}

static void enqueue_final_positions(const NveCtx &c, cudaStream_t st)
{
    k_final_positions<<<(c.N + 255) / 256, 256, 0, st>>>(c.r, c.pa.r_alt, c.N, c.ctl);
}

// Work before and after the loop (fused NVE: first kick-drift / final copy;
// Nose-Hoover chain: opening half-step / closing velocity factor).
static void enqueue_loop_pre(const NveCtx &c, int cond, cudaStream_t st)
{
    if (c.fused) enqueue_kick_drift(c, cond, st);
    if (c.nhc) k_nhc_begin<<<1, 1024, 0, st>>>(c.v, c.N, c.pa.mass, c.pa.nhc, c.pa.nhc_M, c.nhc_reset);
}

static void enqueue_loop_post(const NveCtx &c, cudaStream_t st)
{
    if (c.fused) enqueue_final_positions(c, st);
    if (c.nhc) k_nhc_end<<<(c.N + 255) / 256, 256, 0, st>>>(c.v, c.N, c.pa.nhc, c.pa.nhc_M);
}

// ---------------------------------------------------------------------------
// The whole NVE loop as one CUDA graph: a WHILE node whose body is one step,
// with the rebuild chain under an IF node.  The kick-drift kernel's last
// block sets the IF condition from the device rebuild flag; the force
// kernel's last block advances the step counter and sets the WHILE
// condition.  Fused loop: the first kick-drift runs before the WHILE node
// (and sets the first IF condition), the body is IF(rebuild) + the fused
// force kernel, whose last block also sets the next IF condition, and a copy
// after the loop returns the final positions to the caller's buffer.  No
// host involvement per step and no launches of an idle rebuild chain.
// Graphs are cached per argument set and device.
// ---------------------------------------------------------------------------
struct NveGraph {
    NveCtx key;
    int device;
    cudaGraph_t graph;
    cudaGraphExec_t exec;
};

static std::vector<NveGraph> g_nve_graphs;
static std::mutex g_nve_mu;

static cudaGraphNodeParams *zeroed_params(unsigned char *raw)
{
    memset(raw, 0, sizeof(cudaGraphNodeParams));
    return reinterpret_cast<cudaGraphNodeParams *>(raw);
}

static md_status build_nve_graph(const NveCtx &c0, NveGraph &out)
{
    NveCtx c = c0;
    cudaGraph_t g = nullptr;
    JMD_CUDA_TRY(cudaGraphCreate(&g, 0));
    cudaGraphConditionalHandle hw, hi;
    JMD_CUDA_TRY(cudaGraphConditionalHandleCreate(&hw, g, 1u, cudaGraphCondAssignDefault));
    JMD_CUDA_TRY(cudaGraphConditionalHandleCreate(&hi, g, 0u, cudaGraphCondAssignDefault));
    alignas(cudaGraphNodeParams) unsigned char wraw[sizeof(cudaGraphNodeParams)];
    cudaGraphNodeParams *wp = zeroed_params(wraw);
    wp->type = cudaGraphNodeTypeConditional;
    wp->conditional.handle = hw;
    wp->conditional.type = cudaGraphCondTypeWhile;
    wp->conditional.size = 1;
    cudaStream_t cs = nullptr, cs2 = nullptr;
    JMD_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    JMD_CUDA_TRY(cudaStreamCreateWithFlags(&cs2, cudaStreamNonBlocking));
    c.cond_if = (unsigned long long)hi;
    c.pa.cond_while = (unsigned long long)hw;
    c.pa.use_cond = 1;
    if (c.fused) c.pa.cond_if = (unsigned long long)hi;
    cudaGraphNode_t wn;
    if (c.fused || c.nhc) {
        // top level: loop prologue -> WHILE -> loop epilogue
        JMD_CUDA_TRY(cudaStreamBeginCaptureToGraph(cs, g, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
        enqueue_loop_pre(c, 1, cs);
        cudaStreamCaptureStatus tst;
        cudaGraph_t tg = nullptr;
        const cudaGraphNode_t *tdeps = nullptr;
        size_t tnd = 0;
        JMD_CUDA_TRY(cudaStreamGetCaptureInfo(cs, &tst, nullptr, &tg, &tdeps, nullptr, &tnd));
        JMD_CUDA_TRY(cudaGraphAddNode(&wn, tg, tdeps, nullptr, tnd, wp));
        JMD_CUDA_TRY(cudaStreamUpdateCaptureDependencies(cs, &wn, nullptr, 1, cudaStreamSetCaptureDependencies));
        enqueue_loop_post(c, cs);
        JMD_CUDA_TRY(cudaStreamEndCapture(cs, &g));
    } else {
        JMD_CUDA_TRY(cudaGraphAddNode(&wn, g, nullptr, nullptr, 0, wp));
    }
    cudaGraph_t body = wp->conditional.phGraph_out[0];

    JMD_CUDA_TRY(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    if (!c.fused) enqueue_kick_drift(c, 1, cs);

    cudaStreamCaptureStatus cst;
    cudaGraph_t cg = nullptr;
    const cudaGraphNode_t *deps = nullptr;
    size_t nd = 0;
    JMD_CUDA_TRY(cudaStreamGetCaptureInfo(cs, &cst, nullptr, &cg, &deps, nullptr, &nd));
    alignas(cudaGraphNodeParams) unsigned char iraw[sizeof(cudaGraphNodeParams)];
    cudaGraphNodeParams *ip = zeroed_params(iraw);
    ip->type = cudaGraphNodeTypeConditional;
    ip->conditional.handle = hi;
    ip->conditional.type = cudaGraphCondTypeIf;
    ip->conditional.size = 1;
    cudaGraphNode_t in;
    JMD_CUDA_TRY(cudaGraphAddNode(&in, cg, deps, nullptr, nd, ip));
    JMD_CUDA_TRY(cudaStreamUpdateCaptureDependencies(cs, &in, nullptr, 1, cudaStreamSetCaptureDependencies));
    cudaGraph_t ibody = ip->conditional.phGraph_out[0];
    JMD_CUDA_TRY(cudaStreamBeginCaptureToGraph(cs2, ibody, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    NbrArgs na = c.na;
    na.gated = 0;
    enqueue_rebuild_chain(na, c.ncell_total, cs2);
    JMD_CUDA_TRY(cudaStreamEndCapture(cs2, &ibody));

    enqueue_forces(c.pa, c.dim, c.pot, c.fused ? 2 : 1, cs);
    if (c.nhc) enqueue_nhc_update(c, cs);
    JMD_CUDA_TRY(cudaStreamEndCapture(cs, &body));
    cudaStreamDestroy(cs2);
    cudaStreamDestroy(cs);

    cudaGraphExec_t ex = nullptr;
    JMD_CUDA_TRY(cudaGraphInstantiate(&ex, g, 0));
    out.key = c0;
    out.graph = g;
    out.exec = ex;
    return MD_OK;
}

static md_status nve_graph_run(const NveCtx &c, int nsteps, uint32_t step0, unsigned long long seed,
                               cudaStream_t st)
{
    int dev = 0;
    JMD_CUDA_TRY(cudaGetDevice(&dev));
    cudaGraphExec_t ex = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_nve_mu);
        for (auto &e : g_nve_graphs)
            if (e.device == dev && memcmp(&e.key, &c, sizeof(NveCtx)) == 0) ex = e.exec;
        if (!ex) {
            NveGraph ng;
            memset(&ng, 0, sizeof(ng));
            md_status s = build_nve_graph(c, ng);
            if (s != MD_OK) return s;
            ng.device = dev;
            g_nve_graphs.push_back(ng);
            ex = ng.exec;
        }
    }
    k_loop_init<<<1, 1, 0, st>>>(c.ctl, (uint32_t)nsteps, step0, seed);
    JMD_CUDA_TRY(cudaGraphLaunch(ex, st));
    JMD_CUDA_TRY(cudaGetLastError());
    return MD_OK;
}

void enqueue_gd_step(const md_space *s, float *d_r, const float *d_f, const md_nbr *nb, float eta, cudaStream_t st)
{
    Box box = make_box(s);
    int g = (nb->N + 255) / 256;
    uint32_t *ctl = ws_ptrs(nb).ctl;
    if (s->dim == 3)
        k_gd_step<3><<<g, 256, 0, st>>>((float4 *)d_r, (const float4 *)d_f, (const float4 *)nb->rref, nb->N, eta, box,
                                        nb->half_skin2, ctl);
    else
        k_gd_step<2><<<g, 256, 0, st>>>((float4 *)d_r, (const float4 *)d_f, (const float4 *)nb->rref, nb->N, eta, box,
                                        nb->half_skin2, ctl);
}

}  // namespace jmd

using namespace jmd;

static int g_fuse_nve = 1;   // md_set_nve_fusion

static md_status run_dynamics(const md_space *s, const md_pot *p, float *d_r, float *d_v, float *d_f, float mass,
                              float dt, int nsteps, md_nbr *nb, double *d_PE, double *d_KE, int use_graph,
                              uint32_t *d_status, cudaStream_t st, int langevin, float gamma, float kT,
                              unsigned long long seed, uint32_t step0, double *d_nhc = nullptr, int nhc_M = 0,
                              double *d_H = nullptr, int nhc_reset = 1)
{
    if (!s || !p || !d_r || !d_v || !d_f || !nb || nsteps < 0 || !(mass > 0.0f)) return MD_ERR_INVALID;
    if (s->dim != nb->dim || !nb->ws || !nb->rref) return MD_ERR_INVALID;
    if (p->kind != MD_LJ && p->kind != MD_SOFT_SPHERE && p->kind != MD_SW && p->kind != MD_BP && p->kind != MD_GNN)
        return MD_ERR_INVALID;
    if (langevin && (s->dim != 3 || !(gamma >= 0.0f) || !(kT >= 0.0f))) return MD_ERR_INVALID;
    // plans with tiles: NVE of pair potentials runs on the tile engine
    if (!langevin && !d_nhc && (nb->flags & MD_NBR_TILES) && tiles_enabled(s, nb, p))
        return run_tiled_nve(s, p, d_r, d_v, d_f, mass, dt, nsteps, nb, d_PE, d_KE, use_graph, d_status, st);
    NveCtx c;
    memset(&c, 0, sizeof(c));   // the graph cache compares contexts bytewise
    c.box = make_box(s);
    c.dim = s->dim;
    c.N = nb->N;
    c.r = (float4 *)d_r;
    c.v = (float4 *)d_v;
    c.f = (float4 *)d_f;
    c.rref = (float4 *)nb->rref;
    c.hdm = 0.5f * dt / mass;
    c.dt = dt;
    c.half_skin2 = nb->half_skin2;
    c.ctl = ws_ptrs(nb).ctl;
    c.na = make_nbr_args(s, d_r, nb, d_status, 1);
    c.na.wrapped = 1;   // the kick-drift kernels keep positions inside the box
    c.ncell_total = nb->ncell_total;
    if (!make_pair_args(s, p, d_r, nb, d_f, c.pa)) return MD_ERR_INVALID;
    c.pa.v = (float4 *)d_v;
    c.pa.half_dt_over_m = c.hdm;
    c.pa.mass = mass;
    c.pa.E_out = d_PE;
    c.pa.KE_out = d_KE;
    c.pa.series = 1;
    c.pa.status = d_status;
    c.pot = p->kind;
    c.langevin = langevin;
    if (d_nhc) {
        c.nhc = 1;
        c.pa.nhc = d_nhc;
        c.pa.nhc_M = nhc_M;
        c.pa.H_out = d_H;
        c.nhc_reset = nhc_reset;
    }
    if (langevin) {
        double e = exp(-(double)gamma * (double)dt);
        c.c1 = (float)e;
        c.c2 = (float)sqrt((1.0 - e * e) * (double)kT / (double)mass);
    }
    // pair potentials in NVE: kick-drift fused into the force kernel,
    // positions alternating with the workspace buffer
    c.fused = (!langevin && !c.nhc && (p->kind == MD_LJ || p->kind == MD_SOFT_SPHERE) && g_fuse_nve) ? 1 : 0;
    if (c.fused) {
        const WsPtrs w = ws_ptrs(nb);
        c.pa.r_alt = w.ralt;
        c.pa.rref = (const float4 *)nb->rref;
        c.pa.dt = dt;
        c.pa.half_skin2 = nb->half_skin2;
        c.na.r_alt = w.ralt;
    }
    if (nsteps == 0) return MD_OK;
    if (use_graph) return nve_graph_run(c, nsteps, step0, seed, st);
    k_loop_init<<<1, 1, 0, st>>>(c.ctl, (uint32_t)nsteps, step0, seed);
    enqueue_loop_pre(c, 0, st);
    for (int k = 0; k < nsteps; ++k) enqueue_nve_step(c, st);
    enqueue_loop_post(c, st);
    JMD_CUDA_TRY(cudaGetLastError());
    return MD_OK;
}

extern "C" md_status md_integrate_nve(const md_space *s, const md_pot *p, float *d_r, float *d_v, float *d_f,
                                      float mass, float dt, int nsteps, md_nbr *nb, double *d_PE, double *d_KE,
                                      int use_graph, uint32_t *d_status, md_stream_t stream)
{
    return run_dynamics(s, p, d_r, d_v, d_f, mass, dt, nsteps, nb, d_PE, d_KE, use_graph, d_status,
                        (cudaStream_t)stream, 0, 0.0f, 0.0f, 0ull, 0u);
}

// Nose-Hoover chain state on the host side: masses and constants; the chain
// positions and velocities are zeroed when reset.
__global__ void k_nhc_setup(double *nhc, int M, double gkT, double kT, double tau, double dt, int reset)
{
    count_launch();
    if (reset)
        for (int k = 0; k < 2 * M; ++k) nhc[k] = 0.0;
    nhc[2 * M] = gkT * tau * tau;
    for (int k = 1; k < M; ++k) nhc[2 * M + k] = kT * tau * tau;
    nhc[3 * M + NHC_GKT] = gkT;
    nhc[3 * M + NHC_KT] = kT;
    nhc[3 * M + NHC_DT] = dt;
}

extern "C" size_t md_nhc_state_doubles(int M) { return (M >= 1 && M <= NHC_MAXM) ? (size_t)nhc_words(M) : 0; }

extern "C" md_status md_integrate_nhc(const md_space *s, const md_pot *p, float *d_r, float *d_v, float *d_f,
                                      float mass, float dt, float kT, float tau, int M, int nsteps, md_nbr *nb,
                                      double *d_therm, int reset, double *d_PE, double *d_KE, double *d_H,
                                      int use_graph, uint32_t *d_status, md_stream_t stream)
{
    if (!d_therm || M < 1 || M > NHC_MAXM || !(kT > 0.0f) || !(tau > 0.0f) || !nb) return MD_ERR_INVALID;
    const double gkT = (double)(s ? s->dim : 0) * (double)nb->N * (double)kT;
    cudaStream_t st = (cudaStream_t)stream;
    k_nhc_setup<<<1, 1, 0, st>>>(d_therm, M, gkT, (double)kT, (double)tau, (double)dt, reset);
    JMD_CUDA_TRY(cudaGetLastError());
    return run_dynamics(s, p, d_r, d_v, d_f, mass, dt, nsteps, nb, d_PE, d_KE, use_graph, d_status, st, 0, 0.0f,
                        0.0f, 0ull, 0u, d_therm, M, d_H, reset ? 1 : 0);
}

extern "C" md_status md_set_nve_fusion(int on)
{
    if (on != 0 && on != 1) return MD_ERR_INVALID;
    g_fuse_nve = on;
    return MD_OK;
}

extern "C" md_status md_integrate_langevin(const md_space *s, const md_pot *p, float *d_r, float *d_v, float *d_f,
                                           float mass, float dt, float gamma, float kT, uint64_t seed,
                                           uint32_t step0, int nsteps, md_nbr *nb, double *d_PE, double *d_KE,
                                           int use_graph, uint32_t *d_status, md_stream_t stream)
{
    return run_dynamics(s, p, d_r, d_v, d_f, mass, dt, nsteps, nb, d_PE, d_KE, use_graph, d_status,
                        (cudaStream_t)stream, 1, gamma, kT, (unsigned long long)seed, step0);
}

extern "C" md_status md_minimize(const md_space *s, const md_pot *p, int kind, float step, int nsteps, float *d_r,
                                 float *d_f, md_nbr *nb, double *d_E, uint32_t *d_status, md_stream_t stream)
{
    if (!s || !p || !d_r || !d_f || !nb || nsteps < 0 || kind != 0) return MD_ERR_INVALID;
    if (s->dim != nb->dim || !nb->ws || !nb->rref) return MD_ERR_INVALID;
    if (p->kind != MD_LJ && p->kind != MD_SOFT_SPHERE) return MD_ERR_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    PairArgs pa;
    if (!make_pair_args(s, p, d_r, nb, d_f, pa)) return MD_ERR_INVALID;
    pa.E_out = d_E;
    pa.series = d_E ? 1 : 0;
    pa.status = d_status;
    NbrArgs na = make_nbr_args(s, d_r, nb, d_status, 1);
    uint32_t *ctl = ws_ptrs(nb).ctl;
    k_loop_init<<<1, 1, 0, st>>>(ctl, (uint32_t)(nsteps + 1), 0u, 0ull);
    if (g_loop_graphs) {
        // the same kernels in the same order as the host loop below, as one
        // graph: WHILE { forces, step (with the displacement check),
        // IF(rebuild) { rebuild chain } }
        struct Key {
            int tag, dim, kind;
            float step;
            md_space space;
            md_nbr nb;
            PairArgs pa;
            NbrArgs na;
            float *r;
            const float *f;
        } key;
        memset(&key, 0, sizeof(key));
        key.tag = 0x47442d31;   // GD-1
        key.dim = s->dim;
        key.kind = p->kind;
        key.step = step;
        key.space = *s;
        key.nb = *nb;
        key.pa = pa;
        key.na = na;
        key.r = d_r;
        key.f = d_f;
        md_status e = run_graph_loop(&key, sizeof(key), ctl, nsteps,
                                     [&](LoopBuilder &lb) {
                                         enqueue_pair(pa, s->dim, p->kind, 0, lb.cs);
                                         enqueue_gd_step(s, d_r, d_f, nb, step, lb.cs);
                                         return lb.rebuild_if(na, nb->ncell_total);
                                     },
                                     st);
        if (e != MD_OK) return e;
    } else {
        for (int t = 0; t < nsteps; ++t) {
            enqueue_pair(pa, s->dim, p->kind, 0, st);
            enqueue_gd_step(s, d_r, d_f, nb, step, st);
            enqueue_rebuild_chain(na, nb->ncell_total, st);
        }
    }
    enqueue_pair(pa, s->dim, p->kind, 0, st);
    JMD_CUDA_TRY(cudaGetLastError());
    return MD_OK;
}
