// fire.cu -- FIRE minimisation (Sec. 3.3.1; Bitzek, Koskinen, Gahler,
// Moseler, Gumbsch, PRL 97, 170201 (2006)), unit mass, unwrapped
// coordinates as in gradient descent.
//
// One step, in the order of the published algorithm:
//   k_fire_drift   v += dt/2 F;  r += dt v;  displacement check
//   rebuild chain  (only when some particle moved > skin/2)
//   k_pair         F(r), U(r)
//   k_fire_power   v += dt/2 F; FP64 sums P = F.v, |v|^2, |F|^2; the last
//                  block applies the FIRE rules to (dt, alpha, npos) and
//                  leaves the mixing coefficients for
//   k_fire_mix     v = (1 - alpha) v + alpha |v| F/|F|, or v = 0 when P <= 0
// The scalar state lives in a small caller-owned device buffer, so a
// minimisation can be continued across calls.
#include "common.cuh"
#include "kernels.cuh"

namespace jmd {

struct FireHdr {
    double dt, alpha;          // current time step and mixing factor
    double P, vv, ff;          // sums of the last step (FP64)
    float keep, scale;         // mixing of the last step: v = keep v + scale F
    int npos, freeze;          // consecutive P > 0 steps; 1: the last step froze v
    unsigned ticket;
    int pad;
};
constexpr int FIRE_BLOCKS = 296;   // power-kernel grid (2 per SM), grid-stride

__host__ __device__ inline size_t fire_state_bytes() { return 256 + sizeof(double) * 3 * FIRE_BLOCKS; }

__global__ void k_fire_init(FireHdr *h, md_fire_params fp)
{
    count_launch();
    h->dt = fp.dt_start;
    h->alpha = fp.alpha_start;
    h->P = h->vv = h->ff = 0.0;
    h->keep = 1.0f;
    h->scale = 0.0f;
    h->npos = 0;
    h->freeze = 0;
    h->ticket = 0u;
}

template <int DIM>
__global__ void __launch_bounds__(256) k_fire_drift(float4 *r, float4 *v, const float4 *f, const float4 *rref, int N,
                                                    const FireHdr *h, Box box, float half_skin2, uint32_t *ctl)
{
    count_launch();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    bool mv = false;
    if (i < N) {
        const float dt = (float)h->dt, hdt = 0.5f * dt;
        float4 fi = f[i], vi = v[i], ri = r[i];
        vi.x += hdt * fi.x;
        vi.y += hdt * fi.y;
        ri.x += dt * vi.x;
        ri.y += dt * vi.y;
        if (DIM == 3) {
            vi.z += hdt * fi.z;
            ri.z += dt * vi.z;
        }
        v[i] = vi;
        r[i] = ri;
        float dx, dy, dz;
        mv = dist2_rn<DIM>(ri, rref[i], box, dx, dy, dz) > half_skin2;
    }
    if (__any_sync(0xffffffffu, mv) && (threadIdx.x & 31) == 0) ctl[CTL_REBUILD] = 1u;
}

template <int DIM>
__global__ void __launch_bounds__(256) k_fire_power(float4 *v, const float4 *f, int N, FireHdr *h, md_fire_params fp,
                                                    uint32_t *status, FireStep *rec)
{
    count_launch();
    __shared__ double sh[3][8];
    __shared__ bool last;
    double *part = reinterpret_cast<double *>(reinterpret_cast<char *>(h) + 256);
    const float hdt = 0.5f * (float)h->dt;
    float P = 0.f, vv = 0.f, ff = 0.f;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        const float4 fi = f[i];
        float4 vi = v[i];
        vi.x += hdt * fi.x;
        vi.y += hdt * fi.y;
        if (DIM == 3) vi.z += hdt * fi.z;
        v[i] = vi;
        P += fi.x * vi.x + fi.y * vi.y + (DIM == 3 ? fi.z * vi.z : 0.f);
        vv += vi.x * vi.x + vi.y * vi.y + (DIM == 3 ? vi.z * vi.z : 0.f);
        ff += fi.x * fi.x + fi.y * fi.y + (DIM == 3 ? fi.z * fi.z : 0.f);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        P += __shfl_xor_sync(0xffffffffu, P, o);
        vv += __shfl_xor_sync(0xffffffffu, vv, o);
        ff += __shfl_xor_sync(0xffffffffu, ff, o);
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        sh[0][w] = P;
        sh[1][w] = vv;
        sh[2][w] = ff;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s[3] = {0.0, 0.0, 0.0};
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k)
            for (int c = 0; c < 3; ++c) s[c] += sh[c][k];
        for (int c = 0; c < 3; ++c) part[3 * blockIdx.x + c] = s[c];
        __threadfence();
        last = atomicAdd(&h->ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    // partials summed by the whole last block (fixed order), then the FIRE
    // rules in one thread
    double S[3] = {0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
        for (int c = 0; c < 3; ++c) S[c] += ((volatile double *)part)[3 * b + c];
    block_sums_f64<3>(S, &sh[0][0], 8);
    if (threadIdx.x != 0) return;
    h->ticket = 0u;
    if (!isfinite(S[0]) || !isfinite(S[1]) || !isfinite(S[2])) raise_status(status, MD_ERR_NONFINITE);
    const double alpha = h->alpha;
    h->P = S[0];
    h->vv = S[1];
    h->ff = S[2];
    h->keep = (float)(1.0 - alpha);
    h->scale = S[2] > 0.0 ? (float)(alpha * sqrt(S[1]) / sqrt(S[2])) : 0.0f;
    if (rec) {   // what this step used: its time step, mixing and decision
        rec->dt = (float)h->dt;
        rec->alpha = (float)alpha;
        rec->keep = h->keep;
        rec->freeze = S[0] > 0.0 ? 0 : 1;
    }
    if (S[0] > 0.0) {
        h->freeze = 0;
        h->npos += 1;
        if (h->npos > fp.n_min) {
            h->dt = fmin(h->dt * (double)fp.f_inc, (double)fp.dt_max);
            h->alpha = alpha * (double)fp.f_alpha;
        }
    } else {
        h->freeze = 1;
        h->dt *= (double)fp.f_dec;
        h->alpha = (double)fp.alpha_start;
        h->npos = 0;
    }
}

template <int DIM>
__global__ void __launch_bounds__(256) k_fire_mix(float4 *v, const float4 *f, int N, const FireHdr *h)
{
    count_launch();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const float4 fi = f[i];
    float4 vi = v[i];
    if (h->freeze) {
        vi.x = vi.y = vi.z = 0.f;
    } else {
        const float keep = h->keep, scale = h->scale;
        vi.x = keep * vi.x + scale * fi.x;
        vi.y = keep * vi.y + scale * fi.y;
        if (DIM == 3) vi.z = keep * vi.z + scale * fi.z;
    }
    v[i] = vi;
}

}  // namespace jmd

using namespace jmd;

extern "C" size_t md_fire_state_bytes(void) { return fire_state_bytes(); }

namespace jmd {

md_status fire_params_ok(const md_fire_params *fp)
{
    if (!(fp->dt_start > 0.f) || !(fp->dt_max >= fp->dt_start) || !(fp->f_inc >= 1.f) || !(fp->f_dec > 0.f) ||
        !(fp->f_dec < 1.f) || !(fp->alpha_start >= 0.f) || !(fp->alpha_start < 1.f) || !(fp->f_alpha > 0.f) ||
        !(fp->f_alpha <= 1.f) || fp->n_min < 0)
        return MD_ERR_INVALID;
    return MD_OK;
}

void enqueue_fire_init(void *state, const md_fire_params &fp, cudaStream_t st)
{
    k_fire_init<<<1, 1, 0, st>>>((FireHdr *)state, fp);
}

// One FIRE step: drift, rebuild (gated, or under an IF node), forces,
// power and rules (recorded into rec when given), mixing.
md_status enqueue_fire_step(const FireCtx &c, FireStep *rec, cudaStream_t cs, LoopBuilder *lb)
{
    FireHdr *h = (FireHdr *)c.state;
    const int g = (c.N + 255) / 256, gp = g < FIRE_BLOCKS ? g : FIRE_BLOCKS;
    if (c.dim == 3) k_fire_drift<3><<<g, 256, 0, cs>>>(c.r, c.v, c.f, c.rref, c.N, h, c.box, c.hs2, c.ctl);
    else k_fire_drift<2><<<g, 256, 0, cs>>>(c.r, c.v, c.f, c.rref, c.N, h, c.box, c.hs2, c.ctl);
    if (lb) {
        md_status e = lb->rebuild_if(c.na, c.ncell);
        if (e != MD_OK) return e;
    } else {
        enqueue_rebuild_chain(c.na, c.ncell, cs);
    }
    enqueue_pair(c.pa, c.dim, c.kind, 0, cs);
    if (c.dim == 3) {
        k_fire_power<3><<<gp, 256, 0, cs>>>(c.v, c.f, c.N, h, c.prm, c.status, rec);
        k_fire_mix<3><<<g, 256, 0, cs>>>(c.v, c.f, c.N, h);
    } else {
        k_fire_power<2><<<gp, 256, 0, cs>>>(c.v, c.f, c.N, h, c.prm, c.status, rec);
        k_fire_mix<2><<<g, 256, 0, cs>>>(c.v, c.f, c.N, h);
    }
    return MD_OK;
}

bool make_fire_ctx(const md_space *s, const md_pot *p, const md_fire_params *fp, float *d_r, float *d_v, float *d_f,
                   md_nbr *nb, void *d_state, uint32_t *d_status, FireCtx &c)
{
    if (!make_pair_args(s, p, d_r, nb, d_f, c.pa)) return false;
    c.pa.status = d_status;
    c.na = make_nbr_args(s, d_r, nb, d_status, 1);
    WsPtrs w = ws_ptrs(nb);
    c.ctl = w.ctl;
    c.state = d_state;
    c.box = make_box(s);
    c.N = nb->N;
    c.dim = s->dim;
    c.kind = p->kind;
    c.r = (float4 *)d_r;
    c.v = (float4 *)d_v;
    c.f = (float4 *)d_f;
    c.rref = (const float4 *)nb->rref;
    c.hs2 = nb->half_skin2;
    c.ncell = nb->ncell_total;
    c.prm = *fp;
    c.status = d_status;
    return true;
}

}  // namespace jmd

extern "C" md_status md_minimize_fire(const md_space *s, const md_pot *p, const md_fire_params *fp, int nsteps,
                                      float *d_r, float *d_v, float *d_f, md_nbr *nb, void *d_state, int restart,
                                      double *d_E, uint32_t *d_status, md_stream_t stream)
{
    if (!s || !p || !fp || !d_r || !d_v || !d_f || !nb || !d_state || nsteps < 0) return MD_ERR_INVALID;
    if ((uintptr_t)d_state & 255u) return MD_ERR_INVALID;
    if (s->dim != nb->dim || !nb->ws || !nb->rref) return MD_ERR_INVALID;
    if (p->kind != MD_LJ && p->kind != MD_SOFT_SPHERE) return MD_ERR_INVALID;
    if (fire_params_ok(fp) != MD_OK) return MD_ERR_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    FireCtx c;
    if (!make_fire_ctx(s, p, fp, d_r, d_v, d_f, nb, d_state, d_status, c)) return MD_ERR_INVALID;
    c.pa.E_out = d_E;
    c.pa.series = d_E ? 1 : 0;
    const int N = c.N;
    enqueue_loop_init(c.ctl, (uint32_t)(nsteps + 1), st);
    if (restart) {
        JMD_CUDA_TRY(cudaMemsetAsync(d_v, 0, sizeof(float4) * (size_t)N, st));
        enqueue_fire_init(d_state, *fp, st);
    }
    enqueue_pair(c.pa, c.dim, c.kind, 0, st);
    if (g_loop_graphs) {
        struct Key {
            int tag;
            FireCtx c;
        } key;
        memset(&key, 0, sizeof(key));
        key.tag = 0x46495245;   // FIRE
        key.c = c;
        md_status e = run_graph_loop(&key, sizeof(key), c.ctl, nsteps,
                                     [&](LoopBuilder &lb) { return enqueue_fire_step(c, nullptr, lb.cs, &lb); }, st);
        if (e != MD_OK) return e;
    } else {
        for (int t = 0; t < nsteps; ++t) enqueue_fire_step(c, nullptr, st, nullptr);
    }
    JMD_CUDA_TRY(cudaGetLastError());
    return MD_OK;
}

extern "C" md_status md_fire_state_read(const void *d_state, double *out3, md_stream_t stream)
{
    if (!d_state || !out3) return MD_ERR_INVALID;
    FireHdr hh;
    cudaStream_t st = (cudaStream_t)stream;
    JMD_CUDA_TRY(cudaMemcpyAsync(&hh, d_state, sizeof(hh), cudaMemcpyDeviceToHost, st));
    JMD_CUDA_TRY(cudaStreamSynchronize(st));
    out3[0] = hh.dt;
    out3[1] = hh.alpha;
    out3[2] = (double)hh.npos;
    return MD_OK;
}
