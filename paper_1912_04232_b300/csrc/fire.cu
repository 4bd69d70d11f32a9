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
                                                    uint32_t *status)
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
    if (!last || threadIdx.x != 0) return;
    __threadfence();
    // the FIRE rules, one thread, partials summed in block order
    double S[3] = {0.0, 0.0, 0.0};
    for (int b = 0; b < (int)gridDim.x; ++b)
        for (int c = 0; c < 3; ++c) S[c] += ((volatile double *)part)[3 * b + c];
    h->ticket = 0u;
    if (!isfinite(S[0]) || !isfinite(S[1]) || !isfinite(S[2])) raise_status(status, MD_ERR_NONFINITE);
    const double alpha = h->alpha;
    h->P = S[0];
    h->vv = S[1];
    h->ff = S[2];
    h->keep = (float)(1.0 - alpha);
    h->scale = S[2] > 0.0 ? (float)(alpha * sqrt(S[1]) / sqrt(S[2])) : 0.0f;
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

extern "C" md_status md_minimize_fire(const md_space *s, const md_pot *p, const md_fire_params *fp, int nsteps,
                                      float *d_r, float *d_v, float *d_f, md_nbr *nb, void *d_state, int restart,
                                      double *d_E, uint32_t *d_status, md_stream_t stream)
{
    if (!s || !p || !fp || !d_r || !d_v || !d_f || !nb || !d_state || nsteps < 0) return MD_ERR_INVALID;
    if ((uintptr_t)d_state & 255u) return MD_ERR_INVALID;
    if (s->dim != nb->dim || !nb->ws || !nb->rref) return MD_ERR_INVALID;
    if (p->kind != MD_LJ && p->kind != MD_SOFT_SPHERE) return MD_ERR_INVALID;
    if (!(fp->dt_start > 0.f) || !(fp->dt_max >= fp->dt_start) || !(fp->f_inc >= 1.f) || !(fp->f_dec > 0.f) ||
        !(fp->f_dec < 1.f) || !(fp->alpha_start >= 0.f) || !(fp->alpha_start < 1.f) || !(fp->f_alpha > 0.f) ||
        !(fp->f_alpha <= 1.f) || fp->n_min < 0)
        return MD_ERR_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    PairArgs pa;
    if (!make_pair_args(s, p, d_r, nb, d_f, pa)) return MD_ERR_INVALID;
    pa.E_out = d_E;
    pa.series = d_E ? 1 : 0;
    pa.status = d_status;
    NbrArgs na = make_nbr_args(s, d_r, nb, d_status, 1);
    WsPtrs w = ws_ptrs(nb);
    FireHdr *h = (FireHdr *)d_state;
    const Box box = make_box(s);
    const int N = nb->N, g = (N + 255) / 256;
    const int gp = g < FIRE_BLOCKS ? g : FIRE_BLOCKS;
    float4 *r = (float4 *)d_r, *v = (float4 *)d_v, *f = (float4 *)d_f;
    enqueue_loop_init(w.ctl, (uint32_t)(nsteps + 1), st);
    if (restart) {
        JMD_CUDA_TRY(cudaMemsetAsync(d_v, 0, sizeof(float4) * (size_t)N, st));
        k_fire_init<<<1, 1, 0, st>>>(h, *fp);
    }
    enqueue_pair(pa, s->dim, p->kind, 0, st);
    const int dim = s->dim, kind = p->kind;
    const float4 *rref = (const float4 *)nb->rref;
    const float hs2 = nb->half_skin2;
    const int ncell = nb->ncell_total;
    const md_fire_params prm = *fp;
    // one step: drift, rebuild (gated, or under an IF node), forces, power, mixing
    auto step = [&](cudaStream_t cs, LoopBuilder *lb) -> md_status {
        if (dim == 3) k_fire_drift<3><<<g, 256, 0, cs>>>(r, v, f, rref, N, h, box, hs2, w.ctl);
        else k_fire_drift<2><<<g, 256, 0, cs>>>(r, v, f, rref, N, h, box, hs2, w.ctl);
        if (lb) {
            md_status e = lb->rebuild_if(na, ncell);
            if (e != MD_OK) return e;
        } else {
            enqueue_rebuild_chain(na, ncell, cs);
        }
        enqueue_pair(pa, dim, kind, 0, cs);
        if (dim == 3) {
            k_fire_power<3><<<gp, 256, 0, cs>>>(v, f, N, h, prm, d_status);
            k_fire_mix<3><<<g, 256, 0, cs>>>(v, f, N, h);
        } else {
            k_fire_power<2><<<gp, 256, 0, cs>>>(v, f, N, h, prm, d_status);
            k_fire_mix<2><<<g, 256, 0, cs>>>(v, f, N, h);
        }
        return MD_OK;
    };
    if (g_loop_graphs) {
        struct Key {
            int tag, dim, kind, N;
            PairArgs pa;
            NbrArgs na;
            const void *r, *v, *f, *h, *rref;
            md_fire_params prm;
            Box box;
            float hs2;
            uint32_t *status;
        } key;
        memset(&key, 0, sizeof(key));
        key.tag = 0x46495245;   // FIRE
        key.dim = dim;
        key.kind = kind;
        key.N = N;
        key.pa = pa;
        key.na = na;
        key.r = r;
        key.v = v;
        key.f = f;
        key.h = h;
        key.rref = rref;
        key.prm = prm;
        key.box = box;
        key.hs2 = hs2;
        key.status = d_status;
        md_status e = run_graph_loop(&key, sizeof(key), w.ctl, nsteps,
                                     [&](LoopBuilder &lb) { return step(lb.cs, &lb); }, st);
        if (e != MD_OK) return e;
    } else {
        for (int t = 0; t < nsteps; ++t) step(st, nullptr);
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
