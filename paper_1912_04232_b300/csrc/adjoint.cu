// adjoint.cu -- differentiating the final energy of a gradient-descent
// minimisation with respect to the small-disk diameter D (Sec. 4.2, App. A).
//
// Bidisperse disks: particles i < nA have diameter D, the rest dB; the box
// edge L(D) keeps the packing fraction fixed (the caller passes L and
// L' = dL/dD).  r_0 = L s_0, r_{t+1} = r_t + eta F(r_t; D), E = U(r_T; D).
// Reverse mode, hand-written:
//   lambda_T = grad U(r_T) = -F(r_T),   g = dU/dD |_{r_T}
//   for t = T-1 .. 0:   g += eta lambda_{t+1} . dF/dD |_{r_t}
//                       lambda_t = lambda_{t+1} - eta H(r_t) lambda_{t+1}
//   g += L' lambda_0 . s_0
// with H the Hessian of U (pair blocks h = u'' e e^T + (u'/r)(I - e e^T))
// and dd_ij/dD = -n_ij L' for the minimum image d_ij = r_i - r_j - n_ij L.
// States are kept only every K steps (K ~ sqrt(T)); each segment is
// recomputed from its checkpoint in the backward sweep.  The neighbor list
// runs in canonical mode (sorted rows, serial pair sums), so forces -- and
// hence the recomputed states -- do not depend on when the list was
// rebuilt: the result is bit-identical for every K.
#include <cmath>

#include "common.cuh"
#include "kernels.cuh"

namespace jmd {

struct AdjArgs {
    Box box;
    int N, cap, nA;
    const float4 *r;
    const int32_t *nbr, *cnt;
    const float4 *lam_in;
    float4 *lam_out;
    const float4 *f;
    const float4 *s0;
    float eta, eps, alpha, Lp;
    double scale;      // factor applied to the block sums before accumulation
    double *target;    // += scale * sum_i value_i (fixed order, last block)
    uint32_t *ctl;
    double2 *partials;
};

// target += scale * sum over blocks (FP64, fixed order, by the last block).
__device__ __forceinline__ void accumulate_f64(double v, const AdjArgs &a)
{
    __shared__ double sh[32];
    __shared__ bool last;
    double b = block_sum_f64(v, sh);
    if (threadIdx.x == 0) {
        a.partials[blockIdx.x] = make_double2(b, 0.0);
        __threadfence();
        unsigned t = atomicAdd(&a.ctl[CTL_TICKET], 1u);
        last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double s = 0.0;
    for (int k = threadIdx.x; k < (int)gridDim.x; k += blockDim.x) s += ((const volatile double *)(a.partials + k))[0];
    s = block_sum_f64(s, sh);
    if (threadIdx.x == 0) {
        a.ctl[CTL_TICKET] = 0u;
        *a.target += a.scale * s;
    }
}

struct SoftTerms {
    float ur, urr, us, urs;
};

// u = (eps/alpha) x^alpha, x = 1 - r/s, and its r / s derivatives.
__device__ __forceinline__ SoftTerms soft_terms(float r, float s, float eps, float alpha)
{
    SoftTerms t;
    float x = 1.0f - r / s;
    float xa1 = alpha == 2.0f ? x : __powf(x, alpha - 1.0f);
    float xa2 = alpha == 2.0f ? 1.0f : __powf(x, alpha - 2.0f);
    float is = 1.0f / s;
    t.ur = -eps * is * xa1;
    t.urr = eps * is * is * (alpha - 1.0f) * xa2;
    t.us = eps * xa1 * r * is * is;
    t.urs = eps * is * is * (xa1 - (alpha - 1.0f) * xa2 * r * is);
    return t;
}

// One backward step at r_t: lambda_out = lambda_in - eta H lambda_in and
// target += eta * sum_i lambda_in_i . dF_i/dD.  Thread per particle, row
// order (canonical list).
__global__ void __launch_bounds__(256) k_adjoint_step(AdjArgs a)
{
    count_launch();
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    float acc = 0.0f;
    if (i < a.N) {
        const float4 ri = a.r[i];
        const float4 li = a.lam_in[i];
        int n = a.cnt[i];
        n = n < a.cap ? n : a.cap;
        const int32_t *row = a.nbr + (size_t)i * a.cap;
        float hx = 0.f, hy = 0.f, gx = 0.f, gy = 0.f;
        for (int k = 0; k < n; ++k) {
            const int j = row[k];
            const float4 rj = a.r[j];
            float dx, dy, dz;
            float r2 = dist2_rn<2>(ri, rj, a.box, dx, dy, dz);
            float sg = 0.5f * (ri.w + rj.w);
            if (!(r2 < sg * sg)) continue;
            float rr = sqrtf(r2);
            float ex = dx / rr, ey = dy / rr;
            SoftTerms t = soft_terms(rr, sg, a.eps, a.alpha);
            float c = t.ur / rr;
            float h00 = t.urr * ex * ex + c * (1.0f - ex * ex);
            float h01 = (t.urr - c) * ex * ey;
            float h11 = t.urr * ey * ey + c * (1.0f - ey * ey);
            const float4 lj = a.lam_in[j];
            float lx = li.x - lj.x, ly = li.y - lj.y;
            hx += h00 * lx + h01 * ly;
            hy += h01 * lx + h11 * ly;
            // image integers of the minimum image
            float nx = rintf(__fmul_rn(__fsub_rn(ri.x, rj.x), a.box.Linv[0]));
            float ny = rintf(__fmul_rn(__fsub_rn(ri.y, rj.y), a.box.Linv[1]));
            float ds = 0.5f * (float)((i < a.nA) + (j < a.nA));
            // dF_i/dD = -[u_rs ds e + h (-n L')]
            float px = -nx * a.Lp, py = -ny * a.Lp;
            gx -= t.urs * ds * ex + h00 * px + h01 * py;
            gy -= t.urs * ds * ey + h01 * px + h11 * py;
        }
        a.lam_out[i] = make_float4(li.x - a.eta * hx, li.y - a.eta * hy, 0.f, 0.f);
        acc = li.x * gx + li.y * gy;
    }
    accumulate_f64((double)acc, a);
}

// lambda_T = -F(r_T) and target += dU/dD |_{r_T} (each pair counted once:
// half of the full-row sum).
__global__ void __launch_bounds__(256) k_adjoint_final(AdjArgs a)
{
    count_launch();
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    float acc = 0.0f;
    if (i < a.N) {
        const float4 ri = a.r[i];
        const float4 fi = a.f[i];
        a.lam_out[i] = make_float4(-fi.x, -fi.y, 0.f, 0.f);
        int n = a.cnt[i];
        n = n < a.cap ? n : a.cap;
        const int32_t *row = a.nbr + (size_t)i * a.cap;
        for (int k = 0; k < n; ++k) {
            const int j = row[k];
            const float4 rj = a.r[j];
            float dx, dy, dz;
            float r2 = dist2_rn<2>(ri, rj, a.box, dx, dy, dz);
            float sg = 0.5f * (ri.w + rj.w);
            if (!(r2 < sg * sg)) continue;
            float rr = sqrtf(r2);
            SoftTerms t = soft_terms(rr, sg, a.eps, a.alpha);
            float nx = rintf(__fmul_rn(__fsub_rn(ri.x, rj.x), a.box.Linv[0]));
            float ny = rintf(__fmul_rn(__fsub_rn(ri.y, rj.y), a.box.Linv[1]));
            float ds = 0.5f * (float)((i < a.nA) + (j < a.nA));
            acc += 0.5f * (t.us * ds + t.ur * (dx * (-nx * a.Lp) + dy * (-ny * a.Lp)) / rr);
        }
    }
    accumulate_f64((double)acc, a);
}

// target += L' sum_i lambda_0_i . s0_i
__global__ void __launch_bounds__(256) k_adjoint_initial(AdjArgs a)
{
    count_launch();
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    float acc = 0.0f;
    if (i < a.N) {
        float4 l = a.lam_in[i], s = a.s0[i];
        acc = a.Lp * (l.x * s.x + l.y * s.y);
    }
    accumulate_f64((double)acc, a);
}

// r_0 = L s_0 with diameters D (i < nA) or dB in the w column.
__global__ void k_adjoint_init_pos(float4 *r, const float4 *s0, int N, int nA, float L, float D, float dB,
                                   double *out)
{
    count_launch();
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) {
        out[0] = 0.0;
        out[1] = 0.0;
    }
    if (i < N) {
        float4 s = s0[i];
        r[i] = make_float4(L * s.x, L * s.y, 0.0f, i < nA ? D : dB);
    }
}

}  // namespace jmd

using namespace jmd;

extern "C" size_t md_adjoint_workspace_size(int N, int T, int K)
{
    if (N < 1 || T < 1 || K < 1) return 0;
    size_t nseg = (size_t)((T + K - 1) / K);
    return (nseg + (size_t)K + 2) * (size_t)N * sizeof(float4);
}

extern "C" md_status md_minimize_adjoint(const md_space *s, const md_pot *p, md_nbr *nb, const float *d_s0, int nA,
                                         float D, float dB, float Lp, float eta, int T, int K, float *d_r, float *d_f,
                                         void *d_ws, double *d_out, uint32_t *d_status, md_stream_t stream)
{
    if (!s || !p || !nb || !d_s0 || !d_r || !d_f || !d_ws || !d_out) return MD_ERR_INVALID;
    if (s->dim != 2 || nb->dim != 2 || p->kind != MD_SOFT_SPHERE || T < 1 || K < 1 || K > T) return MD_ERR_INVALID;
    if (!(nb->flags & MD_NBR_CANONICAL) || !nb->ws || !nb->rref || nA < 0 || nA > nb->N) return MD_ERR_INVALID;
    const float smax = D > dB ? D : dB;
    if (nb->r_cut < smax) return MD_ERR_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    const int N = nb->N;
    const size_t sN = (size_t)N;
    float4 *ws = (float4 *)d_ws;
    const int nseg = (T + K - 1) / K;
    float4 *ckpt = ws;                       // [nseg][N]
    float4 *seg = ws + (size_t)nseg * sN;    // [K][N]
    float4 *lamA = seg + (size_t)K * sN;     // [N]
    float4 *lamB = lamA + sN;                // [N]
    float4 *r = (float4 *)d_r;
    const int g = (N + 255) / 256;

    PairArgs pa;
    if (!make_pair_args(s, p, d_r, nb, d_f, pa)) return MD_ERR_INVALID;
    pa.status = d_status;
    NbrArgs na = make_nbr_args(s, d_r, nb, d_status, 1);
    WsPtrs w = ws_ptrs(nb);

    AdjArgs aa;
    memset(&aa, 0, sizeof(aa));
    aa.box = make_box(s);
    aa.N = N;
    aa.cap = nb->cap;
    aa.nA = nA;
    aa.r = r;
    aa.nbr = nb->nbr;
    aa.cnt = nb->cnt;
    aa.f = (const float4 *)d_f;
    aa.s0 = (const float4 *)d_s0;
    aa.eta = eta;
    aa.eps = p->eps;
    aa.alpha = p->alpha;
    aa.Lp = Lp;
    aa.target = d_out + 1;
    aa.ctl = w.ctl;
    aa.partials = w.partials;
    if (g > w.max_blocks) return MD_ERR_INVALID;

    // forward: r_0 = L s_0, T gradient-descent steps, checkpoints every K
    k_adjoint_init_pos<<<g, 256, 0, st>>>(r, (const float4 *)d_s0, N, nA, s->L[0], D, dB, d_out);
    md_status stt = md_neighbor_list_build(s, d_r, nb, d_status, stream);
    if (stt != MD_OK) return stt;
    for (int t = 0; t < T; ++t) {
        if (t % K == 0)
            JMD_CUDA_TRY(cudaMemcpyAsync(ckpt + (size_t)(t / K) * sN, r, sN * sizeof(float4),
                                         cudaMemcpyDeviceToDevice, st));
        enqueue_pair(pa, 2, MD_SOFT_SPHERE, 0, st);
        enqueue_gd_step(s, d_r, d_f, nb, eta, st);
        enqueue_rebuild_chain(na, nb->ncell_total, st);
    }
    // E_final and F(r_T), then lambda_T and dU/dD at r_T
    PairArgs pe = pa;
    pe.E_out = d_out;
    enqueue_pair(pe, 2, MD_SOFT_SPHERE, 0, st);
    aa.lam_out = lamA;
    aa.scale = 1.0;
    k_adjoint_final<<<g, 256, 0, st>>>(aa);

    // backward sweep, segment by segment
    float4 *lin = lamA, *lout = lamB;
    aa.scale = (double)eta;
    for (int k = nseg - 1; k >= 0; --k) {
        const int t0 = k * K, t1 = (t0 + K < T) ? t0 + K : T;
        JMD_CUDA_TRY(cudaMemcpyAsync(r, ckpt + (size_t)k * sN, sN * sizeof(float4), cudaMemcpyDeviceToDevice, st));
        stt = md_neighbor_list_build(s, d_r, nb, d_status, stream);
        if (stt != MD_OK) return stt;
        for (int t = t0; t < t1; ++t) {
            JMD_CUDA_TRY(cudaMemcpyAsync(seg + (size_t)(t - t0) * sN, r, sN * sizeof(float4),
                                         cudaMemcpyDeviceToDevice, st));
            if (t + 1 < t1) {   // the last state of the segment needs no step
                enqueue_pair(pa, 2, MD_SOFT_SPHERE, 0, st);
                enqueue_gd_step(s, d_r, d_f, nb, eta, st);
                enqueue_rebuild_chain(na, nb->ncell_total, st);
            }
        }
        for (int t = t1 - 1; t >= t0; --t) {
            float *rt = (float *)(seg + (size_t)(t - t0) * sN);
            stt = md_neighbor_list_build(s, rt, nb, d_status, stream);
            if (stt != MD_OK) return stt;
            aa.r = (const float4 *)rt;
            aa.lam_in = lin;
            aa.lam_out = lout;
            k_adjoint_step<<<g, 256, 0, st>>>(aa);
            float4 *tmp = lin;
            lin = lout;
            lout = tmp;
        }
    }
    aa.lam_in = lin;
    aa.scale = 1.0;
    k_adjoint_initial<<<g, 256, 0, st>>>(aa);
    JMD_CUDA_TRY(cudaGetLastError());
    return MD_OK;
}
