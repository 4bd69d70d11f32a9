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

// Row i of the Hessian applied to w, (H w)_i, and dF_i/dD, at positions
// a.r (canonical row order, so the sums have a fixed order).
__device__ __forceinline__ void hess_row(const AdjArgs &a, int i, const float4 *w, float &hx, float &hy, float &gx,
                                         float &gy)
{
    const float4 ri = a.r[i];
    const float4 wi = w[i];
    int n = a.cnt[i];
    n = n < a.cap ? n : a.cap;
    const int32_t *row = a.nbr + (size_t)i * a.cap;
    hx = hy = gx = gy = 0.f;
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
        const float4 wj = w[j];
        float lx = wi.x - wj.x, ly = wi.y - wj.y;
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
        const float4 li = a.lam_in[i];
        float hx, hy, gx, gy;
        hess_row(a, i, a.lam_in, hx, hy, gx, gy);
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

// ---------------------------------------------------------------------------
// FIRE (Sec. 3.3.1; Bitzek et al. 2006) through the packing, reverse mode.
// Step q, with its time step, mixing factor alpha and decision held fixed
// (h = dt/2, keep = 1 - alpha):
//   v_a = v_q + h F(r_q);  r_{q+1} = r_q + dt v_a;  F' = F(r_{q+1});
//   v_b = v_a + h F';  v_{q+1} = keep v_b + alpha |v_b| F'/|F'|  (P > 0),  0  (P <= 0)
// Given the adjoints (lr', lv') of (r_{q+1}, v_{q+1}), with n_v = |v_b|,
// n_f = |F'|, c = F'.lv':
//   g_vb = keep lv' + alpha c v_b / (n_v n_f)
//   g_F' = (alpha n_v / n_f) lv' - alpha n_v c F' / n_f^3 + h g_vb
//   g_r' = lr' - H(r_{q+1}) g_F',       dE/dD += g_F' . dF/dD |_{r_{q+1}}
//   lv_q = g_va = g_vb + dt g_r',       lr_q = g_r' - h H(r_q) g_va
// The two products with H(r_q) (this step's h g_va and step q-1's g_F')
// are taken together: each state gets one Hessian product with the
// direction w = (pending h g_va) + g_F'.
// ---------------------------------------------------------------------------
struct FaArgs {
    AdjArgs a;                    // a.r: positions of state q+1 (list built there)
    const float4 *vq, *fq, *fn;   // v_q, F(r_q), F(r_{q+1})
    const FireStep *rec;          // step q
    float4 *lam_v, *lam_rp, *w_pend, *gvb, *wtot;
    double *scal;                 // |v_b|^2, |F'|^2, F'.lv'
    int final_state;              // 1: state 0, direction w_pend, no step
};

__device__ __forceinline__ float4 fa_vb(const FaArgs &f, int i, float hdt)
{
    const float4 fq = f.fq[i], fn = f.fn[i];
    float4 v = f.vq[i];
    v.x += hdt * fq.x;
    v.y += hdt * fq.y;
    v.x += hdt * fn.x;
    v.y += hdt * fn.y;
    return v;
}

__global__ void __launch_bounds__(256) k_fa_sums(FaArgs f)
{
    count_launch();
    __shared__ double sh[3][8];
    __shared__ bool last;
    const float hdt = 0.5f * f.rec->dt;
    float vv = 0.f, ff = 0.f, fl = 0.f;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < f.a.N) {
        const float4 vb = fa_vb(f, i, hdt), fn = f.fn[i], lv = f.lam_v[i];
        vv = vb.x * vb.x + vb.y * vb.y;
        ff = fn.x * fn.x + fn.y * fn.y;
        fl = fn.x * lv.x + fn.y * lv.y;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        vv += __shfl_xor_sync(0xffffffffu, vv, o);
        ff += __shfl_xor_sync(0xffffffffu, ff, o);
        fl += __shfl_xor_sync(0xffffffffu, fl, o);
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        sh[0][w] = vv;
        sh[1][w] = ff;
        sh[2][w] = fl;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s0 = 0.0, s1 = 0.0, s2 = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
            s0 += sh[0][k];
            s1 += sh[1][k];
            s2 += sh[2][k];
        }
        f.a.partials[2 * blockIdx.x] = make_double2(s0, s1);
        f.a.partials[2 * blockIdx.x + 1] = make_double2(s2, 0.0);
        __threadfence();
        last = atomicAdd(&f.a.ctl[CTL_TICKET], 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double S[3] = {0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
        const volatile double *p = (const volatile double *)(f.a.partials + 2 * b);
        S[0] += p[0];
        S[1] += p[1];
        S[2] += p[2];
    }
    __shared__ double shs[3][8];
    block_sums_f64<3>(S, &shs[0][0], 8);
    const double S0 = S[0], S1 = S[1], S2 = S[2];
    if (threadIdx.x != 0) return;
    f.a.ctl[CTL_TICKET] = 0u;
    f.scal[0] = S0;
    f.scal[1] = S1;
    f.scal[2] = S2;
}

__global__ void __launch_bounds__(256) k_fa_dir(FaArgs f)
{
    count_launch();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= f.a.N) return;
    const FireStep rs = *f.rec;
    const float hdt = 0.5f * rs.dt;
    float4 g = make_float4(0.f, 0.f, 0.f, 0.f), gF = g;
    if (!rs.freeze) {
        const double nv = sqrt(f.scal[0]), nf = sqrt(f.scal[1]), c = f.scal[2];
        const float4 vb = fa_vb(f, i, hdt), fn = f.fn[i], lv = f.lam_v[i];
        const float a1 = (nv > 0.0 && nf > 0.0) ? (float)(rs.alpha * c / (nv * nf)) : 0.0f;
        g.x = rs.keep * lv.x + a1 * vb.x;
        g.y = rs.keep * lv.y + a1 * vb.y;
        if (nf > 0.0) {
            const float b1 = (float)(rs.alpha * nv / nf), b2 = (float)(rs.alpha * nv * c / (nf * nf * nf));
            gF.x = b1 * lv.x - b2 * fn.x;
            gF.y = b1 * lv.y - b2 * fn.y;
        }
        gF.x += hdt * g.x;
        gF.y += hdt * g.y;
    }
    f.gvb[i] = g;
    const float4 wp = f.w_pend[i];
    f.wtot[i] = make_float4(wp.x + gF.x, wp.y + gF.y, 0.f, 0.f);
}

__global__ void __launch_bounds__(256) k_fa_hvp(FaArgs f)
{
    count_launch();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const float4 *w = f.final_state ? f.w_pend : f.wtot;
    float acc = 0.0f;
    if (i < f.a.N) {
        float hx, hy, gx, gy;
        hess_row(f.a, i, w, hx, hy, gx, gy);
        const float4 wi = w[i], lr = f.lam_rp[i];
        const float ox = lr.x - hx, oy = lr.y - hy;
        acc = wi.x * gx + wi.y * gy;
        f.lam_rp[i] = make_float4(ox, oy, 0.f, 0.f);
        if (!f.final_state) {
            const FireStep rs = *f.rec;
            const float4 gb = f.gvb[i];
            const float vx = gb.x + rs.dt * ox, vy = gb.y + rs.dt * oy;
            f.lam_v[i] = make_float4(vx, vy, 0.f, 0.f);
            f.w_pend[i] = make_float4(0.5f * rs.dt * vx, 0.5f * rs.dt * vy, 0.f, 0.f);
        }
    }
    accumulate_f64((double)acc, f.a);
}

}  // namespace jmd

using namespace jmd;

extern "C" size_t md_adjoint_workspace_size(int N, int T, int K)
{
    if (N < 1 || T < 1 || K < 1) return 0;
    size_t nseg = (size_t)((T + K - 1) / K);
    return (nseg + (size_t)K + 2) * (size_t)N * sizeof(float4);
}

// The list for positions x at a point of the reverse sweep.  Host launches
// rebuild it; inside a captured graph the displacement check decides, under a
// conditional node.  The list is canonical, so a particle's force and Hessian
// products are functions of the positions alone and both give the same bits.
static md_status list_for(const md_space *s, const float *x, md_nbr *nb, uint32_t *d_status, cudaStream_t st,
                          LoopBuilder *lb)
{
    if (!lb) return md_neighbor_list_build(s, x, nb, d_status, (md_stream_t)st);
    enqueue_check_disp(s, x, nb, st);
    return lb->rebuild_if(make_nbr_args(s, x, nb, d_status, 1), nb->ncell_total);
}

static md_status gd_adjoint_body(const md_space *s, const md_pot *p, md_nbr *nb, const float *d_s0, int nA, float D,
                                 float dB, float Lp, float eta, int T, int K, float *d_r, float *d_f, void *d_ws,
                                 double *d_out, uint32_t *d_status, cudaStream_t st, LoopBuilder *lb)
{
    if (!s || !p || !nb || !d_s0 || !d_r || !d_f || !d_ws || !d_out) return MD_ERR_INVALID;
    if (s->dim != 2 || nb->dim != 2 || p->kind != MD_SOFT_SPHERE || T < 1 || K < 1 || K > T) return MD_ERR_INVALID;
    if (!(nb->flags & MD_NBR_CANONICAL) || !nb->ws || !nb->rref || nA < 0 || nA > nb->N) return MD_ERR_INVALID;
    const float smax = D > dB ? D : dB;
    if (nb->r_cut < smax) return MD_ERR_INVALID;
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
    md_status stt = md_neighbor_list_build(s, d_r, nb, d_status, (md_stream_t)st);
    if (stt != MD_OK) return stt;
    for (int t = 0; t < T; ++t) {
        if (t % K == 0)
            JMD_CUDA_TRY(cudaMemcpyAsync(ckpt + (size_t)(t / K) * sN, r, sN * sizeof(float4),
                                         cudaMemcpyDeviceToDevice, st));
        enqueue_pair(pa, 2, MD_SOFT_SPHERE, 0, st);
        enqueue_gd_step(s, d_r, d_f, nb, eta, st);
        if (lb) {
            stt = lb->rebuild_if(na, nb->ncell_total);
            if (stt != MD_OK) return stt;
        } else {
            enqueue_rebuild_chain(na, nb->ncell_total, st);
        }
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
        stt = md_neighbor_list_build(s, d_r, nb, d_status, (md_stream_t)st);
        if (stt != MD_OK) return stt;
        for (int t = t0; t < t1; ++t) {
            JMD_CUDA_TRY(cudaMemcpyAsync(seg + (size_t)(t - t0) * sN, r, sN * sizeof(float4),
                                         cudaMemcpyDeviceToDevice, st));
            if (t + 1 < t1) {   // the last state of the segment needs no step
                enqueue_pair(pa, 2, MD_SOFT_SPHERE, 0, st);
                enqueue_gd_step(s, d_r, d_f, nb, eta, st);
                if (lb) {
                    stt = lb->rebuild_if(na, nb->ncell_total);
                    if (stt != MD_OK) return stt;
                } else {
                    enqueue_rebuild_chain(na, nb->ncell_total, st);
                }
            }
        }
        for (int t = t1 - 1; t >= t0; --t) {
            float *rt = (float *)(seg + (size_t)(t - t0) * sN);
            stt = list_for(s, rt, nb, d_status, st, lb);
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

namespace {
struct FaWs {
    size_t state, ckpt_rv, ckpt_h, seg, adj, fin, hist, scal, total;
};
FaWs fa_ws(int N, int T, int K)
{
    FaWs w;
    const size_t sN = (size_t)N, nseg = (size_t)((T + K - 1) / K), f4 = sizeof(float4);
    size_t o = 0;
    w.state = o;   o = align256(o + md_fire_state_bytes());
    w.ckpt_rv = o; o = align256(o + nseg * 2 * sN * f4);
    w.ckpt_h = o;  o = align256(o + nseg * 256);
    w.seg = o;     o = align256(o + 3 * (size_t)(K + 1) * sN * f4);
    w.adj = o;     o = align256(o + 5 * sN * f4);
    w.fin = o;     o = align256(o + 3 * sN * f4);
    w.hist = o;    o = align256(o + (size_t)T * sizeof(FireStep));
    w.scal = o;    o = align256(o + 4 * sizeof(double));
    w.total = o;
    return w;
}
}  // namespace

extern "C" size_t md_fire_adjoint_workspace_size(int N, int T, int K)
{
    if (N < 1 || T < 1 || K < 1 || K > T) return 0;
    return fa_ws(N, T, K).total;
}

static md_status fire_adjoint_body(const md_space *s, const md_pot *p, const md_fire_params *fp, md_nbr *nb,
                                   const float *d_s0, int nA, float D, float dB, float Lp, int T, int K, float *d_r,
                                   float *d_v, float *d_f, void *d_ws, double *d_out, uint32_t *d_status,
                                   cudaStream_t st, LoopBuilder *lb)
{
    if (!s || !p || !fp || !nb || !d_s0 || !d_r || !d_v || !d_f || !d_ws || !d_out) return MD_ERR_INVALID;
    if (s->dim != 2 || nb->dim != 2 || p->kind != MD_SOFT_SPHERE || T < 1 || K < 1 || K > T) return MD_ERR_INVALID;
    if (!(nb->flags & MD_NBR_CANONICAL) || !nb->ws || !nb->rref || nA < 0 || nA > nb->N) return MD_ERR_INVALID;
    if ((uintptr_t)d_ws & 255u) return MD_ERR_INVALID;
    if (fire_params_ok(fp) != MD_OK) return MD_ERR_INVALID;
    const float smax = D > dB ? D : dB;
    if (nb->r_cut < smax) return MD_ERR_INVALID;
    const int N = nb->N;
    const size_t sN = (size_t)N, f4 = sizeof(float4);
    const FaWs L = fa_ws(N, T, K);
    unsigned char *b = (unsigned char *)d_ws;
    void *state = b + L.state;
    float4 *ckrv = (float4 *)(b + L.ckpt_rv);
    unsigned char *ckh = b + L.ckpt_h;
    float4 *seg = (float4 *)(b + L.seg);          // [K+1][3][N]: r, v, F
    float4 *adj = (float4 *)(b + L.adj);
    float4 *fin = (float4 *)(b + L.fin);           // r_T, v_T, F(r_T)
    FireStep *hist = (FireStep *)(b + L.hist);
    double *scal = (double *)(b + L.scal);
    const int g = (N + 255) / 256;
    WsPtrs w = ws_ptrs(nb);
    if (2 * g > w.max_blocks) return MD_ERR_INVALID;

    FireCtx c;
    if (!make_fire_ctx(s, p, fp, d_r, d_v, d_f, nb, state, d_status, c)) return MD_ERR_INVALID;
    float4 *r = (float4 *)d_r, *v = (float4 *)d_v, *fr = (float4 *)d_f;
    auto seg_at = [&](int k, int which) { return seg + ((size_t)k * 3 + which) * sN; };

    AdjArgs aa;
    memset(&aa, 0, sizeof(aa));
    aa.box = make_box(s);
    aa.N = N;
    aa.cap = nb->cap;
    aa.nA = nA;
    aa.nbr = nb->nbr;
    aa.cnt = nb->cnt;
    aa.s0 = (const float4 *)d_s0;
    aa.eps = p->eps;
    aa.alpha = p->alpha;
    aa.Lp = Lp;
    aa.target = d_out + 1;
    aa.ctl = w.ctl;
    aa.partials = w.partials;
    aa.scale = 1.0;

    // forward: r_0 = L s_0 from rest, T FIRE steps (each step's rules
    // recorded), checkpoints of (r, v, FIRE state) every K steps
    k_adjoint_init_pos<<<g, 256, 0, st>>>(r, (const float4 *)d_s0, N, nA, s->L[0], D, dB, d_out);
    JMD_CUDA_TRY(cudaMemsetAsync(d_v, 0, sN * f4, st));
    enqueue_fire_init(state, *fp, st);
    md_status stt = md_neighbor_list_build(s, d_r, nb, d_status, (md_stream_t)st);
    if (stt != MD_OK) return stt;
    enqueue_pair(c.pa, 2, MD_SOFT_SPHERE, 0, st);
    for (int t = 0; t < T; ++t) {
        if (t % K == 0) {
            const size_t k = (size_t)(t / K);
            JMD_CUDA_TRY(cudaMemcpyAsync(ckrv + 2 * k * sN, r, sN * f4, cudaMemcpyDeviceToDevice, st));
            JMD_CUDA_TRY(cudaMemcpyAsync(ckrv + (2 * k + 1) * sN, v, sN * f4, cudaMemcpyDeviceToDevice, st));
            JMD_CUDA_TRY(cudaMemcpyAsync(ckh + 256 * k, state, 256, cudaMemcpyDeviceToDevice, st));
        }
        stt = enqueue_fire_step(c, hist + t, st, lb);
        if (stt != MD_OK) return stt;
    }
    // E = U(r_T); lambda_r(T) = -F(r_T), dU/dD at r_T; lambda_v(T) = 0
    PairArgs pe = c.pa;
    pe.E_out = d_out;
    enqueue_pair(pe, 2, MD_SOFT_SPHERE, 0, st);
    float4 *lam_v = adj, *lam_rp = adj + sN, *w_pend = adj + 2 * sN, *gvb = adj + 3 * sN, *wtot = adj + 4 * sN;
    aa.r = r;
    aa.f = fr;
    aa.lam_out = lam_rp;
    k_adjoint_final<<<g, 256, 0, st>>>(aa);
    JMD_CUDA_TRY(cudaMemsetAsync(lam_v, 0, sN * f4, st));
    JMD_CUDA_TRY(cudaMemsetAsync(w_pend, 0, sN * f4, st));
    JMD_CUDA_TRY(cudaMemcpyAsync(fin, r, sN * f4, cudaMemcpyDeviceToDevice, st));
    JMD_CUDA_TRY(cudaMemcpyAsync(fin + sN, v, sN * f4, cudaMemcpyDeviceToDevice, st));
    JMD_CUDA_TRY(cudaMemcpyAsync(fin + 2 * sN, fr, sN * f4, cudaMemcpyDeviceToDevice, st));

    FaArgs fa;
    memset(&fa, 0, sizeof(fa));
    fa.a = aa;
    fa.lam_v = lam_v;
    fa.lam_rp = lam_rp;
    fa.w_pend = w_pend;
    fa.gvb = gvb;
    fa.wtot = wtot;
    fa.scal = scal;

    // backward, segment by segment: replay from the checkpoint keeping every
    // state (r, v, F), then the reverse steps
    const int nseg = (T + K - 1) / K;
    for (int k = nseg - 1; k >= 0; --k) {
        const int t0 = k * K, t1 = (t0 + K < T) ? t0 + K : T;
        JMD_CUDA_TRY(cudaMemcpyAsync(r, ckrv + 2 * (size_t)k * sN, sN * f4, cudaMemcpyDeviceToDevice, st));
        JMD_CUDA_TRY(cudaMemcpyAsync(v, ckrv + (2 * (size_t)k + 1) * sN, sN * f4, cudaMemcpyDeviceToDevice, st));
        JMD_CUDA_TRY(cudaMemcpyAsync(state, ckh + 256 * (size_t)k, 256, cudaMemcpyDeviceToDevice, st));
        stt = md_neighbor_list_build(s, d_r, nb, d_status, (md_stream_t)st);
        if (stt != MD_OK) return stt;
        enqueue_pair(c.pa, 2, MD_SOFT_SPHERE, 0, st);
        for (int t = t0; t <= t1; ++t) {
            if (t > t0) {
                stt = enqueue_fire_step(c, nullptr, st, lb);
                if (stt != MD_OK) return stt;
            }
            JMD_CUDA_TRY(cudaMemcpyAsync(seg_at(t - t0, 0), r, sN * f4, cudaMemcpyDeviceToDevice, st));
            JMD_CUDA_TRY(cudaMemcpyAsync(seg_at(t - t0, 1), v, sN * f4, cudaMemcpyDeviceToDevice, st));
            JMD_CUDA_TRY(cudaMemcpyAsync(seg_at(t - t0, 2), fr, sN * f4, cudaMemcpyDeviceToDevice, st));
        }
        for (int q = t1 - 1; q >= t0; --q) {
            float *rn = (float *)seg_at(q + 1 - t0, 0);
            stt = list_for(s, rn, nb, d_status, st, lb);
            if (stt != MD_OK) return stt;
            fa.a.r = (const float4 *)rn;
            fa.vq = seg_at(q - t0, 1);
            fa.fq = seg_at(q - t0, 2);
            fa.fn = seg_at(q + 1 - t0, 2);
            fa.rec = hist + q;
            fa.final_state = 0;
            k_fa_sums<<<g, 256, 0, st>>>(fa);
            k_fa_dir<<<g, 256, 0, st>>>(fa);
            k_fa_hvp<<<g, 256, 0, st>>>(fa);
        }
        if (k == 0) {
            // state 0: its pending Hessian product, then r_0 = L(D) s_0
            float *r0 = (float *)seg_at(0, 0);
            stt = list_for(s, r0, nb, d_status, st, lb);
            if (stt != MD_OK) return stt;
            fa.a.r = (const float4 *)r0;
            fa.final_state = 1;
            k_fa_hvp<<<g, 256, 0, st>>>(fa);
        }
    }
    aa.lam_in = lam_rp;
    k_adjoint_initial<<<g, 256, 0, st>>>(aa);
    // leave r_T, v_T, F(r_T) in the caller's buffers
    JMD_CUDA_TRY(cudaMemcpyAsync(r, fin, sN * f4, cudaMemcpyDeviceToDevice, st));
    JMD_CUDA_TRY(cudaMemcpyAsync(v, fin + sN, sN * f4, cudaMemcpyDeviceToDevice, st));
    JMD_CUDA_TRY(cudaMemcpyAsync(fr, fin + 2 * sN, sN * f4, cudaMemcpyDeviceToDevice, st));
    JMD_CUDA_TRY(cudaGetLastError());
    return MD_OK;
}

// A loop builder on a stream that is being captured: conditional rebuild
// nodes go into the graph under capture (their bodies captured on a second
// stream).
static md_status with_loop_builder(md_nbr *nb, cudaStream_t cs, const std::function<md_status(LoopBuilder *)> &f)
{
    LoopBuilder lb;
    cudaStreamCaptureStatus cst;
    JMD_CUDA_TRY(cudaStreamGetCaptureInfo(cs, &cst, nullptr, &lb.graph, nullptr, nullptr, nullptr));
    if (cst != cudaStreamCaptureStatusActive || !lb.graph) return MD_ERR_CUDA;
    lb.cs = cs;
    lb.ctl = ws_ptrs(nb).ctl;
    JMD_CUDA_TRY(cudaStreamCreateWithFlags(&lb.cs2, cudaStreamNonBlocking));
    const md_status r = f(&lb);
    cudaStreamDestroy(lb.cs2);
    return r;
}

// Box of the bidisperse packing (App. A): nA disks of diameter D and N - nA
// of diameter dB in a square of packing fraction phi,
//   L(D) = sqrt((nA pi D^2 / 4 + (N - nA) pi dB^2 / 4) / phi),
//   dL/dD = pi nA D / (4 phi L).
static bool packing_box(int N, int nA, double D, double dB, double phi, double *L, double *Lp)
{
    if (N < 1 || nA < 0 || nA > N || !(D > 0.0) || !(dB > 0.0) || !(phi > 0.0)) return false;
    const double pi = 3.14159265358979323846;
    const double area = (nA * pi * D * D + (N - nA) * pi * dB * dB) / 4.0;
    *L = sqrt(area / phi);
    *Lp = pi * nA * D / (4.0 * phi * *L);
    return true;
}

// The packing's box must be the space the caller planned its list in: its
// edges equal L(D) (to the FP32 rounding of the box and of D).
static bool packing_space_ok(const md_space *s, int N, int nA, float D, float dB, double phi, float *Lp)
{
    double L = 0.0, lp = 0.0;
    if (!s || s->dim != 2 || !packing_box(N, nA, (double)D, (double)dB, phi, &L, &lp)) return false;
    if (fabs(s->L64[0] - L) > 1e-6 * L || fabs(s->L64[1] - L) > 1e-6 * L) return false;
    *Lp = (float)lp;
    return true;
}

// The adjoints' launch sequences are fixed by their arguments (step count,
// checkpoint schedule), so each call runs as one captured graph, cached per
// argument set (md_set_loop_graphs(0): host launches).  Same kernels, same
// order, same bits.
extern "C" md_status md_minimize_adjoint(const md_space *s, const md_pot *p, md_nbr *nb, const float *d_s0, int nA,
                                         float D, float dB, double phi, float eta, int T, int K, float *d_r,
                                         float *d_f, void *d_ws, double *d_out, uint32_t *d_status,
                                         md_stream_t stream)
{
    cudaStream_t st = (cudaStream_t)stream;
    float Lp = 0.0f;
    if (!nb || !packing_space_ok(s, nb->N, nA, D, dB, phi, &Lp)) return MD_ERR_INVALID;
    if (!s || !p || !nb || !g_loop_graphs)
        return gd_adjoint_body(s, p, nb, d_s0, nA, D, dB, Lp, eta, T, K, d_r, d_f, d_ws, d_out, d_status, st,
                               nullptr);
    struct Key {
        int tag, nA, T, K;
        float D, dB, Lp, eta;
        md_space s;
        md_pot p;
        md_nbr nb;
        const void *s0, *r, *f, *ws, *out, *status;
    } key;
    memset(&key, 0, sizeof(key));
    key.tag = 0x4144474a;
    key.nA = nA;
    key.T = T;
    key.K = K;
    key.D = D;
    key.dB = dB;
    key.Lp = Lp;
    key.eta = eta;
    key.s = *s;
    key.p = *p;
    key.nb = *nb;
    key.s0 = d_s0;
    key.r = d_r;
    key.f = d_f;
    key.ws = d_ws;
    key.out = d_out;
    key.status = d_status;
    return run_captured_call(&key, sizeof(key), [&](cudaStream_t cs) {
        return with_loop_builder(nb, cs, [&](LoopBuilder *lb) {
            return gd_adjoint_body(s, p, nb, d_s0, nA, D, dB, Lp, eta, T, K, d_r, d_f, d_ws, d_out, d_status, cs, lb);
        });
    }, st);
}

extern "C" md_status md_minimize_fire_adjoint(const md_space *s, const md_pot *p, const md_fire_params *fp,
                                              md_nbr *nb, const float *d_s0, int nA, float D, float dB, double phi,
                                              int T, int K, float *d_r, float *d_v, float *d_f, void *d_ws,
                                              double *d_out, uint32_t *d_status, md_stream_t stream)
{
    cudaStream_t st = (cudaStream_t)stream;
    float Lp = 0.0f;
    if (!nb || !packing_space_ok(s, nb->N, nA, D, dB, phi, &Lp)) return MD_ERR_INVALID;
    if (!s || !p || !fp || !nb || !g_loop_graphs)
        return fire_adjoint_body(s, p, fp, nb, d_s0, nA, D, dB, Lp, T, K, d_r, d_v, d_f, d_ws, d_out, d_status, st,
                                 nullptr);
    struct Key {
        int tag, nA, T, K;
        float D, dB, Lp;
        md_space s;
        md_pot p;
        md_fire_params fp;
        md_nbr nb;
        const void *s0, *r, *v, *f, *ws, *out, *status;
    } key;
    memset(&key, 0, sizeof(key));
    key.tag = 0x46414457;
    key.nA = nA;
    key.T = T;
    key.K = K;
    key.D = D;
    key.dB = dB;
    key.Lp = Lp;
    key.s = *s;
    key.p = *p;
    key.fp = *fp;
    key.nb = *nb;
    key.s0 = d_s0;
    key.r = d_r;
    key.v = d_v;
    key.f = d_f;
    key.ws = d_ws;
    key.out = d_out;
    key.status = d_status;
    return run_captured_call(&key, sizeof(key), [&](cudaStream_t cs) {
        return with_loop_builder(nb, cs, [&](LoopBuilder *lb) {
            return fire_adjoint_body(s, p, fp, nb, d_s0, nA, D, dB, Lp, T, K, d_r, d_v, d_f, d_ws, d_out, d_status, cs,
                                     lb);
        });
    }, st);
}

extern "C" md_status md_packing_space(int N, int nA, double D, double dB, double phi, md_space *out, double *dLdD)
{
    double L = 0.0, lp = 0.0;
    if (!out || !packing_box(N, nA, D, dB, phi, &L, &lp)) return MD_ERR_INVALID;
    const double box[2] = {L, L};
    const md_status e = md_space_periodic(2, box, out);
    if (e != MD_OK) return e;
    if (dLdD) *dLdD = lp;
    return MD_OK;
}
