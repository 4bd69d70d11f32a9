// pair.cu -- pair energies and forces over the neighbor list (Sec. 3.2.2,
// 3.3.2): U = 1/2 sum_{i != j} u(r_ij), F_i = -sum_j u'(r_ij) d_ij / r_ij.
//
// Gather form: a group of TPP threads owns particle i, strides over its
// sorted row, gathers float4 neighbor positions and reduces F_i and e_i with
// shuffles.  Every pair is visited from both sides (full list, no Newton's
// third law), so no atomics are needed and the result is deterministic.
//
// Fused variant (KICK): after F_i is known the group leader applies the
// closing half-kick v += dt/2 F/m of velocity Verlet and the block emits
// FP64 partial sums of potential and kinetic energy; the last block to
// finish (ticket) adds the partials in a fixed order.
#include "common.cuh"
#include "kernels.cuh"

namespace jmd {

template <int DIM, int TPP, int POT, int KICK>
__global__ void __launch_bounds__(256) k_pair(PairArgs a)
{
    count_launch();
    __shared__ double sh[8];
    __shared__ bool last;
    int gid = blockIdx.x * blockDim.x + threadIdx.x;
    int i = gid / TPP;
    int lg = threadIdx.x & (TPP - 1);
    bool valid = i < a.N;
    float fx = 0.f, fy = 0.f, fz = 0.f, e = 0.f;
    float4 ri = make_float4(0.f, 0.f, 0.f, 0.f);
    if (valid) {
        ri = a.r[i];
        int n = a.cnt[i];
        n = n < a.cap ? n : a.cap;
        const int32_t *row = a.nbr + (size_t)i * a.cap;
        for (int k = lg; k < n; k += TPP) {
            int j = __ldg(row + k);
            float4 rj = __ldg(a.r + j);
            float dx, dy, dz;
            float r2 = dist2_rn<DIM>(ri, rj, a.box, dx, dy, dz);
            if (POT == MD_LJ) {
                if (r2 < a.rc2) {
                    float ir2 = __fdividef(1.0f, r2);
                    float s2 = a.sigma2 * ir2;
                    float s6 = s2 * s2 * s2;
                    float fr = a.c24eps * ir2 * s6 * (2.0f * s6 - 1.0f);
                    fx += fr * dx;
                    fy += fr * dy;
                    fz += fr * dz;
                    e += a.c4eps * s6 * (s6 - 1.0f) - a.e_shift;
                }
            } else {  // soft sphere, s_ij = (w_i + w_j)/2
                float sg = 0.5f * (ri.w + rj.w);
                if (r2 < sg * sg) {
                    float rr = sqrtf(r2);
                    float isg = __fdividef(1.0f, sg);
                    float x = 1.0f - rr * isg;
                    float xa1, ua;
                    if (a.alpha == 2.0f) {
                        xa1 = x;
                        ua = 0.5f * x * x;
                    } else {
                        xa1 = __powf(x, a.alpha - 1.0f);
                        ua = xa1 * x / a.alpha;
                    }
                    // F_i += (eps/s) x^(alpha-1) d / r
                    float fr = a.eps * isg * xa1 * __fdividef(1.0f, rr);
                    fx += fr * dx;
                    fy += fr * dy;
                    fz += fr * dz;
                    e += a.eps * ua;
                }
            }
        }
    }
#pragma unroll
    for (int o = TPP / 2; o > 0; o >>= 1) {
        fx += __shfl_xor_sync(0xffffffffu, fx, o);
        fy += __shfl_xor_sync(0xffffffffu, fy, o);
        fz += __shfl_xor_sync(0xffffffffu, fz, o);
        e += __shfl_xor_sync(0xffffffffu, e, o);
    }
    double pe = 0.0, ke = 0.0;
    if (valid && lg == 0) {
        float ei = 0.5f * e;
        a.f[i] = make_float4(fx, fy, fz, ei);
        pe = (double)ei;
        if (KICK) {
            float4 v = a.v[i];
            v.x += a.half_dt_over_m * fx;
            v.y += a.half_dt_over_m * fy;
            if (DIM == 3) v.z += a.half_dt_over_m * fz;
            a.v[i] = v;
            float v2 = v.x * v.x + v.y * v.y + v.z * v.z;
            ke = 0.5 * (double)a.mass * (double)v2;
        }
    }
    if (!a.E_out && !KICK) return;
    double bpe = block_sum_f64(pe, sh);
    double bke = KICK ? block_sum_f64(ke, sh) : 0.0;
    if (threadIdx.x == 0) {
        a.partials[blockIdx.x] = make_double2(bpe, bke);
        __threadfence();
        unsigned t = atomicAdd(&a.ctl[CTL_TICKET], 1u);
        last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double spe = 0.0, ske = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
        const volatile double *p = (const volatile double *)(a.partials + b);
        spe += p[0];
        ske += p[1];
    }
    spe = block_sum_f64(spe, sh);
    ske = block_sum_f64(ske, sh);
    if (threadIdx.x == 0) {
        a.ctl[CTL_TICKET] = 0u;
        if (!isfinite(spe) || !isfinite(ske)) raise_status(a.status, MD_ERR_NONFINITE);
        unsigned step = a.series ? a.ctl[CTL_STEP] : 0u;
        if (a.E_out) a.E_out[step] = spe;
        if (a.KE_out) a.KE_out[step] = ske;
        if (a.series) a.ctl[CTL_STEP] = step + 1u;
        if (a.use_cond)
            cudaGraphSetConditional((cudaGraphConditionalHandle)a.cond_while,
                                    (step + 1u < a.ctl[CTL_NSTEPS]) ? 1u : 0u);
    }
}

template <int DIM, int TPP, int POT, int KICK>
static void launch_pair_t(const PairArgs &a, cudaStream_t st)
{
    k_pair<DIM, TPP, POT, KICK><<<pair_blocks(a.N, TPP), 256, 0, st>>>(a);
}

template <int DIM, int POT, int KICK>
static void launch_pair_tpp(const PairArgs &a, cudaStream_t st)
{
    switch (a.tpp) {
    case 4: launch_pair_t<DIM, 4, POT, KICK>(a, st); break;
    case 16: launch_pair_t<DIM, 16, POT, KICK>(a, st); break;
    case 32: launch_pair_t<DIM, 32, POT, KICK>(a, st); break;
    default: launch_pair_t<DIM, 8, POT, KICK>(a, st); break;
    }
}

void enqueue_pair(const PairArgs &a, int dim, int pot, int kick, cudaStream_t st)
{
    if (dim == 3) {
        if (pot == MD_LJ) kick ? launch_pair_tpp<3, MD_LJ, 1>(a, st) : launch_pair_tpp<3, MD_LJ, 0>(a, st);
        else kick ? launch_pair_tpp<3, MD_SOFT_SPHERE, 1>(a, st) : launch_pair_tpp<3, MD_SOFT_SPHERE, 0>(a, st);
    } else {
        if (pot == MD_LJ) kick ? launch_pair_tpp<2, MD_LJ, 1>(a, st) : launch_pair_tpp<2, MD_LJ, 0>(a, st);
        else kick ? launch_pair_tpp<2, MD_SOFT_SPHERE, 1>(a, st) : launch_pair_tpp<2, MD_SOFT_SPHERE, 0>(a, st);
    }
}

int pair_blocks(int N, int tpp) { return (int)(((long long)N * tpp + 255) / 256); }

static int g_tpp = 8;

bool make_pair_args(const md_space *s, const md_pot *p, const float *d_r, const md_nbr *nb, float *d_f, PairArgs &a)
{
    if (!s || !p || !d_r || !nb || !d_f || !nb->nbr || !nb->cnt || !nb->ws) return false;
    if (p->kind != MD_LJ && p->kind != MD_SOFT_SPHERE) return false;
    memset(&a, 0, sizeof(a));
    a.box = make_box(s);
    a.N = nb->N;
    a.cap = nb->cap;
    a.r = (const float4 *)d_r;
    a.nbr = nb->nbr;
    a.cnt = nb->cnt;
    a.f = (float4 *)d_f;
    WsPtrs w = ws_ptrs(nb);
    a.ctl = w.ctl;
    a.partials = w.partials;
    a.tpp = g_tpp;
    if (p->kind == MD_LJ) {
        if (p->r_cut > nb->r_list) return false;
        float rc = p->r_cut;
        a.rc2 = rc * rc;
        a.sigma2 = p->sigma * p->sigma;
        a.c24eps = 24.0f * p->eps;
        a.c4eps = 4.0f * p->eps;
        a.e_shift = p->e_shift;
    } else {
        a.eps = p->eps;
        a.alpha = p->alpha;
    }
    return pair_blocks(a.N, a.tpp) <= w.max_blocks;
}

}  // namespace jmd

using namespace jmd;

extern "C" md_status md_set_pair_tpp(int tpp)
{
    if (tpp != 4 && tpp != 8 && tpp != 16 && tpp != 32) return MD_ERR_INVALID;
    g_tpp = tpp;
    return MD_OK;
}

extern "C" md_status md_energy_forces(const md_space *s, const md_pot *p, const float *d_r, const md_nbr *nb,
                                      float *d_f, double *d_E, uint32_t *d_status, md_stream_t stream)
{
    if (!p || !s || !nb) return MD_ERR_INVALID;
    if (s->dim != nb->dim) return MD_ERR_INVALID;
    if (p->kind == MD_SW) return md_energy_forces_sw(s, p, d_r, nb, d_f, d_E, d_status, stream);
    PairArgs a;
    if (!make_pair_args(s, p, d_r, nb, d_f, a)) return MD_ERR_INVALID;
    a.E_out = d_E;
    a.status = d_status;
    enqueue_pair(a, s->dim, p->kind, 0, (cudaStream_t)stream);
    JMD_CUDA_TRY(cudaGetLastError());
    return MD_OK;
}
