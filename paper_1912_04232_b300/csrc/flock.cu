// flock.cu -- the flocking energy model (Sec. 4.3 and its appendix) on the
// periodic neighbor list.
//
// Boid i: position R_i, heading theta_i, N_i = (cos, sin) theta_i.  With
// rho(r; Rc) = (1 - r/Rc)^a / a below Rc and each unordered pair once:
//   E_align = sum J_al rho(r_ij; R_al) (1 - N_i.N_j)^2  (turns boids only)
//   E_avoid = sum J_av rho(r_ij; R_av)
//   E_coh   = sum_i J_co/2 (1 - u_i.N_i)^2, u_i towards the mean offset of
//             the boids within R_co (turns boids only)
//   E_obst  = sum_i sum_o J_ob rho(|R_o - R_i|; D_o) (1 + N_i.w_io)^2, w_io
//             the unit vector from the boid to disk obstacle o
//   E_flee  = the obstacle form against each predator (range R_fl)
// and forward Euler R_i += dt (v N_i - dE/dR_i), theta_i -= dt dE/dtheta_i.
// Predators minimise their own energy: the cohesion form towards the boids
// within R_ch (heading only) plus the obstacles (k_predator_scan over slabs
// of boids, k_predator_step per predator).  They sprint (speed x sprint_factor) in
// the steps s with s mod sprint_period < sprint_steps, s counted from 0 in
// each call.
//
// k_flock_step: a group of TPP lanes per boid gathers its row of the list
// (float4 = x, y, cos theta, sin theta, so no pair needs a sine), reduces
// the sums with shuffles, adds cohesion and obstacles, and writes the new
// state to the other buffer (every boid reads its neighbours' old state);
// the headings are updated in place by their owners.  The displacement
// check for the list and the FP64 energy of the state before the step are
// fused in.
#include <algorithm>

#include "common.cuh"
#include "kernels.cuh"

namespace jmd {

struct FlockArgs {
    Box box;
    int N, cap, n_obs;
    md_flock_params p;
    float dt;
    const float4 *b;        // x, y, cos theta, sin theta (this step)
    float4 *b_out;          // the next step
    float *theta;           // headings, updated in place
    const float *obs;       // n_obs x 3: x, y, radius
    const float4 *pred;     // n_pred predators this step: x, y, theta, energy of the previous state
    float4 *pred_out;       // the next step (w: its energy in this state)
    int n_pred;
    const int32_t *nbr, *cnt;
    const float4 *rref;
    float half_skin2;
    uint32_t *ctl;
    double2 *partials;
    double *E_out;
    uint32_t *status;
};

__device__ __forceinline__ float fl_rho(float r, float Rc, float a)
{
    if (!(r < Rc)) return 0.0f;
    const float x = 1.0f - r / Rc;
    return a == 2.0f ? 0.5f * x * x : __powf(x, a) / a;
}
__device__ __forceinline__ float fl_rho_d(float r, float Rc, float a)
{
    if (!(r < Rc)) return 0.0f;
    const float x = 1.0f - r / Rc;
    return -(a == 2.0f ? x : __powf(x, a - 1.0f)) / Rc;
}

// The disk form J rho(r; D) (1 + N.w)^2 of an agent at (x, y), heading
// (ci, si), against a disk at (ox, oy): adds energy and the gradient in the
// agent's variables.
__device__ __forceinline__ void fl_disk(const FlockArgs &a, float x, float y, float ci, float si, float ox, float oy,
                                        float D, float J, float &e, float &gx, float &gy, float &gth)
{
    const float dx = min_image_rn(ox, x, a.box.L[0], a.box.Linv[0]);
    const float dy = min_image_rn(oy, y, a.box.L[1], a.box.Linv[1]);
    const float r = sqrtf(dx * dx + dy * dy);
    if (!(r > 0.0f && r < D)) return;
    const float wx = dx / r, wy = dy / r;
    const float nw = ci * wx + si * wy, q = 1.0f + nw;
    const float rh = fl_rho(r, D, a.p.alpha), rhd = fl_rho_d(r, D, a.p.alpha);
    e += J * rh * q * q;
    gth += 2.0f * J * rh * q * (-si * wx + ci * wy);
    gx += J * (rhd * (-wx) * q * q + rh * 2.0f * q * (-(ci - nw * wx) / r));
    gy += J * (rhd * (-wy) * q * q + rh * 2.0f * q * (-(si - nw * wy) / r));
}

// The cohesion form J/2 (1 - u.N)^2 from summed offsets (cx, cy) of n
// agents: adds energy and the heading gradient.
__device__ __forceinline__ void fl_heading(float cx, float cy, float n, float ci, float si, float J, float &e,
                                           float &gth)
{
    if (!(n > 0.0f)) return;
    const float mx = cx / n, my = cy / n;
    const float m = sqrtf(mx * mx + my * my);
    if (!(m > 0.0f)) return;
    const float ux = mx / m, uy = my / m;
    const float un = ux * ci + uy * si, up = -ux * si + uy * ci;
    e += 0.5f * J * (1.0f - un) * (1.0f - un);
    gth += -J * (1.0f - un) * up;
}

template <int TPP>
__global__ void __launch_bounds__(256) k_flock_step(FlockArgs a)
{
    count_launch();
    __shared__ double sh[8];
    __shared__ bool last;
    const int lg = threadIdx.x & (TPP - 1);
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) / TPP;
    const bool valid = i < a.N;
    const md_flock_params &p = a.p;
    float gth = 0.f, gx = 0.f, gy = 0.f, cx = 0.f, cy = 0.f, nco = 0.f, e = 0.f;
    float4 bi = make_float4(0.f, 0.f, 1.f, 0.f);
    if (valid) {
        bi = a.b[i];
        int n = a.cnt[i];
        n = n < a.cap ? n : a.cap;
        const int32_t *row = a.nbr + (size_t)i * a.cap;
        for (int k = lg; k < n; k += TPP) {
            const int j = __ldg(row + k);
            const float4 bj = __ldg(a.b + j);
            float dx, dy, dz;
            const float r2 = dist2_rn<2>(bi, bj, a.box, dx, dy, dz);
            const float r = sqrtf(r2);
            const float c = bi.z * bj.z + bi.w * bj.w;       // cos(theta_i - theta_j)
            const float s = bi.w * bj.z - bi.z * bj.w;       // sin(theta_i - theta_j)
            if (r < p.R_align) {
                const float rh = fl_rho(r, p.R_align, p.alpha);
                e += 0.5f * p.J_align * rh * (1.0f - c) * (1.0f - c);
                gth += 2.0f * p.J_align * rh * (1.0f - c) * s;
            }
            if (r < p.R_avoid && r > 0.0f) {
                e += 0.5f * p.J_avoid * fl_rho(r, p.R_avoid, p.alpha);
                const float g = p.J_avoid * fl_rho_d(r, p.R_avoid, p.alpha) / r;
                gx += g * dx;
                gy += g * dy;
            }
            if (r < p.R_cohesion) {
                cx -= dx;
                cy -= dy;
                nco += 1.0f;
            }
        }
    }
#pragma unroll
    for (int o = TPP / 2; o > 0; o >>= 1) {
        gth += __shfl_xor_sync(0xffffffffu, gth, o);
        gx += __shfl_xor_sync(0xffffffffu, gx, o);
        gy += __shfl_xor_sync(0xffffffffu, gy, o);
        cx += __shfl_xor_sync(0xffffffffu, cx, o);
        cy += __shfl_xor_sync(0xffffffffu, cy, o);
        nco += __shfl_xor_sync(0xffffffffu, nco, o);
        e += __shfl_xor_sync(0xffffffffu, e, o);
    }
    bool mv = false;
    if (valid && lg == 0) {
        const float ci = bi.z, si = bi.w;
        fl_heading(cx, cy, nco, ci, si, p.J_cohesion, e, gth);
        for (int o = 0; o < a.n_obs; ++o)
            fl_disk(a, bi.x, bi.y, ci, si, __ldg(a.obs + 3 * o), __ldg(a.obs + 3 * o + 1), __ldg(a.obs + 3 * o + 2),
                    p.J_obstacle, e, gx, gy, gth);
        for (int q = 0; q < a.n_pred; ++q) {
            const float4 pq = a.pred[q];
            fl_disk(a, bi.x, bi.y, ci, si, pq.x, pq.y, p.R_flee, p.J_flee, e, gx, gy, gth);
        }
        float th = a.theta[i];
        const float x = wrap_coord(bi.x + a.dt * (p.speed * ci - gx), a.box.L[0], a.box.Linv[0]);
        const float y = wrap_coord(bi.y + a.dt * (p.speed * si - gy), a.box.L[1], a.box.Linv[1]);
        th -= a.dt * gth;
        float sn, cs;
        sincosf(th, &sn, &cs);
        a.theta[i] = th;
        const float4 bo = make_float4(x, y, cs, sn);
        a.b_out[i] = bo;
        float ddx, ddy, ddz;
        mv = dist2_rn<2>(bo, a.rref[i], a.box, ddx, ddy, ddz) > a.half_skin2;
    } else {
        e = 0.0f;
    }
    if (__any_sync(0xffffffffu, mv) && (threadIdx.x & 31) == 0) a.ctl[CTL_REBUILD] = 1u;
    if (!a.E_out) {
        if (blockIdx.x == 0 && threadIdx.x == 0) a.ctl[CTL_STEP] += 1u;   // the step count (sprints)
        return;
    }
    // FP64 energy of the state before the step: warp (FP32), block and grid
    // (FP64, fixed order by the last block)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = (double)e;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];
        a.partials[blockIdx.x] = make_double2(s, 0.0);
        __threadfence();
        last = atomicAdd(&a.ctl[CTL_TICKET], 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    // the block partials summed by the whole last block (fixed order)
    double E = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) E += ((volatile double *)(a.partials + b))[0];
    E = block_sum_f64(E, sh);
    if (threadIdx.x != 0) return;
    for (int q = 0; q < a.n_pred; ++q) E += (double)a.pred_out[q].w;
    a.ctl[CTL_TICKET] = 0u;
    if (!isfinite(E)) raise_status(a.status, MD_ERR_NONFINITE);
    const unsigned step = a.ctl[CTL_STEP];
    a.E_out[step] = E;
    a.ctl[CTL_STEP] = step + 1u;
}

// Chase sums, in two kernels so that the scan of the boids fills the GPU and
// the sums keep a fixed order: k_predator_scan block s takes the boids of
// slab s and writes, per predator q, the summed offsets R_i - R_q of the
// boids within R_ch and their count to ppart[q * S + s]; k_predator_step
// (one warp per predator) adds the S slabs, then takes the predator's chase
// and obstacle energy and gradient and its forward-Euler step into pred_out
// (w = its energy in the state before the step).
__global__ void __launch_bounds__(256) k_predator_scan(FlockArgs a, float4 *ppart, int S)
{
    count_launch();
    __shared__ float sh[3][8];
    const int s = blockIdx.x;
    const int chunk = (a.N + S - 1) / S;
    const int i0 = s * chunk, i1 = min(a.N, i0 + chunk);
    const float R2 = a.p.R_chase * a.p.R_chase;
    for (int q = 0; q < a.n_pred; ++q) {
        const float4 pq = a.pred[q];
        float cx = 0.f, cy = 0.f, n = 0.f;
        for (int i = i0 + (int)threadIdx.x; i < i1; i += blockDim.x) {
            const float4 bi = a.b[i];
            const float dx = min_image_rn(bi.x, pq.x, a.box.L[0], a.box.Linv[0]);
            const float dy = min_image_rn(bi.y, pq.y, a.box.L[1], a.box.Linv[1]);
            if (dx * dx + dy * dy < R2) {
                cx += dx;
                cy += dy;
                n += 1.0f;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            cx += __shfl_xor_sync(0xffffffffu, cx, o);
            cy += __shfl_xor_sync(0xffffffffu, cy, o);
            n += __shfl_xor_sync(0xffffffffu, n, o);
        }
        if ((threadIdx.x & 31) == 0) {
            sh[0][threadIdx.x >> 5] = cx;
            sh[1][threadIdx.x >> 5] = cy;
            sh[2][threadIdx.x >> 5] = n;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            cx = cy = n = 0.f;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
                cx += sh[0][w];
                cy += sh[1][w];
                n += sh[2][w];
            }
            ppart[(size_t)q * S + s] = make_float4(cx, cy, n, 0.f);
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(32) k_predator_step(FlockArgs a, const float4 *ppart, int S)
{
    count_launch();
    const int q = blockIdx.x;
    const float4 pq = a.pred[q];
    float cx = 0.f, cy = 0.f, n = 0.f;
    for (int s = (int)threadIdx.x; s < S; s += 32) {
        const float4 v = ppart[(size_t)q * S + s];
        cx += v.x;
        cy += v.y;
        n += v.z;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        cx += __shfl_xor_sync(0xffffffffu, cx, o);
        cy += __shfl_xor_sync(0xffffffffu, cy, o);
        n += __shfl_xor_sync(0xffffffffu, n, o);
    }
    if (threadIdx.x != 0) return;
    float sn, cs;
    sincosf(pq.z, &sn, &cs);
    float e = 0.f, gx = 0.f, gy = 0.f, gth = 0.f;
    fl_heading(cx, cy, n, cs, sn, a.p.J_chase, e, gth);
    for (int o = 0; o < a.n_obs; ++o)
        fl_disk(a, pq.x, pq.y, cs, sn, __ldg(a.obs + 3 * o), __ldg(a.obs + 3 * o + 1), __ldg(a.obs + 3 * o + 2),
                a.p.J_obstacle, e, gx, gy, gth);
    const uint32_t step = *(const volatile uint32_t *)&a.ctl[CTL_STEP];
    const float vp = (a.p.sprint_period > 0 && (int)(step % (uint32_t)a.p.sprint_period) < a.p.sprint_steps)
                         ? a.p.predator_speed * a.p.sprint_factor
                         : a.p.predator_speed;
    const float x = wrap_coord(pq.x + a.dt * (vp * cs - gx), a.box.L[0], a.box.Linv[0]);
    const float y = wrap_coord(pq.y + a.dt * (vp * sn - gy), a.box.L[1], a.box.Linv[1]);
    a.pred_out[q] = make_float4(x, y, pq.z - a.dt * gth, e);
}

// (x, y) from the caller's positions, (cos, sin) of the headings.
__global__ void __launch_bounds__(256) k_flock_init(float4 *b, const float *theta, int N)
{
    count_launch();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    float sn, cs;
    sincosf(theta[i], &sn, &cs);
    float4 bi = b[i];
    bi.z = cs;
    bi.w = sn;
    b[i] = bi;
}

}  // namespace jmd

using namespace jmd;

extern "C" md_status md_flock_run(const md_space *s, const md_flock_params *prm, const float *d_obs, int n_obs,
                                  float *d_pred, float *d_pred_alt, int n_pred, float *d_b, float *d_theta,
                                  float *d_b_alt, float dt, int nsteps, md_nbr *nb, double *d_E, uint32_t *d_status,
                                  md_stream_t stream)
{
    if (!s || !prm || !d_b || !d_theta || !d_b_alt || !nb || nsteps < 0 || n_obs < 0 || n_pred < 0)
        return MD_ERR_INVALID;
    if ((n_obs > 0 && !d_obs) || (n_pred > 0 && (!d_pred || !d_pred_alt))) return MD_ERR_INVALID;
    if (s->dim != 2 || nb->dim != 2 || !nb->nbr || !nb->cnt || !nb->ws || !nb->rref || !nbr_layout_ok(nb))
        return MD_ERR_INVALID;
    const float rmax = fmaxf(prm->R_align, fmaxf(prm->R_avoid, prm->R_cohesion));
    if (!(rmax > 0.0f) || rmax > nb->r_cut || !(prm->alpha >= 1.0f) || !(dt > 0.0f)) return MD_ERR_INVALID;
    if (prm->sprint_period < 0 || prm->sprint_steps < 0) return MD_ERR_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    const WsPtrs w = ws_ptrs(nb);
    const int N = nb->N;
    FlockArgs a;
    memset(&a, 0, sizeof(a));
    a.box = make_box(s);
    a.N = N;
    a.cap = nb->cap;
    a.n_obs = n_obs;
    a.p = *prm;
    a.dt = dt;
    a.theta = d_theta;
    a.obs = d_obs;
    a.n_pred = n_pred;
    a.pred = (const float4 *)d_pred;   // (the graph key holds both predator buffers)
    a.pred_out = (float4 *)d_pred_alt;
    a.nbr = nb->nbr;
    a.cnt = nb->cnt;
    a.rref = (const float4 *)nb->rref;
    a.half_skin2 = nb->half_skin2;
    a.ctl = w.ctl;
    a.partials = w.partials;
    a.E_out = d_E;
    a.status = d_status;
    constexpr int TPP = 4;
    const int grid = (int)(((long long)N * TPP + 255) / 256);
    if (d_E && grid > w.max_blocks) return MD_ERR_INVALID;
    // the chase partials borrow the energy partials (free until k_flock_step)
    if (n_pred > w.max_blocks) return MD_ERR_INVALID;
    const int S = n_pred > 0 ? std::max(1, std::min((N + 255) / 256, w.max_blocks / n_pred)) : 1;
    float4 *ppart = (float4 *)w.partials;
    enqueue_loop_init(w.ctl, (uint32_t)nsteps, st);
    k_flock_init<<<(N + 255) / 256, 256, 0, st>>>((float4 *)d_b, d_theta, N);
    NbrArgs na[2] = {make_nbr_args(s, d_b_alt, nb, d_status, 1), make_nbr_args(s, d_b, nb, d_status, 1)};
    float4 *buf[2] = {(float4 *)d_b, (float4 *)d_b_alt};
    float4 *pbuf[2] = {(float4 *)d_pred, (float4 *)d_pred_alt};
    const int ncell = nb->ncell_total;
    // step t: the state in buf[t & 1] moves to the other buffer; the list is
    // rebuilt (if needed) on the new positions
    auto step = [&](int t, cudaStream_t cs, LoopBuilder *lb) -> md_status {
        FlockArgs at = a;
        at.b = buf[t & 1];
        at.b_out = buf[(t + 1) & 1];
        at.pred = pbuf[t & 1];
        at.pred_out = pbuf[(t + 1) & 1];
        if (n_pred > 0) {
            k_predator_scan<<<S, 256, 0, cs>>>(at, ppart, S);
            k_predator_step<<<n_pred, 32, 0, cs>>>(at, ppart, S);
        }
        k_flock_step<TPP><<<grid, 256, 0, cs>>>(at);
        if (lb) return lb->rebuild_if(na[t & 1], ncell);
        enqueue_rebuild_chain(na[t & 1], ncell, cs);
        return MD_OK;
    };
    int done = 0;
    if (g_loop_graphs && nsteps >= 2) {
        // graph loop of two steps per iteration (the buffers trade places)
        struct Key {
            int tag;
            FlockArgs a;
            NbrArgs na0, na1;
            int ncell;
        } key;
        memset(&key, 0, sizeof(key));
        key.tag = 0x464c4f43;   // FLOC
        key.a = a;
        key.na0 = na[0];
        key.na1 = na[1];
        key.ncell = ncell;
        md_status e = run_graph_loop(&key, sizeof(key), w.ctl, nsteps / 2,
                                     [&](LoopBuilder &lb) {
                                         md_status e0 = step(0, lb.cs, &lb);
                                         return e0 != MD_OK ? e0 : step(1, lb.cs, &lb);
                                     },
                                     st);
        if (e != MD_OK) return e;
        done = nsteps / 2 * 2;
    }
    for (int t = done; t < nsteps; ++t) step(t, st, nullptr);
    if (nsteps & 1) {
        JMD_CUDA_TRY(cudaMemcpyAsync(d_b, d_b_alt, sizeof(float4) * (size_t)N, cudaMemcpyDeviceToDevice, st));
        if (n_pred > 0)
            JMD_CUDA_TRY(cudaMemcpyAsync(d_pred, d_pred_alt, sizeof(float4) * (size_t)n_pred,
                                         cudaMemcpyDeviceToDevice, st));
    }
    JMD_CUDA_TRY(cudaGetLastError());
    return MD_OK;
}
