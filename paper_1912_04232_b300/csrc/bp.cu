// bp.cu -- Behler-Parrinello symmetry-function descriptors (Sec. 3.2.4, 4.1)
// and the two gathers that tie them to forces and to training.
//
//   f_c(r) = (cos(pi r / R_c) + 1) / 2,  R_c = 3.77 A
//   radial   G_m  = sum_j exp(-eta_r (r_ij - R_m)^2) f_c(r_ij),   R_m = 2 + 0.25 (m-1), m = 1..8
//   angular  G_zl = 2^(1-z) sum_{j<k} (1 + l cos theta_jik)^z exp(-eta_a (r_ij^2 + r_ik^2)) f_c f_c,
//            z in {1, 2, 4, 16}, l in {+1, -1}
//
// k_bp_desc   : G [N][16], four atoms per warp (pairs and triplets over eight lanes)
// k_bp_force  : F_k = -sum_i sum_m e_im dG_im/dr_k with e = dE/dG from the
//               network; gather form (self terms, pair terms of the
//               neighbors, triplets centred on each neighbor with k as a
//               leg), four atoms per warp, eight lanes each, no atomics
// k_bp_jvp    : v_im = sum_k dG_im/dr_k . dF_k (the descriptor Jacobian
//               applied to a per-atom vector field): the input of the
//               force-loss gradient, gathered over the atom's own pairs and
//               triplets
#include "common.cuh"
#include "kernels.cuh"
#include "bp.cuh"
#include "reduce.cuh"
#include "bp_terms.cuh"

namespace jmd {

constexpr int BP_WARPS = 8;

// The angular terms' gradients contracted with a weight per column:
// g_u = sum_col e_col dt_col/du and g_w = sum_col e_col dt_col/dw for the
// triplet with legs u, w (|u|, |w| < R_c).  Each column is
// t = 2^(1-z) (1 + l cos)^z B with B = exp(-eta_a (|u|^2 + |w|^2)) f_c f_c, so
// dt/du = (dt/dcos) dcos/du + (dt/dB) dB/du and the sums over columns fold
// into two scalars, sum e dt/dcos and sum e dt/dB, before the vectors.
__device__ __forceinline__ void angular_grad(const BpConst &c, float ux, float uy, float uz, float ru, float wx,
                                             float wy, float wz, float rw, const float e[8], float gu[3], float gw[3])
{
    const float iu = 1.0f / ru, iw = 1.0f / rw;
    const float cs = (ux * wx + uy * wy + uz * wz) * iu * iw;
    float fu, dfu, fw, dfw;
    fcut(c, ru, fu, dfu);
    fcut(c, rw, fw, dfw);
    const float ex = __expf(-c.eta_a * (ru * ru + rw * rw));
    const float B = ex * fu * fw;
    const float bu = -2.0f * c.eta_a * B + ex * dfu * fw * iu;   // dB/du = bu u
    const float bw = -2.0f * c.eta_a * B + ex * fu * dfw * iw;   // dB/dw = bw w
    const float zs[4] = {1.0f, 2.0f, 4.0f, 16.0f};
    const float pref[4] = {1.0f, 0.5f, 0.125f, 1.0f / 32768.0f};   // 2^(1 - z)
    float A = 0.0f, Bs = 0.0f;   // sum e dt/dcos, sum e dt/dB
#pragma unroll
    for (int l = 0; l < 2; ++l) {
        const float lam = l == 0 ? 1.0f : -1.0f;
        float pz[4], pzm1[4];
        powers(1.0f + lam * cs, pz, pzm1);
#pragma unroll
        for (int zi = 0; zi < 4; ++zi) {
            const float ec = e[2 * zi + l];
            A += ec * pref[zi] * zs[zi] * pzm1[zi] * lam;
            Bs += ec * pref[zi] * pz[zi];
        }
    }
    A *= B;
    const float iuw = iu * iw;
    gu[0] = A * (wx * iuw - cs * ux * iu * iu) + Bs * bu * ux;
    gu[1] = A * (wy * iuw - cs * uy * iu * iu) + Bs * bu * uy;
    gu[2] = A * (wz * iuw - cs * uz * iu * iu) + Bs * bu * uz;
    gw[0] = A * (ux * iuw - cs * wx * iw * iw) + Bs * bw * wx;
    gw[1] = A * (uy * iuw - cs * wy * iw * iw) + Bs * bw * wy;
    gw[2] = A * (uz * iuw - cs * wz * iw * iw) + Bs * bw * wz;
}

// The angular terms' directional derivatives: out[col] += dt_col/du . a +
// dt_col/dw . b for the triplet with legs u, w.  With dt/du = (dt/dcos)
// dcos/du + (dt/dB) dB/du, the vector parts are the same for all columns, so
// they reduce to two scalars first: X = dcos/du . a + dcos/dw . b and
// Y = dB/du . a + dB/dw . b.
__device__ __forceinline__ void angular_dir(const BpConst &c, float ux, float uy, float uz, float ru, float wx,
                                            float wy, float wz, float rw, float ax, float ay, float az, float bx,
                                            float by, float bz, float *out)
{
    const float iu = 1.0f / ru, iw = 1.0f / rw;
    const float cs = (ux * wx + uy * wy + uz * wz) * iu * iw;
    float fu, dfu, fw, dfw;
    fcut(c, ru, fu, dfu);
    fcut(c, rw, fw, dfw);
    const float ex = __expf(-c.eta_a * (ru * ru + rw * rw));
    const float B = ex * fu * fw;
    const float bu = -2.0f * c.eta_a * B + ex * dfu * fw * iu;
    const float bw = -2.0f * c.eta_a * B + ex * fu * dfw * iw;
    const float iuw = iu * iw;
    const float ua = ux * ax + uy * ay + uz * az, ub = ux * bx + uy * by + uz * bz;
    const float wa = wx * ax + wy * ay + wz * az, wb = wx * bx + wy * by + wz * bz;
    const float X = (wa * iuw - cs * ua * iu * iu) + (ub * iuw - cs * wb * iw * iw);
    const float Y = bu * ua + bw * wb;
    const float zs[4] = {1.0f, 2.0f, 4.0f, 16.0f};
    const float pref[4] = {1.0f, 0.5f, 0.125f, 1.0f / 32768.0f};   // 2^(1 - z)
#pragma unroll
    for (int l = 0; l < 2; ++l) {
        const float lam = l == 0 ? 1.0f : -1.0f;
        float pz[4], pzm1[4];
        powers(1.0f + lam * cs, pz, pzm1);
#pragma unroll
        for (int zi = 0; zi < 4; ++zi)
            out[2 * zi + l] += pref[zi] * zs[zi] * pzm1[zi] * lam * B * X + pref[zi] * pz[zi] * Y;
    }
}

// Neighbors of atom i inside R_c into the warp's shared list
// (j, u = r_j - r_i, |u|); returns the count (clamped, overflow flagged).
__device__ __forceinline__ int gather_within(const BpArgs &a, const BpConst &c, int i, const float4 &ri, int *nj,
                                             float4 *nd)
{
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    int n = a.cnt[i];
    n = n < a.cap ? n : a.cap;
    const int32_t *row = a.nbr + (size_t)i * a.cap;
    const int base = a.sys_n ? (i / a.sys_n) * a.sys_n : 0;
    int m = 0;
    for (int k0 = 0; k0 < n; k0 += 32) {
        int k = k0 + lane;
        bool in = false;
        int j = 0;
        float dx = 0.f, dy = 0.f, dz = 0.f, r2 = 0.f;
        if (k < n) {
            j = row[k] + base;
            float4 rj = __ldg(a.r + j);
            r2 = dist2_rn<3>(rj, ri, a.box, dx, dy, dz);
            in = r2 < c.rc2;
        }
        unsigned mk = __ballot_sync(0xffffffffu, in);
        int pos = m + __popc(mk & lt);
        if (in && pos < BP_MAXN) {
            nj[pos] = j;
            nd[pos] = make_float4(dx, dy, dz, sqrtf(r2));
        }
        m += __popc(mk);
    }
    if (m > BP_MAXN) {
        if (lane == 0) raise_status(a.status, MD_ERR_NBR_OVERFLOW);
        m = BP_MAXN;
    }
    __syncwarp();
    return m;
}

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Descriptors with DESC_GROUP lanes per atom (a silicon atom has about five
// partners inside R_c, so a whole warp per atom would leave most lanes idle);
// desc_group (bp_terms.cuh) does one atom per group.
constexpr int DESC_GROUP = 8;
constexpr int DESC_PER_WARP = 32 / DESC_GROUP;

__global__ void __launch_bounds__(BP_WARPS * 32) k_bp_desc(BpArgs a)
{
    count_launch();
    __shared__ float4 nd[BP_WARPS][DESC_PER_WARP][BP_MAXN];
    const BpConst c = bp_const();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int grp = lane / DESC_GROUP, gl = lane % DESC_GROUP;
    const unsigned gmask = ((1u << DESC_GROUP) - 1u) << (grp * DESC_GROUP);
    const unsigned below = (1u << lane) - 1u;
    float4 *ndg = nd[w][grp];
    const int step = gridDim.x * BP_WARPS * DESC_PER_WARP;
    // every lane runs every trip (group ballots and sums are warp-wide);
    // atoms past the end carry an empty list
    for (int i0 = (blockIdx.x * BP_WARPS + w) * DESC_PER_WARP; i0 < a.N; i0 += step) {
        const int i = i0 + grp;
        const bool valid = i < a.N;
        float G[16];
        desc_group<DESC_GROUP>(a, c, i, valid, ndg, gl, gmask, below, G);
        if (valid && gl == 0) {
            float4 *o = reinterpret_cast<float4 *>(a.G + (size_t)i * 16);
            o[0] = make_float4(G[0], G[1], G[2], G[3]);
            o[1] = make_float4(G[4], G[5], G[6], G[7]);
            o[2] = make_float4(G[8], G[9], G[10], G[11]);
            o[3] = make_float4(G[12], G[13], G[14], G[15]);
        }
        __syncwarp();
    }
}

__device__ __forceinline__ void load16(const float *p, float e[16])
{
    const float4 *q = reinterpret_cast<const float4 *>(p);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        float4 v = __ldg(q + k);
        e[4 * k] = v.x;
        e[4 * k + 1] = v.y;
        e[4 * k + 2] = v.z;
        e[4 * k + 3] = v.w;
    }
}

// The queued triplets: centred on atom k (legs s and t of its list;
// F += sum_m e_km (dt/du + dt/dw)), or centred on neighbor j = s with k as a
// leg (t == BP_LEG; the leg from j to k is -u, the other leg w' from j;
// F -= sum_m e_jm dt(-u, w')/d(-u)).  One code path with selected
// coefficients, so a group's mixed queue runs without divergence.  The G
// lanes of a group (lane gl of the group) evaluate its queue.
constexpr unsigned char BP_LEG = 0xff;
template <int G>
__device__ __forceinline__ void bp_queue_terms(const BpArgs &a, const BpConst &c, int k, const int *nj,
                                               const float4 *nd, const unsigned char *qs, const unsigned char *qk,
                                               const float4 *qw, int qn, int gl, float &fx, float &fy, float &fz)
{
    for (int q = gl; q < qn; q += G) {
        const int t = qk[q];
        const bool leg = t == BP_LEG;
        const float4 u = nd[qs[q]];
        const float4 wv = leg ? qw[q] : nd[t];
        const float sg = leg ? -1.0f : 1.0f;   // sign of the first leg and of its term
        const float cw = leg ? 0.0f : 1.0f;    // the second leg's gradient counts for centred triplets only
        const int src = leg ? nj[qs[q]] : k;   // whose dE/dG weights the term
        const float4 *ep = reinterpret_cast<const float4 *>(a.dEdG + (size_t)src * 16 + 8);
        const float4 e0 = __ldg(ep), e1 = __ldg(ep + 1);
        const float ej[8] = {e0.x, e0.y, e0.z, e0.w, e1.x, e1.y, e1.z, e1.w};
        float gu[3], gw[3];
        angular_grad(c, sg * u.x, sg * u.y, sg * u.z, u.w, wv.x, wv.y, wv.z, wv.w, ej, gu, gw);
        fx += sg * gu[0] + cw * gw[0];
        fy += sg * gu[1] + cw * gw[1];
        fz += sg * gu[2] + cw * gw[2];
    }
}

constexpr int BPF_G = 8;                   // lanes per atom of the force gather
constexpr int BPF_PER_WARP = 32 / BPF_G;   // atoms per warp
constexpr int BPF_MAXN = BP_MAXN;          // partners inside R_c kept per atom (more: overflow)
constexpr int BPF_QG = 24;                 // queued triplets per atom between evaluations

// Force gather with BPF_G lanes per atom, BPF_PER_WARP atoms per warp (a
// silicon atom has about five partners inside R_c).  Every lane of a warp
// runs every trip of every loop (group ballots, scans and sums are
// warp-wide); a queue is evaluated when any group's would overflow.
// LISTS 1: the partners come from the lists k_bp_desc stored (this atom's
// and its neighbors'); LISTS 0: from the neighbor rows, tested here.
template <int KICK, int LISTS>
__global__ void __launch_bounds__(BP_WARPS * 32, 4) k_bp_force(BpArgs a)
{
    count_launch();
    __shared__ int nj[BP_WARPS][BPF_PER_WARP][BPF_MAXN];
    __shared__ float4 nd[BP_WARPS][BPF_PER_WARP][BPF_MAXN];
    __shared__ int qpre[BP_WARPS][BPF_PER_WARP][BPF_MAXN + 1];   // neighbors' row offsets in the candidate sweep
    __shared__ unsigned char qs[BP_WARPS][BPF_PER_WARP][BPF_QG];   // queued triplets: first leg
    __shared__ unsigned char qk[BP_WARPS][BPF_PER_WARP][BPF_QG];   // ... second leg of a centred triplet, or BP_LEG
    __shared__ float4 qw[BP_WARPS][BPF_PER_WARP][BPF_QG];          // ... and the other leg (w', |w'|) of a leg triplet
    const BpConst c = bp_const();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int grp = lane / BPF_G, gl = lane % BPF_G;
    const unsigned gmask = ((1u << BPF_G) - 1u) << (grp * BPF_G);
    const unsigned below = (1u << lane) - 1u;
    int *njg = nj[w][grp];
    float4 *ndg = nd[w][grp];
    int *qp = qpre[w][grp];
    unsigned char *qsg = qs[w][grp], *qkg = qk[w][grp];
    float4 *qwg = qw[w][grp];
    float pe_acc = 0.0f, ke_acc = 0.0f;
    const int step = gridDim.x * BP_WARPS * BPF_PER_WARP;
    for (int k0 = (blockIdx.x * BP_WARPS + w) * BPF_PER_WARP; k0 < a.N; k0 += step) {
        const int k = k0 + grp;
        const bool valid = k < a.N;
        const float4 rk = valid ? a.r[k] : make_float4(0.f, 0.f, 0.f, 0.f);
        int n = 0, base = 0;
        const int32_t *row = a.nbr + (size_t)(valid ? k : 0) * a.cap;
        if (valid) {
            n = min(a.cnt[k], a.cap);
            base = a.sys_n ? (k / a.sys_n) * a.sys_n : 0;
        }
        // partners inside R_c, compacted into the group's list
        const int nmax = LISTS ? 0 : __reduce_max_sync(0xffffffffu, n);
        int m = 0;
        if (LISTS) {
            if (valid) m = a.pa.tb_cnt[k];
            for (int s = gl; s < m; s += BPF_G) {
                njg[s] = a.pa.tb_idx[(size_t)k * BP_MAXN + s];
                ndg[s] = a.pa.tb_vec[(size_t)k * BP_MAXN + s];
            }
        }
        for (int c0 = 0; c0 < nmax; c0 += BPF_G) {
            const int kk = c0 + gl;
            bool in = false;
            int j = 0;
            float dx = 0.f, dy = 0.f, dz = 0.f, r2 = 0.f;
            if (kk < n) {
                j = row[kk] + base;
                const float4 rj = __ldg(a.r + j);
                r2 = dist2_rn<3>(rj, rk, a.box, dx, dy, dz);
                in = r2 < c.rc2;
            }
            const unsigned mk = __ballot_sync(0xffffffffu, in) & gmask;
            const int pos = m + __popc(mk & below);
            if (in && pos < BPF_MAXN) {
                njg[pos] = j;
                ndg[pos] = make_float4(dx, dy, dz, sqrtf(r2));
            }
            m += __popc(mk);
        }
        if (m > BPF_MAXN) {
            if (gl == 0) raise_status(a.status, MD_ERR_NBR_OVERFLOW);
            m = BPF_MAXN;
        }
        __syncwarp();
        float fx = 0.f, fy = 0.f, fz = 0.f;
        // self radial + the neighbor's radial term of the same pair:
        // both give (e_km + e_jm) g'_m(r) u/r with u = r_j - r_k
        const int mmax = __reduce_max_sync(0xffffffffu, m);
        for (int s0 = 0; s0 < mmax; s0 += BPF_G) {
            const int s = s0 + gl;
            if (s < m) {
                const float4 u = ndg[s];
                float ek[16], ej[16];
                load16(a.dEdG + (size_t)k * 16, ek);
                load16(a.dEdG + (size_t)njg[s] * 16, ej);
                float g[8], dg[8];
                radial8(c, u.w, g, dg);
                float sc = 0.0f;
#pragma unroll
                for (int q = 0; q < 8; ++q) sc += (ek[q] + ej[q]) * dg[q];
                sc /= u.w;
                fx += sc * u.x;
                fy += sc * u.y;
                fz += sc * u.z;
            }
        }
        // triplets centred on k: F_k += sum_m e_km (dt/du + dt/dw), and
        // triplets centred on neighbor j with k as leg u' = r_k - r_j:
        // F_k -= sum_m e_jm dt(u', w')/du', w' = r_l - r_j, l in N(j), l != k.
        // Both kinds go into the group's shared-memory queue, evaluated with
        // every lane busy: the centred pairs (s1 < s2) first, then the leg
        // candidates (s, l) of all neighbors' rows, swept BPF_G per step,
        // those inside R_c queued with w'.
        int qn = 0;
        auto enqueue = [&](bool in, int q1, int q2, float4 wv) {
            const unsigned mk = __ballot_sync(0xffffffffu, in) & gmask;
            if (__any_sync(0xffffffffu, qn + __popc(mk) > BPF_QG)) {   // some group full: evaluate every queue
                __syncwarp();
                bp_queue_terms<BPF_G>(a, c, k, njg, ndg, qsg, qkg, qwg, qn, gl, fx, fy, fz);
                __syncwarp();
                qn = 0;
            }
            const int pos = qn + __popc(mk & below);
            if (in) {
                qsg[pos] = (unsigned char)q1;
                qkg[pos] = (unsigned char)q2;
                qwg[pos] = wv;
            }
            qn += __popc(mk);
        };
        const int nt = m * (m - 1) / 2;
        const int ntmax = __reduce_max_sync(0xffffffffu, nt);
        for (int t0 = 0; t0 < ntmax; t0 += BPF_G) {
            int t = t0 + gl, s1 = 0;
            const bool in = t < nt;
            if (in)
                while (t >= m - 1 - s1) {   // pair t of (s1 < s2) in row-major order
                    t -= m - 1 - s1;
                    ++s1;
                }
            enqueue(in, s1, s1 + 1 + t, make_float4(0.f, 0.f, 0.f, 0.f));
        }
        int tot = 0;
        for (int s0 = 0; s0 < mmax; s0 += BPF_G) {   // exclusive prefix of the neighbors' row lengths
            const int s = s0 + gl;
            int nn = 0;
            if (s < m) nn = LISTS ? a.pa.tb_cnt[njg[s]] : min(a.cnt[njg[s]], a.cap);
            int incl = nn;
#pragma unroll
            for (int o = 1; o < BPF_G; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, o, BPF_G);
                if (gl >= o) incl += y;
            }
            if (s < m) qp[s] = tot + incl - nn;
            tot += __shfl_sync(0xffffffffu, incl, BPF_G - 1, BPF_G);
        }
        if (gl == 0) qp[m] = tot;
        __syncwarp();
        const int totmax = __reduce_max_sync(0xffffffffu, tot);
        for (int b0 = 0; b0 < totmax; b0 += BPF_G) {
            const int it = b0 + gl;
            bool in = false;
            int s = 0;
            float4 wv = make_float4(0.f, 0.f, 0.f, 0.f);
            if (it < tot) {
                int lo = 0, hi = m - 1;   // last s with qpre[s] <= it
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (qp[mid] <= it) lo = mid;
                    else hi = mid - 1;
                }
                s = lo;
                const int j = njg[s];
                if (LISTS) {
                    // j's partner inside R_c, with w' = r_l - r_j as k_bp_desc computed it
                    const size_t e = (size_t)j * BP_MAXN + (it - qp[s]);
                    if (a.pa.tb_idx[e] != k) {
                        wv = a.pa.tb_vec[e];
                        in = true;
                    }
                } else {
                    const int basej = a.sys_n ? (j / a.sys_n) * a.sys_n : 0;
                    const int l = a.nbr[(size_t)j * a.cap + (it - qp[s])] + basej;
                    if (l != k) {
                        const float4 rj = __ldg(a.r + j), rl = __ldg(a.r + l);
                        float wx, wy, wz;
                        const float w2 = dist2_rn<3>(rl, rj, a.box, wx, wy, wz);
                        in = w2 < c.rc2;
                        wv = make_float4(wx, wy, wz, sqrtf(w2));
                    }
                }
            }
            enqueue(in, s, BP_LEG, wv);
        }
        __syncwarp();
        bp_queue_terms<BPF_G>(a, c, k, njg, ndg, qsg, qkg, qwg, qn, gl, fx, fy, fz);
#pragma unroll
        for (int o = BPF_G / 2; o > 0; o >>= 1) {
            fx += __shfl_xor_sync(0xffffffffu, fx, o);
            fy += __shfl_xor_sync(0xffffffffu, fy, o);
            fz += __shfl_xor_sync(0xffffffffu, fz, o);
        }
        if (valid && gl == 0) {
            const float ei = a.Ei ? a.Ei[k] : 0.0f;
            a.pa.f[k] = make_float4(fx, fy, fz, ei);
            pe_acc += ei;
            if (KICK) {
                float4 v = a.pa.v[k];
                v.x += a.pa.half_dt_over_m * fx;
                v.y += a.pa.half_dt_over_m * fy;
                v.z += a.pa.half_dt_over_m * fz;
                a.pa.v[k] = v;
                ke_acc += 0.5f * a.pa.mass * (v.x * v.x + v.y * v.y + v.z * v.z);
            }
        }
        __syncwarp();
    }
    if (!a.pa.E_out && !KICK) return;
    energy_epilogue(pe_acc, ke_acc, a.pa);
}

// v_im = sum over atom i's pairs and triplets of dG_im/dr . dF (dF [N][4]).
__global__ void __launch_bounds__(BP_WARPS * 32) k_bp_jvp(BpArgs a)
{
    count_launch();
    __shared__ int nj[BP_WARPS][BP_MAXN];
    __shared__ float4 nd[BP_WARPS][BP_MAXN];
    const BpConst c = bp_const();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = blockIdx.x * BP_WARPS + w; i < a.N; i += gridDim.x * BP_WARPS) {
        const float4 ri = a.r[i];
        const int m = gather_within(a, c, i, ri, nj[w], nd[w]);
        const float4 dFi = a.dF[i];
        float v[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) v[q] = 0.0f;
        for (int s = lane; s < m; s += 32) {
            float4 u = nd[w][s];
            float4 dFj = a.dF[nj[w][s]];
            float g[8], dg[8];
            radial8(c, u.w, g, dg);
            float p = ((dFj.x - dFi.x) * u.x + (dFj.y - dFi.y) * u.y + (dFj.z - dFi.z) * u.z) / u.w;
#pragma unroll
            for (int q = 0; q < 8; ++q) v[q] += dg[q] * p;
        }
        for (int t = lane; t < m * m; t += 32) {
            int s1 = t / m, s2 = t - s1 * m;
            if (s1 >= s2) continue;
            float4 u = nd[w][s1], vv = nd[w][s2];
            float4 dFj = a.dF[nj[w][s1]], dFl = a.dF[nj[w][s2]];
            float ax = dFj.x - dFi.x, ay = dFj.y - dFi.y, az = dFj.z - dFi.z;
            float bx = dFl.x - dFi.x, by = dFl.y - dFi.y, bz = dFl.z - dFi.z;
            angular_dir(c, u.x, u.y, u.z, u.w, vv.x, vv.y, vv.z, vv.w, ax, ay, az, bx, by, bz, v + 8);
        }
#pragma unroll
        for (int q = 0; q < 16; ++q) v[q] = warp_sum(v[q]);
        if (lane == 0) {
            float4 *o = reinterpret_cast<float4 *>(a.V + (size_t)i * 16);
            o[0] = make_float4(v[0], v[1], v[2], v[3]);
            o[1] = make_float4(v[4], v[5], v[6], v[7]);
            o[2] = make_float4(v[8], v[9], v[10], v[11]);
            o[3] = make_float4(v[12], v[13], v[14], v[15]);
        }
        __syncwarp();
    }
}

static int bp_grid(int N)
{
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms < 1) sms = 1;
    }
    int groups = (N + BP_WARPS - 1) / BP_WARPS;
    int g = sms * 8;
    return groups < g ? groups : g;
}

void enqueue_bp_desc(const BpArgs &a, cudaStream_t st)
{
    k_bp_desc<<<bp_grid((a.N + DESC_PER_WARP - 1) / DESC_PER_WARP), BP_WARPS * 32, 0, st>>>(a);
}

void enqueue_bp_force(const BpArgs &a, int kick, cudaStream_t st)
{
    const int g = bp_grid((a.N + BPF_PER_WARP - 1) / BPF_PER_WARP);
    if (a.pa.tb_cnt) {
        if (kick) k_bp_force<1, 1><<<g, BP_WARPS * 32, 0, st>>>(a);
        else k_bp_force<0, 1><<<g, BP_WARPS * 32, 0, st>>>(a);
    } else {
        if (kick) k_bp_force<1, 0><<<g, BP_WARPS * 32, 0, st>>>(a);
        else k_bp_force<0, 0><<<g, BP_WARPS * 32, 0, st>>>(a);
    }
}

void enqueue_bp_jvp(const BpArgs &a, cudaStream_t st) { k_bp_jvp<<<bp_grid(a.N), BP_WARPS * 32, 0, st>>>(a); }

void enqueue_mlp_infer(const float *P, const float *norm, const float *G, int N, float *Ei, float *dEdG,
                       cudaStream_t st);
void enqueue_mlp_infer_tc(const float *P, const float *norm, const float *G, int N, float *Ei, float *dEdG,
                          uint32_t *status, cudaStream_t st);

static int g_bp_tc = 0;   // 1: network on the tensor cores (BF16), 0: FP32 CUDA cores
int bp_variant() { return g_bp_tc; }

static BpArgs bp_args_from(const PairArgs &pa)
{
    BpArgs b;
    memset(&b, 0, sizeof(b));
    b.box = pa.box;
    b.N = pa.N;
    b.cap = pa.cap;
    b.sys_n = pa.bp_sys_n;
    b.r = pa.r;
    b.nbr = pa.nbr;
    b.cnt = pa.cnt;
    b.G = pa.bp_G;
    b.dEdG = pa.bp_dEdG;
    b.Ei = pa.bp_Ei;
    b.status = pa.status;
    b.pa = pa;
    return b;
}

// Learned-potential forces: descriptors, network (energy and input
// gradient), force gather (with the closing kick when asked).  On the
// tensor cores the descriptors are computed inside the network kernel (one
// launch, no round trip of G through memory); the FP32 network keeps the
// separate descriptor kernel.
void enqueue_bp_step(const PairArgs &pa, int kick, cudaStream_t st)
{
    BpArgs b = bp_args_from(pa);
    if (g_bp_tc) {
        enqueue_bp_desc_mlp_tc(b, pa.bp_params, pa.bp_norm, pa.bp_Ei, pa.bp_dEdG, pa.status, st);
    } else {
        enqueue_bp_desc(b, st);
        enqueue_mlp_infer(pa.bp_params, pa.bp_norm, pa.bp_G, pa.N, pa.bp_Ei, pa.bp_dEdG, st);
    }
    enqueue_bp_force(b, kick, st);
}

static bool bp_list_ok(const md_space *s, const md_nbr *nb)
{
    return s && nb && s->dim == 3 && nb->dim == 3 && nb->nbr && nb->cnt && nb->r_list >= BP_RC;
}

static BpArgs bp_plain(const md_space *s, const float *d_r, const md_nbr *nb, int sys_n, uint32_t *d_status)
{
    BpArgs b;
    memset(&b, 0, sizeof(b));
    b.box = make_box(s);
    b.N = nb->N;
    b.cap = nb->cap;
    b.sys_n = sys_n;
    b.r = (const float4 *)d_r;
    b.nbr = nb->nbr;
    b.cnt = nb->cnt;
    b.status = d_status;
    return b;
}

}  // namespace jmd

using namespace jmd;

extern "C" md_status md_bp_set_tensor_cores(int on)
{
    g_bp_tc = on ? 1 : 0;
    return MD_OK;
}

extern "C" md_status md_bp_descriptors(const md_space *s, const float *d_r, const md_nbr *nb, int sys_n, float *d_G,
                                       uint32_t *d_status, md_stream_t stream)
{
    if (!bp_list_ok(s, nb) || !d_r || !d_G || sys_n < 0) return MD_ERR_INVALID;
    BpArgs b = bp_plain(s, d_r, nb, sys_n, d_status);
    b.G = d_G;
    enqueue_bp_desc(b, (cudaStream_t)stream);
    JMD_CUDA_TRY(cudaGetLastError());
    return MD_OK;
}

extern "C" md_status md_bp_forces(const md_space *s, const float *d_r, const md_nbr *nb, int sys_n,
                                  const float *d_dEdG, const float *d_Ei, float *d_f, double *d_E, uint32_t *d_status,
                                  md_stream_t stream)
{
    if (!bp_list_ok(s, nb) || !d_r || !d_dEdG || !d_f || sys_n < 0 || !nb->ws) return MD_ERR_INVALID;
    if (d_E && !d_Ei) return MD_ERR_INVALID;
    BpArgs b = bp_plain(s, d_r, nb, sys_n, d_status);
    b.dEdG = d_dEdG;
    b.Ei = d_Ei;
    WsPtrs w = ws_ptrs(nb);
    b.pa.f = (float4 *)d_f;
    b.pa.E_out = d_E;
    b.pa.ctl = w.ctl;
    b.pa.partials = w.partials;
    b.pa.status = d_status;
    if (d_E && bp_grid(nb->N) > w.max_blocks) return MD_ERR_INVALID;   // reduction partials
    enqueue_bp_force(b, 0, (cudaStream_t)stream);
    JMD_CUDA_TRY(cudaGetLastError());
    return MD_OK;
}

extern "C" md_status md_bp_jvp(const md_space *s, const float *d_r, const md_nbr *nb, int sys_n, const float *d_dF,
                               float *d_V, uint32_t *d_status, md_stream_t stream)
{
    if (!bp_list_ok(s, nb) || !d_r || !d_dF || !d_V || sys_n < 0) return MD_ERR_INVALID;
    BpArgs b = bp_plain(s, d_r, nb, sys_n, d_status);
    b.dF = (const float4 *)d_dF;
    b.V = d_V;
    enqueue_bp_jvp(b, (cudaStream_t)stream);
    JMD_CUDA_TRY(cudaGetLastError());
    return MD_OK;
}
