// sw.cu -- Stillinger-Weber forces (Sec. 3.3.2; form of Stillinger & Weber 1985):
//   E = sum_{i<j} phi2(r_ij) + sum_i sum_{j<k in N(i)} phi3(r_ij, r_ik, theta_jik)
//   phi2(r) = A eps [B (sigma/r)^p - (sigma/r)^q] exp(sigma/(r - a sigma))
//   phi3    = lambda eps (cos theta - cos0)^2 g(r_ij) g(r_ik),
//   g(r)    = exp(gamma sigma / (r - a sigma)),      all for r < a sigma.
//
// Gather form, eight lanes per atom i (four atoms per warp), no atomics.
// F_i collects
//   (1) the two-body terms of every neighbor j,
//   (2) the triplets centred on i (legs j < k of i's neighbors), and
//   (3) the triplets centred on each neighbor j in which i is a leg
//       (the other leg k runs over j's row); the triplets of (2) and the
//       candidates of (3) inside a*sigma are queued in shared memory first
//       and then evaluated together with every lane busy.
// e_i = 1/2 sum_j phi2(r_ij) + sum_{j<k} phi3(i; j, k), so sum_i e_i = E.
// With partner-list scratch (md_sw_lists_bytes), k_sw_lists first stores
// every atom's partners inside a*sigma (index, r_j - r_i and the one-leg
// factors g, g', 1/r, in row order) and its two-body terms, and k_sw_pl
// takes the triplets from those lists: for (3) it visits only the
// neighbors' partners inside a*sigma instead of testing their whole rows
// (about a third of the entries in silicon at 1000 K and a 0.3 A skin), and
// no triplet recomputes an exponential or a division of its legs.
#include "common.cuh"
#include "kernels.cuh"
#include "reduce.cuh"

namespace jmd {

constexpr int SW_MAXN = SW_LIST_SLOTS;   // neighbors inside a*sigma kept per atom
constexpr int SW_WARPS = 8;

struct SwP {
    float eps, sg, rc, lam, gam, A, B, p, q, c0, rc2;
};

__device__ __forceinline__ SwP sw_params(const PairArgs &a)
{
    SwP P;
    P.eps = a.sw[0];
    P.sg = a.sw[1];
    P.lam = a.sw[3];
    P.gam = a.sw[4];
    P.A = a.sw[5];
    P.B = a.sw[6];
    P.p = a.sw[7];
    P.q = a.sw[8];
    P.c0 = a.sw[9];
    P.rc = a.sw[10];
    P.rc2 = a.sw[11];
    return P;
}

// phi2 and its derivative d phi2 / dr (r < rc)
__device__ __forceinline__ float sw_phi2(const SwP &P, float r, float &dphi)
{
    float sr = P.sg / r;
    float srp = __powf(sr, P.p), srq = __powf(sr, P.q);
    float bra = P.B * srp - srq;
    float dbra = (-P.p * P.B * srp + P.q * srq) / r;
    float x = r - P.rc;
    float ex = expf(P.sg / x);
    float dex = ex * (-P.sg / (x * x));
    dphi = P.A * P.eps * (dbra * ex + bra * dex);
    return P.A * P.eps * bra * ex;
}

// g(r) = exp(gamma sigma / (r - rc)) and g'(r)
__device__ __forceinline__ float sw_g(const SwP &P, float r, float &dg)
{
    float x = r - P.rc;
    float v = expf(P.gam * P.sg / x);
    dg = v * (-P.gam * P.sg / (x * x));
    return v;
}

// Triplet with centre c, legs u = r_a - r_c and w = r_b - r_c (|u|, |w| < rc).
// Returns h and its gradients with respect to u and w.
__device__ __forceinline__ float sw_triplet(const SwP &P, float ux, float uy, float uz, float ru, float wx, float wy,
                                            float wz, float rw, float gu[3], float gw[3])
{
    float iu = 1.0f / ru, iw = 1.0f / rw;
    float c = (ux * wx + uy * wy + uz * wz) * iu * iw;
    float dgu, dgw;
    float g1 = sw_g(P, ru, dgu), g2 = sw_g(P, rw, dgw);
    float cc = c - P.c0;
    float le = P.lam * P.eps;
    float h = le * cc * cc * g1 * g2;
    float dh_dc = 2.0f * le * cc * g1 * g2;
    float dh_dru = le * cc * cc * dgu * g2;
    float dh_drw = le * cc * cc * g1 * dgw;
    float uu[3] = {ux, uy, uz}, ww[3] = {wx, wy, wz};
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        float dc_du = ww[q] * iu * iw - c * uu[q] * iu * iu;
        float dc_dw = uu[q] * iu * iw - c * ww[q] * iw * iw;
        gu[q] = dh_dc * dc_du + dh_dru * uu[q] * iu;
        gw[q] = dh_dc * dc_dw + dh_drw * ww[q] * iw;
    }
    return h;
}

// The queued triplets: centred on the atom (legs s and k of its list:
// F += dh/du + dh/dw, e += h), or centred on neighbor s with the atom as a
// leg (k == SW_LEG; the leg from s to the atom is -u, the other leg w' from
// s: F -= dh(-u, w')/d(-u)).  One code path with selected coefficients, so
// a group's mixed queue runs without divergence.  The G lanes of a group
// (lane gl of the group) evaluate its queue.
constexpr unsigned char SW_LEG = 0xff;
template <int G>
__device__ __forceinline__ void sw_queue_terms(const SwP &P, const float4 *nd, const unsigned char *qs,
                                               const unsigned char *qk, const float4 *qw, int qn, int gl, float &fx,
                                               float &fy, float &fz, float &e)
{
    for (int q = gl; q < qn; q += G) {
        const int k = qk[q];
        const bool leg = k == SW_LEG;
        const float4 a = nd[qs[q]];
        const float4 b = leg ? qw[q] : nd[k];
        const float sg = leg ? -1.0f : 1.0f;
        float gu[3], gw[3];
        const float h = sw_triplet(P, sg * a.x, sg * a.y, sg * a.z, a.w, b.x, b.y, b.z, b.w, gu, gw);
        const float cw = leg ? 0.0f : 1.0f;
        fx += sg * gu[0] + cw * gw[0];
        fy += sg * gu[1] + cw * gw[1];
        fz += sg * gu[2] + cw * gw[2];
        e += cw * h;
    }
}

constexpr int SW_G = 8;                  // lanes per atom
constexpr int SW_PER_WARP = 32 / SW_G;   // atoms per warp
constexpr int SW_QG = 32;                // queued triplets per atom between evaluations

// One group of SW_G lanes per atom, SW_PER_WARP atoms per warp (a silicon
// atom has about five partners inside a*sigma).  Every lane of a warp runs
// every trip of every loop (group ballots, scans and sums are warp-wide);
// a queue is evaluated when any group's would overflow.
// Two-kernel form, pass 1: the atom's row entries inside a*sigma, compacted
// by a group ballot in row order, each with its vector u = r_j - r_i and r,
// and with the one-leg factors of every triplet that has this leg: g(r),
// g'(r) and 1/r; and the atom's two-body force and energy.
__global__ void __launch_bounds__(SW_WARPS * 32) k_sw_lists(PairArgs a)
{
    count_launch();
    const SwP P = sw_params(a);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int grp = lane / SW_G, gl = lane % SW_G;
    const unsigned gmask = ((1u << SW_G) - 1u) << (grp * SW_G);
    const unsigned below = (1u << lane) - 1u;
    const int step = gridDim.x * SW_WARPS * SW_PER_WARP;
    for (int i0 = (blockIdx.x * SW_WARPS + w) * SW_PER_WARP; i0 < a.N; i0 += step) {
        const int i = i0 + grp;
        const bool valid = i < a.N;
        const float4 ri = valid ? a.r[i] : make_float4(0.f, 0.f, 0.f, 0.f);
        int n = 0;
        const int32_t *row = a.nbr + (size_t)(valid ? i : 0) * a.cap;
        if (valid) n = min(a.cnt[i], a.cap);
        const size_t o = (size_t)(valid ? i : 0) * SW_MAXN;
        const int nmax = __reduce_max_sync(0xffffffffu, n);
        int m = 0;
        float fx = 0.f, fy = 0.f, fz = 0.f, e = 0.f;
        for (int k0 = 0; k0 < nmax; k0 += SW_G) {
            const int k = k0 + gl;
            bool in = false;
            int j = 0;
            float dx = 0.f, dy = 0.f, dz = 0.f, r2 = 0.f;
            if (k < n) {
                j = row[k];
                const float4 rj = __ldg(a.r + j);
                r2 = dist2_rn<3>(rj, ri, a.box, dx, dy, dz);   // u = r_j - r_i
                in = r2 < P.rc2;
            }
            const unsigned mk = __ballot_sync(0xffffffffu, in) & gmask;
            const int pos = m + __popc(mk & below);
            if (in) {
                const float r = sqrtf(r2);
                float dphi, dg;
                const float ph = sw_phi2(P, r, dphi);
                const float fr = dphi / r;
                fx += fr * dx;
                fy += fr * dy;
                fz += fr * dz;
                e += 0.5f * ph;
                if (pos < SW_MAXN) {
                    const float g = sw_g(P, r, dg);
                    a.tb_idx[o + pos] = j;
                    a.tb_vec[o + pos] = make_float4(dx, dy, dz, r);
                    a.tb_aux[o + pos] = make_float4(g, dg, 1.0f / r, 0.f);
                }
            }
            m += __popc(mk);
        }
#pragma unroll
        for (int q = SW_G / 2; q > 0; q >>= 1) {
            fx += __shfl_xor_sync(0xffffffffu, fx, q);
            fy += __shfl_xor_sync(0xffffffffu, fy, q);
            fz += __shfl_xor_sync(0xffffffffu, fz, q);
            e += __shfl_xor_sync(0xffffffffu, e, q);
        }
        if (valid && gl == 0) {
            if (m > SW_MAXN) raise_status(a.status, MD_ERR_NBR_OVERFLOW);
            a.tb_cnt[i] = min(m, SW_MAXN);
            a.tb_f2[i] = make_float4(fx, fy, fz, e);
        }
    }
}

// The triplet of sw_triplet with its one-leg factors given: g, g' and 1/r
// of each leg (k_sw_lists computed them with the same expressions, so every
// value is the one sw_triplet computes, bit for bit).
__device__ __forceinline__ float sw_triplet_pre(const SwP &P, float ux, float uy, float uz, float iu, float g1,
                                                float dgu, float wx, float wy, float wz, float iw, float g2, float dgw,
                                                float gu[3], float gw[3])
{
    float c = (ux * wx + uy * wy + uz * wz) * iu * iw;
    float cc = c - P.c0;
    float le = P.lam * P.eps;
    float h = le * cc * cc * g1 * g2;
    float dh_dc = 2.0f * le * cc * g1 * g2;
    float dh_dru = le * cc * cc * dgu * g2;
    float dh_drw = le * cc * cc * g1 * dgw;
    float uu[3] = {ux, uy, uz}, ww[3] = {wx, wy, wz};
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        float dc_du = ww[q] * iu * iw - c * uu[q] * iu * iu;
        float dc_dw = uu[q] * iu * iw - c * ww[q] * iw * iw;
        gu[q] = dh_dc * dc_du + dh_dru * uu[q] * iu;
        gw[q] = dh_dc * dc_dw + dh_drw * ww[q] * iw;
    }
    return h;
}

// Two-kernel form, pass 2: the triplets, from the stored lists.  Centred
// triplets take both legs from the atom's own list; a triplet centred on
// neighbor j with the atom as a leg takes the other leg from j's list
// (queued as its list entry).  The two-body part comes from pass 1.
constexpr int SWL_QG = 32;   // queued triplets per atom between evaluations

template <int KICK>
__global__ void __launch_bounds__(SW_WARPS * 32, 4) k_sw_pl(PairArgs a)
{
    count_launch();
    __shared__ int nj[SW_WARPS][SW_PER_WARP][SW_MAXN];
    __shared__ float4 nd[SW_WARPS][SW_PER_WARP][SW_MAXN];    // (ux, uy, uz, r)
    __shared__ float4 na[SW_WARPS][SW_PER_WARP][SW_MAXN];    // (g, g', 1/r)
    __shared__ int qpre[SW_WARPS][SW_PER_WARP][SW_MAXN + 1];
    __shared__ unsigned char qs[SW_WARPS][SW_PER_WARP][SWL_QG];   // first leg (own list)
    __shared__ unsigned char qk[SW_WARPS][SW_PER_WARP][SWL_QG];   // second leg (own list), or SW_LEG
    __shared__ int qe[SW_WARPS][SW_PER_WARP][SWL_QG];             // ... the other leg's list entry
    const SwP P = sw_params(a);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int grp = lane / SW_G, gl = lane % SW_G;
    const unsigned gmask = ((1u << SW_G) - 1u) << (grp * SW_G);
    const unsigned below = (1u << lane) - 1u;
    int *njg = nj[w][grp];
    float4 *ndg = nd[w][grp], *nag = na[w][grp];
    int *qp = qpre[w][grp];
    unsigned char *qsg = qs[w][grp], *qkg = qk[w][grp];
    int *qeg = qe[w][grp];
    float pe_acc = 0.0f, ke_acc = 0.0f;
    auto terms = [&](int qn, float &fx, float &fy, float &fz, float &e) {
        for (int q = gl; q < qn; q += SW_G) {
            const int k = qkg[q];
            const bool leg = k == SW_LEG;
            const float4 u = ndg[qsg[q]], ua = nag[qsg[q]];
            const float4 v = leg ? a.tb_vec[qeg[q]] : ndg[k];
            const float4 va = leg ? a.tb_aux[qeg[q]] : nag[k];
            const float sg = leg ? -1.0f : 1.0f;
            float gu[3], gw[3];
            const float h = sw_triplet_pre(P, sg * u.x, sg * u.y, sg * u.z, ua.z, ua.x, ua.y, v.x, v.y, v.z, va.z, va.x,
                                           va.y, gu, gw);
            const float cw = leg ? 0.0f : 1.0f;
            fx += sg * gu[0] + cw * gw[0];
            fy += sg * gu[1] + cw * gw[1];
            fz += sg * gu[2] + cw * gw[2];
            e += cw * h;
        }
    };
    const int step = gridDim.x * SW_WARPS * SW_PER_WARP;
    for (int i0 = (blockIdx.x * SW_WARPS + w) * SW_PER_WARP; i0 < a.N; i0 += step) {
        const int i = i0 + grp;
        const bool valid = i < a.N;
        const int m = valid ? a.tb_cnt[i] : 0;
        for (int s = gl; s < m; s += SW_G) {
            const size_t o = (size_t)i * SW_MAXN + s;
            njg[s] = a.tb_idx[o];
            ndg[s] = a.tb_vec[o];
            nag[s] = a.tb_aux[o];
        }
        __syncwarp();
        float fx = 0.f, fy = 0.f, fz = 0.f, e = 0.f;
        int qn = 0;
        auto enqueue = [&](bool in, int q1, int q2, int ge) {
            const unsigned mk = __ballot_sync(0xffffffffu, in) & gmask;
            if (__any_sync(0xffffffffu, qn + __popc(mk) > SWL_QG)) {   // some group full: evaluate every queue
                __syncwarp();
                terms(qn, fx, fy, fz, e);
                __syncwarp();
                qn = 0;
            }
            const int pos = qn + __popc(mk & below);
            if (in) {
                qsg[pos] = (unsigned char)q1;
                qkg[pos] = (unsigned char)q2;
                qeg[pos] = ge;
            }
            qn += __popc(mk);
        };
        // centred pairs (s1 < s2)
        const int nt = m * (m - 1) / 2;
        const int ntmax = __reduce_max_sync(0xffffffffu, nt);
        for (int t0 = 0; t0 < ntmax; t0 += SW_G) {
            int t = t0 + gl, s1 = 0;
            const bool in = t < nt;
            if (in)
                while (t >= m - 1 - s1) {   // pair t of (s1 < s2) in row-major order
                    t -= m - 1 - s1;
                    ++s1;
                }
            enqueue(in, s1, s1 + 1 + t, 0);
        }
        // the neighbors' partners other than this atom
        const int mmax = __reduce_max_sync(0xffffffffu, m);
        int tot = 0;
        for (int s0 = 0; s0 < mmax; s0 += SW_G) {   // exclusive prefix of the neighbors' list lengths
            const int s = s0 + gl;
            const int nn = s < m ? a.tb_cnt[njg[s]] : 0;
            int incl = nn;
#pragma unroll
            for (int o = 1; o < SW_G; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, o, SW_G);
                if (gl >= o) incl += y;
            }
            if (s < m) qp[s] = tot + incl - nn;
            tot += __shfl_sync(0xffffffffu, incl, SW_G - 1, SW_G);
        }
        if (gl == 0) qp[m] = tot;
        __syncwarp();
        const int totmax = __reduce_max_sync(0xffffffffu, tot);
        for (int b0 = 0; b0 < totmax; b0 += SW_G) {
            const int it = b0 + gl;
            bool in = false;
            int s = 0, ge = 0;
            if (it < tot) {
                int lo = 0, hi = m - 1;   // last s with qpre[s] <= it
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (qp[mid] <= it) lo = mid;
                    else hi = mid - 1;
                }
                s = lo;
                ge = njg[s] * SW_MAXN + (it - qp[s]);
                in = a.tb_idx[ge] != i;
            }
            enqueue(in, s, SW_LEG, ge);
        }
        __syncwarp();
        terms(qn, fx, fy, fz, e);
#pragma unroll
        for (int o = SW_G / 2; o > 0; o >>= 1) {
            fx += __shfl_xor_sync(0xffffffffu, fx, o);
            fy += __shfl_xor_sync(0xffffffffu, fy, o);
            fz += __shfl_xor_sync(0xffffffffu, fz, o);
            e += __shfl_xor_sync(0xffffffffu, e, o);
        }
        if (valid && gl == 0) {
            const float4 f2 = a.tb_f2[i];   // two-body part
            fx += f2.x;
            fy += f2.y;
            fz += f2.z;
            e += f2.w;
            a.f[i] = make_float4(fx, fy, fz, e);
            pe_acc += e;
            if (KICK) ke_acc += half_kick<3>(a, i, fx, fy, fz);
        }
        __syncwarp();
    }
    if (!a.E_out && !KICK) return;
    energy_epilogue(pe_acc, ke_acc, a);
}

template <int KICK>
__global__ void __launch_bounds__(SW_WARPS * 32, 4) k_sw(PairArgs a)
{
    count_launch();
    __shared__ int nj[SW_WARPS][SW_PER_WARP][SW_MAXN];
    __shared__ float4 nd[SW_WARPS][SW_PER_WARP][SW_MAXN];   // (ux, uy, uz, r): u = r_j - r_i
    __shared__ int qpre[SW_WARPS][SW_PER_WARP][SW_MAXN + 1];     // neighbors' row offsets in the candidate sweep
    __shared__ unsigned char qs[SW_WARPS][SW_PER_WARP][SW_QG];   // queued triplets: first leg
    __shared__ unsigned char qk[SW_WARPS][SW_PER_WARP][SW_QG];   // ... second leg of a centred triplet, or SW_LEG
    __shared__ float4 qw[SW_WARPS][SW_PER_WARP][SW_QG];          // ... and the other leg (w', |w'|) of a leg triplet
    const SwP P = sw_params(a);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int grp = lane / SW_G, gl = lane % SW_G;
    const unsigned gmask = ((1u << SW_G) - 1u) << (grp * SW_G);
    const unsigned below = (1u << lane) - 1u;
    int *njg = nj[w][grp];
    float4 *ndg = nd[w][grp];
    int *qp = qpre[w][grp];
    unsigned char *qsg = qs[w][grp], *qkg = qk[w][grp];
    float4 *qwg = qw[w][grp];
    float pe_acc = 0.0f, ke_acc = 0.0f;
    const int step = gridDim.x * SW_WARPS * SW_PER_WARP;
    for (int i0 = (blockIdx.x * SW_WARPS + w) * SW_PER_WARP; i0 < a.N; i0 += step) {
        const int i = i0 + grp;
        const bool valid = i < a.N;
        const float4 ri = valid ? a.r[i] : make_float4(0.f, 0.f, 0.f, 0.f);
        int n = 0;
        const int32_t *row = a.nbr + (size_t)(valid ? i : 0) * a.cap;
        if (valid) n = min(a.cnt[i], a.cap);
        // (0) neighbors inside a*sigma, compacted into the group's list
        const int nmax = __reduce_max_sync(0xffffffffu, n);
        int m = 0;
        for (int k0 = 0; k0 < nmax; k0 += SW_G) {
            const int k = k0 + gl;
            bool in = false;
            int j = 0;
            float dx = 0.f, dy = 0.f, dz = 0.f, r2 = 0.f;
            if (k < n) {
                j = row[k];
                const float4 rj = __ldg(a.r + j);
                r2 = dist2_rn<3>(rj, ri, a.box, dx, dy, dz);   // u = r_j - r_i
                in = r2 < P.rc2;
            }
            const unsigned mk = __ballot_sync(0xffffffffu, in) & gmask;
            const int pos = m + __popc(mk & below);
            if (in && pos < SW_MAXN) {
                njg[pos] = j;
                ndg[pos] = make_float4(dx, dy, dz, sqrtf(r2));
            }
            m += __popc(mk);
        }
        if (m > SW_MAXN) {
            if (gl == 0) raise_status(a.status, MD_ERR_NBR_OVERFLOW);
            m = SW_MAXN;
        }
        __syncwarp();
        float fx = 0.f, fy = 0.f, fz = 0.f, e = 0.f;
        // (1) two-body: F_i += phi2'(r) u / r
        const int mmax = __reduce_max_sync(0xffffffffu, m);
        for (int s0 = 0; s0 < mmax; s0 += SW_G) {
            const int s = s0 + gl;
            if (s < m) {
                const float4 u = ndg[s];
                float dphi;
                const float ph = sw_phi2(P, u.w, dphi);
                const float fr = dphi / u.w;
                fx += fr * u.x;
                fy += fr * u.y;
                fz += fr * u.z;
                e += 0.5f * ph;
            }
        }
        // (2) triplets centred on i: F_i += dh/du + dh/dw, e += h, and
        // (3) triplets centred on neighbor j with i as a leg:
        //     u' = r_i - r_j = -u, w' = r_k - r_j; F_i -= dh/du'.
        // Both kinds go into the group's shared-memory queue, evaluated with
        // every lane busy: the centred pairs (s1 < s2) first, then the leg
        // candidates (s, k) of all neighbors' rows, swept SW_G per step,
        // those inside a*sigma queued with w'.
        int qn = 0;
        auto enqueue = [&](bool in, int q1, int q2, float4 wv) {
            const unsigned mk = __ballot_sync(0xffffffffu, in) & gmask;
            if (__any_sync(0xffffffffu, qn + __popc(mk) > SW_QG)) {   // some group full: evaluate every queue
                __syncwarp();
                sw_queue_terms<SW_G>(P, ndg, qsg, qkg, qwg, qn, gl, fx, fy, fz, e);
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
        for (int t0 = 0; t0 < ntmax; t0 += SW_G) {
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
        for (int s0 = 0; s0 < mmax; s0 += SW_G) {   // exclusive prefix of the neighbors' row lengths
            const int s = s0 + gl;
            int nn = 0;
            if (s < m) nn = min(a.cnt[njg[s]], a.cap);
            int incl = nn;
#pragma unroll
            for (int o = 1; o < SW_G; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, o, SW_G);
                if (gl >= o) incl += y;
            }
            if (s < m) qp[s] = tot + incl - nn;
            tot += __shfl_sync(0xffffffffu, incl, SW_G - 1, SW_G);
        }
        if (gl == 0) qp[m] = tot;
        __syncwarp();
        const int totmax = __reduce_max_sync(0xffffffffu, tot);
        for (int b0 = 0; b0 < totmax; b0 += SW_G) {
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
                const int kk = a.nbr[(size_t)j * a.cap + (it - qp[s])];
                if (kk != i) {
                    const float4 rj = __ldg(a.r + j), rk = __ldg(a.r + kk);
                    float wx, wy, wz;
                    const float w2 = dist2_rn<3>(rk, rj, a.box, wx, wy, wz);
                    in = w2 < P.rc2;
                    wv = make_float4(wx, wy, wz, sqrtf(w2));
                }
            }
            enqueue(in, s, SW_LEG, wv);
        }
        __syncwarp();
        sw_queue_terms<SW_G>(P, ndg, qsg, qkg, qwg, qn, gl, fx, fy, fz, e);
#pragma unroll
        for (int o = SW_G / 2; o > 0; o >>= 1) {
            fx += __shfl_xor_sync(0xffffffffu, fx, o);
            fy += __shfl_xor_sync(0xffffffffu, fy, o);
            fz += __shfl_xor_sync(0xffffffffu, fz, o);
            e += __shfl_xor_sync(0xffffffffu, e, o);
        }
        if (valid && gl == 0) {
            a.f[i] = make_float4(fx, fy, fz, e);
            pe_acc += e;
            if (KICK) ke_acc += half_kick<3>(a, i, fx, fy, fz);
        }
        __syncwarp();
    }
    if (!a.E_out && !KICK) return;
    energy_epilogue(pe_acc, ke_acc, a);
}

template <class K>
static int sw_grid(K kern, int N)
{
    int per_sm = 0, sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, SW_WARPS * 32, 0);
    if (per_sm < 1) per_sm = 1;
    if (sms < 1) sms = 1;
    int groups = (N + SW_WARPS * SW_PER_WARP - 1) / (SW_WARPS * SW_PER_WARP);
    int g = per_sm * sms;
    return groups < g ? groups : g;
}

template <class K>
static void launch_full(K kern, int &g_full, const PairArgs &a, cudaStream_t st)
{
    if (!g_full) g_full = sw_grid(kern, 1 << 30);   // resident CTAs of the whole GPU
    const int groups = (a.N + SW_WARPS * SW_PER_WARP - 1) / (SW_WARPS * SW_PER_WARP);
    kern<<<groups < g_full ? groups : g_full, SW_WARPS * 32, 0, st>>>(a);
}

void enqueue_sw(const PairArgs &a, int kick, cudaStream_t st)
{
    static int g0 = 0, g1 = 0, gl = 0, gp0 = 0, gp1 = 0;
    if (a.tb_cnt) {
        launch_full(k_sw_lists, gl, a, st);
        if (kick) launch_full(k_sw_pl<1>, gp1, a, st);
        else launch_full(k_sw_pl<0>, gp0, a, st);
    } else {
        if (kick) launch_full(k_sw<1>, g1, a, st);
        else launch_full(k_sw<0>, g0, a, st);
    }
}

size_t sw_lists_bytes(int N) { return tb_layout(N, SW_MAXN, true).bytes; }

}  // namespace jmd
