// bp_terms.cuh -- the Behler-Parrinello symmetry functions (Sec. 3.2.4,
// 4.1) as device code shared by the descriptor kernel (bp.cu) and the
// tensor-core network that computes its own tile's descriptors (mlp_tc.cu).
//
//   f_c(r) = (cos(pi r / R_c) + 1) / 2,  R_c = 3.77 A
//   radial   G_m  = sum_j exp(-eta_r (r_ij - R_m)^2) f_c(r_ij),   R_m = 2 + 0.25 (m-1), m = 1..8
//   angular  G_zl = 2^(1-z) sum_{j<k} (1 + l cos theta_jik)^z exp(-eta_a (r_ij^2 + r_ik^2)) f_c f_c,
//            z in {1, 2, 4, 16}, l in {+1, -1}
#pragma once

#include "bp.cuh"
#include "common.cuh"
#include "kernels.cuh"

namespace jmd {

constexpr int BP_MAXN = BP_LIST_SLOTS;   // neighbors inside R_c kept per atom

struct BpConst {
    float rc, rc2, eta_r, eta_a, pi_rc;
};

__device__ __forceinline__ BpConst bp_const()
{
    BpConst c;
    c.rc = BP_RC;
    c.rc2 = BP_RC * BP_RC;
    c.eta_r = BP_ETA_R;
    c.eta_a = BP_ETA_A;
    c.pi_rc = 3.14159265358979f / BP_RC;
    return c;
}

__device__ __forceinline__ void fcut(const BpConst &c, float r, float &f, float &df)
{
    float s, co;
    __sincosf(c.pi_rc * r, &s, &co);
    f = 0.5f * (co + 1.0f);
    df = -0.5f * c.pi_rc * s;
}

// radial g_m(r) and dg_m/dr for all 8 centres
__device__ __forceinline__ void radial8(const BpConst &c, float r, float g[8], float dg[8])
{
    float f, df;
    fcut(c, r, f, df);
#pragma unroll
    for (int m = 0; m < 8; ++m) {
        float x = r - (2.0f + 0.25f * m);
        float ex = __expf(-c.eta_r * x * x);
        g[m] = ex * f;
        dg[m] = ex * (df - 2.0f * c.eta_r * x * f);
    }
}

// q^(z-1) and q^z for z in {1, 2, 4, 16} (slot order z-major, l-minor
// handled by the caller)
__device__ __forceinline__ void powers(float q, float pz[4], float pzm1[4])
{
    float q2 = q * q, q4 = q2 * q2, q8 = q4 * q4;
    pz[0] = q;
    pzm1[0] = 1.0f;
    pz[1] = q2;
    pzm1[1] = q;
    pz[2] = q4;
    pzm1[2] = q2 * q;
    pz[3] = q8 * q8;
    pzm1[3] = q8 * q4 * q2 * q;
}

// Angular terms of one triplet (centre at the origin, legs u, w; |u|, |w| < R_c):
// t[8] in column order (z, l) = (1,+) (1,-) (2,+) (2,-) (4,+) ... ; when
// grad != 0 also dt/du, dt/dw for each of the 8 columns.
template <bool GRAD>
__device__ __forceinline__ void angular8(const BpConst &c, float ux, float uy, float uz, float ru, float wx, float wy,
                                         float wz, float rw, float t[8], float du[8][3], float dw[8][3])
{
    float iu = 1.0f / ru, iw = 1.0f / rw;
    float cs = (ux * wx + uy * wy + uz * wz) * iu * iw;
    float fu, dfu, fw, dfw;
    fcut(c, ru, fu, dfu);
    fcut(c, rw, fw, dfw);
    float ex = __expf(-c.eta_a * (ru * ru + rw * rw));
    float B = ex * fu * fw;
    // dB/du = B (-2 eta_a u) + ex dfu fw u/|u|
    float bu = -2.0f * c.eta_a * B + ex * dfu * fw * iu;
    float bw = -2.0f * c.eta_a * B + ex * fu * dfw * iw;
    float dcu[3], dcw[3];
    if (GRAD) {
        dcu[0] = wx * iu * iw - cs * ux * iu * iu;
        dcu[1] = wy * iu * iw - cs * uy * iu * iu;
        dcu[2] = wz * iu * iw - cs * uz * iu * iu;
        dcw[0] = ux * iu * iw - cs * wx * iw * iw;
        dcw[1] = uy * iu * iw - cs * wy * iw * iw;
        dcw[2] = uz * iu * iw - cs * wz * iw * iw;
    }
    const float zs[4] = {1.0f, 2.0f, 4.0f, 16.0f};
    const float pref[4] = {1.0f, 0.5f, 0.125f, 1.0f / 32768.0f};   // 2^(1 - z)
#pragma unroll
    for (int l = 0; l < 2; ++l) {
        float lam = l == 0 ? 1.0f : -1.0f;
        float q = 1.0f + lam * cs;
        float pz[4], pzm1[4];
        powers(q, pz, pzm1);
#pragma unroll
        for (int zi = 0; zi < 4; ++zi) {
            int col = 2 * zi + l;
            t[col] = pref[zi] * pz[zi] * B;
            if (GRAD) {
                float a = pref[zi] * zs[zi] * pzm1[zi] * lam * B;   // dt/dc
                float b = pref[zi] * pz[zi];                          // dt/dB
                du[col][0] = a * dcu[0] + b * bu * ux;
                du[col][1] = a * dcu[1] + b * bu * uy;
                du[col][2] = a * dcu[2] + b * bu * uz;
                dw[col][0] = a * dcw[0] + b * bw * wx;
                dw[col][1] = a * dcw[1] + b * bw * wy;
                dw[col][2] = a * dcw[2] + b * bw * wz;
            }
        }
    }
}

// Descriptors of atom i by the G lanes of one group (lane gl of the group;
// gmask the group's lanes, below the lanes before this one).  The group
// sweeps the atom's row G entries at a time and compacts the partners inside
// R_c (group ballot, row order) into ndg (BP_MAXN slots), storing them in the
// partner lists when the arguments carry them; then it takes the pairs and
// the triplets (s1 < s2, enumerated without the s1 >= s2 slots) over its
// lanes and sums the 16 descriptors over the group (every lane of the group
// ends with the sums).  Every lane of the warp must call it together (the
// trip counts are warp-wide maxima); atoms past the end pass valid = false.
template <int G>
__device__ __forceinline__ void desc_group(const BpArgs &a, const BpConst &c, int i, bool valid, float4 *ndg, int gl,
                                           unsigned gmask, unsigned below, float Gd[16])
{
    const float4 ri = valid ? a.r[i] : make_float4(0.f, 0.f, 0.f, 0.f);
    int n = 0;
    const int32_t *row = nullptr;
    int base = 0;
    if (valid) {
        n = min(a.cnt[i], a.cap);
        row = a.nbr + (size_t)i * a.cap;
        base = a.sys_n ? (i / a.sys_n) * a.sys_n : 0;
    }
    const int nmax = __reduce_max_sync(0xffffffffu, n);
    int m = 0;
    for (int k0 = 0; k0 < nmax; k0 += G) {
        const int k = k0 + gl;
        bool in = false;
        float dx = 0.f, dy = 0.f, dz = 0.f, r2 = 0.f;
        if (k < n) {
            const float4 rj = __ldg(a.r + row[k] + base);
            r2 = dist2_rn<3>(rj, ri, a.box, dx, dy, dz);
            in = r2 < c.rc2;
        }
        const unsigned mk = __ballot_sync(0xffffffffu, in) & gmask;
        const int pos = m + __popc(mk & below);
        if (in && pos < BP_MAXN) {
            const float4 u = make_float4(dx, dy, dz, sqrtf(r2));
            ndg[pos] = u;
            if (a.pa.tb_idx) {   // the partner lists of the force kernel
                a.pa.tb_idx[(size_t)i * BP_MAXN + pos] = row[k] + base;
                a.pa.tb_vec[(size_t)i * BP_MAXN + pos] = u;
            }
        }
        m += __popc(mk);
    }
    if (m > BP_MAXN) {
        if (gl == 0) raise_status(a.status, MD_ERR_NBR_OVERFLOW);
        m = BP_MAXN;
    }
    if (a.pa.tb_cnt && valid && gl == 0) a.pa.tb_cnt[i] = m;
    __syncwarp();
#pragma unroll
    for (int q = 0; q < 16; ++q) Gd[q] = 0.0f;
    const int mmax = __reduce_max_sync(0xffffffffu, m);
    for (int s0 = 0; s0 < mmax; s0 += G) {
        const int s = s0 + gl;
        if (s < m) {
            float g[8], dg[8];
            radial8(c, ndg[s].w, g, dg);
#pragma unroll
            for (int q = 0; q < 8; ++q) Gd[q] += g[q];
        }
    }
    const int nt = m * (m - 1) / 2;
    const int ntmax = __reduce_max_sync(0xffffffffu, nt);
    for (int t0 = 0; t0 < ntmax; t0 += G) {
        int t = t0 + gl;
        if (t < nt) {
            // triplet t of the pairs (s1 < s2) in row-major order
            int s1 = 0;
            while (t >= m - 1 - s1) {
                t -= m - 1 - s1;
                ++s1;
            }
            const int s2 = s1 + 1 + t;
            const float4 u = ndg[s1], v = ndg[s2];
            float tt[8], du[8][3], dw[8][3];
            angular8<false>(c, u.x, u.y, u.z, u.w, v.x, v.y, v.z, v.w, tt, du, dw);
#pragma unroll
            for (int q = 0; q < 8; ++q) Gd[8 + q] += tt[q];
        }
    }
#pragma unroll
    for (int q = 0; q < 16; ++q)
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) Gd[q] += __shfl_xor_sync(0xffffffffu, Gd[q], o);
}

}  // namespace jmd
