// batch.cu -- many independent systems advanced together (the paper's vmap
// over systems, Sec. 4.2): replicas of different sizes, boxes, densities
// and potentials concatenated particle-wise (CSR offsets), each with its
// own cell grid, neighbor rows (global indices), rebuild flag and energy
// series, all advanced by the same kernels -- one CUDA graph launch for the
// whole run.
//
// Per step:
//   k_b_kick_drift   every particle, with its replica's dt, mass and box;
//                    sets the replica's rebuild flag (and a global "any")
//   IF any:          k_b_bin -> k_b_scan (block per replica, segmented) ->
//                    k_b_scatter -> k_b_sort_cells -> k_b_build (block per
//                    cell) -> k_b_finish,
//                    each skipping replicas whose flag is clear
//   k_b_pair<KICK>   forces + closing half-kick, per-particle potential and
//                    kinetic energy into f.w and v.w
//   k_b_energy       block per replica: FP64 sums in fixed order into the
//                    replica's series; the last block advances the step and
//                    sets the graph's WHILE condition (k_b_step alone when
//                    no series is asked for; non-finite forces are reported
//                    by k_b_pair either way)
// Arithmetic per particle is the single-system arithmetic (same pair term,
// lane mapping, shuffle order, kick and drift), so a replica advanced here
// matches the same replica advanced alone with the same tuning, bit for bit.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"

namespace jmd {

struct RepMeta {
    int p0, n;            // particle offset and count
    int c0, nct;          // cell offset and count (cell c0 + nct is the end sentinel)
    int nc[3];
    int kind;             // MD_LJ or MD_SOFT_SPHERE
    Box box;
    float cell_scale[3];
    float rl2, half_skin2;
    float hdm, dt, mass;
    float rc2, sigma2, c24eps, c4eps, e_shift;   // LJ
    float eps, alpha;                            // soft sphere
};

struct BatchDev {
    const RepMeta *meta;
    const int32_t *rep_of;    // [N]
    const int32_t *cell_rep;  // [C]
    int32_t *cell_count, *cell_start, *cell_of, *rank, *atoms_u, *atoms;
    float4 *rsorted;          // cell-ordered positions, particle index in w
    uint32_t *flag;           // [R] rebuild flags
    uint32_t *builds;         // [R] builds per replica
    uint32_t *ctl;            // control words (CTL_*)
    int32_t *nbr, *cnt;
    float4 *rref;
    int N, R, C, cap, tpp;
    int wrapped;              // 1: positions inside [0, L) (the NVE loop wraps them), near-image form in the build
    uint32_t *status;
    // per-replica threads per particle (md_batch_set_class_tpp): the
    // particles grouped by their replica's value (4, 8, 16), counts per
    // group; plist == NULL: one launch over all particles with tpp
    const int32_t *plist;
    int pgroup[3];
    // the particle list of the launch in flight (NULL: particles 0..N-1)
    const int32_t *pl;
    int pn;
};

struct BatchLayout {
    size_t meta, rep_of, cell_rep, cell_count, cell_start, cell_of, rank, atoms_u, atoms, rsorted, flag, builds, ctl,
        plist, total;
};

static BatchLayout batch_layout(int N, int R, int C)
{
    BatchLayout w;
    size_t o = 0;
    w.ctl = o;        o = align256(o + sizeof(uint32_t) * CTL_WORDS);
    w.meta = o;       o = align256(o + sizeof(RepMeta) * (size_t)R);
    w.rep_of = o;     o = align256(o + sizeof(int32_t) * (size_t)N);
    w.cell_rep = o;   o = align256(o + sizeof(int32_t) * (size_t)C);
    w.cell_count = o; o = align256(o + sizeof(int32_t) * (size_t)C);
    w.cell_start = o; o = align256(o + sizeof(int32_t) * (size_t)C);
    w.cell_of = o;    o = align256(o + sizeof(int32_t) * (size_t)N);
    w.rank = o;       o = align256(o + sizeof(int32_t) * (size_t)N);
    w.atoms_u = o;    o = align256(o + sizeof(int32_t) * (size_t)N);
    w.atoms = o;      o = align256(o + sizeof(int32_t) * (size_t)N);
    w.rsorted = o;    o = align256(o + sizeof(float4) * (size_t)N);
    w.flag = o;       o = align256(o + sizeof(uint32_t) * (size_t)R);
    w.builds = o;     o = align256(o + sizeof(uint32_t) * (size_t)R);
    w.plist = o;      o = align256(o + sizeof(int32_t) * (size_t)N);
    w.total = o;
    return w;
}

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------
template <int COND>
__global__ void __launch_bounds__(256) k_b_kick_drift(BatchDev b, float4 *r, float4 *v, const float4 *f,
                                                      unsigned long long cond_if)
{
    count_launch();
    __shared__ bool last;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < b.N) {
        const RepMeta &m = b.meta[b.rep_of[i]];
        float4 fi = f[i], vi = v[i], ri = r[i];
        vi.x += m.hdm * fi.x;
        vi.y += m.hdm * fi.y;
        vi.z += m.hdm * fi.z;
        ri.x = wrap_coord(ri.x + m.dt * vi.x, m.box.L[0], m.box.Linv[0]);
        ri.y = wrap_coord(ri.y + m.dt * vi.y, m.box.L[1], m.box.Linv[1]);
        ri.z = wrap_coord(ri.z + m.dt * vi.z, m.box.L[2], m.box.Linv[2]);
        v[i] = vi;
        r[i] = ri;
        float dx, dy, dz;
        if (dist2_rn<3>(ri, b.rref[i], m.box, dx, dy, dz) > m.half_skin2) {
            b.flag[b.rep_of[i]] = 1u;
            b.ctl[CTL_REBUILD] = 1u;
            if (COND) __threadfence();
        }
    }
    if (COND) {
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            unsigned t = atomicAdd(&b.ctl[CTL_TICKET2], 1u);
            last = (t == gridDim.x - 1);
        }
        __syncthreads();
        if (last && threadIdx.x == 0) {
            __threadfence();
            unsigned any = *(volatile uint32_t *)&b.ctl[CTL_REBUILD];
            b.ctl[CTL_TICKET2] = 0u;
            cudaGraphSetConditional((cudaGraphConditionalHandle)cond_if, any ? 1u : 0u);
        }
    }
}

__device__ __forceinline__ int b_cell_axis(float x, float L, float Linv, float scale, int n)
{
    float y = wrap_coord(x, L, Linv);
    int q = (int)(y * scale);
    return q < 0 ? 0 : (q >= n ? n - 1 : q);
}

__global__ void __launch_bounds__(256) k_b_bin(BatchDev b, const float4 *r)
{
    count_launch();
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    bool act = false;
    int c = -1;
    if (i < b.N) {
        const int rep = b.rep_of[i];
        act = *(volatile uint32_t *)&b.flag[rep] != 0u;
        if (act) {
            const RepMeta &m = b.meta[rep];
            float4 p = r[i];
            if (!isfinite(p.x) || !isfinite(p.y) || !isfinite(p.z)) raise_status(b.status, MD_ERR_NONFINITE);
            int cx = b_cell_axis(p.x, m.box.L[0], m.box.Linv[0], m.cell_scale[0], m.nc[0]);
            int cy = b_cell_axis(p.y, m.box.L[1], m.box.Linv[1], m.cell_scale[1], m.nc[1]);
            int cz = b_cell_axis(p.z, m.box.L[2], m.box.Linv[2], m.cell_scale[2], m.nc[2]);
            c = m.c0 + (cz * m.nc[1] + cy) * m.nc[0] + cx;
        }
    }
    unsigned amask = __ballot_sync(0xffffffffu, act);
    if (!act) return;
    unsigned peers = __match_any_sync(amask, c);
    int lane = threadIdx.x & 31;
    int leader = __ffs(peers) - 1;
    int below = __popc(peers & ((1u << lane) - 1u));
    int base = 0;
    if (lane == leader) base = atomicAdd(&b.cell_count[c], __popc(peers));
    base = __shfl_sync(peers, base, leader);
    b.cell_of[i] = c;
    b.rank[i] = base + below;
}

// block per replica: cell_start = p0 + exclusive scan of its cells; the end
// sentinel gets p0 + n; counts cleared for the next build
__global__ void __launch_bounds__(256) k_b_scan(BatchDev b)
{
    count_launch();
    const int rep = blockIdx.x;
    if (*(volatile uint32_t *)&b.flag[rep] == 0u) return;
    const RepMeta &m = b.meta[rep];
    __shared__ int warp_tot[8];
    int t = threadIdx.x;
    int per = (m.nct + blockDim.x - 1) / blockDim.x;
    int lo = m.c0 + t * per, hi = min(lo + per, m.c0 + m.nct);
    int s = 0;
    for (int q = lo; q < hi; ++q) s += b.cell_count[q];
    int lane = t & 31, w = t >> 5;
    int x = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[w] = x;
    __syncthreads();
    int before = 0;
    for (int k = 0; k < w; ++k) before += warp_tot[k];
    int run = m.p0 + before + x - s;
    for (int q = lo; q < hi; ++q) {
        b.cell_start[q] = run;
        run += b.cell_count[q];
        b.cell_count[q] = 0;
    }
    if (t == 0) b.cell_start[m.c0 + m.nct] = m.p0 + m.n;
}

__global__ void __launch_bounds__(256) k_b_scatter(BatchDev b, const float4 *r)
{
    count_launch();
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= b.N) return;
    if (*(volatile uint32_t *)&b.flag[b.rep_of[i]] == 0u) return;
    int slot = b.cell_start[b.cell_of[i]] + b.rank[i];
    b.atoms_u[slot] = i;
}

// One warp per cell (as the single-system k_sort_cells): members ranked by
// global index, written with their positions (index in w) in that order;
// the positions of this build go to rref.
constexpr int BS_WARPS = 8;
__global__ void __launch_bounds__(BS_WARPS * 32) k_b_sort_cells(BatchDev b, const float4 *r)
{
    count_launch();
    const int lane = threadIdx.x & 31;
    const int q = blockIdx.x * BS_WARPS + (threadIdx.x >> 5);
    if (q >= b.C) return;   // whole warp
    const int rep = b.cell_rep[q];
    if (rep < 0 || *(volatile uint32_t *)&b.flag[rep] == 0u) return;
    const int s0 = b.cell_start[q], n = b.cell_start[q + 1] - s0;
    const int32_t *u = b.atoms_u + s0;
    for (int base = 0; base < n; base += 32) {
        const int k = base + lane;
        const int me = k < n ? u[k] : 0x7fffffff;
        int rk = 0;
        for (int c0 = 0; c0 < n; c0 += 32) {
            int other = (c0 + lane < n) ? u[c0 + lane] : 0x7fffffff;
#pragma unroll 8
            for (int t = 0; t < 32; ++t) rk += (__shfl_sync(0xffffffffu, other, t) < me);
        }
        if (k < n) {
            const float4 p = r[me];
            b.atoms[s0 + rk] = me;
            b.rsorted[s0 + rk] = make_float4(p.x, p.y, p.z, __int_as_float(me));
            b.rref[me] = p;
        }
    }
}

__device__ __forceinline__ int b_axis_cells(int q, int n, int *out)
{
    if (n >= 3) {
        out[0] = q == 0 ? n - 1 : q - 1;
        out[1] = q;
        out[2] = q == n - 1 ? 0 : q + 1;
        return 3;
    }
    if (n == 2) {
        out[0] = 0;
        out[1] = 1;
        return 2;
    }
    out[0] = 0;
    return 1;
}

constexpr int BB_CMAX = 1024;
constexpr int BB_WARPS = 4;

// Dense stencil (more candidates than a block stages): row of particle i by
// one warp straight from the replica's cells, then sorted in the warp's
// shared buffer (CAPP2 >= cap, power of two).  Same decisions as the
// single-system per-warp path.
template <int CAPP2>
__device__ void b_build_row_warp(const BatchDev &b, const RepMeta &m, int i, const float4 &pi, int c, int *row)
{
    const int lane = threadIdx.x & 31;
    const int lc = c - m.c0;
    int cx = lc % m.nc[0];
    int cy = (lc / m.nc[0]) % m.nc[1];
    int cz = lc / (m.nc[0] * m.nc[1]);
    int sx[3], sy[3], sz[3];
    int mx = b_axis_cells(cx, m.nc[0], sx);
    int my = b_axis_cells(cy, m.nc[1], sy);
    int mz = b_axis_cells(cz, m.nc[2], sz);
    int count = 0;
    const unsigned lt = (1u << lane) - 1u;
    for (int zz = 0; zz < mz; ++zz)
        for (int yy = 0; yy < my; ++yy)
            for (int xx = 0; xx < mx; ++xx) {
                int q = m.c0 + (sz[zz] * m.nc[1] + sy[yy]) * m.nc[0] + sx[xx];
                int s0 = b.cell_start[q], s1 = b.cell_start[q + 1];
                for (int s = s0; s < s1; s += 32) {
                    int slot = s + lane;
                    bool hit = false;
                    int j = 0;
                    if (slot < s1) {
                        j = b.atoms[slot];
                        float dx, dy, dz;
                        hit = (j != i) && (dist2_rn<3>(pi, b.rsorted[slot], m.box, dx, dy, dz) < m.rl2);
                    }
                    unsigned mk = __ballot_sync(0xffffffffu, hit);
                    int pos = count + __popc(mk & lt);
                    if (hit && pos < CAPP2) row[pos] = j;
                    count += __popc(mk);
                }
            }
    __syncwarp();
    int n = count < b.cap ? count : b.cap;
    for (int k = n + lane; k < CAPP2; k += 32) row[k] = 0x7fffffff;
    __syncwarp();
    for (int size = 2; size <= CAPP2; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int t = lane; t < CAPP2 / 2; t += 32) {
                int lo = 2 * t - (t & (stride - 1));
                int hi = lo + stride;
                bool up = ((lo & size) == 0);
                int x = row[lo], y = row[hi];
                if ((x > y) == up) {
                    row[lo] = y;
                    row[hi] = x;
                }
            }
            __syncwarp();
        }
    }
    int32_t *out = b.nbr + (size_t)i * b.cap;
    for (int k = lane; k < b.cap; k += 32) out[k] = (k < n) ? row[k] : b.N;
    if (lane == 0) {
        b.cnt[i] = count;
        if (count > b.cap) raise_status(b.status, MD_ERR_NBR_OVERFLOW);
    }
    __syncwarp();
}

// block per (non-sentinel) cell, same candidate order as the single-system
// build: stencil cells in fixed order, ascending global index inside a cell
// (k_b_sort_cells); candidates swept 64 at a time with two ballots.
// Cells whose stencil exceeds the staging capacity set MD_ERR_BOUNDS
// (replica plans keep stencils small; see md_batch_plan).
template <bool NEAR>
__global__ void __launch_bounds__(BB_WARPS * 32) k_b_build(BatchDev b)
{
    count_launch();
    __shared__ float4 spos[BB_CMAX];
    __shared__ int soff[28], sbeg[27], nst;
    const int q = blockIdx.x;
    const int rep = b.cell_rep[q];
    if (rep < 0) return;   // sentinel slot
    if (*(volatile uint32_t *)&b.flag[rep] == 0u) return;
    const RepMeta &m = b.meta[rep];
    const int tid = threadIdx.x;
    const int own_b = b.cell_start[q], own_e = b.cell_start[q + 1];
    if (own_e == own_b) return;
    if (tid < 32) {
        int lq = q - m.c0;
        int cx = lq % m.nc[0];
        int cy = (lq / m.nc[0]) % m.nc[1];
        int cz = lq / (m.nc[0] * m.nc[1]);
        int sx[3], sy[3], sz[3];
        int mx = b_axis_cells(cx, m.nc[0], sx);
        int my = b_axis_cells(cy, m.nc[1], sy);
        int mz = b_axis_cells(cz, m.nc[2], sz);
        int nm = mx * my * mz;
        int cnt = 0;
        if (tid < nm) {
            int xx = tid % mx, yy = (tid / mx) % my, zz = tid / (mx * my);
            int c = m.c0 + (sz[zz] * m.nc[1] + sy[yy]) * m.nc[0] + sx[xx];
            cnt = b.cell_start[c + 1] - b.cell_start[c];
            sbeg[tid] = b.cell_start[c];
        }
        int incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (tid >= o) incl += y;
        }
        if (tid < nm) soff[tid + 1] = incl;
        if (tid == 0) {
            soff[0] = 0;
            nst = nm;
        }
    }
    __syncthreads();
    const int M = soff[nst];
    if (M > BB_CMAX) {
        // per-warp rows; the 16 KB candidate-position array serves as 8 warp
        // buffers of 512 ints
        static_assert(sizeof(spos) >= BB_WARPS * 512 * sizeof(int), "row buffers must fit");
        int *rowbuf = reinterpret_cast<int *>(spos) + (tid >> 5) * 512;
        for (int s = own_b + (tid >> 5); s < own_e; s += BB_WARPS) {
            int i = b.atoms[s];
            float4 pi = b.rsorted[s];
            if (b.cap <= 128) b_build_row_warp<128>(b, m, i, pi, q, rowbuf);
            else if (b.cap <= 256) b_build_row_warp<256>(b, m, i, pi, q, rowbuf);
            else b_build_row_warp<512>(b, m, i, pi, q, rowbuf);
        }
        return;
    }
    // staging: the members are in canonical order already (k_b_sort_cells),
    // padded with NaN positions (which fail every test) to whole sweep steps
    const int lane = tid & 31, warp = tid >> 5;
    for (int mm = warp; mm < nst; mm += BB_WARPS) {
        const int b0 = soff[mm], n = soff[mm + 1] - b0, src = sbeg[mm];
        for (int k = lane; k < n; k += 32) spos[b0 + k] = b.rsorted[src + k];
    }
    const float nan = __int_as_float(0x7fc00000);
    const int Mp = (M + 63) / 64 * 64;
    for (int k = M + tid; k < Mp; k += blockDim.x) spos[k] = make_float4(nan, nan, nan, __int_as_float(-1));
    __syncthreads();
    const unsigned lt = (1u << lane) - 1u;
    for (int s = own_b + warp; s < own_e; s += BB_WARPS) {
        const float4 ri = b.rsorted[s];
        const int i = __float_as_int(ri.w);
        int32_t *out = b.nbr + (size_t)i * b.cap;
        int count = 0;
        for (int k0 = 0; k0 < Mp; k0 += 64) {
            bool hit[2];
            int j[2];
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const float4 c = spos[k0 + 32 * u + lane];
                j[u] = __float_as_int(c.w);
                float dx, dy, dz;
                // NEAR: positions inside the box, where the comparison form
                // gives the bits of the rint form
                const float r2 = NEAR ? dist2_near<3>(ri, c, m.box, dx, dy, dz) : dist2_rn<3>(ri, c, m.box, dx, dy, dz);
                hit[u] = (j[u] != i) && (r2 < m.rl2);
            }
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const unsigned mk = __ballot_sync(0xffffffffu, hit[u]);
                const int pos = count + __popc(mk & lt);
                if (hit[u] && pos < b.cap) out[pos] = j[u];
                count += __popc(mk);
            }
        }
        int n = count < b.cap ? count : b.cap;
        for (int k = n + lane; k < b.cap; k += 32) out[k] = b.N;
        if (lane == 0) {
            b.cnt[i] = count;
            if (count > b.cap) raise_status(b.status, MD_ERR_NBR_OVERFLOW);
        }
    }
}

__global__ void k_b_finish(BatchDev b)
{
    count_launch();
    for (int rep = threadIdx.x; rep < b.R; rep += blockDim.x) {
        if (b.flag[rep]) b.builds[rep] += 1u;
        b.flag[rep] = 0u;
    }
    if (threadIdx.x == 0) b.ctl[CTL_REBUILD] = 0u;
}

__global__ void k_b_flag_all(BatchDev b)
{
    count_launch();
    for (int rep = threadIdx.x; rep < b.R; rep += blockDim.x) b.flag[rep] = 1u;
    if (threadIdx.x == 0) b.ctl[CTL_REBUILD] = 1u;
}

// pair term of one replica's potential (the single-system pair term)
__device__ __forceinline__ void b_pair_term(const RepMeta &m, const float4 &ri, const float4 &rj, float &fx, float &fy,
                                            float &fz, float &e)
{
    float dx, dy, dz;
    float r2 = dist2_rn<3>(ri, rj, m.box, dx, dy, dz);
    if (m.kind == MD_LJ) {
        if (r2 < m.rc2) {
            float ir2 = __fdividef(1.0f, r2);
            float s2 = m.sigma2 * ir2;
            float s6 = s2 * s2 * s2;
            float fr = m.c24eps * ir2 * s6 * (2.0f * s6 - 1.0f);
            fx += fr * dx;
            fy += fr * dy;
            fz += fr * dz;
            e += m.c4eps * s6 * (s6 - 1.0f) - m.e_shift;
        }
    } else {
        float sg = 0.5f * (ri.w + rj.w);
        if (r2 < sg * sg) {
            float rr = sqrtf(r2);
            float isg = __fdividef(1.0f, sg);
            float x = 1.0f - rr * isg;
            float xa1, ua;
            if (m.alpha == 2.0f) {
                xa1 = x;
                ua = 0.5f * x * x;
            } else {
                xa1 = __powf(x, m.alpha - 1.0f);
                ua = xa1 * x / m.alpha;
            }
            float fr = m.eps * isg * xa1 * __fdividef(1.0f, rr);
            fx += fr * dx;
            fy += fr * dy;
            fz += fr * dz;
            e += m.eps * ua;
        }
    }
}

template <int TPP, int KICK>
__global__ void __launch_bounds__(256) k_b_pair(BatchDev b, const float4 *r, float4 *v, float4 *f)
{
    count_launch();
    constexpr int PPB = 256 / TPP;
    const int lg = threadIdx.x & (TPP - 1);
    const int gl = threadIdx.x / TPP;
    const int lim = b.pl ? b.pn : b.N;
    for (int base = blockIdx.x * PPB; base < lim; base += gridDim.x * PPB) {
        const int k = base + gl;
        bool valid = k < lim;
        int i = valid ? (b.pl ? __ldg(b.pl + k) : k) : b.N;
        float fx = 0.f, fy = 0.f, fz = 0.f, e = 0.f;
        const RepMeta *mp = nullptr;
        if (valid) {
            mp = &b.meta[b.rep_of[i]];
            const RepMeta &m = *mp;
            float4 ri = __ldg(r + i);
            int n = __ldg(b.cnt + i);
            n = n < b.cap ? n : b.cap;
            const int32_t *row = b.nbr + (size_t)i * b.cap;
            for (int k0 = lg; k0 < n; k0 += 4 * TPP) {
                const int k1 = k0 + TPP, k2 = k0 + 2 * TPP, k3 = k0 + 3 * TPP;
                int j0 = __ldg(row + k0);
                int j1 = k1 < n ? __ldg(row + k1) : i;
                int j2 = k2 < n ? __ldg(row + k2) : i;
                int j3 = k3 < n ? __ldg(row + k3) : i;
                float4 r0 = __ldg(r + j0);
                float4 r1 = __ldg(r + j1);
                float4 r2 = __ldg(r + j2);
                float4 r3 = __ldg(r + j3);
                b_pair_term(m, ri, r0, fx, fy, fz, e);
                if (k1 < n) b_pair_term(m, ri, r1, fx, fy, fz, e);
                if (k2 < n) b_pair_term(m, ri, r2, fx, fy, fz, e);
                if (k3 < n) b_pair_term(m, ri, r3, fx, fy, fz, e);
            }
        }
#pragma unroll
        for (int o = TPP / 2; o > 0; o >>= 1) {
            fx += __shfl_xor_sync(0xffffffffu, fx, o);
            fy += __shfl_xor_sync(0xffffffffu, fy, o);
            fz += __shfl_xor_sync(0xffffffffu, fz, o);
            e += __shfl_xor_sync(0xffffffffu, e, o);
        }
        if (valid && lg == 0) {
            float ei = 0.5f * e;
            f[i] = make_float4(fx, fy, fz, ei);
            // a blown-up replica is reported here whether or not energies are summed
            if (!(isfinite(fx) && isfinite(fy) && isfinite(fz) && isfinite(ei))) raise_status(b.status, MD_ERR_NONFINITE);
            if (KICK) {
                float4 vi = v[i];
                vi.x += mp->hdm * fx;
                vi.y += mp->hdm * fy;
                vi.z += mp->hdm * fz;
                vi.w = 0.5f * mp->mass * (vi.x * vi.x + vi.y * vi.y + vi.z * vi.z);
                v[i] = vi;
            }
        }
    }
}

// block per replica: PE[rep][step] = sum f.w, KE[rep][step] = sum v.w (FP64,
// fixed order); the last block advances the step counter and, in a graph,
// sets the WHILE condition.
__global__ void __launch_bounds__(256) k_b_energy(BatchDev b, const float4 *v, const float4 *f, double *PE, double *KE,
                                                  int series_len, unsigned long long cond_while, int use_cond)
{
    count_launch();
    __shared__ double sh[2][32];
    __shared__ bool last;
    const int rep = blockIdx.x;
    const RepMeta &m = b.meta[rep];
    double E[2] = {0.0, 0.0};
    for (int k = threadIdx.x; k < m.n; k += blockDim.x) {
        E[0] += (double)f[m.p0 + k].w;
        E[1] += (double)v[m.p0 + k].w;
    }
    block_sums_f64<2>(E, &sh[0][0], 32);
    const double pe = E[0], ke = E[1];
    const unsigned step = b.ctl[CTL_STEP];
    if (threadIdx.x == 0) {
        if (!isfinite(pe) || !isfinite(ke)) raise_status(b.status, MD_ERR_NONFINITE);
        if (PE && (int)step < series_len) PE[(size_t)rep * series_len + step] = pe;
        if (KE && (int)step < series_len) KE[(size_t)rep * series_len + step] = ke;
        __threadfence();
        unsigned t = atomicAdd(&b.ctl[CTL_TICKET], 1u);
        last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        b.ctl[CTL_TICKET] = 0u;
        b.ctl[CTL_STEP] = step + 1u;
        if (use_cond)
            cudaGraphSetConditional((cudaGraphConditionalHandle)cond_while, (step + 1u < b.ctl[CTL_NSTEPS]) ? 1u : 0u);
    }
}

// The loop control of a step without energy series: advance the step
// counter and, in a graph, set the WHILE condition (one thread).
__global__ void k_b_step(BatchDev b, unsigned long long cond_while, int use_cond)
{
    count_launch();
    const unsigned step = b.ctl[CTL_STEP];
    b.ctl[CTL_STEP] = step + 1u;
    if (use_cond)
        cudaGraphSetConditional((cudaGraphConditionalHandle)cond_while, (step + 1u < b.ctl[CTL_NSTEPS]) ? 1u : 0u);
}

__global__ void k_b_loop_init(uint32_t *ctl, uint32_t nsteps)
{
    count_launch();
    ctl[CTL_STEP] = 0u;
    ctl[CTL_NSTEPS] = nsteps;
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct BatchHost {
    std::vector<RepMeta> meta;
    std::vector<int32_t> rep_of, cell_rep;
    cudaGraphExec_t exec = nullptr;
    cudaGraph_t graph = nullptr;
    const void *g_r = nullptr, *g_v = nullptr, *g_f = nullptr, *g_pe = nullptr, *g_ke = nullptr;
    int g_len = -1, g_tpp = 0;
    uint32_t *g_status = nullptr;
    // per-replica threads per particle (md_batch_set_class_tpp)
    bool classes = false;
    int pgroup[3] = {0, 0, 0};   // particles with 4, 8, 16 threads each
    unsigned class_version = 0, g_class_version = 0;
};

static BatchDev batch_dev(const md_batch *bt, uint32_t *status)
{
    BatchLayout w = batch_layout(bt->N, bt->R, bt->ncell_total);
    char *p = (char *)bt->ws;
    BatchDev b;
    memset(&b, 0, sizeof(b));
    b.meta = (const RepMeta *)(p + w.meta);
    b.rep_of = (const int32_t *)(p + w.rep_of);
    b.cell_rep = (const int32_t *)(p + w.cell_rep);
    b.cell_count = (int32_t *)(p + w.cell_count);
    b.cell_start = (int32_t *)(p + w.cell_start);
    b.cell_of = (int32_t *)(p + w.cell_of);
    b.rank = (int32_t *)(p + w.rank);
    b.atoms_u = (int32_t *)(p + w.atoms_u);
    b.atoms = (int32_t *)(p + w.atoms);
    b.rsorted = (float4 *)(p + w.rsorted);
    b.flag = (uint32_t *)(p + w.flag);
    b.builds = (uint32_t *)(p + w.builds);
    b.ctl = (uint32_t *)(p + w.ctl);
    b.nbr = bt->nbr;
    b.cnt = bt->cnt;
    b.rref = (float4 *)bt->rref;
    b.N = bt->N;
    b.R = bt->R;
    b.C = bt->ncell_total;
    b.cap = bt->cap;
    b.tpp = bt->tpp;
    b.status = status;
    const BatchHost *H = (const BatchHost *)bt->host;
    if (H && H->classes) {
        b.plist = (const int32_t *)(p + w.plist);
        for (int k = 0; k < 3; ++k) b.pgroup[k] = H->pgroup[k];
    }
    return b;
}

static void enqueue_b_rebuild(const BatchDev &b, const float4 *r, cudaStream_t st)
{
    int g = (b.N + 255) / 256;
    k_b_bin<<<g, 256, 0, st>>>(b, r);
    k_b_scan<<<b.R, 256, 0, st>>>(b);
    k_b_scatter<<<g, 256, 0, st>>>(b, r);
    k_b_sort_cells<<<(b.C + BS_WARPS - 1) / BS_WARPS, BS_WARPS * 32, 0, st>>>(b, r);
    if (b.wrapped) k_b_build<true><<<b.C, BB_WARPS * 32, 0, st>>>(b);
    else k_b_build<false><<<b.C, BB_WARPS * 32, 0, st>>>(b);
    k_b_finish<<<1, 256, 0, st>>>(b);
}

template <int TPP, int KICK>
static void launch_b_pair(const BatchDev &b, const float4 *r, float4 *v, float4 *f, cudaStream_t st)
{
    static int per_sm = 0, sms = 0;
    if (!per_sm) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_b_pair<TPP, KICK>, 256, 0);
        if (per_sm < 1) per_sm = 1;
    }
    int groups = (int)(((long long)(b.pl ? b.pn : b.N) * TPP + 255) / 256);
    int g = per_sm * sms;
    k_b_pair<TPP, KICK><<<groups < g ? groups : g, 256, 0, st>>>(b, r, v, f);
}

static void enqueue_b_pair_tpp(const BatchDev &b, int tpp, const float4 *r, float4 *v, float4 *f, int kick,
                               cudaStream_t st)
{
    switch (tpp) {
    case 8: kick ? launch_b_pair<8, 1>(b, r, v, f, st) : launch_b_pair<8, 0>(b, r, v, f, st); break;
    case 16: kick ? launch_b_pair<16, 1>(b, r, v, f, st) : launch_b_pair<16, 0>(b, r, v, f, st); break;
    default: kick ? launch_b_pair<4, 1>(b, r, v, f, st) : launch_b_pair<4, 0>(b, r, v, f, st); break;
    }
}

// One launch with bt->tpp over all particles, or (per-replica threads per
// particle) one launch per nonempty group of the particle list.
static void enqueue_b_pair(const BatchDev &b0, const float4 *r, float4 *v, float4 *f, int kick, cudaStream_t st)
{
    if (!b0.plist) {
        enqueue_b_pair_tpp(b0, b0.tpp, r, v, f, kick, st);
        return;
    }
    const int tpps[3] = {4, 8, 16};
    int off = 0;
    for (int g = 0; g < 3; ++g) {
        if (b0.pgroup[g] > 0) {
            BatchDev b = b0;
            b.pl = b0.plist + off;
            b.pn = b0.pgroup[g];
            enqueue_b_pair_tpp(b, tpps[g], r, v, f, kick, st);
        }
        off += b0.pgroup[g];
    }
}

static md_status b_graph(BatchHost &H, const BatchDev &b0, float4 *r, float4 *v, float4 *f, double *PE, double *KE,
                         int len)
{
    BatchDev b = b0;
    cudaGraph_t g = nullptr;
    JMD_CUDA_TRY(cudaGraphCreate(&g, 0));
    cudaGraphConditionalHandle hw, hi;
    JMD_CUDA_TRY(cudaGraphConditionalHandleCreate(&hw, g, 1u, cudaGraphCondAssignDefault));
    JMD_CUDA_TRY(cudaGraphConditionalHandleCreate(&hi, g, 0u, cudaGraphCondAssignDefault));
    alignas(cudaGraphNodeParams) unsigned char wraw[sizeof(cudaGraphNodeParams)];
    memset(wraw, 0, sizeof(wraw));
    cudaGraphNodeParams *wp = reinterpret_cast<cudaGraphNodeParams *>(wraw);
    wp->type = cudaGraphNodeTypeConditional;
    wp->conditional.handle = hw;
    wp->conditional.type = cudaGraphCondTypeWhile;
    wp->conditional.size = 1;
    cudaGraphNode_t wn;
    JMD_CUDA_TRY(cudaGraphAddNode(&wn, g, nullptr, nullptr, 0, wp));
    cudaGraph_t body = wp->conditional.phGraph_out[0];
    cudaStream_t cs = nullptr, cs2 = nullptr;
    JMD_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    JMD_CUDA_TRY(cudaStreamCreateWithFlags(&cs2, cudaStreamNonBlocking));
    JMD_CUDA_TRY(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    int gk = (b.N + 255) / 256;
    k_b_kick_drift<1><<<gk, 256, 0, cs>>>(b, r, v, f, (unsigned long long)hi);
    cudaStreamCaptureStatus cst;
    cudaGraph_t cg = nullptr;
    const cudaGraphNode_t *deps = nullptr;
    size_t nd = 0;
    JMD_CUDA_TRY(cudaStreamGetCaptureInfo(cs, &cst, nullptr, &cg, &deps, nullptr, &nd));
    alignas(cudaGraphNodeParams) unsigned char iraw[sizeof(cudaGraphNodeParams)];
    memset(iraw, 0, sizeof(iraw));
    cudaGraphNodeParams *ip = reinterpret_cast<cudaGraphNodeParams *>(iraw);
    ip->type = cudaGraphNodeTypeConditional;
    ip->conditional.handle = hi;
    ip->conditional.type = cudaGraphCondTypeIf;
    ip->conditional.size = 1;
    cudaGraphNode_t in;
    JMD_CUDA_TRY(cudaGraphAddNode(&in, cg, deps, nullptr, nd, ip));
    JMD_CUDA_TRY(cudaStreamUpdateCaptureDependencies(cs, &in, nullptr, 1, cudaStreamSetCaptureDependencies));
    cudaGraph_t ibody = ip->conditional.phGraph_out[0];
    JMD_CUDA_TRY(cudaStreamBeginCaptureToGraph(cs2, ibody, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    enqueue_b_rebuild(b, r, cs2);
    JMD_CUDA_TRY(cudaStreamEndCapture(cs2, &ibody));
    enqueue_b_pair(b, r, v, f, 1, cs);
    if (PE || KE) k_b_energy<<<b.R, 256, 0, cs>>>(b, v, f, PE, KE, len, (unsigned long long)hw, 1);
    else k_b_step<<<1, 1, 0, cs>>>(b, (unsigned long long)hw, 1);
    JMD_CUDA_TRY(cudaStreamEndCapture(cs, &body));
    cudaStreamDestroy(cs2);
    cudaStreamDestroy(cs);
    cudaGraphExec_t ex = nullptr;
    JMD_CUDA_TRY(cudaGraphInstantiate(&ex, g, 0));
    if (H.exec) cudaGraphExecDestroy(H.exec);
    if (H.graph) cudaGraphDestroy(H.graph);
    H.exec = ex;
    H.graph = g;
    return MD_OK;
}

}  // namespace jmd

using namespace jmd;

extern "C" md_status md_batch_plan(const md_replica_desc *reps, int R, int cap, md_batch *out)
{
    if (!reps || !out || R < 1 || cap < 1 || cap > 512) return MD_ERR_INVALID;
    BatchHost *H = new BatchHost();
    int p = 0, c = 0;
    for (int k = 0; k < R; ++k) {
        const md_replica_desc &d = reps[k];
        if (d.N < 1 || !(d.L > 0.0) || (d.kind != MD_LJ && d.kind != MD_SOFT_SPHERE) || !(d.mass > 0.0f)) {
            delete H;
            return MD_ERR_INVALID;
        }
        md_space s;
        double box[3] = {d.L, d.L, d.L};
        md_space_periodic(3, box, &s);
        md_nbr nb;
        md_status st = md_nbr_plan(&s, d.N, d.r_cut, d.skin, cap, &nb);
        if (st != MD_OK) {
            delete H;
            return st;
        }
        RepMeta m;
        memset(&m, 0, sizeof(m));
        m.p0 = p;
        m.n = d.N;
        m.c0 = c;
        if (d.cell_mult > 1.0f) {
            // larger cells: side >= cell_mult r_list (the plan's margin kept)
            nb.ncell_total = 1;
            for (int a = 0; a < 3; ++a) {
                int n = (int)floor(d.L / ((double)nb.r_list * (double)d.cell_mult * (1.0 + 1e-4)));
                nb.ncell[a] = n < 1 ? 1 : n;
                nb.cell_scale[a] = (float)((double)nb.ncell[a] / d.L);
                nb.ncell_total *= nb.ncell[a];
            }
        }
        m.nct = nb.ncell_total;
        for (int a = 0; a < 3; ++a) {
            m.nc[a] = nb.ncell[a];
            m.cell_scale[a] = nb.cell_scale[a];
        }
        m.kind = d.kind;
        m.box = make_box(&s);
        m.rl2 = nb.r_list2;
        m.half_skin2 = nb.half_skin2;
        m.dt = d.dt;
        m.mass = d.mass;
        m.hdm = 0.5f * d.dt / d.mass;
        if (d.kind == MD_LJ) {
            m.rc2 = d.r_cut * d.r_cut;
            m.sigma2 = d.sigma * d.sigma;
            m.c24eps = 24.0f * d.eps;
            m.c4eps = 4.0f * d.eps;
            m.e_shift = d.e_shift;
        } else {
            m.eps = d.eps;
            m.alpha = d.alpha;
        }
        H->meta.push_back(m);
        for (int i = 0; i < d.N; ++i) H->rep_of.push_back(k);
        for (int q = 0; q < nb.ncell_total; ++q) H->cell_rep.push_back(k);
        H->cell_rep.push_back(-1);   // end sentinel
        p += d.N;
        c += nb.ncell_total + 1;
    }
    md_batch b;
    memset(&b, 0, sizeof(b));
    b.R = R;
    b.N = p;
    b.cap = cap;
    b.ncell_total = c;
    b.tpp = 4;
    b.ws_bytes = batch_layout(p, R, c).total;
    b.host = H;
    *out = b;
    return MD_OK;
}

extern "C" void md_batch_free(md_batch *bt)
{
    if (!bt || !bt->host) return;
    BatchHost *H = (BatchHost *)bt->host;
    if (H->exec) cudaGraphExecDestroy(H->exec);
    if (H->graph) cudaGraphDestroy(H->graph);
    delete H;
    bt->host = nullptr;
}

extern "C" md_status md_batch_bind(md_batch *bt, int32_t *d_nbr, int32_t *d_cnt, float *d_rref, void *d_ws,
                                   md_stream_t stream)
{
    if (!bt || !bt->host || !d_nbr || !d_cnt || !d_rref || !d_ws || ((uintptr_t)d_ws & 255u)) return MD_ERR_INVALID;
    BatchHost *H = (BatchHost *)bt->host;
    bt->nbr = d_nbr;
    bt->cnt = d_cnt;
    bt->rref = d_rref;
    bt->ws = d_ws;
    BatchLayout w = batch_layout(bt->N, bt->R, bt->ncell_total);
    char *p = (char *)d_ws;
    cudaStream_t st = (cudaStream_t)stream;
    JMD_CUDA_TRY(cudaMemcpyAsync(p + w.meta, H->meta.data(), sizeof(RepMeta) * H->meta.size(),
                                 cudaMemcpyHostToDevice, st));
    JMD_CUDA_TRY(cudaMemcpyAsync(p + w.rep_of, H->rep_of.data(), sizeof(int32_t) * H->rep_of.size(),
                                 cudaMemcpyHostToDevice, st));
    JMD_CUDA_TRY(cudaMemcpyAsync(p + w.cell_rep, H->cell_rep.data(), sizeof(int32_t) * H->cell_rep.size(),
                                 cudaMemcpyHostToDevice, st));
    JMD_CUDA_TRY(cudaMemsetAsync(p + w.cell_count, 0, sizeof(int32_t) * (size_t)bt->ncell_total, st));
    JMD_CUDA_TRY(cudaMemsetAsync(p + w.ctl, 0, sizeof(uint32_t) * CTL_WORDS, st));
    JMD_CUDA_TRY(cudaMemsetAsync(p + w.flag, 0, sizeof(uint32_t) * (size_t)bt->R * 2, st));
    JMD_CUDA_TRY(cudaStreamSynchronize(st));   // host vectors stay alive anyway; keep bind synchronous
    return MD_OK;
}

extern "C" md_status md_batch_build(md_batch *bt, const float *d_r, uint32_t *d_status, md_stream_t stream)
{
    if (!bt || !bt->ws || !d_r) return MD_ERR_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    BatchDev b = batch_dev(bt, d_status);
    k_b_flag_all<<<1, 256, 0, st>>>(b);
    enqueue_b_rebuild(b, (const float4 *)d_r, st);
    JMD_CUDA_TRY(cudaGetLastError());
    return MD_OK;
}

extern "C" md_status md_batch_forces(md_batch *bt, const float *d_r, float *d_f, uint32_t *d_status,
                                     md_stream_t stream)
{
    if (!bt || !bt->ws || !d_r || !d_f) return MD_ERR_INVALID;
    BatchDev b = batch_dev(bt, d_status);
    enqueue_b_pair(b, (const float4 *)d_r, nullptr, (float4 *)d_f, 0, (cudaStream_t)stream);
    JMD_CUDA_TRY(cudaGetLastError());
    return MD_OK;
}

extern "C" md_status md_batch_run_nve(md_batch *bt, float *d_r, float *d_v, float *d_f, int nsteps, double *d_PE,
                                      double *d_KE, int use_graph, uint32_t *d_status, md_stream_t stream)
{
    if (!bt || !bt->ws || !bt->host || !d_r || !d_v || !d_f || nsteps < 0) return MD_ERR_INVALID;
    if (nsteps == 0) return MD_OK;
    BatchHost *H = (BatchHost *)bt->host;
    cudaStream_t st = (cudaStream_t)stream;
    BatchDev b = batch_dev(bt, d_status);
    b.wrapped = 1;   // every rebuild in the loop follows a kick-drift, which wraps the positions
    float4 *r = (float4 *)d_r, *v = (float4 *)d_v, *f = (float4 *)d_f;
    if (use_graph) {
        if (!H->exec || H->g_r != d_r || H->g_v != d_v || H->g_f != d_f || H->g_pe != d_PE || H->g_ke != d_KE ||
            H->g_len != nsteps || H->g_tpp != bt->tpp || H->g_status != d_status ||
            H->g_class_version != H->class_version) {
            md_status s = b_graph(*H, b, r, v, f, d_PE, d_KE, nsteps);
            if (s != MD_OK) return s;
            H->g_r = d_r;
            H->g_v = d_v;
            H->g_f = d_f;
            H->g_pe = d_PE;
            H->g_ke = d_KE;
            H->g_len = nsteps;
            H->g_tpp = bt->tpp;
            H->g_status = d_status;
            H->g_class_version = H->class_version;
        }
        k_b_loop_init<<<1, 1, 0, st>>>(b.ctl, (uint32_t)nsteps);
        JMD_CUDA_TRY(cudaGraphLaunch(H->exec, st));
    } else {
        k_b_loop_init<<<1, 1, 0, st>>>(b.ctl, (uint32_t)nsteps);
        int gk = (b.N + 255) / 256;
        for (int s = 0; s < nsteps; ++s) {
            k_b_kick_drift<0><<<gk, 256, 0, st>>>(b, r, v, f, 0ull);
            enqueue_b_rebuild(b, r, st);   // kernels skip replicas with clear flags
            enqueue_b_pair(b, r, v, f, 1, st);
            if (d_PE || d_KE) k_b_energy<<<b.R, 256, 0, st>>>(b, v, f, d_PE, d_KE, nsteps, 0ull, 0);
            else k_b_step<<<1, 1, 0, st>>>(b, 0ull, 0);
        }
    }
    JMD_CUDA_TRY(cudaGetLastError());
    return MD_OK;
}

extern "C" md_status md_batch_set_class_tpp(md_batch *bt, const int *tpp_of_rep, md_stream_t stream)
{
    if (!bt || !bt->host || !bt->ws) return MD_ERR_INVALID;
    BatchHost *H = (BatchHost *)bt->host;
    ++H->class_version;
    if (!tpp_of_rep) {
        H->classes = false;
        return MD_OK;
    }
    std::vector<int32_t> list;
    list.reserve((size_t)bt->N);
    const int tpps[3] = {4, 8, 16};
    for (int k = 0; k < bt->R; ++k)
        if (tpp_of_rep[k] != 4 && tpp_of_rep[k] != 8 && tpp_of_rep[k] != 16) return MD_ERR_INVALID;
    for (int g = 0; g < 3; ++g) {
        const size_t before = list.size();
        for (int k = 0; k < bt->R; ++k)
            if (tpp_of_rep[k] == tpps[g])
                for (int i = 0; i < H->meta[k].n; ++i) list.push_back(H->meta[k].p0 + i);
        H->pgroup[g] = (int)(list.size() - before);
    }
    BatchLayout w = batch_layout(bt->N, bt->R, bt->ncell_total);
    cudaStream_t st = (cudaStream_t)stream;
    JMD_CUDA_TRY(cudaMemcpyAsync((char *)bt->ws + w.plist, list.data(), sizeof(int32_t) * list.size(),
                                 cudaMemcpyHostToDevice, st));
    JMD_CUDA_TRY(cudaStreamSynchronize(st));
    H->classes = true;
    return MD_OK;
}

extern "C" md_status md_batch_stats(const md_batch *bt, uint32_t *h_builds, md_stream_t stream)
{
    if (!bt || !bt->ws || !h_builds) return MD_ERR_INVALID;
    BatchLayout w = batch_layout(bt->N, bt->R, bt->ncell_total);
    cudaStream_t st = (cudaStream_t)stream;
    JMD_CUDA_TRY(cudaMemcpyAsync(h_builds, (char *)bt->ws + w.builds, sizeof(uint32_t) * (size_t)bt->R,
                                 cudaMemcpyDeviceToHost, st));
    JMD_CUDA_TRY(cudaStreamSynchronize(st));
    return MD_OK;
}

// Autotuner: time `probe` graph steps for each threads-per-particle choice
// on the caller's state (restored between trials from d_scratch, which must
// hold 2 N float4) and keep the fastest; the choice is cached in a small
// JSON file keyed by the replica sizes.
extern "C" md_status md_batch_autotune(md_batch *bt, float *d_r, float *d_v, float *d_f, void *d_scratch, int probe,
                                       const char *cache_path, int *tpp_out, md_stream_t stream)
{
    if (!bt || !bt->host || !d_r || !d_v || !d_f || !d_scratch || probe < 1) return MD_ERR_INVALID;
    BatchHost *H = (BatchHost *)bt->host;
    // key: FNV-1a over replica sizes and kinds
    unsigned long long key = 1469598103934665603ull;
    for (const RepMeta &m : H->meta) {
        key = (key ^ (unsigned long long)m.n) * 1099511628211ull;
        key = (key ^ (unsigned long long)m.kind) * 1099511628211ull;
    }
    char keystr[32];
    snprintf(keystr, sizeof(keystr), "%016llx", key);
    if (cache_path) {
        FILE *fp = fopen(cache_path, "r");
        if (fp) {
            char buf[4096];
            size_t n = fread(buf, 1, sizeof(buf) - 1, fp);
            fclose(fp);
            buf[n] = 0;
            std::string s(buf);
            std::string pat = std::string("\"") + keystr + "\": ";
            size_t at = s.find(pat);
            if (at != std::string::npos) {
                int t = atoi(s.c_str() + at + pat.size());
                if (t == 4 || t == 8 || t == 16) {
                    bt->tpp = t;
                    if (tpp_out) *tpp_out = t;
                    return MD_OK;
                }
            }
        }
    }
    cudaStream_t st = (cudaStream_t)stream;
    size_t bytes = sizeof(float4) * (size_t)bt->N;
    float4 *save = (float4 *)d_scratch;
    JMD_CUDA_TRY(cudaMemcpyAsync(save, d_r, bytes, cudaMemcpyDeviceToDevice, st));
    JMD_CUDA_TRY(cudaMemcpyAsync(save + bt->N, d_v, bytes, cudaMemcpyDeviceToDevice, st));
    const int cand[3] = {4, 8, 16};
    float best = 1e30f;
    int best_t = bt->tpp;
    cudaEvent_t e0, e1;
    JMD_CUDA_TRY(cudaEventCreate(&e0));
    JMD_CUDA_TRY(cudaEventCreate(&e1));
    for (int c = 0; c < 3; ++c) {
        bt->tpp = cand[c];
        JMD_CUDA_TRY(cudaMemcpyAsync(d_r, save, bytes, cudaMemcpyDeviceToDevice, st));
        JMD_CUDA_TRY(cudaMemcpyAsync(d_v, save + bt->N, bytes, cudaMemcpyDeviceToDevice, st));
        md_status s = md_batch_build(bt, d_r, nullptr, stream);
        if (s == MD_OK) s = md_batch_forces(bt, d_r, d_f, nullptr, stream);
        if (s == MD_OK) s = md_batch_run_nve(bt, d_r, d_v, d_f, probe, nullptr, nullptr, 1, nullptr, stream);  // warm
        if (s != MD_OK) return s;
        JMD_CUDA_TRY(cudaEventRecord(e0, st));
        s = md_batch_run_nve(bt, d_r, d_v, d_f, probe, nullptr, nullptr, 1, nullptr, stream);
        if (s != MD_OK) return s;
        JMD_CUDA_TRY(cudaEventRecord(e1, st));
        JMD_CUDA_TRY(cudaEventSynchronize(e1));
        float ms = 0.f;
        JMD_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
        if (ms < best) {
            best = ms;
            best_t = cand[c];
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    JMD_CUDA_TRY(cudaMemcpyAsync(d_r, save, bytes, cudaMemcpyDeviceToDevice, st));
    JMD_CUDA_TRY(cudaMemcpyAsync(d_v, save + bt->N, bytes, cudaMemcpyDeviceToDevice, st));
    JMD_CUDA_TRY(cudaStreamSynchronize(st));
    bt->tpp = best_t;
    if (tpp_out) *tpp_out = best_t;
    if (cache_path) {
        FILE *fp = fopen(cache_path, "w");
        if (fp) {
            fprintf(fp, "{\"%s\": %d}\n", keystr, best_t);
            fclose(fp);
        }
    }
    return MD_OK;
}
