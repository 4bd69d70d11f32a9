// nbr.cu -- cell-list binning and Verlet neighbor-list build (Sec. 3.2.3).
//
// Rebuild chain (every kernel can be gated by the device rebuild flag, so the
// chain can sit in a stream and cost only an early exit when no particle has
// moved more than skin/2; inside the NVE graph it sits under an IF node and
// runs ungated):
//   k_bin_count : cell of each particle; warp-aggregated atomic histogram
//                 (one atomic per distinct cell per warp); the returned
//                 offset is the particle's rank inside its cell
//   k_scan      : exclusive scan of the histogram -> cell_start (1 CTA);
//                 zeroes the histogram for the next build
//   k_scatter   : counting-sort scatter of the particle indices (the order
//                 inside a cell is the atomics' arrival order)
//   k_sort_cells: one warp per cell puts its members in ascending particle
//                 order and writes the cell-ordered float4 positions, so the
//                 candidate order is fixed once per build
//   k_build_cells: one CTA per cell stages its stencil's candidates in
//                 shared memory and sweeps them with ballot compaction into
//                 padded int32 rows
#include <cmath>

#include "cells.cuh"
#include "common.cuh"
#include "kernels.cuh"

namespace jmd {

__device__ __forceinline__ int cell_axis(float x, float L, float Linv, float scale, int n)
{
    float y = wrap_coord(x, L, Linv);
    int q = (int)(y * scale);
    return q < 0 ? 0 : (q >= n ? n - 1 : q);
}

// Positions the chain bins and stages: r, or in the fused NVE loop the buffer
// of the current step (odd steps in r_alt).
__device__ __forceinline__ const float4 *chain_positions(const NbrArgs &a)
{
    return (a.r_alt && (*(volatile uint32_t *)&a.ws.ctl[CTL_STEP] & 1u)) ? a.r_alt : a.r;
}

__device__ __forceinline__ bool chain_active(const NbrArgs &a)
{
    return !a.gated || *(volatile uint32_t *)&a.ws.ctl[CTL_REBUILD] != 0u;
}

__global__ void __launch_bounds__(256) k_bin_count(NbrArgs a)
{
    count_launch();
    if (!chain_active(a)) return;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    bool act = i < a.N;
    int c = -1;
    if (act) {
        float4 p = chain_positions(a)[i];
        // a non-finite coordinate would silently drop out of every pair test
        if (!isfinite(p.x) || !isfinite(p.y) || !isfinite(p.z)) raise_status(a.status, MD_ERR_NONFINITE);
        int cx = cell_axis(p.x, a.box.L[0], a.box.Linv[0], a.cell_scale[0], a.nc[0]);
        int cy = cell_axis(p.y, a.box.L[1], a.box.Linv[1], a.cell_scale[1], a.nc[1]);
        int cz = a.dim == 3 ? cell_axis(p.z, a.box.L[2], a.box.Linv[2], a.cell_scale[2], a.nc[2]) : 0;
        c = (cz * a.nc[1] + cy) * a.nc[0] + cx;
    }
    unsigned amask = __ballot_sync(0xffffffffu, act);
    if (!act) return;
    unsigned peers = __match_any_sync(amask, c);
    int lane = threadIdx.x & 31;
    int leader = __ffs(peers) - 1;
    int below = __popc(peers & ((1u << lane) - 1u));
    int base = 0;
    if (lane == leader) base = atomicAdd(&a.ws.cell_count[c], __popc(peers));
    base = __shfl_sync(peers, base, leader);
    a.ws.cell_of[i] = c;
    a.ws.rank[i] = base + below;
}

// Exclusive scan over ncell counts by one CTA of 1024 threads; each thread
// owns a contiguous chunk.  Also clears the histogram for the next build.
__global__ void __launch_bounds__(1024) k_scan(NbrArgs a, int ncell)
{
    count_launch();
    if (!chain_active(a)) return;
    __shared__ int warp_tot[32];
    int t = threadIdx.x;
    int per = (ncell + blockDim.x - 1) / blockDim.x;
    int b = t * per, e = min(b + per, ncell);
    int s = 0;
    for (int q = b; q < e; ++q) s += a.ws.cell_count[q];
    int lane = t & 31, w = t >> 5;
    int x = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[w] = x;
    __syncthreads();
    if (w == 0) {
        int v = (lane < (int)(blockDim.x >> 5)) ? warp_tot[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += y;
        }
        warp_tot[lane] = v;   // inclusive over warps
    }
    __syncthreads();
    int run = x - s + (w > 0 ? warp_tot[w - 1] : 0);
    for (int q = b; q < e; ++q) {
        a.ws.cell_start[q] = run;
        run += a.ws.cell_count[q];
        a.ws.cell_count[q] = 0;
    }
    if (t == blockDim.x - 1) a.ws.cell_start[ncell] = warp_tot[(blockDim.x >> 5) - 1];
}

__global__ void __launch_bounds__(256) k_scatter(NbrArgs a)
{
    count_launch();
    if (!chain_active(a)) return;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.N) return;
    int slot = a.ws.cell_start[a.ws.cell_of[i]] + a.ws.rank[i];
    a.ws.atoms_u[slot] = i;
}

// One warp per cell: rank every member by particle index against the whole
// cell (shuffles, 32 members per pass) and write the members and their
// positions in that order, the particle index in the w lane.  Every stencil that visits the cell then reads
// it already in canonical order.
constexpr int SORT_WARPS = 8;
__global__ void __launch_bounds__(SORT_WARPS * 32) k_sort_cells(NbrArgs a, int ncell)
{
    count_launch();
    if (!chain_active(a)) return;
    const int lane = threadIdx.x & 31;
    const int q = blockIdx.x * SORT_WARPS + (threadIdx.x >> 5);
    if (q >= ncell) return;   // whole warp
    const int b = a.ws.cell_start[q], n = a.ws.cell_start[q + 1] - b;
    const int32_t *u = a.ws.atoms_u + b;
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
            const float4 p = chain_positions(a)[me];
            a.ws.atoms[b + rk] = me;
            a.ws.rsorted[b + rk] = make_float4(p.x, p.y, p.z, __int_as_float(me));   // index in w
            a.rref[me] = p;   // positions of this build (displacement check)
        }
    }
}

// Per-axis stencil cells with duplicates (fewer than 3 cells) removed.
__device__ __forceinline__ int axis_cells(int q, int n, int *out)
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

// Ascending bitonic sort of row[0..n) by one warp; row has CAPP2 (power of
// two) slots, the tail is padded with INT_MAX first.
template <int CAPP2>
__device__ __forceinline__ void warp_sort_row(int *row, int n)
{
    const int lane = threadIdx.x & 31;
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
}

// Canonical mode: sort each finished row ascending (one warp per row).
template <int CAPP2>
__global__ void __launch_bounds__(256) k_sort_rows(NbrArgs a)
{
    count_launch();
    if (!chain_active(a)) return;
    __shared__ int buf[8][CAPP2];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = blockIdx.x * 8 + w; i < a.N; i += gridDim.x * 8) {
        int n = a.cnt[i];
        n = n < a.cap ? n : a.cap;
        int32_t *row = a.nbr + (size_t)i * a.cap;
        for (int k = lane; k < n; k += 32) buf[w][k] = row[k];
        __syncwarp();
        warp_sort_row<CAPP2>(buf[w], n);
        for (int k = lane; k < n; k += 32) row[k] = buf[w][k];
        __syncwarp();
    }
}

// Row of particle i found by one warp scanning the stencil cells directly
// from global memory, then bitonic-sorted in the warp's shared buffer
// (CAPP2 >= cap, power of two).  Used for cells whose stencil holds more
// candidates than the block-staged path can keep in shared memory.
template <int DIM, int CAPP2>
__device__ void build_row_warp(const NbrArgs &a, int i, int c, int *row)
{
    const int lane = threadIdx.x & 31;
    float4 ri = chain_positions(a)[i];
    int cx = c % a.nc[0];
    int cy = (c / a.nc[0]) % a.nc[1];
    int cz = c / (a.nc[0] * a.nc[1]);
    int sx[3], sy[3], sz[3];
    int mx = axis_cells(cx, a.nc[0], sx);
    int my = axis_cells(cy, a.nc[1], sy);
    int mz = DIM == 3 ? axis_cells(cz, a.nc[2], sz) : 1;
    if (DIM != 3) sz[0] = 0;
    int count = 0;
    const unsigned lt = (1u << lane) - 1u;
    for (int zz = 0; zz < mz; ++zz)
        for (int yy = 0; yy < my; ++yy)
            for (int xx = 0; xx < mx; ++xx) {
                int q = (sz[zz] * a.nc[1] + sy[yy]) * a.nc[0] + sx[xx];
                int b = a.ws.cell_start[q], e = a.ws.cell_start[q + 1];
                for (int s = b; s < e; s += 32) {
                    int slot = s + lane;
                    bool hit = false;
                    int j = 0;
                    if (slot < e) {
                        j = a.ws.atoms[slot];
                        float4 rj = a.ws.rsorted[slot];
                        float dx, dy, dz;
                        hit = (j != i) && (dist2_rn<DIM>(ri, rj, a.box, dx, dy, dz) < a.r_list2);
                    }
                    unsigned m = __ballot_sync(0xffffffffu, hit);
                    int pos = count + __popc(m & lt);
                    if (hit && pos < CAPP2) row[pos] = j;
                    count += __popc(m);
                }
            }
    __syncwarp();
    int n = count < a.cap ? count : a.cap;
    warp_sort_row<CAPP2>(row, n);
    int32_t *out = a.nbr + (size_t)i * a.cap;
    for (int k = lane; k < a.cap; k += 32) out[k] = (k < n) ? row[k] : a.N;
    if (lane == 0) {
        a.cnt[i] = count;
        a.rref[i] = ri;
        if (count > a.cap) raise_status(a.status, MD_ERR_NBR_OVERFLOW);
        atomicMax(&a.ws.ctl[CTL_MAXCNT], (uint32_t)count);
    }
    __syncwarp();
}

// ---------------------------------------------------------------------------
// Neighbor-list build: one CTA per cell.  The candidates of the cell's
// stencil (cells.cuh) are copied into shared memory in canonical order with
// the particle index in the w lane (k_sort_cells), and padded with NaN
// positions to whole sweep steps (a NaN fails every distance test, so the
// sweep needs no bounds check).  Each warp takes particles of the cell and
// sweeps the candidates 128 at a time (four ballots), writing hits straight
// into the padded int32 row and, when the list keeps local rows, each hit's
// index into the staged array into the 16-bit row.  The row order is a
// deterministic function of the positions and the cell grid.
// ---------------------------------------------------------------------------
constexpr int BUILD_WARPS = 4;
constexpr int BUILD_CHUNK = 128;  // candidates per sweep step (BUILD_CHUNK / 32 per lane)
static_assert(STAGE_CMAX % BUILD_CHUNK == 0, "the padding must fit the staging buffer");
__device__ __forceinline__ int padded_m(int M) { return (M + BUILD_CHUNK - 1) / BUILD_CHUNK * BUILD_CHUNK; }

// Rows of the cell's particles p = warp, warp + BUILD_WARPS, ...  The
// distance form, all with the same bits: MODE 2, no stencil cell wraps, so
// rint(t * Linv) = 0 and the plain difference is the nearest-image
// displacement; MODE 1, positions inside [0, L) (min_image_near); MODE 0,
// the general formula.
template <int DIM, int MODE, bool LOCAL>
__device__ __forceinline__ int build_sweep(const NbrArgs &a, const float4 *cand, const uint16_t *lidx,
                                           const StencilInfo &inf)
{
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const int M = padded_m(inf.soff[inf.nst]);
    int wmax = 0;
    for (int p = threadIdx.x >> 5; p < inf.own_n; p += BUILD_WARPS) {
        const float4 ri = cand[inf.own_off + p];
        const int i = __float_as_int(ri.w);
        int count = 0;
        int32_t *out = a.nbr + (size_t)i * a.cap;
        uint16_t *lout = LOCAL ? a.lrow + (size_t)i * a.cap : nullptr;
        for (int k0 = 0; k0 < M; k0 += BUILD_CHUNK) {
            constexpr int BU = BUILD_CHUNK / 32;
            bool hit[BU];
            int j[BU];
#pragma unroll
            for (int u = 0; u < BU; ++u) {
                const float4 c = cand[k0 + 32 * u + lane];
                j[u] = __float_as_int(c.w);
                float dx, dy, dz;
                const float r2 = MODE == 2   ? dist2_inner<DIM>(ri, c, dx, dy, dz)
                                 : MODE == 1 ? dist2_near<DIM>(ri, c, a.box, dx, dy, dz)
                                             : dist2_rn<DIM>(ri, c, a.box, dx, dy, dz);
                hit[u] = (j[u] != i) && (r2 < a.r_list2);
            }
#pragma unroll
            for (int u = 0; u < BU; ++u) {
                const unsigned mk = __ballot_sync(0xffffffffu, hit[u]);
                const int pos = count + __popc(mk & lt);
                if (hit[u] && pos < a.cap) {
                    out[pos] = j[u];
                    if (LOCAL) lout[pos] = lidx[k0 + 32 * u + lane];
                }
                count += __popc(mk);
            }
        }
        const int n = count < a.cap ? count : a.cap;
        for (int k = n + lane; k < a.cap; k += 32) {
            out[k] = a.N;
            if (LOCAL) lout[k] = LROW_PAD;
        }
        if (lane == 0) {
            a.cnt[i] = count;
            if (count > a.cap) raise_status(a.status, MD_ERR_NBR_OVERFLOW);
            wmax = count > wmax ? count : wmax;
        }
    }
    return wmax;
}

template <int DIM>
__global__ void __launch_bounds__(BUILD_WARPS * 32) k_build_cells(NbrArgs a)
{
    count_launch();
    if (!chain_active(a)) return;
    __shared__ float4 cand[STAGE_CMAX];
    __shared__ uint16_t lidx[STAGE_CMAX];   // each staged candidate's index in the block region
    __shared__ StencilInfo inf;
    __shared__ RegionInfo reg;
    __shared__ int sreg[27];                // region offset of each stencil cell
    __shared__ int wsum[1];
    __shared__ int bmax;
    const int q = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (warp == 0) {
        int beg, cnt;
        stencil_locate<DIM>(a.nc, a.ws.cell_start, q, lane, beg, cnt);
        stencil_publish<DIM>(a.nc, a.wrapped, q, lane, beg, cnt, inf);
    }
    if (tid == 0) bmax = 0;
    __syncthreads();
    if (inf.own_n == 0) return;   // whole CTA: empty cell
    const int M = inf.soff[inf.nst];
    // local rows: the region of the cell's block (cells.cuh); the force
    // kernel stages the same region when it holds at most REGION_CMAX
    bool local = a.lrow != nullptr && region_grid_ok(a.nc, DIM) && M <= STAGE_CMAX;
    if (local) {
        const int cx = q % a.nc[0], cy = (q / a.nc[0]) % a.nc[1], cz = q / (a.nc[0] * a.nc[1]);
        region_locate<DIM>(a.nc, a.ws.cell_start, cx >> 1, cy >> 1, cz >> 1, reg, wsum);
        local = reg.roff[reg.nreg] <= REGION_CMAX;
        if (tid < inf.nst) {
            // stencil cell (xx, yy, zz) of the cell at region position (px, py, pz)
            const int xx = tid % 3, yy = (tid / 3) % 3, zz = tid / 9;
            const int px = (cx & 1) + 1, py = (cy & 1) + 1, pz = DIM == 3 ? (cz & 1) + 1 : 1;
            const int ri = ((DIM == 3 ? pz + zz - 1 : 0) * reg.ey + (py + yy - 1)) * reg.ex + (px + xx - 1);
            sreg[tid] = reg.roff[ri];
        }
        __syncthreads();
    }
    int wmax = 0;
    if (M > STAGE_CMAX) {
        // dense stencil: per-warp rows straight from global memory with the
        // rows' own sort (int32 rows only); the candidate buffer holds 512
        // ints per warp
        static_assert(sizeof(cand) >= BUILD_WARPS * 512 * sizeof(int), "row buffers must fit");
        int *rowbuf = reinterpret_cast<int *>(cand) + warp * 512;
        for (int p = warp; p < inf.own_n; p += BUILD_WARPS) {
            const int i = a.ws.atoms[inf.own_beg + p];
            if (a.cap <= 128) build_row_warp<DIM, 128>(a, i, q, rowbuf);
            else if (a.cap <= 256) build_row_warp<DIM, 256>(a, i, q, rowbuf);
            else build_row_warp<DIM, 512>(a, i, q, rowbuf);
        }
    } else {
        for (int m = warp; m < inf.nst; m += BUILD_WARPS) {
            const int b0 = inf.soff[m], n = inf.soff[m + 1] - b0;
            const float4 *src = a.ws.rsorted + inf.sbeg[m];
            for (int k = lane; k < n; k += 32) {
                cand[b0 + k] = src[k];
                if (local) lidx[b0 + k] = (uint16_t)(sreg[m] + k);
            }
        }
        const float nan = __int_as_float(0x7fc00000);
        for (int k = M + tid; k < padded_m(M); k += BUILD_WARPS * 32)
            cand[k] = make_float4(nan, nan, nan, __int_as_float(-1));
        __syncthreads();
        // the local-row stores are a template switch, so the plain sweep
        // carries no branch for them
        if (local)
            wmax = inf.inner   ? build_sweep<DIM, 2, true>(a, cand, lidx, inf)
                   : a.wrapped ? build_sweep<DIM, 1, true>(a, cand, lidx, inf)
                               : build_sweep<DIM, 0, true>(a, cand, lidx, inf);
        else
            wmax = inf.inner   ? build_sweep<DIM, 2, false>(a, cand, nullptr, inf)
                   : a.wrapped ? build_sweep<DIM, 1, false>(a, cand, nullptr, inf)
                               : build_sweep<DIM, 0, false>(a, cand, nullptr, inf);
    }
    // one atomic per CTA for the largest row count
    if (lane == 0 && wmax > 0) atomicMax(&bmax, wmax);
    __syncthreads();
    if (tid == 0 && bmax > 0) atomicMax(&a.ws.ctl[CTL_MAXCNT], (uint32_t)bmax);
}

// Sets the rebuild flag if any particle moved more than skin/2 (minimum
// image) since the last build.
template <int DIM>
__global__ void __launch_bounds__(256) k_check_disp(const float4 *r, const float4 *rref, int N, Box box,
                                                    float half_skin2, uint32_t *ctl)
{
    count_launch();
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    bool mv = false;
    if (i < N) {
        float dx, dy, dz;
        mv = dist2_rn<DIM>(r[i], rref[i], box, dx, dy, dz) > half_skin2;
    }
    if (__any_sync(0xffffffffu, mv) && (threadIdx.x & 31) == 0) ctl[CTL_REBUILD] = 1u;
}

__global__ void k_set_flag(uint32_t *ctl, uint32_t v)
{
    count_launch();
    ctl[CTL_REBUILD] = v;
}

// Counts a finished build and clears the rebuild flag (single thread).
__global__ void k_finish_build(uint32_t *ctl)
{
    count_launch();
    if (ctl[CTL_REBUILD] != 0u) {
        unsigned long long *b = (unsigned long long *)&ctl[CTL_BUILDS_LO];
        *b += 1ull;
    }
    ctl[CTL_REBUILD] = 0u;
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
NbrArgs make_nbr_args(const md_space *s, const float *d_r, const md_nbr *nb, uint32_t *d_status, int gated)
{
    NbrArgs a;
    memset(&a, 0, sizeof(a));
    a.box = make_box(s);
    a.N = nb->N;
    a.cap = nb->cap;
    a.dim = nb->dim;
    for (int k = 0; k < 3; ++k) {
        a.nc[k] = nb->ncell[k];
        a.cell_scale[k] = nb->cell_scale[k];
    }
    a.r_list2 = nb->r_list2;
    a.r = (const float4 *)d_r;
    a.nbr = nb->nbr;
    a.lrow = ws_ptrs(nb).lrow;
    a.cnt = nb->cnt;
    a.rref = (float4 *)nb->rref;
    a.ws = ws_ptrs(nb);
    a.status = d_status;
    a.gated = gated;
    a.canonical = (nb->flags & MD_NBR_CANONICAL) ? 1 : 0;
    return a;
}

// Only the cell list of the rebuild chain (binning, counting sort, members
// in ascending order per cell): atoms / cell_start for the spatial sort.
void enqueue_cell_binning(const NbrArgs &a, int ncell_total, cudaStream_t st)
{
    int tb = 256, nb = (a.N + tb - 1) / tb;
    k_bin_count<<<nb, tb, 0, st>>>(a);
    k_scan<<<1, 1024, 0, st>>>(a, ncell_total);
    k_scatter<<<nb, tb, 0, st>>>(a);
    k_sort_cells<<<(ncell_total + SORT_WARPS - 1) / SORT_WARPS, SORT_WARPS * 32, 0, st>>>(a, ncell_total);
}

// Enqueue the (gated or ungated) rebuild chain.  The flag is consumed by
// k_finish_build at the end.
void enqueue_rebuild_chain(const NbrArgs &a, int ncell_total, cudaStream_t st)
{
    int tb = 256, nb = (a.N + tb - 1) / tb;
    k_bin_count<<<nb, tb, 0, st>>>(a);
    k_scan<<<1, 1024, 0, st>>>(a, ncell_total);
    k_scatter<<<nb, tb, 0, st>>>(a);
    k_sort_cells<<<(ncell_total + SORT_WARPS - 1) / SORT_WARPS, SORT_WARPS * 32, 0, st>>>(a, ncell_total);
    if (a.dim == 3) k_build_cells<3><<<ncell_total, BUILD_WARPS * 32, 0, st>>>(a);
    else k_build_cells<2><<<ncell_total, BUILD_WARPS * 32, 0, st>>>(a);
    if (a.canonical) {
        int g = (a.N + 7) / 8;
        g = g < 4096 ? g : 4096;
        if (a.cap <= 64) k_sort_rows<64><<<g, 256, 0, st>>>(a);
        else if (a.cap <= 128) k_sort_rows<128><<<g, 256, 0, st>>>(a);
        else if (a.cap <= 256) k_sort_rows<256><<<g, 256, 0, st>>>(a);
        else k_sort_rows<512><<<g, 256, 0, st>>>(a);
    }
    k_finish_build<<<1, 1, 0, st>>>(a.ws.ctl);
}

void enqueue_check_disp(const md_space *s, const float *d_r, const md_nbr *nb, cudaStream_t st)
{
    WsPtrs w = ws_ptrs(nb);
    int tb = 256, g = (nb->N + tb - 1) / tb;
    Box box = make_box(s);
    if (nb->dim == 3)
        k_check_disp<3><<<g, tb, 0, st>>>((const float4 *)d_r, (const float4 *)nb->rref, nb->N, box, nb->half_skin2,
                                          w.ctl);
    else
        k_check_disp<2><<<g, tb, 0, st>>>((const float4 *)d_r, (const float4 *)nb->rref, nb->N, box, nb->half_skin2,
                                          w.ctl);
}

static bool nbr_ready(const md_nbr *nb)
{
    return nb && nb->nbr && nb->cnt && nb->rref && nb->ws && nb->N > 0 && nb->cap > 0 && nb->cap <= 512 &&
           nbr_layout_ok(nb);
}

}  // namespace jmd

using namespace jmd;

extern "C" md_status md_nbr_plan(const md_space *s, int N, float r_cut, float skin, int cap, md_nbr *out)
{
    if (!s || !out || N < 1 || cap < 1 || cap > 512 || !(r_cut > 0.0f) || !(skin >= 0.0f) ||
        (s->dim != 2 && s->dim != 3))
        return MD_ERR_INVALID;
    md_nbr nb;
    memset(&nb, 0, sizeof(nb));
    nb.dim = s->dim;
    nb.N = N;
    nb.cap = cap;
    nb.r_cut = r_cut;
    nb.skin = skin;
    float rl = r_cut + skin;
    nb.r_list = rl;
    nb.r_list2 = rl * rl;
    float hs = 0.5f * skin;
    nb.half_skin2 = hs * hs;
    nb.ncell_total = 1;
    for (int k = 0; k < 3; ++k) {
        nb.ncell[k] = 1;
        nb.cell_scale[k] = 0.0f;
        if (k < s->dim) {
            if ((double)s->L[k] < 2.0 * (double)rl) return MD_ERR_BOX_TOO_SMALL;
            // cells of side >= r_list with a margin above FP32 rounding of
            // coordinates and of the membership test
            int n = (int)floor((double)s->L[k] / ((double)rl * (1.0 + 1e-4)));
            nb.ncell[k] = n < 1 ? 1 : n;
            nb.cell_scale[k] = (float)((double)nb.ncell[k] / (double)s->L[k]);
        }
        nb.ncell_total *= nb.ncell[k];
    }
    nb.flags = 0;
    nb.ws_bytes = ws_layout(N, nb.ncell_total, cap, 0).total;
    *out = nb;
    return MD_OK;
}

extern "C" md_status md_nbr_set_flags(md_nbr *nb, int flags)
{
    if (!nb || (flags & ~(MD_NBR_CANONICAL | MD_NBR_LOCAL_ROWS | MD_NBR_TILES))) return MD_ERR_INVALID;
    if ((flags & MD_NBR_CANONICAL) && (flags & (MD_NBR_LOCAL_ROWS | MD_NBR_TILES))) return MD_ERR_INVALID;
    if ((flags & MD_NBR_LOCAL_ROWS) && (flags & MD_NBR_TILES)) return MD_ERR_INVALID;
    if ((flags & MD_NBR_TILES) && !tiles_plan_ok(nullptr, nb)) return MD_ERR_INVALID;
    nb->flags = flags;
    nb->ws_bytes = ws_layout(nb->N, nb->ncell_total, nb->cap, flags, nb->ncell).total;
    return MD_OK;
}

extern "C" md_status md_nbr_bind(md_nbr *nb, int32_t *d_nbr, int32_t *d_cnt, float *d_rref, void *d_ws,
                                 md_stream_t stream)
{
    if (!nb || !d_nbr || !d_cnt || !d_rref || !d_ws) return MD_ERR_INVALID;
    if (!nbr_layout_ok(nb)) return MD_ERR_INVALID;
    if (((uintptr_t)d_ws & 255u) || ((uintptr_t)d_rref & 15u) || ((uintptr_t)d_nbr & 15u)) return MD_ERR_INVALID;
    nb->nbr = d_nbr;
    nb->cnt = d_cnt;
    nb->rref = d_rref;
    nb->ws = d_ws;
    WsPtrs w = ws_ptrs(nb);
    cudaStream_t st = (cudaStream_t)stream;
    JMD_CUDA_TRY(cudaMemsetAsync(w.ctl, 0, sizeof(uint32_t) * CTL_WORDS, st));
    JMD_CUDA_TRY(cudaMemsetAsync(w.cell_count, 0, sizeof(int32_t) * (size_t)nb->ncell_total, st));
    if (nb->flags & MD_NBR_TILES) {
        // the tile engine's histogram must start at zero; its cell starts at
        // zero describe an empty system until the first import
        const WsLayout wl = ws_layout(nb->N, nb->ncell_total, nb->cap, nb->flags, nb->ncell);
        TilePlan tp;
        const int nt = tile_geometry(nb->N, nb->ncell, tp) ? tp.ntiles : 0;
        const TileLayout tl = tile_layout(nb->N, 8 * nb->ncell_total, nb->cap, nt);
        char *tb = (char *)d_ws + wl.tiles;
        // histogram, cell starts and tile tables (zero tables stage nothing)
        JMD_CUDA_TRY(cudaMemsetAsync(tb + tl.hcount, 0, tl.bsum - tl.hcount, st));
    }
    return MD_OK;
}

extern "C" md_status md_neighbor_list_build(const md_space *s, const float *d_r, md_nbr *nb, uint32_t *d_status,
                                            md_stream_t stream)
{
    if (!s || !d_r || !nbr_ready(nb) || s->dim != nb->dim) return MD_ERR_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    WsPtrs w = ws_ptrs(nb);
    k_set_flag<<<1, 1, 0, st>>>(w.ctl, 1u);
    NbrArgs a = make_nbr_args(s, d_r, nb, d_status, 1);
    enqueue_rebuild_chain(a, nb->ncell_total, st);
    JMD_CUDA_TRY(cudaGetLastError());
    return MD_OK;
}

extern "C" md_status md_neighbor_list_update(const md_space *s, const float *d_r, md_nbr *nb, uint32_t *d_status,
                                             md_stream_t stream)
{
    if (!s || !d_r || !nbr_ready(nb) || s->dim != nb->dim) return MD_ERR_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    enqueue_check_disp(s, d_r, nb, st);
    NbrArgs a = make_nbr_args(s, d_r, nb, d_status, 1);
    enqueue_rebuild_chain(a, nb->ncell_total, st);
    JMD_CUDA_TRY(cudaGetLastError());
    return MD_OK;
}

extern "C" md_status md_nbr_stats(const md_nbr *nb, int64_t *builds, int32_t *max_count, md_stream_t stream)
{
    if (!nbr_ready(nb)) return MD_ERR_INVALID;
    WsPtrs w = ws_ptrs(nb);
    uint32_t h[CTL_WORDS];
    cudaStream_t st = (cudaStream_t)stream;
    JMD_CUDA_TRY(cudaMemcpyAsync(h, w.ctl, sizeof(h), cudaMemcpyDeviceToHost, st));
    JMD_CUDA_TRY(cudaStreamSynchronize(st));
    if (builds) *builds = (int64_t)(((uint64_t)h[CTL_BUILDS_HI] << 32) | h[CTL_BUILDS_LO]);
    if (max_count) *max_count = (int32_t)h[CTL_MAXCNT];
    return MD_OK;
}
