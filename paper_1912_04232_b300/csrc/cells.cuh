// cells.cuh -- the stencil of one cell of the cell list (Sec. 3.2.3), shared
// by the neighbor build and the cell-centred force kernel.
//
// The cells of a cell's stencil, in canonical order: z, y, x offsets
// ascending (-1, 0, +1 with periodic wrap), duplicates removed on axes with
// fewer than three cells.  With the members of every cell in ascending
// particle order (k_sort_cells), concatenating the stencil cells gives the
// "staged" candidate array of the cell; an index into it is a local index.
#pragma once

#include "common.cuh"

namespace jmd {

struct StencilInfo {
    int soff[28];          // prefix of the stencil cells' counts (soff[nst] = M)
    int sbeg[27];          // first slot of each stencil cell
    int nst;               // stencil cells
    int own_off, own_n;    // the cell's own members in the staged array
    int own_beg;           // ... and their first slot
    int inner;             // no stencil cell wraps (and positions inside [0, L))
};

// Stencil cells of one axis: offset o of coordinate c among n cells; the
// own cell's offset.
__device__ __forceinline__ int axis_count(int n) { return n >= 3 ? 3 : n; }
__device__ __forceinline__ int axis_cell(int c, int n, int o)
{
    if (n >= 3) {
        int x = c + o - 1;
        return x < 0 ? x + n : (x >= n ? x - n : x);
    }
    return o;
}
__device__ __forceinline__ int axis_own(int c, int n) { return n >= 3 ? 1 : (n == 2 ? c : 0); }

// Lane m of one warp: first slot and count of stencil cell m of cell q.
template <int DIM>
__device__ __forceinline__ void stencil_locate(const int *nc, const int32_t *cell_start, int q, int lane, int &beg,
                                               int &cnt)
{
    const int cx = q % nc[0], cy = (q / nc[0]) % nc[1], cz = q / (nc[0] * nc[1]);
    const int mx = axis_count(nc[0]), my = axis_count(nc[1]), mz = DIM == 3 ? axis_count(nc[2]) : 1;
    beg = 0;
    cnt = 0;
    if (lane < mx * my * mz) {
        const int xx = lane % mx, yy = (lane / mx) % my, zz = lane / (mx * my);
        const int c =
            ((DIM == 3 ? axis_cell(cz, nc[2], zz) : 0) * nc[1] + axis_cell(cy, nc[1], yy)) * nc[0] + axis_cell(cx, nc[0], xx);
        beg = cell_start[c];
        cnt = cell_start[c + 1] - beg;
    }
}

// The same warp: prefix of the located counts and the rest of the cell's
// info.  wrapped: positions are inside [0, L) (enables `inner`).
template <int DIM>
__device__ __forceinline__ void stencil_publish(const int *nc, int wrapped, int q, int lane, int beg, int cnt,
                                                StencilInfo &inf)
{
    const int cx = q % nc[0], cy = (q / nc[0]) % nc[1], cz = q / (nc[0] * nc[1]);
    const int mx = axis_count(nc[0]), my = axis_count(nc[1]), mz = DIM == 3 ? axis_count(nc[2]) : 1;
    const int m = mx * my * mz;
    const int own = ((DIM == 3 ? axis_own(cz, nc[2]) : 0) * my + axis_own(cy, nc[1])) * mx + axis_own(cx, nc[0]);
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    const int own_off = __shfl_sync(0xffffffffu, incl - cnt, own);
    const int own_n = __shfl_sync(0xffffffffu, cnt, own);
    const int own_beg = __shfl_sync(0xffffffffu, beg, own);
    if (lane < m) {
        inf.soff[lane + 1] = incl;
        inf.sbeg[lane] = beg;
    }
    if (lane == 0) {
        bool inner = wrapped != 0;
        const int cc[3] = {cx, cy, cz};
#pragma unroll
        for (int d = 0; d < DIM; ++d) inner = inner && nc[d] >= 5 && cc[d] >= 1 && cc[d] <= nc[d] - 2;
        inf.soff[0] = 0;
        inf.nst = m;
        inf.own_off = own_off;
        inf.own_n = own_n;
        inf.own_beg = own_beg;
        inf.inner = inner ? 1 : 0;
    }
}

// Candidates a CTA stages per cell; cells whose stencil holds more take the
// per-particle paths with global (int32) rows.
constexpr int STAGE_CMAX = 1024;

// ---------------------------------------------------------------------------
// Cell blocks and their regions (local rows).  Along each axis the cells are
// grouped in blocks of two (the last block of an odd axis holds one); the
// region of a block is the block grown by one cell on each side, 4 (or 3)
// cells per axis with periodic wrap, which contains the stencil of every
// cell of the block.  With at least 4 cells on every axis the region's cells
// are distinct.  The region's cells are taken in (z, y, x) order, members in
// ascending particle order; a local row entry is the partner's index in this
// concatenation.
// ---------------------------------------------------------------------------
constexpr int REGION_CMAX = 2048;   // particles a force CTA stages per block
constexpr int REGION_CELLS = 64;    // 4 x 4 x 4

__host__ __device__ __forceinline__ int blocks_along(int n) { return (n + 1) / 2; }
// cells of block b's region along an axis of n cells
__device__ __forceinline__ int region_extent(int b, int n) { return (2 * b + 1 < n) ? 4 : 3; }
// region cell o of block b (o = 0 is the cell before the block)
__device__ __forceinline__ int region_cell(int b, int n, int o)
{
    int x = 2 * b - 1 + o;
    return x < 0 ? x + n : (x >= n ? x - n : x);
}
// local rows need distinct region cells: at least 4 cells on every used axis
__host__ __device__ __forceinline__ bool region_grid_ok(const int *nc, int dim)
{
    return nc[0] >= 4 && nc[1] >= 4 && (dim < 3 || nc[2] >= 4);
}

struct RegionInfo {
    int ex, ey, ez;         // region extent in cells
    int nreg;               // ex * ey * ez
    int roff[REGION_CELLS + 1];   // prefix of the region cells' counts
    int rbeg[REGION_CELLS];       // first slot of each region cell
};

// Two warps (lanes t = 0..63 of threads 0..63): counts and first slots of
// the region cells of block (bx, by, bz), prefix into inf.roff.  Called by
// every thread of the CTA (contains __syncthreads); inf is shared.
template <int DIM>
__device__ __forceinline__ void region_locate(const int *nc, const int32_t *cell_start, int bx, int by, int bz,
                                              RegionInfo &inf, int *wsum)
{
    const int t = threadIdx.x;
    const int ex = region_extent(bx, nc[0]), ey = region_extent(by, nc[1]);
    const int ez = DIM == 3 ? region_extent(bz, nc[2]) : 1;
    const int nreg = ex * ey * ez;
    int cnt = 0;
    if (t < REGION_CELLS) {
        int beg = 0;
        if (t < nreg) {
            const int rx = t % ex, ry = (t / ex) % ey, rz = t / (ex * ey);
            const int c = ((DIM == 3 ? region_cell(bz, nc[2], rz) : 0) * nc[1] + region_cell(by, nc[1], ry)) * nc[0] +
                          region_cell(bx, nc[0], rx);
            beg = cell_start[c];
            cnt = cell_start[c + 1] - beg;
        }
        inf.rbeg[t] = beg;
        int incl = cnt;
        const int lane = t & 31;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        inf.roff[t + 1] = incl;   // within the warp; the second warp adds the first's total below
        if (t == 31) wsum[0] = incl;
    }
    if (t == 0) {
        inf.roff[0] = 0;
        inf.ex = ex;
        inf.ey = ey;
        inf.ez = ez;
        inf.nreg = nreg;
    }
    __syncthreads();
    if (t >= 32 && t < REGION_CELLS) inf.roff[t + 1] += wsum[0];
    __syncthreads();
}

// Local-row padding value (no candidate has this index).
constexpr uint16_t LROW_PAD = 0xffffu;

}  // namespace jmd
