// tiles.cu -- the tile engine: velocity-Verlet NVE for Lennard-Jones and
// soft-sphere particles in 3-D (Sec. 3.3.1) on neighbor lists (Sec. 3.2.3)
// laid out for shared memory.
//
// Data layout (MD_NBR_TILES scratch, see common.cuh tile_layout):
//   * half-cells: 2 x 2 x 2 per cell of the list's grid (side >= r_list/2),
//     index h = (hz * Hy + hy) * Hx + hx;
//   * particles live in memory in half-cell order (slots), members of a
//     half-cell by ascending caller index; every rebuild re-sorts them, and
//     ids[slot] is the caller's index;
//   * a tile is a column of 1 x t x t half-cells; its region is the tile
//     grown by two half-cells on each side (periodic), 5 x (t+4) x (t+4)
//     half-cells in (z, y, x) order.  A row (fixed y, z) of the region is a
//     run of 5 consecutive half-cells along x, i.e. one or two contiguous
//     slot ranges;
//   * a particle's row holds 16-bit indices into its tile's region (the
//     partners, then the sentinel index reg_cap up to the longest row of its
//     warp rounded up to 8); cnt[slot] = the number of partners.  The step
//     kernels stage each region copy at its periodic image (shift codes in
//     the tile's table), so every partner's nearest-image vector is the
//     plain difference of staged positions.
//
// Rebuild chain (under the loop's IF node, or gated by the rebuild flag):
//   k_t_bin     wrap-free half-cell of every particle, warp-aggregated
//               atomic histogram, rank inside the half-cell
//   k_t_scan1/2/3  exclusive scan of the histogram (blocks, block totals,
//               add), clearing the histogram
//   k_t_scatter counting-sort scatter of the source slots
//   k_t_place   members of each half-cell by ascending caller index;
//               positions (wrapped), velocities, ids and build positions
//               written to the other buffer set
//   k_t_build   one CTA per tile: stage the region (bulk copies), then one
//               thread per own particle tests the x-pruned runs of its
//               5 x 5 x 5 half-cell window and writes its row
//   k_t_finish  switches the buffer sets, counts the build
// Step:
//   k_t_step    one CTA per tile: stage the region (bulk copies), forces
//               from shared memory, closing half-kick, next kick-drift
//               (positions not wrapped between rebuilds), displacement
//               check, FP64 energies (fixed order, last block)
#include <cmath>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"

namespace jmd {

// Self-checks of the staging and row indices (built with -DJMD_TILE_CHECKS):
// a failed check counts itself in ctl[32 + id], raises MD_ERR_BOUNDS and
// skips the access.
#ifdef JMD_TILE_CHECKS
#define TCHECK(a, cond, id) ((cond) ? true : (atomicAdd(&(a).ctl[32 + (id)], 1u), raise_status((a).status, MD_ERR_BOUNDS), false))
#else
#define TCHECK(a, cond, id) true
#endif

constexpr int TT = 256;                                          // threads per CTA of every tile kernel
constexpr int NQ_MAX = (TILE_XMAX + 4) * (TILE_TMAX + 4) * (TILE_TMAX + 4);   // region half-cells
constexpr int OWN_MAX = TILE_OWN_MAX;                            // own half-cells of a tile

struct TileArgs {
    Box box;
    int N, cap;
    int H[3], tx, ty, tz, ntx, nty, ntz, ntiles, reg_cap, nhc;
    float hscale[3];
    float r_list2, half_skin2;
    int32_t *hcount, *hstart, *bsum, *key, *rank, *tmp;
    float4 *rb0, *rb1, *vb0, *vb1;
    int32_t *pb0, *pb1;
    float4 *rref, *fs;
    uint32_t *cnt;
    uint16_t *rows;
    uint4 *sent;          // a row chunk of eight sentinel entries (written by every build)
    int32_t *tab;         // per-tile tables (TILE_TAB_WORDS each)
    uint32_t *ctl;
    double2 *partials;
    uint32_t *status;
    // caller arrays (import / export)
    const float4 *r_in, *v_in, *f_in;
    float4 *r_out, *v_out, *f_out, *rref_out;
    int32_t *nbr_out, *cnt_out;
    int export_rows;
    // potential
    int pot;
    float rc2, e_shift, eps, alpha;
    float lj_f12, lj_f6, lj_e12, lj_e6;   // 48 eps sigma^12, 24 eps sigma^6, 4 eps sigma^12, 4 eps sigma^6
    // integration and reductions
    float hdm, dt, mass;
    double *E_out, *KE_out;
    int series;
    unsigned long long cond_while, cond_if;
    int use_cond;
    int gated;    // 1: the chain runs only if ctl[CTL_REBUILD] != 0
    int import;   // 1: the chain reads the caller's arrays
    int variant;  // lanes per particle of the step kernel (part of a cached graph's key)
};

// ---------------------------------------------------------------------------
// device helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool t_active(const TileArgs &a)
{
    return !a.gated || *(volatile uint32_t *)&a.ctl[CTL_REBUILD] != 0u;
}
__device__ __forceinline__ uint32_t t_sel(const TileArgs &a) { return *(volatile uint32_t *)&a.ctl[CTL_TSEL]; }
__device__ __forceinline__ float4 *t_r(const TileArgs &a, uint32_t b) { return b ? a.rb1 : a.rb0; }
__device__ __forceinline__ float4 *t_v(const TileArgs &a, uint32_t b) { return b ? a.vb1 : a.vb0; }
__device__ __forceinline__ int32_t *t_p(const TileArgs &a, uint32_t b) { return b ? a.pb1 : a.pb0; }
__device__ __forceinline__ int wrapi(int x, int n) { return x < 0 ? x + n : (x >= n ? x - n : x); }

__device__ __forceinline__ int h_axis(float x, float L, float Linv, float scale, int n)
{
    const float y = wrap_coord(x, L, Linv);
    const int q = (int)(y * scale);
    return q < 0 ? 0 : (q >= n ? n - 1 : q);
}

__device__ __forceinline__ uint32_t ld_nc_u32(const uint16_t *p)
{
    uint32_t v;
    asm volatile("ld.global.nc.L1::no_allocate.b32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}

// Tile geometry: own half-cells x0..x0+nx-1, y0..y0+ny-1, z0..z0+nz-1; the
// region is RX x RY x RZ half-cells from (x0-2, y0-2, z0-2), periodic.
struct TGeo {
    int x0, y0, z0, nx, ny, nz, RX, RY, RZ, nq, nown;
};
__device__ __forceinline__ TGeo t_geo(const TileArgs &a, int b)
{
    TGeo g;
    const int ix = b % a.ntx, r = b / a.ntx;
    const int iy = r % a.nty, iz = r / a.nty;
    g.x0 = ix * a.tx;
    g.y0 = iy * a.ty;
    g.z0 = iz * a.tz;
    g.nx = min(a.tx, a.H[0] - g.x0);
    g.ny = min(a.ty, a.H[1] - g.y0);
    g.nz = min(a.tz, a.H[2] - g.z0);
    g.RX = g.nx + 4;
    g.RY = g.ny + 4;
    g.RZ = g.nz + 4;
    g.nq = g.RX * g.RY * g.RZ;
    g.nown = g.nx * g.ny * g.nz;
    return g;
}
// Global half-cell of region half-cell q.
__device__ __forceinline__ int t_hglob(const TileArgs &a, const TGeo &g, int q)
{
    const int xl = q % g.RX, yl = (q / g.RX) % g.RY, zl = q / (g.RX * g.RY);
    const int gx = wrapi(g.x0 - 2 + xl, a.H[0]);
    const int gy = wrapi(g.y0 - 2 + yl, a.H[1]);
    const int gz = wrapi(g.z0 - 2 + zl, a.H[2]);
    return (gz * a.H[1] + gy) * a.H[0] + gx;
}
// Region half-cell of own half-cell k.
__device__ __forceinline__ int t_ownq(const TGeo &g, int k)
{
    const int xo = k % g.nx, yo = (k / g.nx) % g.ny, zo = k / (g.nx * g.ny);
    return (2 + xo) + g.RX * ((2 + yo) + g.RY * (2 + zo));
}

// Shared tables of the step kernels (the build adds the region's
// half-cell offsets, TileSm).
struct TileStepSm {
    int own_off[OWN_MAX + 1];      // own half-cell -> first own particle (prefix)
    int own_slot[OWN_MAX];         // own half-cell -> first slot
    int own_loc[OWN_MAX];          // own half-cell -> first local index
    int total;
    int nown;
    int ok;
    unsigned char *kmap;   // own particle -> own half-cell (dynamic shared memory after the positions)
    unsigned long long bar;        // mbarrier of the bulk copies
};

struct TileSm {
    int hoff[NQ_MAX + 1];          // region half-cell -> first local index (exclusive prefix)
    int own_off[OWN_MAX + 1];      // own half-cell -> first own particle (prefix)
    int own_slot[OWN_MAX];         // own half-cell -> first slot
    int own_loc[OWN_MAX];          // own half-cell -> first local index
    int wtot[TT / 32];
    int total;
    int nown;
    int ok;
    unsigned char *kmap;   // own particle -> own half-cell (dynamic shared memory after the positions)
    unsigned long long bar;        // mbarrier of the bulk copies
};

__device__ __forceinline__ uint32_t sm_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(sm_addr(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(sm_addr(bar)), "r"(bytes) : "memory");
}
// try_wait may suspend the thread until the phase completes, for at most
// the hint (20 us), so the bounded wait below spins little.
__device__ __forceinline__ bool mbar_test(unsigned long long *bar, unsigned phase)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(sm_addr(bar)), "r"(phase), "r"(20000u)
        : "memory");
    return ok != 0;
}
// Bulk copy of `bytes` (multiple of 16, both addresses 16-byte aligned)
// from global to shared memory, completing on `bar`.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, unsigned long long *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     sm_addr(dst)),
                 "l"(src), "r"(bytes), "r"(sm_addr(bar))
                 : "memory");
}

// Block-wide exclusive scan of one int per thread (TT threads); returns the
// thread's exclusive prefix, the total in *tot (all threads).
__device__ __forceinline__ int block_excl_scan(int v, int *wtot, int *tot)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wtot[w] = x;
    __syncthreads();
    if (w == 0) {
        int u = lane < TT / 32 ? wtot[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, u, o);
            if (lane >= o) u += y;
        }
        if (lane < TT / 32) wtot[lane] = u;   // inclusive over warps
    }
    __syncthreads();
    const int ex = x - v + (w > 0 ? wtot[w - 1] : 0);
    *tot = wtot[TT / 32 - 1];
    __syncthreads();
    return ex;
}

// Region of tile g from the cell starts: local offset of every region
// half-cell (sm.hoff, exclusive prefix, total in sm.total) and the own
// half-cells' first slots, local indices and particle prefix.
__device__ void tile_scan(const TileArgs &a, const TGeo &g, TileSm &sm)
{
    const int tid = threadIdx.x;
    constexpr int PER = (NQ_MAX + TT - 1) / TT;
    const int qb = tid * PER;
    int c[PER];
    int s = 0;
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int q = qb + k;
        c[k] = 0;
        if (q < g.nq) {
            const int h = t_hglob(a, g, q);
            c[k] = __ldg(a.hstart + h + 1) - __ldg(a.hstart + h);
        }
        s += c[k];
    }
    int tot;
    int run = block_excl_scan(s, sm.wtot, &tot);
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int q = qb + k;
        if (q < g.nq) sm.hoff[q] = run;
        run += c[k];
    }
    if (tid == 0) {
        sm.hoff[g.nq] = tot;
        sm.total = tot;
    }
    __syncthreads();
    // own half-cells: region (2 + xo, 2 + yo, 2 + zo)
    int oc = 0;
    if (tid < g.nown) {
        const int q = t_ownq(g, tid);
        sm.own_loc[tid] = sm.hoff[q];
        oc = sm.hoff[q + 1] - sm.hoff[q];
        sm.own_slot[tid] = __ldg(a.hstart + t_hglob(a, g, q));
    }
    int otot;
    const int oex = block_excl_scan(oc, sm.wtot, &otot);
    if (tid < g.nown) sm.own_off[tid] = oex;
    if (tid == 0) {
        sm.own_off[g.nown] = otot;
        sm.nown = g.nown;
    }
    __syncthreads();
}

// Own particle p -> its own half-cell (sm.kmap), from the own tables.
template <class SM>
__device__ __forceinline__ void tile_own_map(SM &sm)
{
    for (int k = threadIdx.x; k < sm.nown; k += TT)
        for (int p = sm.own_off[k]; p < sm.own_off[k + 1]; ++p) sm.kmap[p] = (unsigned char)k;
    __syncthreads();
}

// Thread 0 waits (bounded, about a second of SM clocks) for the region's
// bulk copies; on a timeout it raises MD_ERR_TIMEOUT and waits once more for
// the copies still in flight, which target this CTA's shared memory.  The
// other threads wait at the block barrier.  Returns sm.ok (uniform).
template <class SM>
__device__ bool tile_wait(const TileArgs &a, SM &sm)
{
    if (threadIdx.x == 0) {
        bool done = mbar_test(&sm.bar, 0u);
        const long long t0 = clock64();
        while (!done && clock64() - t0 < (2ll << 30)) done = mbar_test(&sm.bar, 0u);
        if (!done) {
            raise_status(a.status, MD_ERR_TIMEOUT);
            const long long t1 = clock64();
            while (!mbar_test(&sm.bar, 0u) && clock64() - t1 < (2ll << 30)) {
            }
        }
        sm.ok = done ? 1 : 0;
    }
    __syncthreads();
    return sm.ok != 0;
}

// Build: after tile_scan, stage the region's positions (one thread per
// region row: the run of half-cells along x is one slot range, or two
// where it wraps, one bulk copy each) and write the tile's table for the
// steps that follow.
// Returns false (uniformly) if the region exceeds the capacity.
__device__ bool tile_stage_build(const TileArgs &a, const TGeo &g, TileSm &sm, const float4 *rsrc, float4 *cand,
                                 int32_t *tab)
{
    const int tid = threadIdx.x;
    const int tot = sm.total;
    if (tid == 0) {
        // the region crosses the box on some axis: some copies need a shift
        const bool wraps = g.x0 < 2 || g.x0 + g.nx + 2 > a.H[0] || g.y0 < 2 || g.y0 + g.ny + 2 > a.H[1] ||
                           g.z0 < 2 || g.z0 + g.nz + 2 > a.H[2];
        tab[0] = tot;
        tab[1] = (2 * g.RY * g.RZ) | (wraps ? 1 << 16 : 0);
        tab[2] = g.nown;
        tab[3] = sm.own_off[g.nown];
    }
    if (tid < g.nown) {
        tab[4 + 2 * TILE_PIECES_MAX + tid] = sm.own_slot[tid];
        tab[4 + 2 * TILE_PIECES_MAX + TILE_OWN_MAX + tid] =
            (int)(((unsigned)sm.own_loc[tid] << 16) | (unsigned)sm.own_off[tid]);
    }
    const bool fits = tot <= a.reg_cap;
    if (!fits) {
        if (tid == 0) raise_status(a.status, MD_ERR_NBR_OVERFLOW);
    } else if (tid == 0) {
        mbar_init(&sm.bar, 1u);
        mbar_expect_tx(&sm.bar, (unsigned)tot * 16u);
    }
    __syncthreads();
    for (int r = tid; r < g.RY * g.RZ; r += TT) {
        const int q0 = g.RX * r;
        // periodic image of the row: code 1 adds L, code 2 subtracts L
        const int uy = g.y0 - 2 + r % g.RY, uz = g.z0 - 2 + r / g.RY;
        const unsigned cyz = (uy < 0 ? 2u : (uy >= a.H[1] ? 1u : 0u)) << 2 |
                             (uz < 0 ? 2u : (uz >= a.H[2] ? 1u : 0u)) << 4;
        int qs = q0;
        int2 pa = make_int2(0, 0), pb = make_int2(0, 0);
        for (int xl = 1; xl <= g.RX; ++xl) {
            const bool brk = xl == g.RX || wrapi(g.x0 - 2 + xl, a.H[0]) == 0;
            if (brk) {
                const int n = sm.hoff[q0 + xl] - sm.hoff[qs];
                const int src = __ldg(a.hstart + t_hglob(a, g, qs));
                if (n > 0) {
                    if (fits && TCHECK(a, sm.hoff[qs] + n <= tot && src >= 0 && src + n <= a.N &&
                                              (sm_addr(cand) & 15u) == 0u, 2))
                        bulk_g2s(cand + sm.hoff[qs], rsrc + src, (unsigned)n * 16u, &sm.bar);
                    // a copy never crosses the x wrap, so one image per copy
                    const int ux = g.x0 - 2 + (qs - q0);
                    const unsigned code = cyz | (ux < 0 ? 2u : (ux >= a.H[0] ? 1u : 0u));
                    const int2 pc = make_int2((int)((unsigned)src | code << TILE_SRC_BITS),
                                              (int)(((unsigned)sm.hoff[qs] << 16) | (unsigned)n));
                    if (pa.y == 0) pa = pc;
                    else pb = pc;
                }
                qs = q0 + xl;
            }
        }
        reinterpret_cast<int2 *>(tab + 4)[2 * r] = pa;
        reinterpret_cast<int2 *>(tab + 4)[2 * r + 1] = pb;
    }
    if (!fits) return false;
    return tile_wait(a, sm);
}

// Step: issue the bulk copies of the region from the tile's table (copies
// and own half-cells as the last build left them); tile_wait completes
// them.  Returns false (uniformly, nothing issued) if the region exceeds
// the capacity (the build raised the overflow).
__device__ bool tile_issue_tab(const TileArgs &a, TileStepSm &sm, const float4 *rsrc, float4 *cand, const int32_t *tab)
{
    const int tid = threadIdx.x;
    const int tot = __ldg(tab + 0), npc = __ldg(tab + 1) & 0xffff, nown = __ldg(tab + 2);
    if (tot > a.reg_cap) return false;
    if (!TCHECK(a, tot >= 0 && npc >= 0 && npc <= TILE_PIECES_MAX && nown >= 0 && nown <= TILE_OWN_MAX &&
                       (sm_addr(cand) & 15u) == 0u && (sm_addr(&sm.bar) & 7u) == 0u, 0))
        return false;
    if (tid == 0) {
        sm.total = tot;
        sm.nown = nown;
        sm.own_off[nown] = __ldg(tab + 3);
        mbar_init(&sm.bar, 1u);
        mbar_expect_tx(&sm.bar, (unsigned)tot * 16u);
    }
    if (tid < nown) {
        sm.own_slot[tid] = __ldg(tab + 4 + 2 * TILE_PIECES_MAX + tid);
        const unsigned w = (unsigned)__ldg(tab + 4 + 2 * TILE_PIECES_MAX + TILE_OWN_MAX + tid);
        sm.own_loc[tid] = (int)(w >> 16);
        sm.own_off[tid] = (int)(w & 0xffffu);
    }
    __syncthreads();
    const int2 *pc = reinterpret_cast<const int2 *>(tab + 4);
    for (int k = tid; k < npc; k += TT) {
        const int2 c = __ldg(pc + k);
        const unsigned n = (unsigned)c.y & 0xffffu;
        const int src = (int)((unsigned)c.x & TILE_SRC_MASK);
        if (n > 0u && TCHECK(a, ((unsigned)c.y >> 16) + n <= (unsigned)tot && src + (int)n <= a.N, 1))
            bulk_g2s(cand + ((unsigned)c.y >> 16), rsrc + src, n * 16u, &sm.bar);
    }
    return true;
}

// After the staging: the copies taken from across the box get their image
// (+-L per axis, from the copy's code), so that every staged partner's
// nearest-image vector is the plain difference.  Tiles whose region does
// not cross the box skip this (uniform, from the table header).
// Subtracting L from a coordinate near L is exact; adding L to one near 0
// rounds once at the precision of L, as the difference of the
// nearest-image form does.
__device__ __forceinline__ void tile_shift(const TileArgs &a, float4 *cand, const int32_t *tab)
{
    const int hdr = __ldg(tab + 1);
    if (!(hdr >> 16)) return;
    const int npc = hdr & 0xffff;
    const int2 *pc = reinterpret_cast<const int2 *>(tab + 4);
    for (int k = threadIdx.x; k < npc; k += TT) {
        const int2 c = __ldg(pc + k);
        const unsigned code = (unsigned)c.x >> TILE_SRC_BITS;
        if (!code) continue;
        const float sx = (code & 1u) ? a.box.L[0] : ((code & 2u) ? -a.box.L[0] : 0.0f);
        const float sy = (code & 4u) ? a.box.L[1] : ((code & 8u) ? -a.box.L[1] : 0.0f);
        const float sz = (code & 16u) ? a.box.L[2] : ((code & 32u) ? -a.box.L[2] : 0.0f);
        const unsigned o = (unsigned)c.y >> 16, n = (unsigned)c.y & 0xffffu;
        for (unsigned e = 0; e < n; ++e) {
            float4 p = cand[o + e];
            p.x += sx;
            p.y += sy;
            p.z += sz;
            cand[o + e] = p;
        }
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// rebuild chain
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(TT) k_t_bin(TileArgs a)
{
    count_launch();
    if (!t_active(a)) return;
    const int i = blockIdx.x * TT + threadIdx.x;
    const bool act = i < a.N;
    int h = 0;
    if (act) {
        const float4 p = a.import ? a.r_in[i] : t_r(a, t_sel(a) & 1u)[i];
        if (!isfinite(p.x) || !isfinite(p.y) || !isfinite(p.z)) raise_status(a.status, MD_ERR_NONFINITE);
        const int hx = h_axis(p.x, a.box.L[0], a.box.Linv[0], a.hscale[0], a.H[0]);
        const int hy = h_axis(p.y, a.box.L[1], a.box.Linv[1], a.hscale[1], a.H[1]);
        const int hz = h_axis(p.z, a.box.L[2], a.box.Linv[2], a.hscale[2], a.H[2]);
        h = (hz * a.H[1] + hy) * a.H[0] + hx;
    }
    const unsigned amask = __ballot_sync(0xffffffffu, act);
    if (!act) return;
    const unsigned peers = __match_any_sync(amask, h);
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(peers) - 1;
    const int below = __popc(peers & ((1u << lane) - 1u));
    int base = 0;
    if (lane == leader) base = atomicAdd(&a.hcount[h], __popc(peers));
    base = __shfl_sync(peers, base, leader);
    a.key[i] = h;
    a.rank[i] = base + below;
}

// Block-local exclusive scan of TSCAN_ITEMS counts (1024 threads x 4); the
// block's total to bsum; the histogram is cleared for the next build.
__global__ void __launch_bounds__(1024) k_t_scan1(TileArgs a)
{
    count_launch();
    if (!t_active(a)) return;
    __shared__ int wt[32];
    const int base = blockIdx.x * TSCAN_ITEMS + threadIdx.x * 4;
    int c[4], s = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        c[k] = base + k < a.nhc ? a.hcount[base + k] : 0;
        s += c[k];
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int x = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wt[w] = x;
    __syncthreads();
    if (w == 0) {
        int u = wt[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, u, o);
            if (lane >= o) u += y;
        }
        wt[lane] = u;
    }
    __syncthreads();
    int run = x - s + (w > 0 ? wt[w - 1] : 0);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (base + k < a.nhc) {
            a.hstart[base + k] = run;
            a.hcount[base + k] = 0;
        }
        run += c[k];
    }
    if (threadIdx.x == 1023) a.bsum[blockIdx.x] = wt[31];
}

// Exclusive scan of the nb block totals (one CTA, nb <= 4096); the grand
// total to hstart[nhc].
__global__ void __launch_bounds__(1024) k_t_scan2(TileArgs a, int nb)
{
    count_launch();
    if (!t_active(a)) return;
    __shared__ int wt[32];
    const int base = threadIdx.x * 4;
    int c[4], s = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        c[k] = base + k < nb ? a.bsum[base + k] : 0;
        s += c[k];
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int x = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wt[w] = x;
    __syncthreads();
    if (w == 0) {
        int u = wt[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, u, o);
            if (lane >= o) u += y;
        }
        wt[lane] = u;
    }
    __syncthreads();
    int run = x - s + (w > 0 ? wt[w - 1] : 0);
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (base + k < nb) a.bsum[base + k] = run;
        run += c[k];
    }
    if (threadIdx.x == 1023) a.hstart[a.nhc] = wt[31];
}

__global__ void __launch_bounds__(TT) k_t_scan3(TileArgs a)
{
    count_launch();
    if (!t_active(a)) return;
    const int i = blockIdx.x * TT + threadIdx.x;
    if (i < a.nhc) a.hstart[i] += a.bsum[i / TSCAN_ITEMS];
}

__global__ void __launch_bounds__(TT) k_t_scatter(TileArgs a)
{
    count_launch();
    if (!t_active(a)) return;
    const int i = blockIdx.x * TT + threadIdx.x;
    if (i < a.N) a.tmp[a.hstart[a.key[i]] + a.rank[i]] = i;
}

// Members of each half-cell by ascending caller index: the rank of a member
// is the number of members of its half-cell with a smaller index.  Writes
// the other buffer set (positions wrapped into [0, L), build positions).
__global__ void __launch_bounds__(TT) k_t_place(TileArgs a)
{
    count_launch();
    if (!t_active(a)) return;
    const int q = blockIdx.x * TT + threadIdx.x;
    if (q >= a.N) return;
    const uint32_t sel = t_sel(a);
    const uint32_t rc = sel & 1u, vc = (sel >> 1) & 1u;
    const int32_t *pc = t_p(a, vc);
    const int s = a.tmp[q];
    const int h = a.key[s];
    const int b = a.hstart[h], e = a.hstart[h + 1];
    const int id = a.import ? s : pc[s];
    int rk = 0;
    for (int m = b; m < e; ++m) {
        const int s2 = a.tmp[m];
        const int id2 = a.import ? s2 : pc[s2];
        rk += id2 < id ? 1 : 0;
    }
    const int d = b + rk;
    float4 p = a.import ? a.r_in[s] : t_r(a, rc)[s];
    p.x = wrap_coord(p.x, a.box.L[0], a.box.Linv[0]);
    p.y = wrap_coord(p.y, a.box.L[1], a.box.Linv[1]);
    p.z = wrap_coord(p.z, a.box.L[2], a.box.Linv[2]);
    t_r(a, rc ^ 1u)[d] = p;
    a.rref[d] = p;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (a.import) {
        if (a.v_in) v = a.v_in[s];
        a.fs[d] = a.f_in ? a.f_in[s] : make_float4(0.f, 0.f, 0.f, 0.f);
    } else {
        v = t_v(a, vc)[s];
    }
    t_v(a, vc ^ 1u)[d] = v;
    t_p(a, vc ^ 1u)[d] = id;
}

// Row of one own particle, one thread per particle.  Its candidates are the
// region's half-cells of its 5 x 5 x 5 window; for each (y, z) row of the
// window the run of x that can hold a partner is one contiguous local range
// (half-cells farther than r_list from the particle, with a margin above
// FP32 rounding, are skipped: rows entirely, and up to two on each end of a
// run).  Partners collect eight at a time in registers (a 16-bit shift
// register of four words) and go out as one 16-byte store.  The row is then
// padded with the sentinel index (reg_cap, a far-away position the step
// kernels place after the region) up to the warp's longest row rounded up
// to 8, so that the step's thread-per-particle loop, whose warps are these
// warps, runs without masks.  The region is staged with its copies at their
// periodic image, so a partner is decided on the plain difference of staged
// positions: r^2 = dz^2 + (dy^2 + dx^2) with FMAs, strict < r_list^2.  This
// rounds differently from the nearest-image formula of the int32 build only
// for pairs within an ulp of r_list.  Needs cap % 8 == 0.
__device__ __forceinline__ int build_thread(const TileArgs &a, const TGeo &g, const TileSm &sm, const float4 *cand,
                                            int k, int loc, int slot, bool valid)
{
    const float wx = a.box.L[0] / (float)a.H[0], wy = a.box.L[1] / (float)a.H[1], wz = a.box.L[2] / (float)a.H[2];
    const float lim2 = a.r_list2 * 1.0002f + 1e-4f;
    const float4 ri = valid ? cand[loc] : make_float4(0.f, 0.f, 0.f, 0.f);
    const int xl = 2 + k % g.nx, yl = 2 + (k / g.nx) % g.ny, zl = 2 + k / (g.nx * g.ny);
    uint16_t *row = a.rows + (size_t)slot * a.cap;
    uint32_t w0 = 0u, w1 = 0u, w2 = 0u, w3 = 0u;   // shift register of the last eight entries
    int nb = 0, n0 = 0;
    // distance from the particle to region half-cell c along an axis (origin
    // o, width w): zero inside, else to the nearer face
    auto gap = [&](float x, int o, int c, float w) {
        const float lo = (float)(o - 2 + c) * w;
        return fmaxf(0.f, fmaxf(lo - x, x - (lo + w)));
    };
    auto push = [&](uint32_t j) {
        w0 = __funnelshift_r(w0, w1, 16);
        w1 = __funnelshift_r(w1, w2, 16);
        w2 = __funnelshift_r(w2, w3, 16);
        w3 = (w3 >> 16) | (j << 16);
    };
    const float gx0 = gap(ri.x, g.x0, xl - 2, wx), gx1 = gap(ri.x, g.x0, xl - 1, wx);
    const float gx3 = gap(ri.x, g.x0, xl + 1, wx), gx4 = gap(ri.x, g.x0, xl + 2, wx);
    for (int zr = zl - 2; zr <= zl + 2; ++zr) {
        const float gz = gap(ri.z, g.z0, zr, wz);
        for (int yr = yl - 2; yr <= yl + 2; ++yr) {
            const float gy = gap(ri.y, g.y0, yr, wy);
            const float rem = lim2 - gy * gy - gz * gz;
            // x-run of this row that can hold a partner (the particle's own
            // column always; one or two more on each side)
            const int xa = gx0 * gx0 <= rem ? xl - 2 : (gx1 * gx1 <= rem ? xl - 1 : xl);
            const int xb = gx4 * gx4 <= rem ? xl + 2 : (gx3 * gx3 <= rem ? xl + 1 : xl);
            const int base = g.RX * (yr + g.RY * zr);
            const int beg = sm.hoff[base + xa];
            const int end = (valid && rem >= 0.f) ? sm.hoff[base + xb + 1] : beg;
            for (int j = beg; j < end; ++j) {
                const float4 cj = cand[j];
                const float dx = ri.x - cj.x, dy = ri.y - cj.y, dz = ri.z - cj.z;
                const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
                if (r2 < a.r_list2 && j != loc) {
                    push((uint32_t)j);
                    if (++nb == 8) {
                        if (n0 + 8 <= a.cap) *reinterpret_cast<uint4 *>(row + n0) = make_uint4(w0, w1, w2, w3);
                        n0 += 8;
                        nb = 0;
                    }
                }
            }
        }
    }
    const int n = n0 + nb;
    const int wmax = __reduce_max_sync(0xffffffffu, valid ? n : 0);
    const int kend = min((wmax + 7) & ~7, a.cap);
    if (valid) {
        const uint32_t sent = (uint32_t)a.reg_cap;
        if (nb > 0) {
            // the pending entries, then sentinels, as one chunk
            for (int m = nb; m < 8; ++m) push(sent);
            if (n0 + 8 <= a.cap) *reinterpret_cast<uint4 *>(row + n0) = make_uint4(w0, w1, w2, w3);
            n0 += 8;
        }
        const uint32_t sw = sent | sent << 16;
        for (int q = n0; q < kend; q += 8) *reinterpret_cast<uint4 *>(row + q) = make_uint4(sw, sw, sw, sw);
        a.cnt[slot] = (uint32_t)min(n, 0xffff);
        if (n > a.cap) raise_status(a.status, MD_ERR_NBR_OVERFLOW);
    }
    return valid ? n : 0;
}

__global__ void __launch_bounds__(TT) k_t_build(TileArgs a)
{
    count_launch();
    if (!t_active(a)) return;
    extern __shared__ __align__(16) float4 cand[];
    __shared__ TileSm sm;
    __shared__ int bmax;
    const TGeo g = t_geo(a, blockIdx.x);
    const uint32_t sel = t_sel(a);
    // the positions k_t_place just wrote (the buffer k_t_finish switches to)
    const float4 *rs = t_r(a, (sel & 1u) ^ 1u);
    if (threadIdx.x == 0) {
        bmax = 0;
        sm.kmap = reinterpret_cast<unsigned char *>(cand + a.reg_cap + 1);
    }
    tile_scan(a, g, sm);
    if (!tile_stage_build(a, g, sm, rs, cand, a.tab + (size_t)blockIdx.x * TILE_TAB_WORDS)) return;
    // the copies from across the box at their periodic image (region
    // half-cell by region half-cell), as the step kernels stage them
    for (int q = threadIdx.x; q < g.nq; q += TT) {
        const int xl = q % g.RX, yl = (q / g.RX) % g.RY, zl = q / (g.RX * g.RY);
        const int ux = g.x0 - 2 + xl, uy = g.y0 - 2 + yl, uz = g.z0 - 2 + zl;
        const float sx = ux < 0 ? -a.box.L[0] : (ux >= a.H[0] ? a.box.L[0] : 0.0f);
        const float sy = uy < 0 ? -a.box.L[1] : (uy >= a.H[1] ? a.box.L[1] : 0.0f);
        const float sz = uz < 0 ? -a.box.L[2] : (uz >= a.H[2] ? a.box.L[2] : 0.0f);
        if (sx == 0.0f && sy == 0.0f && sz == 0.0f) continue;
        for (int e = sm.hoff[q]; e < sm.hoff[q + 1]; ++e) {
            float4 p = cand[e];
            p.x += sx;
            p.y += sy;
            p.z += sz;
            cand[e] = p;
        }
    }
    __syncthreads();
    tile_own_map(sm);
    const int nown = sm.own_off[g.nown];
    int wmax = 0;
    for (int p0 = 0; p0 < nown; p0 += TT) {
        const int p = p0 + threadIdx.x;
        const bool valid = p < nown;
        int k = 0, loc = 0, slot = 0;
        if (valid) {
            k = sm.kmap[p];
            const int t = p - sm.own_off[k];
            loc = sm.own_loc[k] + t;
            slot = sm.own_slot[k] + t;
        }
        const int n = build_thread(a, g, sm, cand, k, loc, slot, valid);
        wmax = max(wmax, n);
    }
    wmax = __reduce_max_sync(0xffffffffu, wmax);
    if ((threadIdx.x & 31) == 0 && wmax > 0) atomicMax(&bmax, wmax);
    __syncthreads();
    if (threadIdx.x == 0 && bmax > 0) atomicMax(&a.ctl[CTL_MAXCNT], (uint32_t)bmax);
}

// Switches to the buffer set the chain wrote and counts the build.
__global__ void k_t_finish(TileArgs a)
{
    count_launch();
    if (!t_active(a)) return;
    a.ctl[CTL_TSEL] ^= 3u;
    const uint32_t sw = (uint32_t)a.reg_cap * 0x10001u;
    *a.sent = make_uint4(sw, sw, sw, sw);
    unsigned long long *b = (unsigned long long *)&a.ctl[CTL_BUILDS_LO];
    *b += 1ull;
    a.ctl[CTL_REBUILD] = 0u;
}

// ---------------------------------------------------------------------------
// forces and the fused step
// ---------------------------------------------------------------------------
// 1/x by the PTX approximate reciprocal (at most 1 ulp from the rounded
// quotient; subnormal results flush to zero, which only the sentinel's
// r^-6 reaches).
__device__ __forceinline__ float rcp_approx(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// One pair's contribution, branch-free: the cutoff decision (r2 < r_c^2, or
// r2 < sigma_ij^2 for soft spheres) selects the force factor and the
// energy, so divergent warps run no extra branches.  LJ in the form
//   F/r = r^-8 (48 eps sigma^12 r^-6 - 24 eps sigma^6),
//   U   = r^-6 (4 eps sigma^12 r^-6 - 4 eps sigma^6) - U(r_c).
// Any r2 > 0 is safe: the sentinel partner (r2 ~ 3e36) and a masked slot
// (r2 = 3e38) fall outside every cutoff and add exactly zero.
template <int POT>
__device__ __forceinline__ void t_term(const TileArgs &a, float dx, float dy, float dz, float r2, float wi, float wj,
                                       float &fx, float &fy, float &fz, float &e)
{
    if (POT == MD_LJ) {
        const bool in = r2 < a.rc2;
        const float ir2 = rcp_approx(r2);
        const float ir6 = ir2 * ir2 * ir2;
        const float fr = (ir2 * ir6) * fmaf(a.lj_f12, ir6, -a.lj_f6);
        const float ep = fmaf(ir6, fmaf(a.lj_e12, ir6, -a.lj_e6), -a.e_shift);
        const float frs = in ? fr : 0.0f;
        fx = fmaf(frs, dx, fx);
        fy = fmaf(frs, dy, fy);
        fz = fmaf(frs, dz, fz);
        e += in ? ep : 0.0f;
    } else {
        const float sg = 0.5f * (wi + wj);
        const bool in = r2 < sg * sg;
        const float rr = sqrtf(r2);
        const float isg = __fdividef(1.0f, sg);
        const float x = 1.0f - rr * isg;
        float xa1, ua;
        if (a.alpha == 2.0f) {
            xa1 = x;
            ua = 0.5f * x * x;
        } else {
            xa1 = __powf(in ? x : 1.0f, a.alpha - 1.0f);
            ua = xa1 * x / a.alpha;
        }
        const float fr = in ? a.eps * isg * xa1 * __fdividef(1.0f, rr) : 0.0f;
        fx = fmaf(fr, dx, fx);
        fy = fmaf(fr, dy, fy);
        fz = fmaf(fr, dz, fz);
        e += in ? a.eps * ua : 0.0f;
    }
}

// Partner at the staged position rj (the region's copies carry their
// periodic image, so the plain difference is the nearest-image vector).
template <int POT>
__device__ __forceinline__ void t_pair(const TileArgs &a, const float4 &ri, const float4 &rj, float &fx, float &fy,
                                       float &fz, float &e)
{
    const float dx = ri.x - rj.x, dy = ri.y - rj.y, dz = ri.z - rj.z;
    const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
    t_term<POT>(a, dx, dy, dz, r2, ri.w, rj.w, fx, fy, fz, e);
}

// FP64 totals: FP32 per warp, FP64 across warps and (last block, fixed
// order) across blocks; the last block writes the series, advances the step,
// sets the graph conditions and, after a step that moved the particles,
// switches the position buffer.
__device__ __forceinline__ void t_epilogue(float pe_acc, float ke_acc, const TileArgs &a, bool flip,
                                           const int *moved_flag)
{
    __shared__ double sh[2][32];
    __shared__ bool last;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        pe_acc += __shfl_xor_sync(0xffffffffu, pe_acc, o);
        ke_acc += __shfl_xor_sync(0xffffffffu, ke_acc, o);
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        sh[0][w] = (double)pe_acc;
        sh[1][w] = (double)ke_acc;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double bpe = 0.0, bke = 0.0;
        for (int k = 0; k < TT / 32; ++k) {
            bpe += sh[0][k];
            bke += sh[1][k];
        }
        // one rebuild-flag store per block, ordered before the ticket by the
        // fence below (a fence per warp costs much when most particles moved)
        if (moved_flag && *moved_flag) a.ctl[CTL_REBUILD] = 1u;
        a.partials[blockIdx.x] = make_double2(bpe, bke);
        __threadfence();
        const unsigned t = atomicAdd(&a.ctl[CTL_TICKET], 1u);
        last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double S[2] = {0.0, 0.0};
    for (int b = threadIdx.x; b < (int)gridDim.x; b += TT) {
        const volatile double *p = (const volatile double *)(a.partials + b);
        S[0] += p[0];
        S[1] += p[1];
    }
    block_sums_f64<2>(S, &sh[0][0], 32);
    if (threadIdx.x == 0) {
        const double spe = S[0], ske = S[1];
        a.ctl[CTL_TICKET] = 0u;
        if (!isfinite(spe) || !isfinite(ske)) raise_status(a.status, MD_ERR_NONFINITE);
        const unsigned step = a.series ? a.ctl[CTL_STEP] : 0u;
        if (a.E_out) a.E_out[step] = spe;
        if (a.KE_out) a.KE_out[step] = ske;
        if (a.series) a.ctl[CTL_STEP] = step + 1u;
        if (flip) a.ctl[CTL_TSEL] ^= 1u;
        if (a.use_cond) {
            cudaGraphSetConditional((cudaGraphConditionalHandle)a.cond_while,
                                    (step + 1u < a.ctl[CTL_NSTEPS]) ? 1u : 0u);
            cudaGraphSetConditional((cudaGraphConditionalHandle)a.cond_if,
                                    *(volatile uint32_t *)&a.ctl[CTL_REBUILD] ? 1u : 0u);
        }
    }
}

// The sentinel partner: rows are padded with index reg_cap, where the step
// kernels put this position; every pair with it lies outside any cutoff.
constexpr float T_FAR = 1e18f;

// End of an own particle's step.  KICK 0: force and per-particle energy into
// fs.  KICK 2, the fused velocity-Verlet step: closing half-kick at the new
// forces, then, unless this is the loop's last step, the next kick and drift
// into the other position buffer (not wrapped) with the displacement check;
// the last step writes the forces instead.
template <int KICK>
__device__ __forceinline__ void t_finish(const TileArgs &a, int s, const float4 &ri, float4 vi, const float4 &rr,
                                         bool more, float fx, float fy, float fz, float ei, float4 *rn, float4 *vv,
                                         float &pe_acc, float &ke_acc, int *moved_any)
{
    pe_acc += ei;
    if (KICK == 0) {
        a.fs[s] = make_float4(fx, fy, fz, ei);
        return;
    }
    vi.x += a.hdm * fx;
    vi.y += a.hdm * fy;
    vi.z += a.hdm * fz;
    ke_acc += 0.5f * a.mass * (vi.x * vi.x + vi.y * vi.y + vi.z * vi.z);
    if (more) {
        vi.x += a.hdm * fx;
        vi.y += a.hdm * fy;
        vi.z += a.hdm * fz;
        float4 r2 = ri;
        r2.x = ri.x + a.dt * vi.x;
        r2.y = ri.y + a.dt * vi.y;
        r2.z = ri.z + a.dt * vi.z;
        rn[s] = r2;
        float dx, dy, dz;
        if (dist2_rn<3>(r2, rr, a.box, dx, dy, dz) > a.half_skin2) *moved_any = 1;
    } else {
        a.fs[s] = make_float4(fx, fy, fz, ei);
    }
    vv[s] = vi;
}

// Own particle p of the tile -> its slot and local index.
__device__ __forceinline__ void t_own(const TileStepSm &sm, int p, int &s, int &li)
{
    const int k = sm.kmap[p];
    const int t = p - sm.own_off[k];
    s = sm.own_slot[k] + t;
    li = sm.own_loc[k] + t;
}

// Step with TPP lanes per particle (tiles of fewer than about 128
// particles).  Each lane prefetches RW row words at fixed positions (so the
// loads need not wait for the count); words at and beyond the count are
// replaced by the sentinel before any use, so every index that reaches
// shared memory is inside the region or the sentinel.
template <int TPP, int KICK>
struct TPre {
    static constexpr int RW = 40 / TPP;   // row words (two entries each) per lane: 80 entries per group
    uint32_t c;
    uint32_t w[RW];
    float4 v, rr;
    int s, li;
};

template <int POT, int TPP, int KICK>
__global__ void __launch_bounds__(TT, 4) k_t_step(TileArgs a)
{
    count_launch();
    extern __shared__ __align__(16) float4 cand[];
    __shared__ TileStepSm sm;
    __shared__ int moved_any;
    using Pre = TPre<TPP, KICK>;
    const uint32_t sel = t_sel(a);
    const uint32_t rcb = sel & 1u;
    const float4 *rc = t_r(a, rcb);
    float4 *rn = t_r(a, rcb ^ 1u);
    float4 *vv = t_v(a, (sel >> 1) & 1u);
    bool more = false;
    if (KICK == 2) {
        const uint32_t step = *(volatile uint32_t *)&a.ctl[CTL_STEP];
        more = step + 1u < *(volatile uint32_t *)&a.ctl[CTL_NSTEPS];
    }
    if (threadIdx.x == 0) {
        sm.kmap = reinterpret_cast<unsigned char *>(cand + a.reg_cap + 1);
        moved_any = 0;
        cand[a.reg_cap] = make_float4(T_FAR, T_FAR, T_FAR, 0.f);
    }
    float pe_acc = 0.f, ke_acc = 0.f;
    const int32_t *tab = a.tab + (size_t)blockIdx.x * TILE_TAB_WORDS;
    if (tile_issue_tab(a, sm, rc, cand, tab) && tile_wait(a, sm)) {
        tile_shift(a, cand, tab);
        tile_own_map(sm);
        const int lg = threadIdx.x & (TPP - 1), gi = threadIdx.x / TPP;
        const int nown = sm.own_off[sm.nown];
        const uint32_t sent = (uint32_t)a.reg_cap, sw = sent * 0x10001u;
        // every lane of a warp runs every trip (the group reductions below
        // are full-warp shuffles); lanes past the tile's last particle
        // carry zeros
        for (int p0 = 0; p0 < nown; p0 += TT / TPP) {
            const int p = p0 + gi;
            const bool valid = p < nown;
            float fx = 0.f, fy = 0.f, fz = 0.f, e = 0.f;
            float4 ri = make_float4(0.f, 0.f, 0.f, 0.f);
            Pre q;
            if (valid) {
                t_own(sm, p, q.s, q.li);
                q.c = __ldg(a.cnt + q.s);
                const uint16_t *row = a.rows + (size_t)q.s * a.cap;
#pragma unroll
                for (int k2 = 0; k2 < Pre::RW; ++k2) {
                    const int wi = lg + k2 * TPP;
                    q.w[k2] = 2 * wi + 1 < a.cap ? ld_nc_u32(row + 2 * wi) : sw;
                }
                if (KICK == 2 && lg == 0) {
                    q.v = vv[q.s];
                    if (more) q.rr = __ldg(a.rref + q.s);
                }
                ri = cand[q.li];
                const int n = min((int)(q.c & 0xffffu), a.cap);
#pragma unroll
                for (int k2 = 0; k2 < Pre::RW; ++k2) {
                    const int e2 = 2 * (lg + k2 * TPP);
                    q.w[k2] = e2 + 1 < n ? q.w[k2] : (e2 < n ? ((q.w[k2] & 0xffffu) | sent << 16) : sw);
                }
#pragma unroll
                for (int k2 = 0; k2 < Pre::RW; ++k2) {
                    if (2 * (lg + k2 * TPP) < n) {
                        t_pair<POT>(a, ri, cand[q.w[k2] & 0xffffu], fx, fy, fz, e);
                        t_pair<POT>(a, ri, cand[q.w[k2] >> 16], fx, fy, fz, e);
                    }
                }
                for (int wi = lg + Pre::RW * TPP; 2 * wi < n; wi += TPP) {   // rows longer than 80
                    uint32_t x = ld_nc_u32(row + 2 * wi);
                    x = 2 * wi + 1 < n ? x : ((x & 0xffffu) | sent << 16);
                    t_pair<POT>(a, ri, cand[x & 0xffffu], fx, fy, fz, e);
                    t_pair<POT>(a, ri, cand[x >> 16], fx, fy, fz, e);
                }
            }
#pragma unroll
            for (int o = TPP / 2; o > 0; o >>= 1) {
                fx += __shfl_xor_sync(0xffffffffu, fx, o);
                fy += __shfl_xor_sync(0xffffffffu, fy, o);
                fz += __shfl_xor_sync(0xffffffffu, fz, o);
                e += __shfl_xor_sync(0xffffffffu, e, o);
            }
            if (valid && lg == 0)
                t_finish<KICK>(a, q.s, ri, q.v, q.rr, more, fx, fy, fz, 0.5f * e, rn, vv, pe_acc, ke_acc,
                               &moved_any);
        }
    }
    t_epilogue(pe_acc, ke_acc, a, KICK == 2 && more, &moved_any);
}

// The same step with one thread per own particle (tiles of a few hundred
// particles fill a CTA in one pass).  Each thread streams its row in 16-byte
// chunks (eight entries, the next chunk fetched while the current one is
// evaluated) up to the warp's longest row rounded up to 8: the build padded
// every row of the warp that far with the sentinel, so no entry is masked.
// Lanes past the tile's last particle read sentinels only.  Needs cap % 8
// == 0.
// (not volatile: the rows are read-only while the step runs, so the
// compiler may schedule the load early)
__device__ __forceinline__ uint4 ld_nc_v4(const void *p)
{
    uint4 v;
    asm("ld.global.nc.L1::no_allocate.v4.u32 {%0, %1, %2, %3}, [%4];"
        : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
        : "l"(p));
    return v;
}

template <int POT>
__device__ __forceinline__ void t_pair_word(const TileArgs &a, const float4 *cand, const float4 &ri, uint32_t w,
                                            float &fx, float &fy, float &fz, float &e)
{
    t_pair<POT>(a, ri, cand[w & 0xffffu], fx, fy, fz, e);
    t_pair<POT>(a, ri, cand[w >> 16], fx, fy, fz, e);
}

template <int POT, int KICK>
__global__ void __launch_bounds__(TT, 4) k_t_step1(TileArgs a)
{
    count_launch();
    extern __shared__ __align__(16) float4 cand[];
    __shared__ TileStepSm sm;
    __shared__ int moved_any;
    const uint32_t sel = t_sel(a);
    const uint32_t rcb = sel & 1u;
    const float4 *rc = t_r(a, rcb);
    float4 *rn = t_r(a, rcb ^ 1u);
    float4 *vv = t_v(a, (sel >> 1) & 1u);
    bool more = false;
    if (KICK == 2) {
        const uint32_t step = *(volatile uint32_t *)&a.ctl[CTL_STEP];
        more = step + 1u < *(volatile uint32_t *)&a.ctl[CTL_NSTEPS];
    }
    if (threadIdx.x == 0) {
        sm.kmap = reinterpret_cast<unsigned char *>(cand + a.reg_cap + 1);
        moved_any = 0;
        cand[a.reg_cap] = make_float4(T_FAR, T_FAR, T_FAR, 0.f);
    }
    float pe_acc = 0.f, ke_acc = 0.f;
    const int32_t *tab = a.tab + (size_t)blockIdx.x * TILE_TAB_WORDS;
    if (tile_issue_tab(a, sm, rc, cand, tab)) {
        // the first pass's counts and first row chunks are fetched while
        // the region's copies are in flight; positions are read after them
        tile_own_map(sm);
        const int nown = sm.own_off[sm.nown];
        bool staged = false;
        for (int p0 = 0; p0 < nown; p0 += TT) {
            const int p = p0 + threadIdx.x;
            const bool valid = p < nown;
            int s = 0, n = 0, li = 0;
            if (valid) {
                t_own(sm, p, s, li);
                n = min((int)(__ldg(a.cnt + s) & 0xffffu), a.cap);
            }
            const uint16_t *row = a.rows + (size_t)s * a.cap;
            const int kend = (__reduce_max_sync(0xffffffffu, n) + 7) & ~7;
            // every load is unconditional: lanes past the tile's last
            // particle, and the chunk after the last, read the sentinel chunk
            uint4 nxt = ld_nc_v4(valid ? (const void *)row : (const void *)a.sent);
            if (p0 == 0) {   // uniform
                staged = tile_wait(a, sm);
                if (staged) tile_shift(a, cand, tab);
            }
            if (!staged) break;
            const float4 ri = valid ? cand[li] : make_float4(0.f, 0.f, 0.f, 0.f);
            float fx = 0.f, fy = 0.f, fz = 0.f, e = 0.f;
            for (int k0 = 0; k0 < kend; k0 += 8) {
                const uint4 cur = nxt;
                nxt = ld_nc_v4((valid && k0 + 8 < kend) ? (const void *)(row + k0 + 8) : (const void *)a.sent);
                t_pair_word<POT>(a, cand, ri, cur.x, fx, fy, fz, e);
                t_pair_word<POT>(a, cand, ri, cur.y, fx, fy, fz, e);
                t_pair_word<POT>(a, cand, ri, cur.z, fx, fy, fz, e);
                t_pair_word<POT>(a, cand, ri, cur.w, fx, fy, fz, e);
            }
            if (valid) {
                float4 vi = make_float4(0.f, 0.f, 0.f, 0.f), rr = vi;
                if (KICK == 2) {
                    vi = vv[s];
                    if (more) rr = __ldg(a.rref + s);
                }
                t_finish<KICK>(a, s, ri, vi, rr, more, fx, fy, fz, 0.5f * e, rn, vv, pe_acc, ke_acc, &moved_any);
            }
        }
        if (nown == 0) tile_wait(a, sm);   // no pass waited for the copies
    }
    t_epilogue(pe_acc, ke_acc, a, KICK == 2 && more, &moved_any);
}

// First half of the loop's first step: v += dt/2 F/m; r += dt v (not
// wrapped), in place; displacement check; the last block hands the rebuild
// decision to the graph's IF node.
__global__ void __launch_bounds__(TT) k_t_kick(TileArgs a)
{
    count_launch();
    __shared__ bool last;
    const uint32_t sel = t_sel(a);
    float4 *r = t_r(a, sel & 1u);
    float4 *v = t_v(a, (sel >> 1) & 1u);
    const int i = blockIdx.x * TT + threadIdx.x;
    bool mv = false;
    if (i < a.N) {
        const float4 f = a.fs[i];
        float4 vi = v[i], ri = r[i];
        vi.x += a.hdm * f.x;
        vi.y += a.hdm * f.y;
        vi.z += a.hdm * f.z;
        ri.x = ri.x + a.dt * vi.x;
        ri.y = ri.y + a.dt * vi.y;
        ri.z = ri.z + a.dt * vi.z;
        v[i] = vi;
        r[i] = ri;
        float dx, dy, dz;
        mv = dist2_rn<3>(ri, a.rref[i], a.box, dx, dy, dz) > a.half_skin2;
    }
    if (__any_sync(0xffffffffu, mv) && (threadIdx.x & 31) == 0) {
        a.ctl[CTL_REBUILD] = 1u;
        __threadfence();
    }
    if (!a.use_cond) return;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned t = atomicAdd(&a.ctl[CTL_TICKET2], 1u);
        last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        const unsigned flag = *(volatile uint32_t *)&a.ctl[CTL_REBUILD];
        a.ctl[CTL_TICKET2] = 0u;
        cudaGraphSetConditional((cudaGraphConditionalHandle)a.cond_if, flag ? 1u : 0u);
    }
}

// Positions (wrapped), velocities, forces and build positions back to the
// caller's order.
__global__ void __launch_bounds__(TT) k_t_export(TileArgs a)
{
    count_launch();
    const int s = blockIdx.x * TT + threadIdx.x;
    if (s >= a.N) return;
    const uint32_t sel = t_sel(a);
    const int id = t_p(a, (sel >> 1) & 1u)[s];
    if (a.r_out) {
        float4 p = t_r(a, sel & 1u)[s];
        p.x = wrap_coord(p.x, a.box.L[0], a.box.Linv[0]);
        p.y = wrap_coord(p.y, a.box.L[1], a.box.Linv[1]);
        p.z = wrap_coord(p.z, a.box.L[2], a.box.Linv[2]);
        a.r_out[id] = p;
    }
    if (a.v_out) a.v_out[id] = t_v(a, (sel >> 1) & 1u)[s];
    if (a.f_out) a.f_out[id] = a.fs[s];
    if (a.export_rows) a.rref_out[id] = a.rref[s];
}

// The tiled rows as the caller's int32 rows (one warp per own particle):
// local index -> region half-cell (binary search) -> slot -> caller index;
// padded with N; counts are the true totals.
__global__ void __launch_bounds__(TT) k_t_rows(TileArgs a)
{
    count_launch();
    __shared__ TileSm sm;
    const TGeo g = t_geo(a, blockIdx.x);
    tile_scan(a, g, sm);
    const uint32_t sel = t_sel(a);
    const int32_t *ids = t_p(a, (sel >> 1) & 1u);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nown = sm.own_off[g.nown];
    for (int p = warp; p < nown; p += TT / 32) {
        int lo = 0, hi = g.nown - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (sm.own_off[mid] <= p) lo = mid;
            else hi = mid - 1;
        }
        const int s = sm.own_slot[lo] + (p - sm.own_off[lo]);
        const int id = ids[s];
        const uint32_t c = a.cnt[s];
        const int n0r = (int)(c & 0xffffu), nsr = (int)(c >> 16);
        const int n0 = min(n0r, a.cap), ns = min(nsr, a.cap - n0);
        const uint16_t *row = a.rows + (size_t)s * a.cap;
        int32_t *out = a.nbr_out + (size_t)id * a.cap;
        for (int k = lane; k < a.cap; k += 32) {
            int v = a.N;
            const int li = k < n0 + ns ? (int)row[k < n0 ? k : a.cap - ns + (k - n0)] : sm.total;
            if (li < sm.total) {   // rows of a tile whose region overflowed were never written
                int ql = 0, qh = g.nq - 1;
                while (ql < qh) {
                    const int mid = (ql + qh + 1) >> 1;
                    if (sm.hoff[mid] <= li) ql = mid;
                    else qh = mid - 1;
                }
                v = ids[__ldg(a.hstart + t_hglob(a, g, ql)) + (li - sm.hoff[ql])];
            }
            out[k] = v;
        }
        if (lane == 0) a.cnt_out[id] = n0r + nsr;
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static int g_tile_tpp = 0;   // 0: by tile size (1 for tiles of >= 128 particles, else 4)

static bool tile_plan(const md_space *s, const md_nbr *nb, TilePlan &tp)
{
    if (!nb || (s && s->dim != 3) || nb->dim != 3 || nb->N < 1 || nb->N > (int)TILE_SRC_MASK || (nb->cap & 7) ||
        nb->cap > 0xffff)
        return false;
    if (!(nb->r_cut > nb->skin)) return false;
    return tile_geometry(nb->N, nb->ncell, tp);
}

static bool tiles_ready(const md_space *s, const md_nbr *nb, TilePlan &tp)
{
    return nb && nb->ws && nb->nbr && nb->cnt && nb->rref && (nb->flags & MD_NBR_TILES) && nbr_layout_ok(nb) &&
           tile_plan(s, nb, tp);
}

static void make_tile_args(const md_space *s, const md_nbr *nb, const TilePlan &tp, uint32_t *d_status, TileArgs &a)
{
    memset(&a, 0, sizeof(a));
    a.box = make_box(s);
    a.N = nb->N;
    a.cap = nb->cap;
    for (int k = 0; k < 3; ++k) {
        a.H[k] = tp.H[k];
        a.hscale[k] = (float)((double)tp.H[k] / (double)s->L[k]);
    }
    a.tx = tp.tx;
    a.ty = tp.ty;
    a.tz = tp.tz;
    a.ntx = tp.ntx;
    a.nty = tp.nty;
    a.ntz = tp.ntz;
    a.ntiles = tp.ntiles;
    a.reg_cap = tp.reg_cap;
    a.nhc = tp.H[0] * tp.H[1] * tp.H[2];
    a.r_list2 = nb->r_list2;
    a.half_skin2 = nb->half_skin2;
    const WsLayout wl = ws_layout(nb->N, nb->ncell_total, nb->cap, nb->flags, nb->ncell);
    const TileLayout tl = tile_layout(nb->N, a.nhc, nb->cap, tp.ntiles);
    char *b = (char *)nb->ws + wl.tiles;
    a.hcount = (int32_t *)(b + tl.hcount);
    a.hstart = (int32_t *)(b + tl.hstart);
    a.bsum = (int32_t *)(b + tl.bsum);
    a.key = (int32_t *)(b + tl.key);
    a.rank = (int32_t *)(b + tl.rank);
    a.tmp = (int32_t *)(b + tl.tmp);
    a.rb0 = (float4 *)(b + tl.r0);
    a.rb1 = (float4 *)(b + tl.r1);
    a.vb0 = (float4 *)(b + tl.v0);
    a.vb1 = (float4 *)(b + tl.v1);
    a.pb0 = (int32_t *)(b + tl.p0);
    a.pb1 = (int32_t *)(b + tl.p1);
    a.rref = (float4 *)(b + tl.rref);
    a.fs = (float4 *)(b + tl.fs);
    a.cnt = (uint32_t *)(b + tl.cnt);
    a.rows = (uint16_t *)(b + tl.rows);
    a.sent = (uint4 *)(b + tl.sent);
    a.tab = (int32_t *)(b + tl.tab);
    const WsPtrs w = ws_ptrs(nb);
    a.ctl = w.ctl;
    a.partials = w.partials;
    a.status = d_status;
}

static bool set_tile_pot(const md_pot *p, const md_nbr *nb, TileArgs &a)
{
    if (!p) return false;
    a.pot = p->kind;
    if (p->kind == MD_LJ) {
        if (!(p->r_cut > 0.0f) || p->r_cut > nb->r_list) return false;
        a.rc2 = p->r_cut * p->r_cut;
        const double s6 = pow((double)p->sigma, 6.0), e = (double)p->eps;
        a.lj_f12 = (float)(48.0 * e * s6 * s6);
        a.lj_f6 = (float)(24.0 * e * s6);
        a.lj_e12 = (float)(4.0 * e * s6 * s6);
        a.lj_e6 = (float)(4.0 * e * s6);
        a.e_shift = p->e_shift;
        return true;
    }
    if (p->kind == MD_SOFT_SPHERE) {
        a.eps = p->eps;
        a.alpha = p->alpha;
        return true;
    }
    return false;
}

// positions of the region and the sentinel, then one byte per own particle (kmap)
static size_t tile_smem(const TileArgs &a) { return ((size_t)a.reg_cap + 1) * sizeof(float4) + (size_t)a.reg_cap + 16; }

template <typename K>
static void tile_smem_attr(K kern)
{
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (TILE_REG_CAP_MAX + 1) * (int)sizeof(float4) + TILE_REG_CAP_MAX + 16);
}

// Dynamic shared memory above 48 KB for the staging kernels, once per
// device, before any launch or capture of them.
static void ensure_tile_attrs()
{
    static std::mutex mu;
    static unsigned long long done = 0ull;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return;
    std::lock_guard<std::mutex> lk(mu);
    if (done & (1ull << dev)) return;
    tile_smem_attr(k_t_build);
    tile_smem_attr(k_t_step<MD_LJ, 4, 0>);
    tile_smem_attr(k_t_step<MD_LJ, 8, 0>);
    tile_smem_attr(k_t_step<MD_LJ, 4, 2>);
    tile_smem_attr(k_t_step<MD_LJ, 8, 2>);
    tile_smem_attr(k_t_step<MD_SOFT_SPHERE, 4, 0>);
    tile_smem_attr(k_t_step<MD_SOFT_SPHERE, 8, 0>);
    tile_smem_attr(k_t_step<MD_SOFT_SPHERE, 4, 2>);
    tile_smem_attr(k_t_step<MD_SOFT_SPHERE, 8, 2>);
    tile_smem_attr(k_t_step1<MD_LJ, 0>);
    tile_smem_attr(k_t_step1<MD_LJ, 2>);
    tile_smem_attr(k_t_step1<MD_SOFT_SPHERE, 0>);
    tile_smem_attr(k_t_step1<MD_SOFT_SPHERE, 2>);
    done |= 1ull << dev;
}

// The rebuild chain (import: from the caller's arrays).
static void enqueue_tile_chain(TileArgs a, int import, int gated, cudaStream_t st)
{
    a.import = import;
    a.gated = gated;
    const int gN = (a.N + TT - 1) / TT;
    const int nb = (a.nhc + TSCAN_ITEMS - 1) / TSCAN_ITEMS;
    k_t_bin<<<gN, TT, 0, st>>>(a);
    k_t_scan1<<<nb, 1024, 0, st>>>(a);
    k_t_scan2<<<1, 1024, 0, st>>>(a, nb);
    k_t_scan3<<<(a.nhc + TT - 1) / TT, TT, 0, st>>>(a);
    k_t_scatter<<<gN, TT, 0, st>>>(a);
    k_t_place<<<gN, TT, 0, st>>>(a);
    k_t_build<<<a.ntiles, TT, tile_smem(a), st>>>(a);
    k_t_finish<<<1, 1, 0, st>>>(a);
}

template <int POT, int TPP, int KICK>
static void launch_step_t(const TileArgs &a, cudaStream_t st)
{
    k_t_step<POT, TPP, KICK><<<a.ntiles, TT, tile_smem(a), st>>>(a);
}

// Lanes per particle of the step kernel for this plan.
static int tile_tpp(const TileArgs &a)
{
    if (g_tile_tpp) return g_tile_tpp;
    const double own = (double)a.N * a.tx * a.ty * a.tz / ((double)a.H[0] * a.H[1] * a.H[2]);
    return own >= 128.0 ? 1 : 4;
}

template <int POT, int KICK>
static void launch_step1(const TileArgs &a, cudaStream_t st)
{
    k_t_step1<POT, KICK><<<a.ntiles, TT, tile_smem(a), st>>>(a);
}

template <int KICK>
static void launch_step(const TileArgs &a, cudaStream_t st)
{
    const int tpp = tile_tpp(a);
    if (a.pot == MD_LJ) {
        if (tpp == 1) launch_step1<MD_LJ, KICK>(a, st);
        else if (tpp == 4) launch_step_t<MD_LJ, 4, KICK>(a, st);
        else launch_step_t<MD_LJ, 8, KICK>(a, st);
    } else {
        if (tpp == 1) launch_step1<MD_SOFT_SPHERE, KICK>(a, st);
        else if (tpp == 4) launch_step_t<MD_SOFT_SPHERE, 4, KICK>(a, st);
        else launch_step_t<MD_SOFT_SPHERE, 8, KICK>(a, st);
    }
}

static void enqueue_tile_export(TileArgs a, float *d_r, float *d_v, float *d_f, const md_nbr *nb, int rows,
                                cudaStream_t st)
{
    a.r_out = (float4 *)d_r;
    a.v_out = (float4 *)d_v;
    a.f_out = (float4 *)d_f;
    a.export_rows = rows;
    a.rref_out = (float4 *)nb->rref;
    a.nbr_out = nb->nbr;
    a.cnt_out = nb->cnt;
    k_t_export<<<(a.N + TT - 1) / TT, TT, 0, st>>>(a);
    if (rows) k_t_rows<<<a.ntiles, TT, 0, st>>>(a);
}

// Cached graphs of the tiled NVE loop: import chain -> first kick ->
// WHILE { IF(rebuild) { chain } -> fused step } -> export.
struct TileGraph {
    TileArgs key;
    int device;
    cudaGraphExec_t exec;
};
static std::vector<TileGraph> g_tile_graphs;
static std::mutex g_tile_mu;

static cudaGraphNodeParams *zparams(unsigned char *raw)
{
    memset(raw, 0, sizeof(cudaGraphNodeParams));
    return reinterpret_cast<cudaGraphNodeParams *>(raw);
}

static md_status build_tile_graph(const TileArgs &a0, const md_nbr *nb, float *d_r, float *d_v, float *d_f,
                                  cudaGraphExec_t *out)
{
    TileArgs a = a0;
    cudaGraph_t g = nullptr;
    JMD_CUDA_TRY(cudaGraphCreate(&g, 0));
    cudaGraphConditionalHandle hw, hi;
    JMD_CUDA_TRY(cudaGraphConditionalHandleCreate(&hw, g, 1u, cudaGraphCondAssignDefault));
    JMD_CUDA_TRY(cudaGraphConditionalHandleCreate(&hi, g, 0u, cudaGraphCondAssignDefault));
    a.cond_while = (unsigned long long)hw;
    a.cond_if = (unsigned long long)hi;
    a.use_cond = 1;
    cudaStream_t cs = nullptr, cs2 = nullptr;
    JMD_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    JMD_CUDA_TRY(cudaStreamCreateWithFlags(&cs2, cudaStreamNonBlocking));
    JMD_CUDA_TRY(cudaStreamBeginCaptureToGraph(cs, g, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    enqueue_tile_chain(a, 1, 0, cs);
    k_t_kick<<<(a.N + TT - 1) / TT, TT, 0, cs>>>(a);
    alignas(cudaGraphNodeParams) unsigned char wraw[sizeof(cudaGraphNodeParams)];
    cudaGraphNodeParams *wp = zparams(wraw);
    wp->type = cudaGraphNodeTypeConditional;
    wp->conditional.handle = hw;
    wp->conditional.type = cudaGraphCondTypeWhile;
    wp->conditional.size = 1;
    cudaStreamCaptureStatus cst;
    cudaGraph_t cg = nullptr;
    const cudaGraphNode_t *deps = nullptr;
    size_t nd = 0;
    JMD_CUDA_TRY(cudaStreamGetCaptureInfo(cs, &cst, nullptr, &cg, &deps, nullptr, &nd));
    cudaGraphNode_t wn;
    JMD_CUDA_TRY(cudaGraphAddNode(&wn, cg, deps, nullptr, nd, wp));
    JMD_CUDA_TRY(cudaStreamUpdateCaptureDependencies(cs, &wn, nullptr, 1, cudaStreamSetCaptureDependencies));
    enqueue_tile_export(a, d_r, d_v, d_f, nb, 1, cs);
    JMD_CUDA_TRY(cudaStreamEndCapture(cs, &g));
    cudaGraph_t body = wp->conditional.phGraph_out[0];

    JMD_CUDA_TRY(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    alignas(cudaGraphNodeParams) unsigned char iraw[sizeof(cudaGraphNodeParams)];
    cudaGraphNodeParams *ip = zparams(iraw);
    ip->type = cudaGraphNodeTypeConditional;
    ip->conditional.handle = hi;
    ip->conditional.type = cudaGraphCondTypeIf;
    ip->conditional.size = 1;
    JMD_CUDA_TRY(cudaStreamGetCaptureInfo(cs, &cst, nullptr, &cg, &deps, nullptr, &nd));
    cudaGraphNode_t in;
    JMD_CUDA_TRY(cudaGraphAddNode(&in, cg, deps, nullptr, nd, ip));
    JMD_CUDA_TRY(cudaStreamUpdateCaptureDependencies(cs, &in, nullptr, 1, cudaStreamSetCaptureDependencies));
    cudaGraph_t ibody = ip->conditional.phGraph_out[0];
    JMD_CUDA_TRY(cudaStreamBeginCaptureToGraph(cs2, ibody, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    enqueue_tile_chain(a, 0, 0, cs2);
    JMD_CUDA_TRY(cudaStreamEndCapture(cs2, &ibody));
    launch_step<2>(a, cs);
    JMD_CUDA_TRY(cudaStreamEndCapture(cs, &body));
    cudaStreamDestroy(cs2);
    cudaStreamDestroy(cs);
    cudaGraphExec_t ex = nullptr;
    JMD_CUDA_TRY(cudaGraphInstantiate(&ex, g, 0));
    cudaGraphDestroy(g);
    *out = ex;
    return MD_OK;
}

// md_integrate_nve on the tile engine (LJ / soft sphere, 3-D).
md_status run_tiled_nve(const md_space *s, const md_pot *p, float *d_r, float *d_v, float *d_f, float mass, float dt,
                        int nsteps, md_nbr *nb, double *d_PE, double *d_KE, int use_graph, uint32_t *d_status,
                        cudaStream_t st)
{
    TilePlan tp;
    if (!tiles_ready(s, nb, tp)) return MD_ERR_INVALID;
    TileArgs a;
    ensure_tile_attrs();
    make_tile_args(s, nb, tp, d_status, a);
    if (!set_tile_pot(p, nb, a)) return MD_ERR_INVALID;
    a.r_in = (const float4 *)d_r;
    a.v_in = (const float4 *)d_v;
    a.f_in = (const float4 *)d_f;
    a.hdm = 0.5f * dt / mass;
    a.dt = dt;
    a.mass = mass;
    a.E_out = d_PE;
    a.KE_out = d_KE;
    a.series = 1;
    a.variant = tile_tpp(a);
    if (nsteps == 0) return MD_OK;
    const uint32_t *ctl = a.ctl;
    if (use_graph) {
        int dev = 0;
        JMD_CUDA_TRY(cudaGetDevice(&dev));
        cudaGraphExec_t ex = nullptr;
        {
            std::lock_guard<std::mutex> lk(g_tile_mu);
            for (auto &e : g_tile_graphs)
                if (e.device == dev && memcmp(&e.key, &a, sizeof(TileArgs)) == 0) ex = e.exec;
            if (!ex) {
                md_status e = build_tile_graph(a, nb, d_r, d_v, d_f, &ex);
                if (e != MD_OK) return e;
                TileGraph tg;
                memset(&tg, 0, sizeof(tg));
                tg.key = a;
                tg.device = dev;
                tg.exec = ex;
                g_tile_graphs.push_back(tg);
            }
        }
        enqueue_loop_init(const_cast<uint32_t *>(ctl), (uint32_t)nsteps, st);
        JMD_CUDA_TRY(cudaGraphLaunch(ex, st));
        JMD_CUDA_TRY(cudaGetLastError());
        return MD_OK;
    }
    enqueue_loop_init(const_cast<uint32_t *>(ctl), (uint32_t)nsteps, st);
    enqueue_tile_chain(a, 1, 0, st);
    k_t_kick<<<(a.N + TT - 1) / TT, TT, 0, st>>>(a);
    for (int k = 0; k < nsteps; ++k) {
        enqueue_tile_chain(a, 0, 1, st);
        launch_step<2>(a, st);
    }
    enqueue_tile_export(a, d_r, d_v, d_f, nb, 1, st);
    JMD_CUDA_TRY(cudaGetLastError());
    return MD_OK;
}

bool tiles_enabled(const md_space *s, const md_nbr *nb, const md_pot *p)
{
    TilePlan tp;
    return p && (p->kind == MD_LJ || p->kind == MD_SOFT_SPHERE) && tiles_ready(s, nb, tp);
}

bool tiles_plan_ok(const md_space *s, const md_nbr *nb)
{
    TilePlan tp;
    return tile_plan(s, nb, tp);
}

}  // namespace jmd

using namespace jmd;

extern "C" md_status md_set_tile_tpp(int tpp)
{
    if (tpp != 0 && tpp != 1 && tpp != 4 && tpp != 8) return MD_ERR_INVALID;
    g_tile_tpp = tpp;
    return MD_OK;
}

extern "C" md_status md_tiles_info(const md_space *s, const md_nbr *nb, int32_t *out)
{
    TilePlan tp;
    if (!out || !tile_plan(s, nb, tp)) return MD_ERR_INVALID;
    out[0] = tp.H[0];
    out[1] = tp.H[1];
    out[2] = tp.H[2];
    out[3] = tp.tx;
    out[4] = tp.ty;
    out[5] = tp.tz;
    out[6] = tp.ntiles;
    out[7] = tp.reg_cap;
    return MD_OK;
}

extern "C" md_status md_tiles_import(const md_space *s, const float *d_r, const float *d_v, const float *d_f,
                                     md_nbr *nb, uint32_t *d_status, md_stream_t stream)
{
    TilePlan tp;
    if (!d_r || !tiles_ready(s, nb, tp)) return MD_ERR_INVALID;
    TileArgs a;
    ensure_tile_attrs();
    make_tile_args(s, nb, tp, d_status, a);
    a.r_in = (const float4 *)d_r;
    a.v_in = (const float4 *)d_v;
    a.f_in = (const float4 *)d_f;
    enqueue_tile_chain(a, 1, 0, (cudaStream_t)stream);
    JMD_CUDA_TRY(cudaGetLastError());
    return MD_OK;
}

extern "C" md_status md_tiles_forces(const md_space *s, const md_pot *p, md_nbr *nb, double *d_E, uint32_t *d_status,
                                     md_stream_t stream)
{
    TilePlan tp;
    if (!tiles_ready(s, nb, tp)) return MD_ERR_INVALID;
    TileArgs a;
    ensure_tile_attrs();
    make_tile_args(s, nb, tp, d_status, a);
    if (!set_tile_pot(p, nb, a)) return MD_ERR_INVALID;
    a.E_out = d_E;
    launch_step<0>(a, (cudaStream_t)stream);
    JMD_CUDA_TRY(cudaGetLastError());
    return MD_OK;
}

extern "C" md_status md_tiles_export(const md_space *s, md_nbr *nb, float *d_r, float *d_v, float *d_f, int rows,
                                     md_stream_t stream)
{
    TilePlan tp;
    if (!tiles_ready(s, nb, tp)) return MD_ERR_INVALID;
    TileArgs a;
    make_tile_args(s, nb, tp, nullptr, a);
    enqueue_tile_export(a, d_r, d_v, d_f, nb, rows ? 1 : 0, (cudaStream_t)stream);
    JMD_CUDA_TRY(cudaGetLastError());
    return MD_OK;
}

extern "C" md_status md_tiles_steps(const md_space *s, const md_pot *p, md_nbr *nb, float mass, float dt, int nsteps,
                                    double *d_PE, double *d_KE, uint32_t *d_status, md_stream_t stream)
{
    TilePlan tp;
    if (!tiles_ready(s, nb, tp) || nsteps < 0 || !(mass > 0.0f)) return MD_ERR_INVALID;
    TileArgs a;
    ensure_tile_attrs();
    make_tile_args(s, nb, tp, d_status, a);
    if (!set_tile_pot(p, nb, a)) return MD_ERR_INVALID;
    if (nsteps == 0) return MD_OK;
    a.hdm = 0.5f * dt / mass;
    a.dt = dt;
    a.mass = mass;
    a.E_out = d_PE;
    a.KE_out = d_KE;
    a.series = 1;
    cudaStream_t st = (cudaStream_t)stream;
    enqueue_loop_init(a.ctl, (uint32_t)nsteps, st);
    k_t_kick<<<(a.N + TT - 1) / TT, TT, 0, st>>>(a);
    for (int k = 0; k < nsteps; ++k) launch_step<2>(a, st);
    JMD_CUDA_TRY(cudaGetLastError());
    return MD_OK;
}
