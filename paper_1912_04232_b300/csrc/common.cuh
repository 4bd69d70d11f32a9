// common.cuh -- device helpers shared by the libjmd kernels (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>
#include <math.h>

#include "../../include/jmd.h"

namespace jmd {

// ---------------------------------------------------------------------------
// Control words at the head of every neighbor-list workspace.
// ---------------------------------------------------------------------------
enum CtlWord : int {
    CTL_REBUILD = 0,     // 1 -> the gated rebuild chain runs
    CTL_TICKET = 1,      // last-block ticket of the energy reductions
    CTL_MAXCNT = 2,      // largest row count seen by any build
    CTL_STEP = 3,        // device step counter of the running loop
    CTL_BUILDS_LO = 4,   // number of builds (64-bit, two words)
    CTL_BUILDS_HI = 5,
    CTL_TICKET2 = 6,     // second ticket (displacement-check hand-off)
    CTL_NSTEPS = 7,      // loop length for device-side loop control
    CTL_SEED_LO = 8,     // Langevin noise key (64 bits)
    CTL_SEED_HI = 9,
    CTL_STEP0 = 10,      // noise counter of the loop's first step
    CTL_ITER = 11,       // iteration counter of a graph loop (graphloop.cu)
    CTL_NITER = 12,      // its length
    CTL_TSEL = 13,       // tile engine: bit 0 current position buffer, bit 1 current velocity / id buffer
    CTL_WORDS = 64
};

struct Box {
    float L[3];
    float Linv[3];
};

__host__ __device__ inline Box make_box(const md_space *s)
{
    Box b;
    for (int k = 0; k < 3; ++k) {
        b.L[k] = s->L[k];
        b.Linv[k] = s->Linv[k];
    }
    return b;
}

// Nearest-image component, every operation rounded separately (Sec. 3.2.1):
//   t = a - b;  d = t - L * rint(t * Linv)
__device__ __forceinline__ float min_image_rn(float a, float b, float L, float Linv)
{
    float t = __fsub_rn(a, b);
    float n = rintf(__fmul_rn(t, Linv));
    return __fsub_rn(t, __fmul_rn(L, n));
}

// The same displacement for |t * Linv| < 1.5, which holds whenever both
// positions lie inside [0, L) (or a little outside): rint(u) can then only
// be -1, 0 or 1 and is decided by two comparisons (rint(+-0.5) = 0, so the
// tests are strict), and t - L*n is formed with the same single rounding
// (L*n is exactly -L, 0 or L).  The bits equal min_image_rn's for every such
// input; it avoids the round-to-integer conversion.
__device__ __forceinline__ float min_image_near(float a, float b, float L, float Linv)
{
    const float t = __fsub_rn(a, b);
    const float u = __fmul_rn(t, Linv);
    const float s = u > 0.5f ? L : (u < -0.5f ? -L : 0.0f);
    return __fsub_rn(t, s);
}

// Squared nearest-image distance, r2 = (dx*dx + dy*dy) + dz*dz, no FMA.
// This exact expression decides every pair-membership test (neighbor list
// and cutoffs) so the decision is reproducible bit for bit.
template <int DIM>
__device__ __forceinline__ float dist2_rn(const float4 &a, const float4 &b, const Box &bx, float &dx, float &dy,
                                          float &dz)
{
    dx = min_image_rn(a.x, b.x, bx.L[0], bx.Linv[0]);
    dy = min_image_rn(a.y, b.y, bx.L[1], bx.Linv[1]);
    float r2 = __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy));
    if (DIM == 3) {
        dz = min_image_rn(a.z, b.z, bx.L[2], bx.Linv[2]);
        r2 = __fadd_rn(r2, __fmul_rn(dz, dz));
    } else {
        dz = 0.0f;
    }
    return r2;
}

// dist2_rn for positions inside [0, L) (min_image_near on every axis).
template <int DIM>
__device__ __forceinline__ float dist2_near(const float4 &a, const float4 &b, const Box &bx, float &dx, float &dy,
                                            float &dz)
{
    dx = min_image_near(a.x, b.x, bx.L[0], bx.Linv[0]);
    dy = min_image_near(a.y, b.y, bx.L[1], bx.Linv[1]);
    float r2 = __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy));
    if (DIM == 3) {
        dz = min_image_near(a.z, b.z, bx.L[2], bx.Linv[2]);
        r2 = __fadd_rn(r2, __fmul_rn(dz, dz));
    } else {
        dz = 0.0f;
    }
    return r2;
}

// Squared distance for a particle whose every list partner is its unwrapped
// image (the particle lies at least r_list + skin from each face): then
// rint(t * Linv) = 0 and the nearest-image formula above reduces to d = t
// exactly, so the same bits come out without the wrap arithmetic.
template <int DIM>
__device__ __forceinline__ float dist2_inner(const float4 &a, const float4 &b, float &dx, float &dy, float &dz)
{
    dx = __fsub_rn(a.x, b.x);
    dy = __fsub_rn(a.y, b.y);
    float r2 = __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy));
    if (DIM == 3) {
        dz = __fsub_rn(a.z, b.z);
        r2 = __fadd_rn(r2, __fmul_rn(dz, dz));
    } else {
        dz = 0.0f;
    }
    return r2;
}

// Row entries streamed past L1 (L1 is left to the gathered positions).
__device__ __forceinline__ int ld_stream(const int32_t *p)
{
    int v;
    asm volatile("ld.global.nc.L1::no_allocate.b32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ int ld_stream_u16(const uint16_t *p)
{
    unsigned short v;
    asm volatile("ld.global.nc.L1::no_allocate.u16 %0, [%1];" : "=h"(v) : "l"(p));
    return v;
}

// Wrap a coordinate into [0, L): x - L floor(x Linv), folded once more if
// rounding left it on the boundary.
__device__ __forceinline__ float wrap_coord(float x, float L, float Linv)
{
    float y = x - L * floorf(x * Linv);
    if (y >= L) y -= L;
    if (y < 0.0f) y = 0.0f;
    return y;
}

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) from its published
// definition: ten rounds of
//   (c0, c1, c2, c3) -> (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0))
// with M0 = 0xD2511F53, M1 = 0xCD9E8D57 and the key advanced by
// (0x9E3779B9, 0xBB67AE85) between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        unsigned hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        unsigned hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
        k.x += 0x9E3779B9u;
        k.y += 0xBB67AE85u;
    }
    return c;
}

// Three standard normals for particle i at noise step s: one Philox block
// with counter (i, s, 0, 0); uniforms u = ((x >> 8) + 1) 2^-24 in (0, 1];
// Box-Muller on (u0, u1) and (u2, u3).
__device__ __forceinline__ float3 normal3(unsigned i, unsigned s, uint2 key)
{
    uint4 x = philox4x32_10(make_uint4(i, s, 0u, 0u), key);
    const float sc = 1.0f / 16777216.0f;
    float u0 = (float)((x.x >> 8) + 1u) * sc, u1 = (float)((x.y >> 8) + 1u) * sc;
    float u2 = (float)((x.z >> 8) + 1u) * sc, u3 = (float)((x.w >> 8) + 1u) * sc;
    float ra = sqrtf(-2.0f * logf(u0)), rb = sqrtf(-2.0f * logf(u2));
    float s1, c1, s3, c3;
    sincospif(2.0f * u1, &s1, &c1);
    sincospif(2.0f * u3, &s3, &c3);
    return make_float3(ra * c1, ra * s1, rb * c3);
}

__device__ __forceinline__ void raise_status(uint32_t *st, uint32_t bits)
{
    if (st) atomicOr(st, bits);
}

// One atomic per kernel launch: block 0 / thread 0 counts the launch, so the
// library can report exactly how many of its kernels ran (graph bodies
// included).  Each translation unit has its own counter (no relocatable
// device code); a static registrar adds the unit's reader to a host list
// that md_launch_count() sums.
static __device__ unsigned long long g_kernel_launches = 0ull;
__device__ __forceinline__ void count_launch()
{
    if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) atomicAdd(&g_kernel_launches, 1ull);
}

typedef unsigned long long (*launch_reader_t)(void);
void register_launch_reader(launch_reader_t f);
static unsigned long long tu_launches(void)
{
    unsigned long long v = 0ull;
    if (cudaMemcpyFromSymbol(&v, g_kernel_launches, sizeof(v)) != cudaSuccess) return 0ull;
    return v;
}
namespace {
struct LaunchRegistrar {
    LaunchRegistrar() { register_launch_reader(&tu_launches); }
};
static LaunchRegistrar g_launch_registrar;
}  // namespace

// Fixed-order FP64 block sum (all threads participate, result valid in
// thread 0).  `sh` needs blockDim.x/32 doubles.
__device__ __forceinline__ double block_sum_f64(double v, double *sh)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    double s = 0.0;
    if (w == 0) {
        int nw = blockDim.x >> 5;
        s = (l < nw) ? sh[l] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    }
    return s;
}

// K block sums at once, each in the order of block_sum_f64 (same bits): the
// K dependency chains interleave (an FP64 add has a long latency on this
// GPU), and the block synchronises twice instead of 2K times.  sh holds K
// rows of `stride` >= blockDim.x / 32 doubles.  Results valid in warp 0.
template <int K>
__device__ __forceinline__ void block_sums_f64(double (&v)[K], double *sh, int stride)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int c = 0; c < K; ++c) v[c] += __shfl_xor_sync(0xffffffffu, v[c], o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
    __syncthreads();
    if (l == 0)
#pragma unroll
        for (int c = 0; c < K; ++c) sh[c * stride + w] = v[c];
    __syncthreads();
#pragma unroll
    for (int c = 0; c < K; ++c) v[c] = (w == 0 && l < nw) ? sh[c * stride + l] : 0.0;
    if (w == 0) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int c = 0; c < K; ++c) v[c] += __shfl_xor_sync(0xffffffffu, v[c], o);
    }
}

// ---------------------------------------------------------------------------
// Workspace layout of a neighbor list (all offsets 256-byte aligned).
// ---------------------------------------------------------------------------
struct WsLayout {
    size_t ctl, cell_count, cell_start, cell_of, rank, atoms_u, atoms, rsorted, ralt, partials, lrow, tiles, total;
    int max_blocks;
};

__host__ inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Partner lists of the three-body potentials (caller-owned scratch): per
// atom the count of partners inside the potential's cutoff, their indices
// and displacement vectors (dx, dy, dz, r) = r_j - r_i, S slots per atom, in
// the order of the atom's neighbor row; with AUX (Stillinger-Weber) also
// each slot's one-leg factors and each atom's two-body force and energy.
struct TbLayout {
    size_t cnt, idx, vec, aux, f2, bytes;
};
__host__ inline TbLayout tb_layout(int N, int S, bool aux)
{
    TbLayout t;
    size_t o = 0;
    t.cnt = o;  o = align256(o + sizeof(int32_t) * (size_t)N);
    t.idx = o;  o = align256(o + sizeof(int32_t) * (size_t)N * S);
    t.vec = o;  o = align256(o + 4 * sizeof(float) * (size_t)N * S);
    t.aux = o;  o = aux ? align256(o + 4 * sizeof(float) * (size_t)N * S) : o;
    t.f2 = o;   o = aux ? align256(o + 4 * sizeof(float) * (size_t)N) : o;
    t.bytes = o;
    return t;
}

// Scratch of the tile engine (MD_NBR_TILES), offsets from its own start.
// nhc = half-cells (2 x 2 x 2 per cell of the list's grid).
constexpr int TSCAN_ITEMS = 4096;       // half-cells per block of the histogram scan
constexpr int TILE_TMAX = 8;            // largest tile extent (half-cells) along y and z
constexpr int TILE_XMAX = 2;            // ... and along x
constexpr int TILE_PIECES_MAX = 2 * (TILE_TMAX + 4) * (TILE_TMAX + 4);   // two copies per region row
constexpr int TILE_OWN_MAX = TILE_XMAX * TILE_TMAX * TILE_TMAX;          // own half-cells
// Per-tile table written by each build and read by every step: region
// total, copies, own half-cells, own particles; the copies (source slot,
// destination offset << 16 | count); the own half-cells (first slot,
// first local index << 16 | first own particle).
// The copy's source slot carries its periodic image in the top bits: two
// bits per axis (1: +L, 2: -L), so slots need N < 2^26.  The header's
// copy count carries a flag (bit 16) when any copy has an image.
constexpr int TILE_TAB_WORDS = 4 + 2 * TILE_PIECES_MAX + 2 * TILE_OWN_MAX;
constexpr int TILE_SRC_BITS = 26;
constexpr unsigned TILE_SRC_MASK = (1u << TILE_SRC_BITS) - 1u;
constexpr int TILE_REG_CAP_MAX = 12800;  // region capacity limit (particles, 200 KB of shared memory)
constexpr int TILE_SLOTS = 4 * 148;      // resident tile CTAs of a B300 (148 SMs, 4 per SM) for the shape choice

struct TilePlan {
    int H[3];
    int tx, ty, tz, ntx, nty, ntz, ntiles, reg_cap;
};

// Tile geometry of N particles on a list grid of ncell cells per axis:
// half-cells H = 2 ncell; tiles of tx x ty x tz half-cells (tx in {1, 2},
// ty, tz in {2, 4, 6, 8}, region = tile grown by 2 on each side, which must
// not wrap onto itself).  The shape minimises a cost model of the step
// kernel in particle units: waves of TILE_SLOTS CTAs times the per-tile
// work (own particles + 0.08 x staged region particles + 40 fixed).
// Region capacity 1.25x the mean region count plus 128.
__host__ inline bool tile_geometry(int N, const int *ncell, TilePlan &tp)
{
    for (int k = 0; k < 3; ++k) {
        if (ncell[k] < 3) return false;
        tp.H[k] = 2 * ncell[k];
    }
    const double hc = (double)tp.H[0] * tp.H[1] * tp.H[2];
    if (hc > (double)TSCAN_ITEMS * 4096.0) return false;
    const int cx[2] = {2, 1}, cyz[4] = {8, 6, 4, 2};
    double best = -1.0;
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 4; ++b)
            for (int c = 0; c < 4; ++c) {
                const int tx = cx[a], ty = cyz[b], tz = cyz[c];
                if (tx + 4 > tp.H[0] || ty + 4 > tp.H[1] || tz + 4 > tp.H[2]) continue;
                const int ntx = (tp.H[0] + tx - 1) / tx, nty = (tp.H[1] + ty - 1) / ty, ntz = (tp.H[2] + tz - 1) / tz;
                const long long nt = (long long)ntx * nty * ntz;
                if (nt > (long long)(N / 4 + 64)) continue;   // FP64 partials of the energy reduction
                const double own = (double)N * tx * ty * tz / hc;
                const double reg = (double)N * (tx + 4) * (ty + 4) * (tz + 4) / hc;
                const double waves = (double)((nt + TILE_SLOTS - 1) / TILE_SLOTS);
                const double cost = waves * (own + 0.08 * reg + 40.0);
                int cap = (int)ceil(1.25 * reg) + 128;
                cap = (cap + 31) & ~31;
                if (cap > TILE_REG_CAP_MAX) continue;
                if (best < 0.0 || cost < best) {
                    best = cost;
                    tp.tx = tx;
                    tp.ty = ty;
                    tp.tz = tz;
                    tp.ntx = ntx;
                    tp.nty = nty;
                    tp.ntz = ntz;
                    tp.ntiles = (int)nt;
                    tp.reg_cap = cap;
                }
            }
    return best >= 0.0;
}

struct TileLayout {
    size_t hcount, hstart, bsum, key, rank, tmp, r0, r1, v0, v1, p0, p1, rref, fs, cnt, tab, rows, sent, total;
};
__host__ inline TileLayout tile_layout(int N, int nhc, int cap, int ntiles)
{
    TileLayout t;
    size_t o = 0;
    const size_t n = (size_t)N;
    t.hcount = o;  o = align256(o + sizeof(int32_t) * (size_t)nhc);
    t.hstart = o;  o = align256(o + sizeof(int32_t) * ((size_t)nhc + 1));
    t.tab = o;     o = align256(o + sizeof(int32_t) * (size_t)TILE_TAB_WORDS * (size_t)ntiles);
    t.bsum = o;    o = align256(o + sizeof(int32_t) * ((size_t)nhc / TSCAN_ITEMS + 2));
    t.key = o;     o = align256(o + sizeof(int32_t) * n);
    t.rank = o;    o = align256(o + sizeof(int32_t) * n);
    t.tmp = o;     o = align256(o + sizeof(int32_t) * n);
    t.r0 = o;      o = align256(o + sizeof(float4) * n);
    t.r1 = o;      o = align256(o + sizeof(float4) * n);
    t.v0 = o;      o = align256(o + sizeof(float4) * n);
    t.v1 = o;      o = align256(o + sizeof(float4) * n);
    t.p0 = o;      o = align256(o + sizeof(int32_t) * n);
    t.p1 = o;      o = align256(o + sizeof(int32_t) * n);
    t.rref = o;    o = align256(o + sizeof(float4) * n);
    t.fs = o;      o = align256(o + sizeof(float4) * n);
    t.cnt = o;     o = align256(o + sizeof(uint32_t) * n);
    t.rows = o;    o = align256(o + sizeof(uint16_t) * n * (size_t)cap);
    t.sent = o;    o = align256(o + 16);   // one 16-byte row chunk of sentinel entries
    t.total = o;
    return t;
}

// Scratch of a neighbor list; the 16-bit local rows only with MD_NBR_LOCAL_ROWS.
__host__ inline WsLayout ws_layout(int N, int ncell_total, int cap, int flags, const int *ncell = nullptr)
{
    WsLayout w;
    size_t o = 0;
    w.ctl = o;          o = align256(o + sizeof(uint32_t) * CTL_WORDS);
    w.cell_count = o;   o = align256(o + sizeof(int32_t) * (size_t)ncell_total);
    w.cell_start = o;   o = align256(o + sizeof(int32_t) * ((size_t)ncell_total + 1));
    w.cell_of = o;      o = align256(o + sizeof(int32_t) * (size_t)N);
    w.rank = o;         o = align256(o + sizeof(int32_t) * (size_t)N);
    w.atoms_u = o;      o = align256(o + sizeof(int32_t) * (size_t)N);
    w.atoms = o;        o = align256(o + sizeof(int32_t) * (size_t)N);
    w.rsorted = o;      o = align256(o + sizeof(float4) * (size_t)N);
    w.ralt = o;         o = align256(o + sizeof(float4) * (size_t)N);
    w.max_blocks = N / 4 + 64;
    w.partials = o;     o = align256(o + sizeof(double2) * (size_t)w.max_blocks);
    w.lrow = o;
    if (flags & MD_NBR_LOCAL_ROWS) o = align256(o + sizeof(uint16_t) * (size_t)N * (size_t)cap);
    w.tiles = o;
    if (flags & MD_NBR_TILES) {
        TilePlan tp;
        const int nt = (ncell && tile_geometry(N, ncell, tp)) ? tp.ntiles : 0;
        o = align256(o + tile_layout(N, 8 * ncell_total, cap, nt).total);
    }
    w.total = o;
    return w;
}

struct WsPtrs {
    uint32_t *ctl;
    int32_t *cell_count, *cell_start, *cell_of, *rank, *atoms_u, *atoms;
    float4 *rsorted;
    float4 *ralt;     // second position buffer of the fused NVE step
    double2 *partials;
    uint16_t *lrow;   // NULL without MD_NBR_LOCAL_ROWS
    int max_blocks;
};

__host__ inline WsPtrs ws_ptrs(const md_nbr *nb)
{
    WsLayout w = ws_layout(nb->N, nb->ncell_total, nb->cap, nb->flags, nb->ncell);
    char *b = (char *)nb->ws;
    WsPtrs p;
    p.ctl = (uint32_t *)(b + w.ctl);
    p.cell_count = (int32_t *)(b + w.cell_count);
    p.cell_start = (int32_t *)(b + w.cell_start);
    p.cell_of = (int32_t *)(b + w.cell_of);
    p.rank = (int32_t *)(b + w.rank);
    p.atoms_u = (int32_t *)(b + w.atoms_u);
    p.atoms = (int32_t *)(b + w.atoms);
    p.rsorted = (float4 *)(b + w.rsorted);
    p.ralt = (float4 *)(b + w.ralt);
    p.partials = (double2 *)(b + w.partials);
    p.lrow = (nb->flags & MD_NBR_LOCAL_ROWS) ? (uint16_t *)(b + w.lrow) : nullptr;
    p.max_blocks = w.max_blocks;
    return p;
}

// The plan's flags are valid and its layout fits the bound scratch (guards
// against flags changed after md_nbr_set_flags / md_nbr_bind).
__host__ inline bool nbr_layout_ok(const md_nbr *nb)
{
    if (nb->flags & ~(MD_NBR_CANONICAL | MD_NBR_LOCAL_ROWS | MD_NBR_TILES)) return false;
    if ((nb->flags & MD_NBR_CANONICAL) && (nb->flags & (MD_NBR_LOCAL_ROWS | MD_NBR_TILES))) return false;
    if ((nb->flags & MD_NBR_LOCAL_ROWS) && (nb->flags & MD_NBR_TILES)) return false;
    return ws_layout(nb->N, nb->ncell_total, nb->cap, nb->flags, nb->ncell).total <= nb->ws_bytes;
}

// Host-side CUDA error to status.
#define JMD_CUDA_TRY(expr)                                                                              \
    do {                                                                                                \
        cudaError_t _e = (expr);                                                                        \
        if (_e != cudaSuccess) return MD_ERR_CUDA;                                                      \
    } while (0)

}  // namespace jmd
