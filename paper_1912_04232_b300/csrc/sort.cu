// sort.cu -- spatial reordering of the particles along a Z-order (Morton)
// curve over the neighbor list's cell grid.
//
// The pair-force kernels gather every neighbor's position through L1; how
// often a gathered line is still there depends on how close in memory the
// particles that are close in space are.  A run that starts from a lattice
// has that order, but diffusion destroys it; with particles in random order
// the LJ force kernel at N = 256,000 takes 1.7x as long.  Sorting restores
// the order: cells are taken along the Z-order curve of their coordinates,
// and each cell's members in ascending old index, so the permutation is a
// deterministic function of the positions and the grid.  Inside a cell the
// relative order of the members does not change, so the rows of the list
// rebuilt by the sort hold the same partners in the same order and the
// forces keep their bits; later rebuilds order a cell's members by the new
// indices, so a trajectory agrees with the unsorted one to the rounding of
// reordered sums.
//
// Steps: bin the positions (the cell-list part of the rebuild chain), put
// each cell's member count at its Z-order key, exclusive scan over the keys
// (two-level, tiles of 4,096), copy each cell's members to its offset (the
// permutation), gather r and v through the scratch, rebuild the list.
#include <cstring>

#include "common.cuh"
#include "kernels.cuh"

namespace jmd {

constexpr int SCAN_TILE = 4096;           // keys per scan block (1,024 threads x 4)
constexpr int SORT_MAX_KEYS = 1 << 24;    // 256^3 cells in 3-D, 4,096^2 in 2-D

static int next_pow2(int n)
{
    int p = 1;
    while (p < n) p <<= 1;
    return p;
}

// Z-order key: bit b of x, y (and z) at positions dim*b, dim*b + 1 (+ 2).
// Built in 64 bits (the shifts of the top bits pass 32); the grid limit
// keeps every key below 2^24.
__device__ __forceinline__ uint32_t zorder_key(int cx, int cy, int cz, int dim)
{
    uint64_t k = 0u;
#pragma unroll
    for (int b = 0; b < 12; ++b) {
        k |= (uint64_t)((cx >> b) & 1) << (dim * b);
        k |= (uint64_t)((cy >> b) & 1) << (dim * b + 1);
        if (dim == 3) k |= (uint64_t)((cz >> b) & 1) << (3 * b + 2);
    }
    return (uint32_t)k;
}

__device__ __forceinline__ uint32_t cell_key(int c, const int *nc, int dim)
{
    const int cx = c % nc[0], cy = (c / nc[0]) % nc[1], cz = c / (nc[0] * nc[1]);
    return zorder_key(cx, cy, cz, dim);
}

struct SortArgs {
    int N, ncell, dim, nkeys, ntiles;
    int nc[3];
    const int32_t *cell_start, *atoms;
    uint32_t *keys;    // [nkeys]: member count, then exclusive offset
    uint32_t *tsum;    // [ntiles]
    int32_t *perm;     // [N]: new index -> old index
};

__global__ void __launch_bounds__(256) k_sort_counts(SortArgs a)
{
    count_launch();
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < a.ncell) a.keys[cell_key(c, a.nc, a.dim)] = (uint32_t)(a.cell_start[c + 1] - a.cell_start[c]);
}

// Exclusive scan inside each tile of SCAN_TILE keys; the tile totals go to
// tsum.
__global__ void __launch_bounds__(1024) k_sort_scan_tiles(uint32_t *x, int n, uint32_t *tsum)
{
    count_launch();
    __shared__ uint32_t wsum[32];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const size_t base = (size_t)blockIdx.x * SCAN_TILE + 4 * (size_t)t;
    uint32_t v[4], s = 0u;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        v[k] = (base + k < (size_t)n) ? x[base + k] : 0u;
        s += v[k];
    }
    uint32_t incl = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) wsum[w] = incl;
    __syncthreads();
    if (w == 0) {
        uint32_t ws = wsum[lane], wi = ws;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        wsum[lane] = wi - ws;   // exclusive over the warps
        if (lane == 31) tsum[blockIdx.x] = wi;
    }
    __syncthreads();
    uint32_t run = wsum[w] + incl - s;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (base + k < (size_t)n) x[base + k] = run;
        run += v[k];
    }
}

// Exclusive scan of the tile totals (at most SCAN_TILE of them), one block.
__global__ void __launch_bounds__(1024) k_sort_scan_totals(uint32_t *tsum, int ntiles)
{
    count_launch();
    __shared__ uint32_t wsum[32];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    uint32_t v[4], s = 0u;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int i = 4 * t + k;
        v[k] = i < ntiles ? tsum[i] : 0u;
        s += v[k];
    }
    uint32_t incl = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) wsum[w] = incl;
    __syncthreads();
    if (w == 0) {
        uint32_t ws = wsum[lane], wi = ws;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        wsum[lane] = wi - ws;
    }
    __syncthreads();
    uint32_t run = wsum[w] + incl - s;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int i = 4 * t + k;
        if (i < ntiles) tsum[i] = run;
        run += v[k];
    }
}

__global__ void __launch_bounds__(1024) k_sort_scan_add(uint32_t *x, int n, const uint32_t *tsum)
{
    count_launch();
    const uint32_t off = tsum[blockIdx.x];
    const size_t base = (size_t)blockIdx.x * SCAN_TILE;
    for (int k = threadIdx.x; k < SCAN_TILE; k += blockDim.x)
        if (base + k < (size_t)n) x[base + k] += off;
}

// One warp per cell: its members, already in ascending old index, go to the
// cell's offset in Z order.
__global__ void __launch_bounds__(256) k_sort_perm(SortArgs a)
{
    count_launch();
    const int c = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (c >= a.ncell) return;
    const int b = a.cell_start[c], n = a.cell_start[c + 1] - b;
    const uint32_t off = a.keys[cell_key(c, a.nc, a.dim)];
    for (int k = lane; k < n; k += 32) a.perm[off + k] = a.atoms[b + k];
}

__global__ void __launch_bounds__(256) k_sort_gather(float4 *dst, const float4 *src, const int32_t *perm, int N)
{
    count_launch();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) dst[i] = src[perm[i]];
}

struct SortLayout {
    size_t keys, tsum, tmp, total;
    int nkeys, ntiles;
};

// 0 keys: the grid is too large to sort.
static SortLayout sort_layout(const md_nbr *nb)
{
    SortLayout L;
    memset(&L, 0, sizeof(L));
    int P = 1;
    for (int k = 0; k < nb->dim; ++k) {
        const int p = next_pow2(nb->ncell[k]);
        P = p > P ? p : P;
    }
    long long nkeys = 1;
    for (int k = 0; k < nb->dim; ++k) nkeys *= P;
    if (nkeys > SORT_MAX_KEYS) return L;
    L.nkeys = (int)nkeys;
    L.ntiles = (L.nkeys + SCAN_TILE - 1) / SCAN_TILE;
    size_t o = 0;
    L.keys = o;
    o = align256(o + sizeof(uint32_t) * (size_t)L.nkeys);
    L.tsum = o;
    o = align256(o + sizeof(uint32_t) * (size_t)L.ntiles);
    L.tmp = o;
    o = align256(o + sizeof(float4) * (size_t)nb->N);
    L.total = o;
    return L;
}

}  // namespace jmd

using namespace jmd;

extern "C" size_t md_sort_scratch_bytes(const md_nbr *nb)
{
    if (!nb || nb->N < 1 || (nb->dim != 2 && nb->dim != 3)) return 0;
    return sort_layout(nb).total;
}

extern "C" md_status md_sort_particles(const md_space *s, md_nbr *nb, float *d_r, float *d_v, int32_t *d_perm,
                                       void *d_scratch, size_t scratch_bytes, uint32_t *d_status, md_stream_t stream)
{
    if (!s || !nb || !d_r || !d_perm || !d_scratch || s->dim != nb->dim) return MD_ERR_INVALID;
    if (!nb->nbr || !nb->cnt || !nb->rref || !nb->ws || nb->N < 1 || !nbr_layout_ok(nb)) return MD_ERR_INVALID;
    if ((uintptr_t)d_scratch & 255u) return MD_ERR_INVALID;
    const SortLayout L = sort_layout(nb);
    if (L.nkeys == 0 || scratch_bytes < L.total) return MD_ERR_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    char *sb = (char *)d_scratch;
    const int N = nb->N;
    NbrArgs na = make_nbr_args(s, d_r, nb, d_status, 0);
    WsPtrs w = ws_ptrs(nb);
    enqueue_cell_binning(na, nb->ncell_total, st);

    SortArgs a;
    memset(&a, 0, sizeof(a));
    a.N = N;
    a.ncell = nb->ncell_total;
    a.dim = nb->dim;
    a.nkeys = L.nkeys;
    a.ntiles = L.ntiles;
    for (int k = 0; k < 3; ++k) a.nc[k] = nb->ncell[k];
    a.cell_start = w.cell_start;
    a.atoms = w.atoms;
    a.keys = (uint32_t *)(sb + L.keys);
    a.tsum = (uint32_t *)(sb + L.tsum);
    a.perm = d_perm;
    JMD_CUDA_TRY(cudaMemsetAsync(a.keys, 0, sizeof(uint32_t) * (size_t)L.nkeys, st));
    k_sort_counts<<<(a.ncell + 255) / 256, 256, 0, st>>>(a);
    k_sort_scan_tiles<<<L.ntiles, 1024, 0, st>>>(a.keys, L.nkeys, a.tsum);
    k_sort_scan_totals<<<1, 1024, 0, st>>>(a.tsum, L.ntiles);
    k_sort_scan_add<<<L.ntiles, 1024, 0, st>>>(a.keys, L.nkeys, a.tsum);
    k_sort_perm<<<(a.ncell + 7) / 8, 256, 0, st>>>(a);
    float4 *tmp = (float4 *)(sb + L.tmp);
    const int g = (N + 255) / 256;
    k_sort_gather<<<g, 256, 0, st>>>(tmp, (const float4 *)d_r, d_perm, N);
    JMD_CUDA_TRY(cudaMemcpyAsync(d_r, tmp, sizeof(float4) * (size_t)N, cudaMemcpyDeviceToDevice, st));
    if (d_v) {
        k_sort_gather<<<g, 256, 0, st>>>(tmp, (const float4 *)d_v, d_perm, N);
        JMD_CUDA_TRY(cudaMemcpyAsync(d_v, tmp, sizeof(float4) * (size_t)N, cudaMemcpyDeviceToDevice, st));
    }
    JMD_CUDA_TRY(cudaGetLastError());
    // the list of the new order
    return md_neighbor_list_build(s, d_r, nb, d_status, stream);
}
