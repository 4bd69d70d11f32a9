// pair.cu -- pair energies and forces over the neighbor list (Sec. 3.2.2,
// 3.3.2): U = 1/2 sum_{i != j} u(r_ij), F_i = -sum_j u'(r_ij) d_ij / r_ij.
//
// Gather form: a group of TPP threads owns particle i, strides over its
// sorted row, gathers float4 neighbor positions and reduces F_i and e_i with
// shuffles.  Every pair is visited from both sides (full list, no Newton's
// third law), so no atomics are needed and the result is deterministic.
//
// Fused variant (KICK): after F_i is known the group leader applies the
// closing half-kick v += dt/2 F/m of velocity Verlet and the block emits
// FP64 partial sums of potential and kinetic energy; the last block to
// finish (ticket) adds the partials in a fixed order.
#include "cells.cuh"
#include "common.cuh"
#include "kernels.cuh"
#include "reduce.cuh"

namespace jmd {

// One neighbor pair: accumulates F_i and the pair energy into the lane's sums.
// (The comparison-based nearest image, which pays off in the issue-bound
// neighbor build, measured slower here, where the gathers bound the time.)
template <int DIM, int POT>
__device__ __forceinline__ void pair_term(const PairArgs &a, const float4 &ri, const float4 &rj, float &fx, float &fy,
                                          float &fz, float &e)
{
    float dx, dy, dz;
    float r2 = dist2_rn<DIM>(ri, rj, a.box, dx, dy, dz);
    // branch-free: the cutoff decision selects the force factor and the
    // energy (a pair outside adds exactly zero), so divergent warps run no
    // extra branch per pair
    if (POT == MD_LJ) {
        const bool in = r2 < a.rc2;
        const float ir2 = __fdividef(1.0f, in ? r2 : 1.0f);
        const float s2 = a.sigma2 * ir2;
        const float s6 = s2 * s2 * s2;
        const float fr = in ? a.c24eps * ir2 * s6 * (2.0f * s6 - 1.0f) : 0.0f;
        fx += fr * dx;
        fy += fr * dy;
        fz += fr * dz;
        e += in ? a.c4eps * s6 * (s6 - 1.0f) - a.e_shift : 0.0f;
    } else {  // soft sphere, s_ij = (w_i + w_j)/2
        const float sg = 0.5f * (ri.w + rj.w);
        const bool in = r2 < sg * sg;
        const float rr = sqrtf(in ? r2 : 1.0f);
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
        // F_i += (eps/s) x^(alpha-1) d / r
        const float fr = in ? a.eps * isg * xa1 * __fdividef(1.0f, rr) : 0.0f;
        fx += fr * dx;
        fy += fr * dy;
        fz += fr * dz;
        e += in ? a.eps * ua : 0.0f;
    }
}

// Bounds-checked entry (CHECK): an index outside [0, N) is reported and
// replaced by i, and its pair is skipped, so a corrupted row never reads
// outside the positions.
__device__ __forceinline__ void check_entry(const PairArgs &a, int i, int &j, bool &ok)
{
    if (ok && (unsigned)j >= (unsigned)a.N) {
        raise_status(a.status, MD_ERR_BOUNDS);
        j = i;
        ok = false;
    }
}

// The lanes of a group take consecutive entries of the row, so one gather
// instruction touches few cache lines; four entries per lane per trip keep
// four gathers in flight; row entries bypass L1.
template <int DIM, int TPP, int POT, bool STREAM, bool CHECK>
__device__ __forceinline__ void pair_loop(const PairArgs &a, const float4 *rp, int i, int n, const int32_t *row,
                                          const float4 &ri, int lg, float &fx, float &fy, float &fz, float &e)
{
    for (int k0 = lg; k0 < n; k0 += 4 * TPP) {
        const int k1 = k0 + TPP, k2 = k0 + 2 * TPP, k3 = k0 + 3 * TPP;
        int j0 = STREAM ? ld_stream(row + k0) : __ldg(row + k0);
        int j1 = k1 < n ? (STREAM ? ld_stream(row + k1) : __ldg(row + k1)) : i;
        int j2 = k2 < n ? (STREAM ? ld_stream(row + k2) : __ldg(row + k2)) : i;
        int j3 = k3 < n ? (STREAM ? ld_stream(row + k3) : __ldg(row + k3)) : i;
        bool ok0 = true, ok1 = k1 < n, ok2 = k2 < n, ok3 = k3 < n;
        if (CHECK) {
            check_entry(a, i, j0, ok0);
            check_entry(a, i, j1, ok1);
            check_entry(a, i, j2, ok2);
            check_entry(a, i, j3, ok3);
        }
        float4 r0 = __ldg(rp + j0);
        float4 r1 = __ldg(rp + j1);
        float4 r2 = __ldg(rp + j2);
        float4 r3 = __ldg(rp + j3);
        if (ok0) pair_term<DIM, POT>(a, ri, r0, fx, fy, fz, e);
        if (ok1) pair_term<DIM, POT>(a, ri, r1, fx, fy, fz, e);
        if (ok2) pair_term<DIM, POT>(a, ri, r2, fx, fy, fz, e);
        if (ok3) pair_term<DIM, POT>(a, ri, r3, fx, fy, fz, e);
    }
}

// Fused NVE step (KICK == 2), lane 0 of particle i's group: the closing
// half-kick of this step (kinetic energy at v(t)), then, unless this is the
// loop's last step, the next step's kick-drift into the other position
// buffer and its displacement check.  The arithmetic repeats half_kick and
// k_kick_drift expression by expression, so the trajectory has the same bits
// as the unfused step.  Returns the kinetic energy; *moved reports the check.
template <int DIM>
__device__ __forceinline__ float kick_kick_drift(const PairArgs &a, int i, float4 ri, float fx, float fy, float fz,
                                                 bool more, float4 *rn, bool *moved)
{
    float4 vi = a.v[i];
    const float4 rr = more ? a.rref[i] : ri;
    vi.x += a.half_dt_over_m * fx;
    vi.y += a.half_dt_over_m * fy;
    if (DIM == 3) vi.z += a.half_dt_over_m * fz;
    const float ke = 0.5f * a.mass * (vi.x * vi.x + vi.y * vi.y + vi.z * vi.z);
    *moved = false;
    if (more) {
        vi.x += a.half_dt_over_m * fx;
        vi.y += a.half_dt_over_m * fy;
        ri.x = wrap_coord(ri.x + a.dt * vi.x, a.box.L[0], a.box.Linv[0]);
        ri.y = wrap_coord(ri.y + a.dt * vi.y, a.box.L[1], a.box.Linv[1]);
        if (DIM == 3) {
            vi.z += a.half_dt_over_m * fz;
            ri.z = wrap_coord(ri.z + a.dt * vi.z, a.box.L[2], a.box.Linv[2]);
        }
        rn[i] = ri;
        float dx, dy, dz;
        *moved = dist2_rn<DIM>(ri, rr, a.box, dx, dy, dz) > a.half_skin2;
    }
    a.v[i] = vi;
    return ke;
}

// Grid-stride over groups of PPB = 256/TPP particles.  Energies accumulate per thread in FP32 over the particles it
// owns, per warp in FP32, across the block's 8 warps in FP64, and across
// blocks in FP64 (fixed order, last block).  KICK: 0 forces only, 1 forces
// and the closing half-kick, 2 the fused step (kick_kick_drift).
template <int DIM, int TPP, int POT, int KICK, int OPT>
__global__ void __launch_bounds__(256) k_pair(PairArgs a)
{
    count_launch();
    constexpr int PPB = 256 / TPP;
    const int lg = threadIdx.x & (TPP - 1);
    const int gl = threadIdx.x / TPP;
    // fused step: this step's positions and the buffer of the next
    const float4 *rc = a.r;
    float4 *rn = nullptr;
    bool more = false;
    if (KICK == 2) {
        const uint32_t step = *(volatile uint32_t *)&a.ctl[CTL_STEP];
        rc = (step & 1u) ? a.r_alt : a.r;
        rn = (step & 1u) ? const_cast<float4 *>(a.r) : a.r_alt;
        more = step + 1u < *(volatile uint32_t *)&a.ctl[CTL_NSTEPS];
    }
    float pe_acc = 0.0f, ke_acc = 0.0f;
    bool moved_any = false;
    for (int base = blockIdx.x * PPB; base < a.N; base += gridDim.x * PPB) {
        int i = base + gl;
        bool valid = i < a.N;
        float fx = 0.f, fy = 0.f, fz = 0.f, e = 0.f;
        float4 ri = make_float4(0.f, 0.f, 0.f, 0.f);
        if (valid) {
            ri = __ldg(rc + i);
            int n = __ldg(a.cnt + i);
            n = n < a.cap ? n : a.cap;
            const int32_t *row = a.nbr + (size_t)i * a.cap;
            pair_loop<DIM, TPP, POT, (OPT & 1) != 0, (OPT & 2) != 0>(a, rc, i, n, row, ri, lg, fx, fy, fz, e);
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
            a.f[i] = make_float4(fx, fy, fz, ei);
            pe_acc += ei;
            if (KICK == 1) ke_acc += half_kick<DIM>(a, i, fx, fy, fz);
            if (KICK == 2) {
                bool mv;
                ke_acc += kick_kick_drift<DIM>(a, i, ri, fx, fy, fz, more, rn, &mv);
                moved_any = moved_any || mv;
            }
        }
    }
    if (KICK == 2 && __any_sync(0xffffffffu, moved_any) && (threadIdx.x & 31) == 0) {
        a.ctl[CTL_REBUILD] = 1u;
        __threadfence();
    }
    if (!a.E_out && !KICK) return;
    energy_epilogue(pe_acc, ke_acc, a);
}

// ---------------------------------------------------------------------------
// Block-centred pair forces (lists with local rows).  One CTA per block of
// 2 x 2 x 2 cells (cells.cuh), grid-stride over the blocks: the positions of
// the block's region (the block grown by one cell, ~64 cells) are gathered
// once into shared memory in the order the build indexed them; then each
// particle's group of TPP lanes reads its 16-bit local row and takes the
// partners from shared memory.  Entries, their order and the arithmetic are
// those of k_pair, so the forces are the same bits.  A block whose region is
// too large to stage, or one of whose cells had a dense stencil (the build
// wrote no local rows there), uses the int32 rows.
// ---------------------------------------------------------------------------
constexpr int PB_THREADS = 256;

template <int DIM, int TPP, int POT>
__device__ __forceinline__ void pair_loop_local(const PairArgs &a, int n, const uint16_t *row, const float4 *cand,
                                                const float4 &ri, int lg, float &fx, float &fy, float &fz, float &e)
{
    for (int k0 = lg; k0 < n; k0 += 4 * TPP) {
        const int k1 = k0 + TPP, k2 = k0 + 2 * TPP, k3 = k0 + 3 * TPP;
        const int j0 = ld_stream_u16(row + k0);
        const int j1 = k1 < n ? ld_stream_u16(row + k1) : 0;
        const int j2 = k2 < n ? ld_stream_u16(row + k2) : 0;
        const int j3 = k3 < n ? ld_stream_u16(row + k3) : 0;
        const float4 r0 = cand[j0], r1 = cand[j1], r2 = cand[j2], r3 = cand[j3];
        pair_term<DIM, POT>(a, ri, r0, fx, fy, fz, e);
        if (k1 < n) pair_term<DIM, POT>(a, ri, r1, fx, fy, fz, e);
        if (k2 < n) pair_term<DIM, POT>(a, ri, r2, fx, fy, fz, e);
        if (k3 < n) pair_term<DIM, POT>(a, ri, r3, fx, fy, fz, e);
    }
}

template <int DIM, int TPP, int POT, int KICK>
__global__ void __launch_bounds__(PB_THREADS) k_pair_block(PairArgs a)
{
    count_launch();
    constexpr int PPP = PB_THREADS / TPP;   // particles per pass
    __shared__ float4 cand[REGION_CMAX];
    __shared__ RegionInfo reg;
    __shared__ int wsum[1];
    __shared__ int own_ri[8], own_off[9], n_own, local_ok;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int lg = tid & (TPP - 1), gl = tid / TPP;
    const float4 *rc = a.r;
    float4 *rn = nullptr;
    bool more = false;
    if (KICK == 2) {
        const uint32_t step = *(volatile uint32_t *)&a.ctl[CTL_STEP];
        rc = (step & 1u) ? a.r_alt : a.r;
        rn = (step & 1u) ? const_cast<float4 *>(a.r) : a.r_alt;
        more = step + 1u < *(volatile uint32_t *)&a.ctl[CTL_NSTEPS];
    }
    const int nbx = blocks_along(a.nc[0]), nby = blocks_along(a.nc[1]);
    const int nbz = DIM == 3 ? blocks_along(a.nc[2]) : 1;
    const int nblk = nbx * nby * nbz;
    float pe_acc = 0.0f, ke_acc = 0.0f;
    bool moved_any = false;
    for (int blk = blockIdx.x; blk < nblk; blk += gridDim.x) {
        const int bx = blk % nbx, by = (blk / nbx) % nby, bz = blk / (nbx * nby);
        region_locate<DIM>(a.nc, a.cell_start, bx, by, bz, reg, wsum);
        if (tid == 0) {
            // own cells are the region's interior; local rows are usable when
            // the region fits and every own cell's stencil was staged
            const int ox = reg.ex - 2, oy = reg.ey - 2, oz = DIM == 3 ? reg.ez - 2 : 1;
            bool ok = reg.roff[reg.nreg] <= REGION_CMAX;
            int k = 0, acc = 0;
            for (int z = 0; z < oz; ++z)
                for (int y = 0; y < oy; ++y)
                    for (int x = 0; x < ox; ++x) {
                        const int zr = DIM == 3 ? z + 1 : 0;
                        const int ri = (zr * reg.ey + (y + 1)) * reg.ex + (x + 1);
                        own_ri[k] = ri;
                        own_off[k] = acc;
                        acc += reg.roff[ri + 1] - reg.roff[ri];
                        int m = 0;
                        for (int dz = (DIM == 3 ? -1 : 0); dz <= (DIM == 3 ? 1 : 0); ++dz)
                            for (int dy = -1; dy <= 1; ++dy) {
                                const int rr = ((zr + dz) * reg.ey + (y + 1 + dy)) * reg.ex + x;   // x-1 .. x+1
                                m += reg.roff[rr + 3] - reg.roff[rr];
                            }
                        ok = ok && m <= STAGE_CMAX;
                        ++k;
                    }
            own_off[k] = acc;
            n_own = k;
            local_ok = ok ? 1 : 0;
        }
        __syncthreads();
        const bool loc = local_ok != 0;
        if (loc) {
            for (int c = warp; c < reg.nreg; c += PB_THREADS / 32) {
                const int b0 = reg.roff[c], nm = reg.roff[c + 1] - b0;
                const int32_t *src = a.atoms + reg.rbeg[c];
                for (int t = lane; t < nm; t += 32) cand[b0 + t] = __ldg(rc + __ldg(src + t));
            }
        }
        __syncthreads();
        const int nown = own_off[n_own];
        for (int p0 = 0; p0 < nown; p0 += PPP) {
            const int p = p0 + gl;
            const bool valid = p < nown;
            float fx = 0.f, fy = 0.f, fz = 0.f, e = 0.f;
            float4 ri = make_float4(0.f, 0.f, 0.f, 0.f);
            int i = 0;
            if (valid) {
                int c = 0;
                while (own_off[c + 1] <= p) ++c;
                const int t = p - own_off[c], rcix = own_ri[c];
                i = __ldg(a.atoms + reg.rbeg[rcix] + t);
                int n = __ldg(a.cnt + i);
                n = n < a.cap ? n : a.cap;
                if (loc) {
                    ri = cand[reg.roff[rcix] + t];
                    pair_loop_local<DIM, TPP, POT>(a, n, a.lrow + (size_t)i * a.cap, cand, ri, lg, fx, fy, fz, e);
                } else {
                    ri = __ldg(rc + i);
                    pair_loop<DIM, TPP, POT, true, false>(a, rc, i, n, a.nbr + (size_t)i * a.cap, ri, lg, fx, fy, fz,
                                                          e);
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
                const float ei = 0.5f * e;
                a.f[i] = make_float4(fx, fy, fz, ei);
                pe_acc += ei;
                if (KICK == 1) ke_acc += half_kick<DIM>(a, i, fx, fy, fz);
                if (KICK == 2) {
                    bool mv;
                    ke_acc += kick_kick_drift<DIM>(a, i, ri, fx, fy, fz, more, rn, &mv);
                    moved_any = moved_any || mv;
                }
            }
        }
        __syncthreads();   // the next block reuses cand, reg and the own lists
    }
    if (KICK == 2 && __any_sync(0xffffffffu, moved_any) && lane == 0) {
        a.ctl[CTL_REBUILD] = 1u;
        __threadfence();
    }
    if (!a.E_out && !KICK) return;
    energy_epilogue(pe_acc, ke_acc, a);
}

template <int DIM, int TPP, int POT, int KICK>
static int pair_block_grid(const PairArgs &a)
{
    static int per_sm = 0, sms = 0;
    if (!per_sm) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pair_block<DIM, TPP, POT, KICK>, PB_THREADS, 0);
        if (per_sm < 1) per_sm = 1;
        if (sms < 1) sms = 1;
    }
    const int nblk = blocks_along(a.nc[0]) * blocks_along(a.nc[1]) * (DIM == 3 ? blocks_along(a.nc[2]) : 1);
    int g = per_sm * sms;
    g = nblk < g ? nblk : g;
    return g < a.max_blocks ? g : a.max_blocks;
}

template <int DIM, int POT, int KICK>
static void launch_pair_block(const PairArgs &a, cudaStream_t st)
{
    switch (a.tpp) {
    case 4: k_pair_block<DIM, 4, POT, KICK><<<pair_block_grid<DIM, 4, POT, KICK>(a), PB_THREADS, 0, st>>>(a); break;
    case 16: k_pair_block<DIM, 16, POT, KICK><<<pair_block_grid<DIM, 16, POT, KICK>(a), PB_THREADS, 0, st>>>(a); break;
    case 32: k_pair_block<DIM, 32, POT, KICK><<<pair_block_grid<DIM, 32, POT, KICK>(a), PB_THREADS, 0, st>>>(a); break;
    default: k_pair_block<DIM, 8, POT, KICK><<<pair_block_grid<DIM, 8, POT, KICK>(a), PB_THREADS, 0, st>>>(a); break;
    }
}

// Blocks per launch: enough resident blocks to fill every SM (grid-stride
// loop inside), never more than there are particle groups.
template <int DIM, int TPP, int POT, int KICK, int OPT>
static int pair_grid(int N)
{
    static int per_sm = 0, sms = 0;
    if (!per_sm) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pair<DIM, TPP, POT, KICK, OPT>, 256, 0);
        if (per_sm < 1) per_sm = 1;
        if (sms < 1) sms = 1;
    }
    int groups = (int)(((long long)N * TPP + 255) / 256);
    int g = per_sm * sms;
    return groups < g ? groups : g;
}

static int g_pair_opt = 1;   // bit 0: stream rows past L1; bit 1: bounds-check row entries

template <int DIM, int TPP, int POT, int KICK>
static void launch_pair_t(const PairArgs &a, cudaStream_t st)
{
    switch (a.opt & 3) {
    case 1: k_pair<DIM, TPP, POT, KICK, 1><<<pair_grid<DIM, TPP, POT, KICK, 1>(a.N), 256, 0, st>>>(a); break;
    case 2: k_pair<DIM, TPP, POT, KICK, 2><<<pair_grid<DIM, TPP, POT, KICK, 2>(a.N), 256, 0, st>>>(a); break;
    case 3: k_pair<DIM, TPP, POT, KICK, 3><<<pair_grid<DIM, TPP, POT, KICK, 3>(a.N), 256, 0, st>>>(a); break;
    default: k_pair<DIM, TPP, POT, KICK, 0><<<pair_grid<DIM, TPP, POT, KICK, 0>(a.N), 256, 0, st>>>(a); break;
    }
}

template <int DIM, int POT, int KICK>
static void launch_pair_tpp(const PairArgs &a, cudaStream_t st)
{
    switch (a.tpp) {
    case 1: launch_pair_t<DIM, 1, POT, KICK>(a, st); break;
    case 4: launch_pair_t<DIM, 4, POT, KICK>(a, st); break;
    case 16: launch_pair_t<DIM, 16, POT, KICK>(a, st); break;
    case 32: launch_pair_t<DIM, 32, POT, KICK>(a, st); break;
    default: launch_pair_t<DIM, 8, POT, KICK>(a, st); break;
    }
}

template <int DIM, int POT>
static void launch_pair_kick(const PairArgs &a, int kick, bool blockk, cudaStream_t st)
{
    if (blockk) {
        if (kick == 2) launch_pair_block<DIM, POT, 2>(a, st);
        else if (kick == 1) launch_pair_block<DIM, POT, 1>(a, st);
        else launch_pair_block<DIM, POT, 0>(a, st);
    } else {
        if (kick == 2) launch_pair_tpp<DIM, POT, 2>(a, st);
        else if (kick == 1) launch_pair_tpp<DIM, POT, 1>(a, st);
        else launch_pair_tpp<DIM, POT, 0>(a, st);
    }
}

// kick: 0 forces only, 1 forces + closing half-kick, 2 the fused NVE step.
// Lists with local rows on grids of >= 4 cells per axis take the
// block-centred kernel, all others the gather kernel over int32 rows.
void enqueue_pair(const PairArgs &a, int dim, int pot, int kick, cudaStream_t st)
{
    const bool blockk = a.lrow != nullptr && region_grid_ok(a.nc, dim);
    if (dim == 3) {
        if (pot == MD_LJ) launch_pair_kick<3, MD_LJ>(a, kick, blockk, st);
        else launch_pair_kick<3, MD_SOFT_SPHERE>(a, kick, blockk, st);
    } else {
        if (pot == MD_LJ) launch_pair_kick<2, MD_LJ>(a, kick, blockk, st);
        else launch_pair_kick<2, MD_SOFT_SPHERE>(a, kick, blockk, st);
    }
}

int pair_blocks(int N, int tpp) { return (int)(((long long)N * tpp + 255) / 256); }

void enqueue_forces(const PairArgs &a, int dim, int pot, int kick, cudaStream_t st)
{
    if (pot == MD_SW) enqueue_sw(a, kick, st);
    else if (pot == MD_BP) enqueue_bp_step(a, kick, st);
    else if (pot == MD_GNN) enqueue_gnn_step(a, kick, st);
    else enqueue_pair(a, dim, pot, kick, st);
}

static int g_tpp = 4;

bool make_pair_args(const md_space *s, const md_pot *p, const float *d_r, const md_nbr *nb, float *d_f, PairArgs &a)
{
    if (!s || !p || !d_r || !nb || !d_f || !nb->nbr || !nb->cnt || !nb->ws || !nbr_layout_ok(nb)) return false;
    if (p->kind != MD_LJ && p->kind != MD_SOFT_SPHERE && p->kind != MD_SW && p->kind != MD_BP && p->kind != MD_GNN)
        return false;
    if ((p->kind == MD_SW || p->kind == MD_BP || p->kind == MD_GNN) && s->dim != 3) return false;
    memset(&a, 0, sizeof(a));
    a.box = make_box(s);
    a.N = nb->N;
    a.cap = nb->cap;
    a.r = (const float4 *)d_r;
    a.nbr = nb->nbr;
    a.cnt = nb->cnt;
    a.f = (float4 *)d_f;
    WsPtrs w = ws_ptrs(nb);
    a.ctl = w.ctl;
    a.partials = w.partials;
    // canonical lists: one thread sums a particle's pairs in row order
    a.tpp = (nb->flags & MD_NBR_CANONICAL) ? 1 : g_tpp;
    a.opt = g_pair_opt;
    a.lrow = w.lrow;
    a.atoms = w.atoms;
    a.cell_start = w.cell_start;
    for (int k = 0; k < 3; ++k) a.nc[k] = nb->ncell[k];
    a.ncell = nb->ncell_total;
    a.max_blocks = w.max_blocks;
    a.variant = bp_variant() | (gnn_variant() << 1);
    if (p->kind == MD_LJ) {
        if (p->r_cut > nb->r_list) return false;
        float rc = p->r_cut;
        a.rc2 = rc * rc;
        a.sigma2 = p->sigma * p->sigma;
        a.c24eps = 24.0f * p->eps;
        a.c4eps = 4.0f * p->eps;
        a.e_shift = p->e_shift;
    } else if (p->kind == MD_SOFT_SPHERE) {
        a.eps = p->eps;
        a.alpha = p->alpha;
    } else if (p->kind == MD_GNN) {
        const md_gnn_model *m = (const md_gnn_model *)p->model;
        if (!gnn_model_ok(m, nb) || (size_t)nb->N * nb->cap >= (size_t)INT32_MAX) return false;
        a.gnn = *m;
    } else if (p->kind == MD_BP) {
        const md_bp_model *m = (const md_bp_model *)p->model;
        if (!m || !m->params || !m->norm || !m->G || !m->dEdG || !m->Ei) return false;
        if (nb->r_list < 3.77f) return false;
        a.bp_params = m->params;
        a.bp_norm = m->norm;
        a.bp_G = m->G;
        a.bp_dEdG = m->dEdG;
        a.bp_Ei = m->Ei;
        a.bp_sys_n = m->sys_n;
        if (m->lists) {   // partner-list scratch of md_bp_lists_bytes(N) bytes
            unsigned char *b = (unsigned char *)m->lists;
            if (((uintptr_t)b & 255u) != 0u) return false;
            const TbLayout t = tb_layout(nb->N, BP_LIST_SLOTS, false);
            a.tb_cnt = (int32_t *)(b + t.cnt);
            a.tb_idx = (int32_t *)(b + t.idx);
            a.tb_vec = (float4 *)(b + t.vec);
        }
    } else {
        for (int k = 0; k < 10; ++k) a.sw[k] = p->sw[k];
        float rc = p->sw[2] * p->sw[1];   // a * sigma
        if (rc > nb->r_list) return false;
        a.sw[10] = rc;
        a.sw[11] = rc * rc;
        if (p->model) {   // partner-list scratch of md_sw_lists_bytes(N) bytes
            unsigned char *b = (unsigned char *)p->model;
            if (((uintptr_t)b & 255u) != 0u || (size_t)nb->N * SW_LIST_SLOTS >= (size_t)INT32_MAX) return false;
            const TbLayout t = tb_layout(nb->N, SW_LIST_SLOTS, true);
            a.tb_cnt = (int32_t *)(b + t.cnt);
            a.tb_idx = (int32_t *)(b + t.idx);
            a.tb_vec = (float4 *)(b + t.vec);
            a.tb_aux = (float4 *)(b + t.aux);
            a.tb_f2 = (float4 *)(b + t.f2);
        }
    }
    return pair_blocks(a.N, a.tpp) <= w.max_blocks;
}

}  // namespace jmd

using namespace jmd;

extern "C" size_t md_sw_lists_bytes(int N) { return N > 0 ? sw_lists_bytes(N) : 0; }

extern "C" size_t md_bp_lists_bytes(int N) { return N > 0 ? tb_layout(N, BP_LIST_SLOTS, false).bytes : 0; }

extern "C" md_status md_set_pair_options(int opt)
{
    if (opt < 0 || opt > 3) return MD_ERR_INVALID;
    g_pair_opt = opt;
    return MD_OK;
}

extern "C" md_status md_set_pair_tpp(int tpp)
{
    if (tpp != 4 && tpp != 8 && tpp != 16 && tpp != 32) return MD_ERR_INVALID;
    g_tpp = tpp;
    return MD_OK;
}

extern "C" md_status md_energy_forces(const md_space *s, const md_pot *p, const float *d_r, const md_nbr *nb,
                                      float *d_f, double *d_E, uint32_t *d_status, md_stream_t stream)
{
    if (!p || !s || !nb) return MD_ERR_INVALID;
    if (s->dim != nb->dim) return MD_ERR_INVALID;
    PairArgs a;
    if (!make_pair_args(s, p, d_r, nb, d_f, a)) return MD_ERR_INVALID;
    a.E_out = d_E;
    a.status = d_status;
    enqueue_forces(a, s->dim, p->kind, 0, (cudaStream_t)stream);
    JMD_CUDA_TRY(cudaGetLastError());
    return MD_OK;
}
