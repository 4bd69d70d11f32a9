// reduce.cuh -- the energy epilogue shared by the force kernels.
//
// Each thread has accumulated FP32 partial potential / kinetic energies over
// the few particles it owns.  They are summed per warp in FP32, across the
// block's warps in FP64 (thread 0), and across blocks in FP64 by the last
// block to finish (atomic ticket, fixed summation order).  The last block
// also writes the per-step series entry, advances the device step counter,
// flags non-finite totals and, inside a graph WHILE loop, sets the loop
// condition.
#pragma once

#include "kernels.cuh"
#include "nhc.cuh"

namespace jmd {

__device__ __forceinline__ void energy_epilogue(float pe_acc, float ke_acc, const PairArgs &a)
{
    __shared__ double sh[2][32];
    __shared__ bool last;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        pe_acc += __shfl_xor_sync(0xffffffffu, pe_acc, o);
        ke_acc += __shfl_xor_sync(0xffffffffu, ke_acc, o);
    }
    const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        sh[0][w] = (double)pe_acc;
        sh[1][w] = (double)ke_acc;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double bpe = 0.0, bke = 0.0;
        for (int k = 0; k < nw; ++k) {
            bpe += sh[0][k];
            bke += sh[1][k];
        }
        a.partials[blockIdx.x] = make_double2(bpe, bke);
        __threadfence();
        unsigned t = atomicAdd(&a.ctl[CTL_TICKET], 1u);
        last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double S[2] = {0.0, 0.0};
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
        const volatile double *p = (const volatile double *)(a.partials + b);
        S[0] += p[0];
        S[1] += p[1];
    }
    block_sums_f64<2>(S, &sh[0][0], 32);
    const double spe = S[0], ske = S[1];
    if (threadIdx.x == 0) {
        a.ctl[CTL_TICKET] = 0u;
        if (!isfinite(spe) || !isfinite(ske)) raise_status(a.status, MD_ERR_NONFINITE);
        unsigned step = a.series ? a.ctl[CTL_STEP] : 0u;
        // Nose-Hoover chain: the totals go to the thermostat state, whose
        // half-steps k_nhc_update takes after this kernel
        if (a.nhc) {
            a.nhc[3 * a.nhc_M + NHC_KRAW] = ske;
            a.nhc[3 * a.nhc_M + NHC_PE] = spe;
        }
        if (a.E_out) a.E_out[step] = spe;
        if (a.KE_out) a.KE_out[step] = ske;
        if (a.series) a.ctl[CTL_STEP] = step + 1u;
        if (a.use_cond)
            cudaGraphSetConditional((cudaGraphConditionalHandle)a.cond_while,
                                    (step + 1u < a.ctl[CTL_NSTEPS]) ? 1u : 0u);
        // fused NVE step: every block has raised (and fenced) the rebuild
        // flag before its ticket, so the last block hands it to the IF node
        if (a.cond_if)
            cudaGraphSetConditional((cudaGraphConditionalHandle)a.cond_if,
                                    *(volatile uint32_t *)&a.ctl[CTL_REBUILD] ? 1u : 0u);
    }
}

// Closing half-kick of velocity Verlet for particle i; returns its kinetic
// energy 1/2 m v^2.
template <int DIM>
__device__ __forceinline__ float half_kick(const PairArgs &a, int i, float fx, float fy, float fz)
{
    float4 v = a.v[i];
    v.x += a.half_dt_over_m * fx;
    v.y += a.half_dt_over_m * fy;
    if (DIM == 3) v.z += a.half_dt_over_m * fz;
    a.v[i] = v;
    return 0.5f * a.mass * (v.x * v.x + v.y * v.y + v.z * v.z);
}

}  // namespace jmd
