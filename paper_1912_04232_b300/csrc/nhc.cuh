// nhc.cuh -- Nose-Hoover chain thermostat (Sec. 3.3.1; Martyna, Klein,
// Tuckerman 1992), device side.  The chain is a handful of scalars, updated
// by one thread (the last block of a force kernel, or k_nhc_begin) and
// applied to the particles as a velocity scale.
//
// State buffer (doubles, caller-owned, nhc_words(M) long):
//   [0, M)      xi_k     chain positions
//   [M, 2M)     w_k      chain velocities p_k / Q_k
//   [2M, 3M)    Q_k      masses: Q_1 = g kT tau^2, Q_k = kT tau^2
//   3M + 0      g kT
//   3M + 1      kT
//   3M + 2      dt
//   3M + 3      closing factor of the last half-step pair, still to apply
//   3M + 4      opening factor of the next step, still to apply
//   3M + 5      kinetic energy after the last closing half-step
//   3M + 6      kinetic energy of the last force kernel (before the half-step)
//   3M + 7      its potential energy
// The factors are applied as (v * closing) * opening, so a run continued
// across calls repeats the arithmetic of an uninterrupted one.
// Half-step: the sweep of Martyna, Tuckerman, Tobias, Klein (1996) with one
// sub-step, "forces" G_1 = (2K - g kT)/Q_1, G_k = (Q_{k-1} w_{k-1}^2 - kT)/Q_k.
#pragma once

namespace jmd {

constexpr int NHC_MAXM = 8;
__host__ __device__ constexpr int nhc_words(int M) { return 3 * M + 8; }
enum { NHC_GKT = 0, NHC_KT = 1, NHC_DT = 2, NHC_SCLOSE = 3, NHC_SOPEN = 4, NHC_K = 5, NHC_KRAW = 6, NHC_PE = 7 };

// iQ: the reciprocal masses (an FP64 division is a long dependent sequence;
// the chain needs six per half-step but only M distinct divisors)
__device__ __forceinline__ double nhc_force(const double *Q, const double *iQ, const double *w, int k, double K,
                                            double gkT, double kT)
{
    return k == 0 ? (2.0 * K - gkT) * iQ[0] : (Q[k - 1] * w[k - 1] * w[k - 1] - kT) * iQ[k];
}

// One thermostat half-step; K (kinetic energy) is rescaled in place and the
// particle velocity factor is returned.
__device__ __forceinline__ double nhc_half_step(double *st, int M, double &K)
{
    double *xi = st, *w = st + M;
    const double *Q = st + 2 * M, *c = st + 3 * M;
    const double gkT = c[NHC_GKT], kT = c[NHC_KT], dt = c[NHC_DT];
    const double q4 = 0.25 * dt, q8 = 0.125 * dt;
    double iQ[NHC_MAXM];
    for (int k = 0; k < M; ++k) iQ[k] = 1.0 / Q[k];
    w[M - 1] += q4 * nhc_force(Q, iQ, w, M - 1, K, gkT, kT);
    for (int k = M - 2; k >= 0; --k) {
        const double e = exp(-q8 * w[k + 1]);
        w[k] = (w[k] * e + q4 * nhc_force(Q, iQ, w, k, K, gkT, kT)) * e;
    }
    const double s = exp(-0.5 * dt * w[0]);
    K *= s * s;
    for (int k = 0; k < M; ++k) xi[k] += 0.5 * dt * w[k];
    for (int k = 0; k < M - 1; ++k) {
        const double e = exp(-q8 * w[k + 1]);
        w[k] = (w[k] * e + q4 * nhc_force(Q, iQ, w, k, K, gkT, kT)) * e;
    }
    w[M - 1] += q4 * nhc_force(Q, iQ, w, M - 1, K, gkT, kT);
    return s;
}

// Energy of the chain: sum_k Q_k w_k^2 / 2 + g kT xi_1 + kT sum_{k>1} xi_k.
__device__ __forceinline__ double nhc_energy(const double *st, int M)
{
    const double *xi = st, *w = st + M, *Q = st + 2 * M, *c = st + 3 * M;
    double e = c[NHC_GKT] * xi[0];
    for (int k = 0; k < M; ++k) e += 0.5 * Q[k] * w[k] * w[k];
    for (int k = 1; k < M; ++k) e += c[NHC_KT] * xi[k];
    return e;
}

}  // namespace jmd
