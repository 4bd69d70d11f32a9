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

#include <type_traits>

namespace jmd {

constexpr int NHC_MAXM = 8;
__host__ __device__ constexpr int nhc_words(int M) { return 3 * M + 8; }
enum { NHC_GKT = 0, NHC_KT = 1, NHC_DT = 2, NHC_SCLOSE = 3, NHC_SOPEN = 4, NHC_K = 5, NHC_KRAW = 6, NHC_PE = 7 };

// e^x for the chain's factors.  Their arguments are -dt w_k / 8 or
// -dt w_1 / 2, small at any sensible dt; for |x| <= 1/64 the Taylor
// polynomial of degree 6 (Horner form, FMAs) is used: its truncation error,
// below |x|^7/7! e^|x| < 5e-17, is under half an ulp of the result, so it
// agrees with a correctly rounded e^x to within rounding of the six FMAs.
// Larger arguments take exp().  On B300 every FP64 operation of this
// one-thread chain is a long dependent latency: six FMAs instead of the
// library routine's longer sequence.
__device__ __forceinline__ double nhc_exp(double x)
{
    if (fabs(x) > 0.015625) return exp(x);
    double p = 1.0 / 720.0;
    p = fma(p, x, 1.0 / 120.0);
    p = fma(p, x, 1.0 / 24.0);
    p = fma(p, x, 1.0 / 6.0);
    p = fma(p, x, 0.5);
    p = fma(p, x, 1.0);
    return fma(p, x, 1.0);
}

// One thermostat half-step of a chain of M (a compile-time length, so the
// chain lives in registers and the sweep's independent exponentials overlap);
// iQ holds the reciprocal masses 1/Q_k.  K (kinetic energy) is rescaled in
// place and the particle velocity factor is returned.
template <int M>
__device__ __forceinline__ double nhc_half_step_m(double *xi, double *w, const double *Q, const double *iQ, double gkT,
                                                  double kT, double dt, double &K)
{
    const double q4 = 0.25 * dt, q8 = 0.125 * dt;
    auto force = [&](int k) {
        return k == 0 ? (2.0 * K - gkT) * iQ[0] : (Q[k - 1] * w[k - 1] * w[k - 1] - kT) * iQ[k];
    };
    w[M - 1] += q4 * force(M - 1);
#pragma unroll
    for (int k = M - 2; k >= 0; --k) {
        const double e = nhc_exp(-q8 * w[k + 1]);
        w[k] = (w[k] * e + q4 * force(k)) * e;
    }
    const double s = nhc_exp(-0.5 * dt * w[0]);
    K *= s * s;
#pragma unroll
    for (int k = 0; k < M; ++k) xi[k] += 0.5 * dt * w[k];
    double e2[M > 1 ? M - 1 : 1];   // w_2 .. w_M do not change before their use below
#pragma unroll
    for (int k = 0; k < M - 1; ++k) e2[k] = nhc_exp(-q8 * w[k + 1]);
#pragma unroll
    for (int k = 0; k < M - 1; ++k) w[k] = (w[k] * e2[k] + q4 * force(k)) * e2[k];
    w[M - 1] += q4 * force(M - 1);
    return s;
}

// The chain state of st in registers for nhc_half_step_m: F(xi, w, Q, iQ)
// runs between the load and the store back.
template <int M, class F>
__device__ __forceinline__ void nhc_with_state(double *st, F &&f)
{
    double xi[M], w[M], Q[M], iQ[M];
#pragma unroll
    for (int k = 0; k < M; ++k) {
        xi[k] = st[k];
        w[k] = st[M + k];
        Q[k] = st[2 * M + k];
    }
#pragma unroll
    for (int k = 0; k < M; ++k) iQ[k] = 1.0 / Q[k];   // independent divisions
    f(xi, w, Q, iQ);
#pragma unroll
    for (int k = 0; k < M; ++k) {
        st[k] = xi[k];
        st[M + k] = w[k];
    }
}

// Runs F<m>() for the runtime chain length M in [1, NHC_MAXM].
template <class F>
__device__ __forceinline__ void nhc_dispatch(int M, F &&f)
{
    switch (M) {
    case 1: f(std::integral_constant<int, 1>()); break;
    case 2: f(std::integral_constant<int, 2>()); break;
    case 3: f(std::integral_constant<int, 3>()); break;
    case 4: f(std::integral_constant<int, 4>()); break;
    case 5: f(std::integral_constant<int, 5>()); break;
    case 6: f(std::integral_constant<int, 6>()); break;
    case 7: f(std::integral_constant<int, 7>()); break;
    default: f(std::integral_constant<int, 8>()); break;
    }
}

// One thermostat half-step on the state buffer (K rescaled in place; the
// velocity factor is returned).
__device__ __forceinline__ double nhc_half_step(double *st, int M, double &K)
{
    const double *c = st + 3 * M;
    const double gkT = c[NHC_GKT], kT = c[NHC_KT], dt = c[NHC_DT];
    double s = 1.0;
    nhc_dispatch(M, [&](auto m) {
        constexpr int MM = decltype(m)::value;
        nhc_with_state<MM>(st, [&](double *xi, double *w, const double *Q, const double *iQ) {
            s = nhc_half_step_m<MM>(xi, w, Q, iQ, gkT, kT, dt, K);
        });
    });
    return s;
}

}  // namespace jmd
