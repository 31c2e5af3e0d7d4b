// kzk_weno.cuh -- WENO5 flux derivative along tau (Sec. 3.3, Eq. 7) and its
// transpose.
//
// Flux of the homogeneous medium: f(u) = -B(sigma) u^2 / 2, split globally
// (Lax-Friedrichs) into f+- = (f +- alpha u)/2 with alpha = B(sigma) * M.
// At interface k+1/2 the upwind part F+ is the Jiang-Shu WENO5 reconstruction
// from f+ at k-2..k+2, the downwind part F- the mirrored one from f- at
// k+3..k-1; the nonlinear term is b_k = -(F_{k+1/2} - F_{k-1/2}) / dtau.
// Jiang-Shu weights omega_r = a_r / sum a, a_r = d_r / (eps + beta_r)^2,
// d = (1/10, 6/10, 3/10); the quotient is formed with one division by
// multiplying numerator and denominator by the three (eps + beta)^2.
#pragma once
#include "kzk_common.cuh"

namespace kzk {

template <typename T>
struct WenoCoef {
    T B;         // B(sigma)
    T alpha;     // LF speed B(sigma) * M
    T eps;       // Jiang-Shu epsilon
    T inv_dtau;  // 1 / dtau
};

// Reconstruction at one interface from v_{-2..2} (upwind side first).
template <typename T>
__device__ __forceinline__ T weno5_rec(T vm2, T vm1, T v0, T v1, T v2, T eps)
{
    const T s6 = T(1) / T(6);
    const T q0 = fma(T(2), vm2, fma(T(-7), vm1, T(11) * v0)) * s6;
    const T q1 = fma(T(-1), vm1, fma(T(5), v0, T(2) * v1)) * s6;
    const T q2 = fma(T(2), v0, fma(T(5), v1, -v2)) * s6;
    const T c13 = T(13) / T(12);
    T s, t;
    s = vm2 - T(2) * vm1 + v0; t = vm2 - T(4) * vm1 + T(3) * v0;
    T b0 = fma(c13 * s, s, T(0.25) * t * t);
    s = vm1 - T(2) * v0 + v1; t = vm1 - v1;
    T b1 = fma(c13 * s, s, T(0.25) * t * t);
    s = v0 - T(2) * v1 + v2; t = T(3) * v0 - T(4) * v1 + v2;
    T b2 = fma(c13 * s, s, T(0.25) * t * t);
    T t0 = eps + b0; t0 *= t0;
    T t1 = eps + b1; t1 *= t1;
    T t2 = eps + b2; t2 *= t2;
    const T a0 = T(0.1) * t1 * t2;
    const T a1 = T(0.6) * t0 * t2;
    const T a2 = T(0.3) * t0 * t1;
    return fma(a0, q0, fma(a1, q1, a2 * q2)) / (a0 + a1 + a2);
}

// b over the points [k0, k0 + Q) of one periodic row u[0..nx) (shared
// memory), written to out[k0 ..).  Also accumulates sum u, sum u^2, max|u|
// and the non-finite count of the owned points.
template <typename T>
__device__ __forceinline__ void weno_row_chunk(const T* __restrict__ u, T* __restrict__ out, int nx,
                                               int k0, int Q, const WenoCoef<T>& c, T& s1, T& s2,
                                               T& mx, int& nf)
{
    const int msk = nx - 1;
    // window: slot s <-> point k - 2 + s for the interface k + 1/2
    T fp[6], fm[6];
    const T half = T(0.5);
#pragma unroll
    for (int s = 0; s < 6; s++) {
        const T v = u[(k0 - 3 + s) & msk];                   // interface k0 - 1/2: k = k0 - 1
        const T f = -half * c.B * v * v;
        fp[s] = half * fma(c.alpha, v, f);
        fm[s] = half * fma(-c.alpha, v, f);
    }
    T Fprev = weno5_rec<T>(fp[0], fp[1], fp[2], fp[3], fp[4], c.eps) +
              weno5_rec<T>(fm[5], fm[4], fm[3], fm[2], fm[1], c.eps);
    for (int i = 0; i < Q; i++) {
        const int k = k0 + i;
#pragma unroll
        for (int s = 0; s < 5; s++) { fp[s] = fp[s + 1]; fm[s] = fm[s + 1]; }
        const T v = u[(k + 3) & msk];
        const T f = -half * c.B * v * v;
        fp[5] = half * fma(c.alpha, v, f);
        fm[5] = half * fma(-c.alpha, v, f);
        const T F = weno5_rec<T>(fp[0], fp[1], fp[2], fp[3], fp[4], c.eps) +
                    weno5_rec<T>(fm[5], fm[4], fm[3], fm[2], fm[1], c.eps);
        out[k] = -(F - Fprev) * c.inv_dtau;
        Fprev = F;
        const T uk = u[k];
        if (isfinite(uk)) {
            s1 += uk;
            s2 = fma(uk, uk, s2);
            mx = fmax(mx, fabs(uk));
        } else {
            nf += 1;
        }
    }
}

}  // namespace kzk
