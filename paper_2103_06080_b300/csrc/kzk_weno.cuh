// kzk_weno.cuh -- WENO5 flux derivative along tau (Sec. 3.3, Eq. 7).
//
// Flux of the homogeneous medium: f(u) = -B(sigma) u^2 / 2, split globally
// (Lax-Friedrichs) into f+- = (f +- alpha u)/2 with alpha = B(sigma) * M.
// At interface k+1/2 the upwind part F+ is the Jiang-Shu WENO5 reconstruction
// from f+ at k-2..k+2, the downwind part F- the mirrored one from f- at
// k+3..k-1; the nonlinear term is b_k = -(F_{k+1/2} - F_{k-1/2}) / dtau.
// Jiang-Shu weights omega_r = a_r / sum a, a_r = d_r / (eps + beta_r)^2,
// d = (1/10, 6/10, 3/10).
//
// Arithmetic organisation (same mathematics, fewer operations):
//  * every smoothness indicator is a function of one 3-point stencil centred
//    at c: with S = f_{c-1} - 2 f_c + f_{c+1}, D = f_{c+1} - f_{c-1},
//      left   13/12 S^2 + 1/4 (D + 2S)^2   (beta_0 of the + side at c+1/2+1,
//                                           beta_2 of the - side at c+1/2),
//      centre 13/12 S^2 + 1/4 D^2          (beta_1),
//      right  13/12 S^2 + 1/4 (D - 2S)^2   (beta_2 of the + side at c-1/2,
//                                           beta_0 of the - side at c-3/2);
//    each is computed once per centre and reused by the three interfaces
//    that need it (a sliding window over the row);
//  * the quotient sum a_r q_r / sum a_r is formed after multiplying numerator
//    and denominator by prod (eps + beta_r)^2, so a_r -> d_r prod_{s != r} t_s,
//    with t0 factored out of the two terms that contain it;
//  * the centred candidate q1 is formed from its stencil, the outer ones from
//    it: q0 - q1 and q2 - q1 are multiples of third differences, i.e. of
//    differences of neighbouring centres' S (two operations each);
//  * the 1/6 of the candidate values q_r is folded into 1/dtau, and common
//    factors of the weights (16 in (eps + beta)^2, 10 in d_r) are dropped;
//  * FP64: both halves F+ and F- and two neighbouring interfaces share one
//    division, which also carries the final scale; FP32: two hardware
//    reciprocals per interface (the product of the denominators could
//    underflow).
#pragma once
#include "kzk_common.cuh"
#include "kzk_fft.cuh"
#include <type_traits>

namespace kzk {

// quotient a / b to about 2 ulp (the FP32 sweep's hardware reciprocal)
__device__ __forceinline__ float fast_div(float a, float b) { return __fdividef(a, b); }

template <typename T>
struct WenoCoef {
    T B;         // B(sigma)
    T alpha;     // LF speed B(sigma) * M (random medium: |c| + B(sigma) M)
    T eps;       // Jiang-Shu epsilon
    T inv_dtau;  // 1 / dtau
    T c;         // random medium: 2 pi U_par of the row (advection along tau)
};

template <typename T, bool PAD>
__device__ __forceinline__ T ld_real(const cx<T>* buf, int k)
{
    const T* p = reinterpret_cast<const T*>(buf);
    return PAD ? p[2 * padx(k >> 1) + (k & 1)] : p[k];
}
template <typename T, bool PAD>
__device__ __forceinline__ void st_real(cx<T>* buf, int k, T v)
{
    T* p = reinterpret_cast<T*>(buf);
    if (PAD) p[2 * padx(k >> 1) + (k & 1)] = v;
    else p[k] = v;
}

// 16 (eps + beta)^2 of the left, centre and right indicators of the stencil
// (fm1, f0, fp1) centred at c, formed as (4 eps + 4 beta)^2: the common factor
// 16 cancels in the weights, and 4 beta = 13/3 S^2 + x^2 needs no 1/4; the
// shared part 13/3 S^2 + 4 eps is formed once.  eps4 = 4 eps (for a flux
// scaled by s, pass 4 s^2 eps: the weights are unchanged).
template <typename T>
__device__ __forceinline__ void indicators(T fm1, T f0, T fp1, T eps4, T& tl, T& tc, T& tr, T& S)
{
    S = fm1 - T(2) * f0 + fp1;
    const T D = fp1 - fm1;
    const T Pe = fma((T(13) / T(3)) * S, S, eps4);
    const T xl = fma(T(2), S, D), xr = fma(T(-2), S, D);
    const T bl = fma(xl, xl, Pe);
    const T bc = fma(D, D, Pe);
    const T br = fma(xr, xr, Pe);
    tl = bl * bl;
    tc = bc * bc;
    tr = br * br;
}

// 6 * numerator and denominator of one reconstruction from its three
// candidate values (times 6) q0 (stencil -2..0), q1 (-1..1), q2 (0..2) and
// the squared shifted indicators t0, t1, t2 of the same stencils.
template <typename T>
__device__ __forceinline__ void rec_parts(T q0, T q1, T q2, T t0, T t1, T t2, T& num6, T& den)
{
    // linear weights 1/10, 6/10, 3/10 scaled by 10 (the factor cancels):
    // a0 = t1 t2, a1 = 6 t0 t2, a2 = 3 t0 t1, with t0 factored out of a1, a2
    const T p12 = t1 * t2, h1 = T(3) * t1, h2 = T(6) * t2;
    den = fma(t0, h2 + h1, p12);
    num6 = fma(p12, q0, t0 * fma(h2, q1, h1 * q2));
}

// Sliding WENO5 sweep over the interfaces k0 - 1/2 .. k0 + Q - 1/2 of a
// periodic line.  load(kk, p, m) gives the split fluxes (scaled: 4 f+ and
// 4 f-) at point kk; store(k, d) receives d = 24 scale (F_{k+1/2} -
// F_{k-1/2}) for k in [k0, k0 + Q) in order (FP64: the factor scale rides on
// the shared division).  eps4: the Jiang-Shu epsilon for that scaling
// (64 eps).  Every smoothness indicator is computed once per stencil centre
// and every interface once.
// QC > 0: Q == QC known at compile time (the interface loop fully unrolled).
template <typename T, int QC = 0, typename Load, typename Store>
__device__ __forceinline__ void weno_sweep(int k0, int Q, T eps4, T scale, Load load, Store store)
{
    T fp[6], fm[6];
    // window slot s <-> point k - 2 + s for interface k + 1/2; start at
    // k = k0 - 1 with the indicators of centres k0 - 2 .. k0 + 0 (pre-roll)
    int k = k0 - 1;
#pragma unroll
    for (int s = 0; s < 5; s++) load(k - 3 + s, fp[s + 1], fm[s + 1]);   // points k0-4 .. k0
    T tLp3, tLp2, tLp1, tCp2, tCp1, tRp1, tLm2, tLm1, tCm1, tx;
    // second differences S_c = f_{c-1} - 2 f_c + f_{c+1} of the centres and
    // their differences dS_c = S_c - S_{c-1} give two of each side's three
    // candidate values from the third (below)
    T Sp0, Sp1, Sp2, Sm0, Sm1, Sm2;
    // centre k0 - 2 (points k0-3, k0-2, k0-1 = slots 2, 3, 4)
    indicators<T>(fp[2], fp[3], fp[4], eps4, tLp2, tx, tx, Sp0);
    indicators<T>(fm[2], fm[3], fm[4], eps4, tx, tx, tx, Sm0);
    // centre k0 - 1 (slots 3, 4, 5)
    indicators<T>(fp[3], fp[4], fp[5], eps4, tLp1, tCp1, tx, Sp1);
    indicators<T>(fm[3], fm[4], fm[5], eps4, tLm1, tx, tx, Sm1);
    // age the history by one centre before computing centre k0
    tLp3 = tLp2; tLp2 = tLp1; tCp2 = tCp1;
    tLm2 = tLm1;
#pragma unroll
    for (int s = 0; s < 5; s++) { fp[s] = fp[s + 1]; fm[s] = fm[s + 1]; }
    load(k0 + 1, fp[5], fm[5]);                                           // slots: points k0-4 .. k0+1
    // centre k0 (slots 3, 4, 5)
    indicators<T>(fp[3], fp[4], fp[5], eps4, tLp1, tCp1, tRp1, Sp2);
    indicators<T>(fm[3], fm[4], fm[5], eps4, tLm1, tCm1, tx, Sm2);
    // at the top of interface k: SpL = S_{k+1}, dpA = dS_k, dpB = dS_{k+1}
    // (+ side), SmL, dmB likewise (- side)
    T SpL = Sp2, dpA = Sp1 - Sp0, dpB = Sp2 - Sp1, SmL = Sm2, dmB = Sm2 - Sm1;
    // invariant at the top of interface k: tX1 = centre k+1, tX2 = centre k,
    // tLp3 = centre k-1; each interface adds centre k+2.  parts(): slide the
    // window by one point and return 6 x the numerator and the denominator of
    // both halves of F_{k+1/2}.
    auto parts = [&](int kk, T& np, T& dp, T& nm, T& dm) {
#pragma unroll
        for (int s = 0; s < 5; s++) { fp[s] = fp[s + 1]; fm[s] = fm[s + 1]; }
        load(kk + 3, fp[5], fm[5]);
        T tLpN, tCpN, tRpN, tLmN, tCmN, tRmN, SpN, SmN;
        indicators<T>(fp[3], fp[4], fp[5], eps4, tLpN, tCpN, tRpN, SpN);
        indicators<T>(fm[3], fm[4], fm[5], eps4, tLmN, tCmN, tRmN, SmN);
        const T dpN = SpN - SpL, dmN = SmN - SmL;
        // candidate values x 6: the centred one directly, the other two from
        // it, q0 - q1 and q2 - q1 being (multiples of) third differences:
        //   + side (f_{k-2} .. f_{k+2}): q0 = q1 - 2 dS_k,     q2 = q1 - dS_{k+1};
        //   - side (mirrored, g_{k+3} .. g_{k-1}): q0 = q1 + 2 dS_{k+2}, q2 = q1 + dS_{k+1}
        const T q1p = fma(T(5), fp[2], fma(T(2), fp[3], -fp[1]));
        const T q1m = fma(T(5), fm[3], fma(T(2), fm[2], -fm[4]));
        // + side: left(k-1), centre(k), right(k+1); - side: right(k+2), centre(k+1), left(k)
        rec_parts<T>(fma(T(-2), dpA, q1p), q1p, q1p - dpB, tLp3, tCp2, tRp1, np, dp);
        rec_parts<T>(fma(T(2), dmN, q1m), q1m, q1m + dmB, tRmN, tCm1, tLm2, nm, dm);
        SpL = SpN; dpA = dpB; dpB = dpN;
        SmL = SmN; dmB = dmN;
        tLp3 = tLp2; tLp2 = tLp1; tLp1 = tLpN;
        tCp2 = tCp1; tCp1 = tCpN;
        tRp1 = tRpN;
        tLm2 = tLm1; tLm1 = tLmN;
        tCm1 = tCmN;
    };
    T np, dp, nm, dm;
    parts(k, np, dp, nm, dm);
    if constexpr (std::is_same<T, double>::value) {
        // F = N / D with N = np dm + nm dp, D = dp dm; two interfaces share one
        // division: scale / (D1 D2) gives both (scaled) quotients
        T Fprev = fma(np, dm, nm * dp) * scale / (dp * dm);
        auto two = [&](int kk) {
            parts(kk, np, dp, nm, dm);
            const T N1 = fma(np, dm, nm * dp), D1 = dp * dm;
            parts(kk + 1, np, dp, nm, dm);
            const T N2 = fma(np, dm, nm * dp), D2 = dp * dm;
            const T inv = scale * (T(1) / (D1 * D2));
            const T F1 = N1 * D2 * inv, F2 = N2 * D1 * inv;
            store(kk, F1 - Fprev);
            store(kk + 1, F2 - F1);
            Fprev = F2;
        };
        if constexpr (QC > 0) {
            static_assert(QC % 2 == 0, "pairs of interfaces");
#pragma unroll
            for (int j = 0; j < QC; j += 2) two(k0 + j);
        } else {
#pragma unroll 1
            for (k = k0; k + 1 < k0 + Q; k += 2) two(k);
            if (k < k0 + Q) {
                parts(k, np, dp, nm, dm);
                store(k, fma(np, dm, nm * dp) * scale / (dp * dm) - Fprev);
            }
        }
    } else {
        // FP32: two hardware reciprocals (the product of the two denominators
        // could underflow)
        T Fprev = fast_div(np, dp) + fast_div(nm, dm);
        if constexpr (QC > 0) {
#pragma unroll
            for (int j = 0; j < QC; j++) {
                parts(k0 + j, np, dp, nm, dm);
                const T F = fast_div(np, dp) + fast_div(nm, dm);
                store(k0 + j, (F - Fprev) * scale);
                Fprev = F;
            }
        } else {
#pragma unroll 2
            for (k = k0; k < k0 + Q; k++) {
                parts(k, np, dp, nm, dm);
                const T F = fast_div(np, dp) + fast_div(nm, dm);
                store(k, (F - Fprev) * scale);
                Fprev = F;
            }
        }
    }
}

// b over the points [k0, k0 + Q) of one periodic row u[0..nx) (shared
// memory, PAD layout), written to out at the same points.  ADV: the flux of
// the random medium, f(u) = -c u - B u^2 / 2 (Eq. 7).  POW2: nx is a power of
// two (the periodic wrap is a mask); otherwise any nx >= 8.
// Q16: Q == 16 and k0 a multiple of 16 (PAD layout): the chunk's 8 complex
// slots never straddle a padding slot, so its points sit at constant offsets
// from the first (real index 2 padx(k0 / 2) + j); only the halo points take
// the general index.
template <typename T, bool PAD, bool ADV = false, bool POW2 = true, bool Q16 = false>
__device__ __forceinline__ void weno_row_chunk(const cx<T>* u, cx<T>* out, int nx, int k0, int Q,
                                               const WenoCoef<T>& c)
{
    static_assert(!Q16 || PAD, "the constant-offset chunk is for the padded layout");
    const int msk = nx - 1;
    auto wrap = [&](int kk) { return POW2 ? (kk & msk) : (kk < 0 ? kk + nx : (kk >= nx ? kk - nx : kk)); };
    const int ib = 2 * padx(k0 >> 1);
    const T* pr = reinterpret_cast<const T*>(u) + ib;
    T* pw = reinterpret_cast<T*>(out) + ib;
    auto rd = [&](int kk) -> T {
        if constexpr (Q16) {
            const int j = kk - k0;
            if (j >= 0 && j < 16) return pr[j];
        }
        return ld_real<T, PAD>(u, wrap(kk));
    };
    // the split fluxes are carried as 4 f+- (no halves):
    //   4 f+ = v (2 (alpha - c) - B v),   4 f- = -v (2 (alpha + c) + B v)
    // so the reconstruction is 4 F, the indicators take 64 eps, and the 1/4
    // joins the 1/6 of the candidate values in the final scale
    const T scale = -c.inv_dtau * (T(1) / T(24));
    const T ap = T(2) * (ADV ? c.alpha - c.c : c.alpha);
    const T am = T(2) * (ADV ? c.alpha + c.c : c.alpha);
    auto load = [&](int kk, T& p, T& m) {
        const T v = rd(kk);
        p = v * fma(-c.B, v, ap);
        m = -v * fma(c.B, v, am);
    };
    auto store = [&](int k, T d) {
        if constexpr (Q16) pw[k - k0] = d;
        else st_real<T, PAD>(out, k, d);
    };
    weno_sweep<T, Q16 ? 16 : 0>(k0, Q, T(64) * c.eps, scale, load, store);
}

// sum u, sum u^2, max|u| and non-finite count of the points [k0, k0 + Q)
// (Q16: Q == 16, k0 a multiple of 16, constant offsets as in weno_row_chunk).
template <typename T, bool PAD, bool Q16 = false>
__device__ __forceinline__ void row_stats(const cx<T>* u, int k0, int Q, T& s1, T& s2, T& mx, int& nf)
{
    // FP64: the finiteness test and the running max |u| on the bit patterns
    // (non-negative doubles order as their bits), off the FP64 pipe
    unsigned long long mb = 0;
    auto acc = [&](T v) {
        if constexpr (std::is_same<T, double>::value) {
            const unsigned long long b = (unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffULL;
            if (b < 0x7ff0000000000000ULL) { s1 += v; s2 = fma(v, v, s2); mb = b > mb ? b : mb; } else { nf += 1; }
        } else {
            if (isfinite(v)) { s1 += v; s2 = fma(v, v, s2); mx = fmax(mx, fabs(v)); } else { nf += 1; }
        }
    };
    if constexpr (Q16) {
        const T* pr = reinterpret_cast<const T*>(u) + 2 * padx(k0 >> 1);
#pragma unroll
        for (int j = 0; j < 16; j++) acc(pr[j]);
    } else {
        for (int k = k0; k < k0 + Q; k++) acc(ld_real<T, PAD>(u, k));
    }
    if constexpr (std::is_same<T, double>::value) mx = fmax(mx, __longlong_as_double((long long)mb));
}

}  // namespace kzk
