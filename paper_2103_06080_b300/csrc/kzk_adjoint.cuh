// kzk_adjoint.cuh -- kernels of the transposed ExpRK22 step.
//
// With P_X u := Re F^{-1}(X o F u) (a real operator for the Hermitian-
// symmetric tables of Eq. 11) one forward step reads
//   b1 = G_n(u),  u* = P_E u + P_{ds Phi1} b1,  b2 = G_{n+1}(u*),
//   u' = u* + P_{ds Phi2}(b2 - b1),
// with G_s(u) = WENO_s(u) + (A(s) - A) d_tau^2 u.  Its transpose, for a
// cotangent lam' of u', is
//   mu2  = P_{conj(ds Phi2)} lam'                     (adjoint C2, column pass)
//   lam* = lam' + J_{G_{n+1}}(u*)^T mu2               (adjoint R2, row pass)
//   lam_lin = P_{conj E} lam*,  nu1 = P_{conj(ds Phi1)} lam* - mu2   (adjoint C1)
//   lam  = lam_lin + J_{G_n}(u)^T nu1                 (adjoint R1, row pass)
// All adjoint arrays use the packed spectral layout of the state (tau-spectrum
// divided by nx), so P_X is a column pass with the conjugated, rescaled table.
//
// WENO transpose: with psi_{k+1/2} = (mu_{k+1} - mu_k)/dtau,
//   (J^T mu)_i = sum_k psi_{k+1/2} dF_{k+1/2}/du_i,
// and for one reconstruction F = sum omega_r q_r, omega_r = a_r / sum a,
// a_r = d_r/(eps + beta_r)^2:
//   dF/dv_j = sum_r omega_r dq_r/dv_j - 2 sum_r omega_r (q_r - F)/(eps + beta_r) dbeta_r/dv_j
// (the derivative through the nonlinear weights), times df+-/du = (-B u +- alpha)/2.
#pragma once
#include "kzk_common.cuh"
#include "kzk_fft.cuh"
#include "kzk_kernels.cuh"

namespace kzk {

// Gradient of one reconstruction w.r.t. v_{-2..2}, scaled: g[j] = 6 w6 dF/dv_j
// (callers pass w6 = w / 6).  With integer-coefficient candidates Q_r = 6 q_r
// and E_r = 4 (eps + beta_r) = eps4 + 13/3 s_r^2 + t_r^2 (s_r, t_r the two
// stencil combinations of beta_r), the Jiang-Shu weights are
// omega_r = a_r / sum a with a_r = d_r prod_{s != r} E_s^2, F6 = sum omega_r Q_r,
// and, since d ln a_r = -2 dE_r / E_r,
//   6 dF = sum_r omega_r dQ_r - 2 sum_r omega_r (Q_r - F6) / E_r dE_r,
//   dE_r = 26/3 s_r ds_r + 2 t_r dt_r.
// In FP64 the four reciprocals (1/sum a, 1/E_r) come from one division,
// r = 1 / (S E0 E1 E2); in FP32 that product can underflow, so they are taken
// separately.
template <typename T>
__device__ __forceinline__ void weno5_grad(T vm2, T vm1, T v0, T v1, T v2, T eps4, T w6, T* g)
{
    const T Q0 = fma(T(2), vm2, fma(T(-7), vm1, T(11) * v0));
    const T Q1 = fma(T(5), v0, fma(T(2), v1, -vm1));
    const T Q2 = fma(T(2), v0, fma(T(5), v1, -v2));
    const T sa = fma(T(-2), vm1, vm2 + v0), ta = fma(T(3), v0, fma(T(-4), vm1, vm2));
    const T sb = fma(T(-2), v0, vm1 + v1), tb = vm1 - v1;
    const T sc = fma(T(-2), v1, v0 + v2), tc = fma(T(3), v0, fma(T(-4), v1, v2));
    const T k13 = T(13) / T(3);
    const T E0 = fma(k13 * sa, sa, fma(ta, ta, eps4));
    const T E1 = fma(k13 * sb, sb, fma(tb, tb, eps4));
    const T E2 = fma(k13 * sc, sc, fma(tc, tc, eps4));
    const T T0 = E0 * E0, T1 = E1 * E1, T2 = E2 * E2;
    // linear weights 1/10, 6/10, 3/10 scaled by 10 (the factor cancels)
    const T a0 = T1 * T2, a1 = T(6) * (T0 * T2), a2 = T(3) * (T0 * T1);
    const T S = a0 + a1 + a2;
    T inv, iE0, iE1, iE2;                                    // 1/S, 1/E_r
    if constexpr (sizeof(T) == 8) {
        const T e01 = E0 * E1, e012 = e01 * E2;
        const T r = T(1) / (S * e012);                       // >= eps^7: fine in FP64
        inv = r * e012;
        const T rS = r * S;
        iE0 = rS * (E1 * E2); iE1 = rS * (E0 * E2); iE2 = rS * e01;
    } else {
        inv = __frcp_rn(S); iE0 = __frcp_rn(E0); iE1 = __frcp_rn(E1); iE2 = __frcp_rn(E2);
    }
    const T o0 = a0 * inv, o1 = a1 * inv, o2 = a2 * inv;     // omega_r
    const T F6 = fma(o0, Q0, fma(o1, Q1, o2 * Q2));
    // -2 omega_r (Q_r - F6) / E_r times the dE_r coefficients 26/3 s_r and 2 t_r
    const T C0 = o0 * (Q0 - F6) * iE0, C1 = o1 * (Q1 - F6) * iE1, C2 = o2 * (Q2 - F6) * iE2;
    const T k52 = T(-52) / T(3);
    const T A0 = (k52 * C0) * sa, B0 = (T(-4) * C0) * ta;
    const T A1 = (k52 * C1) * sb, B1 = (T(-4) * C1) * tb;
    const T A2 = (k52 * C2) * sc, B2 = (T(-4) * C2) * tc;
    g[0] = w6 * fma(T(2), o0, A0 + B0);
    g[1] = w6 * (fma(T(-7), o0, A1 + B1 - o1) - fma(T(2), A0, T(4) * B0));
    g[2] = w6 * (fma(T(11), o0, fma(T(5), o1, T(2) * o2)) + fma(T(3), B0 + B2, A0 + A2) - T(2) * A1);
    g[3] = w6 * (fma(T(2), o1, fma(T(5), o2, A1 - B1)) - fma(T(2), A2, T(4) * B2));
    g[4] = w6 * (A2 + B2 - o2);
}

// The sliding form of weno5_grad for the row sweep.  Every 3-point stencil
// centre c contributes S = f_{c-1} - 2 f_c + f_{c+1}, D = f_{c+1} - f_{c-1}
// and Pe = 13/3 S^2 + eps4 once (with kS = 13/3 S, which also carries the
// s_r-terms of the gradient: -52/3 C s = -4 C kS); a reconstruction takes its
// three stencils' (kS_r, t_r, E_r = t_r^2 + Pe) from the centres it spans,
// the t_r being the combinations D + 2S, -D, 2S - D of weno5_grad's (s, t)
// pairs (mirrored for the downwind side), and its outer candidates from the
// centred one and differences of neighbouring S (third differences), as the
// forward sweep does.
template <typename T>
struct GradCentre {
    T S, D, Pe;
    __device__ __forceinline__ T kS() const { return (T(13) / T(3)) * S; }
};
template <typename T>
__device__ __forceinline__ GradCentre<T> grad_centre(T fm1, T f0, T fp1, T eps4)
{
    GradCentre<T> c;
    c.S = fma(T(-2), f0, fm1 + fp1);
    c.D = fp1 - fm1;
    c.Pe = fma(c.kS(), c.S, eps4);
    return c;
}
template <typename T>
struct GradPart {
    T Q0, Q1, Q2, k0, t0, k1, t1, k2, t2, E0, E1, E2, a0, a1, a2, Ssum, e01, e012;
};
// weights and X = S E0 E1 E2 of one reconstruction from its candidates
// (times 6) and its stencils' (kS, t, Pe)
template <typename T>
__device__ __forceinline__ void grad_prep(GradPart<T>& q, T Q0, T Q1, T Q2, T k0, T t0, T Pe0, T k1, T t1, T Pe1,
                                          T k2, T t2, T Pe2)
{
    q.Q0 = Q0; q.Q1 = Q1; q.Q2 = Q2;
    q.k0 = k0; q.t0 = t0; q.k1 = k1; q.t1 = t1; q.k2 = k2; q.t2 = t2;
    q.E0 = fma(t0, t0, Pe0);
    q.E1 = fma(t1, t1, Pe1);
    q.E2 = fma(t2, t2, Pe2);
    const T T0 = q.E0 * q.E0, T1 = q.E1 * q.E1, T2 = q.E2 * q.E2;
    q.a0 = T1 * T2;
    q.a1 = T(6) * (T0 * T2);
    q.a2 = T(3) * (T0 * T1);
    q.Ssum = q.a0 + q.a1 + q.a2;
    q.e01 = q.E0 * q.E1;
    q.e012 = q.e01 * q.E2;
}
// g[j] = 6 w6 dF/dv_j (as weno5_grad), given r = 1 / (S E0 E1 E2) (FP64); the
// factor w6 rides on the weights' reciprocal (omega_r w6) and so on every
// term of g
template <typename T>
__device__ __forceinline__ void grad_finish(const GradPart<T>& q, T r, T w6, T* g)
{
    T inv, iE0, iE1, iE2;                                    // 1/S and -4/E_r
    if constexpr (sizeof(T) == 8) {
        inv = r * q.e012;
        const T rS = T(-4) * (r * q.Ssum);
        iE0 = rS * (q.E1 * q.E2); iE1 = rS * (q.E0 * q.E2); iE2 = rS * q.e01;
    } else {
        inv = __frcp_rn(q.Ssum);
        iE0 = T(-4) * __frcp_rn(q.E0); iE1 = T(-4) * __frcp_rn(q.E1); iE2 = T(-4) * __frcp_rn(q.E2);
    }
    const T F6 = fma(q.a0, q.Q0, fma(q.a1, q.Q1, q.a2 * q.Q2)) * inv;
    const T wi = w6 * inv;
    const T o0 = q.a0 * wi, o1 = q.a1 * wi, o2 = q.a2 * wi;  // w6 omega_r
    // -4 w6 C_r with C_r = omega_r (Q_r - F6) / E_r; A_r = -52/3 C_r s_r, B_r = -4 C_r t_r (times w6)
    const T C0 = o0 * (q.Q0 - F6) * iE0, C1 = o1 * (q.Q1 - F6) * iE1, C2 = o2 * (q.Q2 - F6) * iE2;
    const T A0 = C0 * q.k0, B0 = C0 * q.t0;
    const T A1 = C1 * q.k1, B1 = C1 * q.t1;
    const T A2 = C2 * q.k2, B2 = C2 * q.t2;
    g[0] = fma(T(2), o0, A0 + B0);
    g[1] = fma(T(-7), o0, A1 + B1 - o1) - fma(T(2), A0, T(4) * B0);
    g[2] = fma(T(11), o0, fma(T(5), o1, T(2) * o2)) + fma(T(3), B0 + B2, A0 + A2) - T(2) * A1;
    g[3] = fma(T(2), o1, fma(T(5), o2, A1 - B1)) - fma(T(2), A2, T(4) * B2);
    g[4] = A2 + B2 - o2;
}

// J_WENO(u)^T mu over the points [k0, k0+Q) of one periodic row (u, mu, g:
// row buffers of nx reals, PAD layout): own-point sums go to g, the two
// contributions left of k0 to spl[0..1] and the three right of k0+Q-1 to
// spr[0..2] (added by the neighbours afterwards).  POW2: nx a power of two
// (the periodic wrap is a mask); otherwise any nx >= 8.
template <typename T, bool PAD = true, bool POW2 = true>
__device__ __forceinline__ void weno_row_chunk_T(const cx<T>* u, const cx<T>* mu, cx<T>* g, T* spl, T* spr,
                                                 int nx, int k0, int Q, const WenoCoef<T>& c)
{
    const int msk = nx - 1;
    auto wrap = [&](int kk) { return POW2 ? (kk & msk) : (kk < 0 ? kk + nx : (kk >= nx ? kk - nx : kk)); };
    const T half = T(0.5);
    const T eps4 = T(4) * c.eps;
    const T inv_dtau6 = c.inv_dtau * (T(1) / T(6));
    T fp[6], fm[6], dp[6], dm[6], acc[6];
    // window slot s <-> point k - 2 + s for interface k + 1/2, starting at k = k0
#pragma unroll
    for (int s = 0; s < 6; s++) {
        const T v = ld_real<T, PAD>(u, wrap(k0 - 2 + s));
        const T f = fma(-c.c, v, -half * c.B * v * v);
        fp[s] = half * fma(c.alpha, v, f);
        fm[s] = half * fma(-c.alpha, v, f);
        dp[s] = half * ((c.alpha - c.c) - c.B * v);
        dm[s] = half * ((-c.alpha - c.c) - c.B * v);
        acc[s] = T(0);
    }
    T mk_ = ld_real<T, PAD>(mu, wrap(k0));
    // stencil centres: + side k0 - 1, k0 (points fp[0..3]); - side k0, k0 + 1 (fm[1..4])
    GradCentre<T> cpA = grad_centre<T>(fp[0], fp[1], fp[2], eps4);   // + side, centre k - 1
    GradCentre<T> cpB = grad_centre<T>(fp[1], fp[2], fp[3], eps4);   // + side, centre k
    GradCentre<T> cmA = grad_centre<T>(fm[1], fm[2], fm[3], eps4);   // - side, centre k
    GradCentre<T> cmB = grad_centre<T>(fm[2], fm[3], fm[4], eps4);   // - side, centre k + 1
    for (int i = 0; i < Q; i++) {
        const int k = k0 + i;
        const T mk1 = ld_real<T, PAD>(mu, wrap(k + 1));
        const T psi6 = (mk1 - mk_) * inv_dtau6;
        mk_ = mk1;
        const GradCentre<T> cpC = grad_centre<T>(fp[2], fp[3], fp[4], eps4);   // + side, centre k + 1
        const GradCentre<T> cmC = grad_centre<T>(fm[3], fm[4], fm[5], eps4);   // - side, centre k + 2
        T gp[5], gm[5];
        // differences of neighbouring S (+ side: S_k - S_{k-1}, S_{k+1} - S_k;
        // - side: S_{k+1} - S_k, S_{k+2} - S_{k+1})
        const T dpAB = cpB.S - cpA.S, dpBC = cpC.S - cpB.S, dmAB = cmB.S - cmA.S, dmBC = cmC.S - cmB.S;
        {
            // candidates x 6: q0 = q1 - 2 (S_k - S_{k-1}), q2 = q1 - (S_{k+1} - S_k)
            const T Q1 = fma(T(5), fp[2], fma(T(2), fp[3], -fp[1]));
            GradPart<T> q;
            grad_prep<T>(q, fma(T(-2), dpAB, Q1), Q1, Q1 - dpBC,
                         cpA.kS(), fma(T(2), cpA.S, cpA.D), cpA.Pe, cpB.kS(), -cpB.D, cpB.Pe,
                         cpC.kS(), fma(T(2), cpC.S, -cpC.D), cpC.Pe);
            // X = S E0 E1 E2 >= eps^7: one FP64 division gives 1/S and the 1/E_r
            grad_finish<T>(q, sizeof(T) == 8 ? T(1) / (q.Ssum * q.e012) : T(0), psi6, gp);
        }
        {
            // mirrored: q0 = q1 + 2 (S_{k+2} - S_{k+1}), q2 = q1 + (S_{k+1} - S_k)
            const T Q1 = fma(T(5), fm[3], fma(T(2), fm[2], -fm[4]));
            GradPart<T> q;
            grad_prep<T>(q, fma(T(2), dmBC, Q1), Q1, Q1 + dmAB,
                         cmC.kS(), fma(T(2), cmC.S, -cmC.D), cmC.Pe, cmB.kS(), cmB.D, cmB.Pe,
                         cmA.kS(), fma(T(2), cmA.S, cmA.D), cmA.Pe);
            grad_finish<T>(q, sizeof(T) == 8 ? T(1) / (q.Ssum * q.e012) : T(0), psi6, gm);
        }
        cpA = cpB; cpB = cpC;
        cmA = cmB; cmB = cmC;
#pragma unroll
        for (int s = 0; s < 5; s++) acc[s] = fma(gp[s], dp[s], acc[s]);
#pragma unroll
        for (int s = 0; s < 5; s++) acc[5 - s] = fma(gm[s], dm[5 - s], acc[5 - s]);
        // point k - 2 is complete
        const int pt = k - 2;
        if (pt < k0) spl[pt - (k0 - 2)] = acc[0];
        else st_real<T, PAD>(g, pt, acc[0]);
#pragma unroll
        for (int s = 0; s < 5; s++) {
            fp[s] = fp[s + 1]; fm[s] = fm[s + 1]; dp[s] = dp[s + 1]; dm[s] = dm[s + 1]; acc[s] = acc[s + 1];
        }
        const T v = ld_real<T, PAD>(u, wrap(k + 4));
        const T f = fma(-c.c, v, -half * c.B * v * v);
        fp[5] = half * fma(c.alpha, v, f);
        fm[5] = half * fma(-c.alpha, v, f);
        dp[5] = half * ((c.alpha - c.c) - c.B * v);
        dm[5] = half * ((-c.alpha - c.c) - c.B * v);
        acc[5] = T(0);
    }
    // remaining points k0+Q-2 .. k0+Q+2 in acc[0..4]
#pragma unroll
    for (int s = 0; s < 5; s++) {
        const int pt = k0 + Q - 2 + s;
        if (pt < k0 + Q) st_real<T, PAD>(g, pt, acc[s]);
        else spr[pt - (k0 + Q)] = acc[s];
    }
}

template <typename T>
struct AdjRowArgs {
    const cx<T>* m;         // cotangent of b (mu2 or nu1), packed spectral
    const T* u;             // state the step linearises at (u* or u^n), physical [batch][ny][nx]
    const cx<T>* l;         // additive term (lam' or lam_lin), packed spectral
    cx<T>* out;             // l + F(J_G(u)^T m) / nx
    const cx<T>* tw;        // exp(-2 pi i k / nx) (real-FFT pre/post-processing)
    const cx<T>* tws;       // staged twiddles of the length-nx/2 FFT
    int log2nx;
    long long inst_stride;
    WenoCoef<T> wc;
    T dA;                   // A(sigma) - A
    T kscale;
    T inv_nx;
    // random medium (nullable): this stage's coefficients (the row's c = 2 pi
    // U_par enters the tau-flux) and the transposed y part, added before the R2C
    const double* med_coef; // [ny][3]
    const T* yT;            // [batch][ny][nx] physical
};

enum AdjRowMode { ADJ_ROW_2 = 0, ADJ_ROW_1 = 1 };

// One row of J_G^T: the physical state row (stored by the forward recompute)
// and the C2R of the cotangent row, WENO5 transpose, R2C, plus the
// absorption-deviation term and the additive row.
// Three padded buffers of nx reals, then the spill slots of the sweep.
// MAXT, MINB: launch bounds (the FP64 kernel for rows of up to 2048 points,
// 128 threads, takes up to 168 registers at the three CTAs per SM its shared
// memory allows anyway, instead of spilling at 128)
template <typename T, int PPT, int MODE, int MAXT = ROW_MAX_THREADS, int MINB = 1>
__global__ void __launch_bounds__(MAXT, MINB) adj_row_kernel(AdjRowArgs<T> a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int nx = 1 << a.log2nx, n = nx >> 1, log2n = a.log2nx - 1;
    const int row = blockIdx.x, inst = blockIdx.y;
    const int bl = row_buf_len(n);
    cx<T>* U = reinterpret_cast<cx<T>*>(smem_raw);
    cx<T>* M = U + bl;
    cx<T>* G = M + bl;
    T* spl = reinterpret_cast<T*>(G + bl);
    T* spr = spl + 2 * nthr;
    const long long base = (long long)inst * a.inst_stride + (long long)row * n;
    const Tw<T> tw{a.tws, nullptr, -1};

    const T* urow = a.u + 2 * base;
    for (int i = tid; i < n; i += nthr) {
        st_real<T, true>(U, 2 * i, __ldcg(urow + 2 * i));
        st_real<T, true>(U, 2 * i + 1, __ldcg(urow + 2 * i + 1));
        M[padx(i)] = __ldcg(a.m + base + i);
    }
    __syncthreads();
    c2r_pre<T, true>(M, n, a.tw, tid, nthr);
    __syncthreads();
    fft_batched<T, PPT, false, true, true>(M, log2n, 0, 1, 0, tw, tid, nthr);

    const int Q = nx / nthr >= 4 ? nx / nthr : 4;
    const int nact = nx / Q;
    const int k0 = tid * Q;
    WenoCoef<T> wc = a.wc;
    if (a.med_coef) {
        const double cj = 2.0 * 3.14159265358979323846 * __ldg(a.med_coef + 3 * row);
        wc.c = (T)cj;
        wc.alpha = (T)(fabs(cj) + (double)a.wc.alpha);
    }
    if (tid < nact) weno_row_chunk_T<T>(U, M, G, spl + 2 * tid, spr + 3 * tid, nx, k0, Q, wc);
    __syncthreads();
    if (tid < nact) {
        const int left = (tid + nact - 1) % nact, right = (tid + 1) % nact;
        // neighbours' spills: right spill of the left neighbour covers k0..k0+2,
        // left spill of the right neighbour covers k0+Q-2, k0+Q-1
        for (int s = 0; s < 3; s++) st_real<T, true>(G, k0 + s, ld_real<T, true>(G, k0 + s) + spr[3 * left + s]);
        st_real<T, true>(G, k0 + Q - 2, ld_real<T, true>(G, k0 + Q - 2) + spl[2 * right + 0]);
        st_real<T, true>(G, k0 + Q - 1, ld_real<T, true>(G, k0 + Q - 1) + spl[2 * right + 1]);
    }
    __syncthreads();
    if (a.yT) {
        const T* yrow = a.yT + 2 * base;
        for (int k = tid; k < nx; k += nthr) st_real<T, true>(G, k, ld_real<T, true>(G, k) + __ldcg(yrow + k));
        __syncthreads();
    }
    fft_batched<T, PPT, false, false, true>(G, log2n, 0, 1, 0, tw, tid, nthr);
    // (A(sigma) - A) k_tau^2 = dA kscale^2 k^2, k^2 an exact integer
    const T dAk = a.dA * a.kscale * a.kscale;
    for (int k = tid; k <= n / 2; k += nthr) {
        cx<T> xk, xnk;
        r2c_post_pair<T, true>(G, n, k, a.tw, xk, xnk);
        xk = scale<T>(xk, a.inv_nx);
        xnk = scale<T>(xnk, a.inv_nx);
        const cx<T> mk0 = __ldcg(a.m + base + k);
        const cx<T> lk = __ldcg(a.l + base + k);
        if (k == 0) {
            xk.y -= dAk * T((long long)n * n) * mk0.y;
            a.out[base] = add<T>(lk, xk);
        } else {
            const T f = dAk * T((long long)k * k);
            xk.x = fma(-f, mk0.x, xk.x);
            xk.y = fma(-f, mk0.y, xk.y);
            a.out[base + k] = add<T>(lk, xk);
            if (2 * k != n) {
                const T g = dAk * T((long long)(n - k) * (n - k));
                const cx<T> mk2 = __ldcg(a.m + base + n - k);
                xnk.x = fma(-g, mk2.x, xnk.x);
                xnk.y = fma(-g, mk2.y, xnk.y);
                a.out[base + n - k] = add<T>(__ldcg(a.l + base + n - k), xnk);
            }
        }
    }
}

template <typename T>
size_t adj_row_smem_bytes(int n, int nthr)
{
    return 3 * (size_t)row_buf_len(n) * sizeof(cx<T>) + 5 * (size_t)nthr * sizeof(T);
}

enum AdjColMode { ADJ_COL_2 = 0, ADJ_COL_1 = 1 };

template <typename T>
struct AdjColArgs {
    const cx<T>* a;     // ADJ_COL_2: lam';  ADJ_COL_1: lam*
    const cx<T>* b;     // ADJ_COL_1: mu2
    cx<T>* out;         // ADJ_COL_2: mu2;   ADJ_COL_1: lam_lin (may alias a)
    cx<T>* out2;        // ADJ_COL_1: nu1
    const cx<T>* Ta;    // ADJ_COL_2: P2';   ADJ_COL_1: E'
    const cx<T>* Tb;    // ADJ_COL_1: P1'
    T sa, sb;           // rescale of conj(Ta), conj(Tb)
    const cx<T>* tw;    // staged twiddles of the length-ny FFT
    int log2ny, log2n, log2tc;
    long long inst_stride;
};

// conj(M) (real for the packed column) applied to value z of a column-FFT'd
// tile; zm is the value at row ny - l (used by the packed column m = 0).
template <typename T>
__device__ __forceinline__ cx<T> conj_mult_entry(cx<T> M, cx<T> z, cx<T> zm, bool packed)
{
    if (!packed) return mulc<T>(z, M);
    const T h = T(0.5) * (M.x + M.y), g = T(0.5) * (M.x - M.y);
    return mk<T>(fma(h, z.x, g * zm.x), fma(h, z.y, -(g * zm.y)));
}

// ADJ_COL_2: out = IFFT(sa conj(Ta) FFT(a)).
// ADJ_COL_1: z = FFT(a); out = IFFT(sa conj(Ta) z); out2 = IFFT(sb conj(Tb) z) - b.
// Same tile organisation as the forward column kernel: padded tiles (two for
// ADJ_COL_1), staged twiddles in shared memory, packed column 0 by pairs.
template <typename T, int PPT, int MODE>
__global__ void __launch_bounds__(col_max_threads<T>(), sizeof(T) == 4 ? 2 : 1) adj_col_kernel(AdjColArgs<T> a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cx<T>* S = reinterpret_cast<cx<T>*>(smem_raw);
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int ny = 1 << a.log2ny, n = 1 << a.log2n, TC = 1 << a.log2tc;
    const int m0 = blockIdx.x * TC, inst = blockIdx.y;
    const long long ibase = (long long)inst * a.inst_stride;
    const int total = ny << a.log2tc;
    cx<T>* tws = reinterpret_cast<cx<T>*>(smem_raw + col_tile_area<T>(ny, a.log2tc, nthr));
    for (int i = tid; i < ny; i += nthr) tws[i] = a.tw[i];
    const Tw<T> tw{tws, nullptr, -1};
    cx<T>* SA = S;
    cx<T>* SB = S + (total + (total >> 4));
    auto gidx = [&](int e) -> long long {
        return ibase + (long long)(e >> a.log2tc) * n + m0 + (e & (TC - 1));
    };

    for (int e = tid; e < total; e += nthr) SA[padx(e)] = __ldcg(a.a + gidx(e));
    __syncthreads();
    fft_batched<T, PPT, true, false, true, false>(SA, a.log2ny, a.log2tc, TC, 1, tw, tid, nthr);
    for (int e = tid; e < total; e += nthr) {
        const int l = e >> a.log2tc, c = e & (TC - 1), m = m0 + c;
        if (m == 0) continue;
        const int lf = l <= (ny >> 1) ? l : ny - l;
        const long long ti = (long long)lf * n + m;
        const cx<T> z = SA[padx(e)];
        if constexpr (MODE == ADJ_COL_1) SB[padx(e)] = mulc<T>(z, scale<T>(a.Tb[ti], a.sb));
        SA[padx(e)] = mulc<T>(z, scale<T>(a.Ta[ti], a.sa));
    }
    if (m0 == 0) {
        for (int l = tid; l <= (ny >> 1); l += nthr) {
            const int lm = (ny - l) & (ny - 1);
            const long long ti = (long long)l * n;
            const int e = padx(l << a.log2tc), em = padx(lm << a.log2tc);
            const cx<T> z = SA[e], zm = SA[em];
            if constexpr (MODE == ADJ_COL_1) {
                const cx<T> Mb = scale<T>(a.Tb[ti], a.sb);
                SB[e] = conj_mult_entry<T>(Mb, z, zm, true);
                if (lm != l) SB[em] = conj_mult_entry<T>(Mb, zm, z, true);
            }
            const cx<T> Ma = scale<T>(a.Ta[ti], a.sa);
            SA[e] = conj_mult_entry<T>(Ma, z, zm, true);
            if (lm != l) SA[em] = conj_mult_entry<T>(Ma, zm, z, true);
        }
    }
    __syncthreads();
    fft_batched<T, PPT, true, true, true, false>(SA, a.log2ny, a.log2tc, TC, 1, tw, tid, nthr);
    if constexpr (MODE == ADJ_COL_1)
        fft_batched<T, PPT, true, true, true, false>(SB, a.log2ny, a.log2tc, TC, 1, tw, tid, nthr);
    for (int e = tid; e < total; e += nthr) {
        const long long g = gidx(e);
        a.out[g] = SA[padx(e)];
        if constexpr (MODE == ADJ_COL_1) a.out2[g] = sub<T>(SB[padx(e)], __ldcg(a.b + g));
    }
}

}  // namespace kzk
