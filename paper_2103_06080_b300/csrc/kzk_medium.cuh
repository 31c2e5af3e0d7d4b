// kzk_medium.cuh -- the random velocity field of Algorithm 1 at one sigma,
// for every row y_j: U_par, U_perp and d U_perp / dy.
//
// With K_n . (sigma, y) lambda = a_n sigma + c_n y (a_n = |K_n| lambda
// cos theta_n, c_n = |K_n| lambda sin theta_n), each mode is
// Re P_nj with P_nj = exp(i (a_n sigma + phi_n)) exp(i c_n y_j): the second
// factor is a plan-time table (FP64, [N][ny]), the first is computed once per
// mode and sigma, so a stage costs one complex product and three FMAs per
// (mode, row) instead of a sine and a cosine:
//   U_par  = sum_n -|U~_n| sin(theta_n) Re P_nj
//   U_perp = sum_n  |U~_n| cos(theta_n) Re P_nj
//   d U_perp / dy = sum_n -|U~_n| cos(theta_n) c_n Im P_nj.
// All in FP64 (the coefficients feed both plan precisions).
#pragma once
#include "kzk_common.cuh"
#include "kzk_weno.cuh"
#include "kzk_adjoint.cuh"

namespace kzk {

constexpr int MED_ROWS = 32;       // rows per CTA
constexpr int MED_GROUPS = 16;     // mode groups per CTA (threads = MED_ROWS * MED_GROUPS)
constexpr int MED_MAX_MODES = 1024;

struct MedArgs {
    const double2* Ty;      // [N][ny]: exp(i c_n y_j)
    const double* a_sig;    // [N]: |K_n| lambda cos(theta_n)
    const double* phase;    // [N]: phi_n
    const double* w;        // [3][N]: -|U~_n| sin(theta_n), |U~_n| cos(theta_n), -|U~_n| cos(theta_n) c_n
    int n_modes, ny;
    double sigma;
    const double* sig;      // nullable: sigma read from device memory (replayed graphs)
    double* coef;           // [ny][3]: U_par, U_perp, d U_perp / dy
    double* bmax;           // [gridDim.x]: max |U_perp| over the CTA's rows
};

__global__ void __launch_bounds__(MED_ROWS * MED_GROUPS) medium_kernel(MedArgs a)
{
    __shared__ double2 eA[MED_MAX_MODES];
    __shared__ double red[3][MED_GROUPS][MED_ROWS];
    __shared__ double mx[MED_ROWS];
    const int tid = threadIdx.x, nthr = blockDim.x;
    for (int n = tid; n < a.n_modes; n += nthr) {
        double s, c;
        sincos(fma(a.a_sig[n], a.sig ? __ldg(a.sig) : a.sigma, a.phase[n]), &s, &c);
        eA[n] = make_double2(c, s);
    }
    __syncthreads();
    const int r = tid % MED_ROWS, g = tid / MED_ROWS;
    const int j = blockIdx.x * MED_ROWS + r;
    double s1 = 0.0, s2 = 0.0, s3 = 0.0;
    if (j < a.ny) {
        const double* w0 = a.w;
        const double* w1 = a.w + a.n_modes;
        const double* w2 = a.w + 2 * a.n_modes;
        for (int n = g; n < a.n_modes; n += MED_GROUPS) {
            const double2 t = __ldg(a.Ty + (long long)n * a.ny + j), e = eA[n];
            const double pr = fma(t.x, e.x, -t.y * e.y), pi = fma(t.x, e.y, t.y * e.x);
            s1 = fma(__ldg(w0 + n), pr, s1);
            s2 = fma(__ldg(w1 + n), pr, s2);
            s3 = fma(__ldg(w2 + n), pi, s3);
        }
    }
    red[0][g][r] = s1;
    red[1][g][r] = s2;
    red[2][g][r] = s3;
    __syncthreads();
    if (g == 0) {
        double t1 = 0.0, t2 = 0.0, t3 = 0.0;
        for (int q = 0; q < MED_GROUPS; q++) { t1 += red[0][q][r]; t2 += red[1][q][r]; t3 += red[2][q][r]; }
        if (j < a.ny) {
            a.coef[3 * j] = t1;
            a.coef[3 * j + 1] = t2;
            a.coef[3 * j + 2] = t3;
        }
        mx[r] = j < a.ny ? fabs(t2) : 0.0;
    }
    __syncthreads();
    if (tid == 0) {
        double m = 0.0;
        for (int q = 0; q < MED_ROWS; q++) m = fmax(m, mx[q]);
        a.bmax[blockIdx.x] = m;
    }
}

// ---------------------------------------------------------------------------
// y-flux of the random medium: b_y = -(G_{j+1/2} - G_{j-1/2}) / dy + (d_y U_perp) u
// with G the WENO5 reconstruction of g = U_perp(y) u split by the global
// Lax-Friedrichs speed alpha_y = max_j |U_perp| (Eq. 7 and the text after it).
// One thread per (column k, chunk of Q rows): a sliding window down the
// column, as the tau sweep of weno_row_chunk slides along a row, so every
// interface is reconstructed once; consecutive threads take consecutive
// columns (coalesced row loads).
// ---------------------------------------------------------------------------
template <typename T>
struct YSweepArgs {
    const T* u;              // physical rows [batch][ny][nx]
    T* by;                   // out: b_y [batch][ny][nx]
    const double* coef;      // [ny][3]: U_par, U_perp, d U_perp / dy
    const double* bmax;      // [n_bmax] partial maxima of |U_perp|
    int n_bmax, nx, ny, Q;
    long long inst_elems;    // nx * ny
    T eps, inv_dy;
};

constexpr int YSWEEP_THREADS = 128;

// The y Lax-Friedrichs speed max_j |U_perp(sigma, y_j)| from the medium
// kernel's per-block partial maxima bmax[0, n): each warp takes a strided
// pass and a shuffle reduction (max is exact in any order, so every warp
// gets the same value).  All 32 lanes of the warp must call it.
__device__ __forceinline__ double bmax_all(const double* bmax, int n)
{
    double m = 0.0;
    for (int i = threadIdx.x & 31; i < n; i += 32) m = fmax(m, __ldg(bmax + i));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    return m;
}

// shared memory of one sweep CTA: Q + 7 rows of YSWEEP_THREADS columns, and
// the split-flux factors and source coefficient of those rows
template <typename T>
__host__ __device__ constexpr size_t ysweep_smem(int Q)
{
    return (size_t)(Q + 7) * (YSWEEP_THREADS + 3) * sizeof(T);
}

template <typename T>
__global__ void __launch_bounds__(YSWEEP_THREADS) ysweep_kernel(YSweepArgs<T> a)
{
    extern __shared__ __align__(16) unsigned char ys_smem[];
    const int tid = threadIdx.x;
    const int k0 = blockIdx.x * YSWEEP_THREADS, k = k0 + tid;
    const int j0 = blockIdx.y * a.Q;
    const int ny = a.ny, nx = a.nx;
    const int Q = min(a.Q, ny - j0);
    const int R = Q + 7;                       // rows j0 - 4 .. j0 + Q + 2
    T* tile = reinterpret_cast<T*>(ys_smem);   // [R][YSWEEP_THREADS]
    T* cp = tile + (size_t)R * YSWEEP_THREADS; // [R]: 2 (U_perp + alpha_y)
    T* cm = cp + R;                            // [R]: 2 (U_perp - alpha_y)
    T* dp = cm + R;                            // [R]: d U_perp / dy
    const double ay = bmax_all(a.bmax, a.n_bmax);
    const T* u = a.u + (long long)blockIdx.z * a.inst_elems;
    // the CTA's rows (periodic in y), every load in flight at once
    for (int idx = tid; idx < R * YSWEEP_THREADS; idx += YSWEEP_THREADS) {
        const int r = idx / YSWEEP_THREADS, c = idx % YSWEEP_THREADS;
        const int row = (((j0 - 4 + r) % ny) + ny) % ny;
        tile[idx] = (k0 + c < nx) ? __ldg(u + (long long)row * nx + k0 + c) : T(0);
    }
    for (int r = tid; r < R; r += YSWEEP_THREADS) {
        const int row = (((j0 - 4 + r) % ny) + ny) % ny;
        const double up = __ldg(a.coef + 3 * row + 1);
        cp[r] = (T)(2.0 * (up + ay));
        cm[r] = (T)(2.0 * (up - ay));
        dp[r] = (T)__ldg(a.coef + 3 * row + 2);
    }
    __syncthreads();
    if (k >= nx) return;
    T* by = a.by + (long long)blockIdx.z * a.inst_elems + k;
    // the split fluxes are carried as 4 g+- = 2 (U_perp +- alpha_y) u
    // (indicators with 64 eps, final scale 1/24: see weno_row_chunk)
    const T scale = -a.inv_dy * (T(1) / T(24));
    const T eps4 = T(64) * a.eps;
    auto load = [&](int jj, T& p, T& m) {
        const int r = jj - (j0 - 4);
        const T v = tile[r * YSWEEP_THREADS + tid];
        p = v * cp[r];
        m = v * cm[r];
    };
    // interfaces j0 - 1/2 .. j0 + Q - 1/2; row j gets the flux difference
    // plus the source (d_y U_perp) u
    auto store = [&](int jj, T d) {
        const int r = jj - (j0 - 4);
        by[(long long)jj * nx] = fma(dp[r], tile[r * YSWEEP_THREADS + tid], d);
    };
    weno_sweep<T>(j0, Q, eps4, scale, load, store);
}

// ---------------------------------------------------------------------------
// Transpose of the y part for the adjoint: yT = J_y(u)^T mu + (d_y U_perp) mu,
// J_y the derivative of -(G_{j+1/2} - G_{j-1/2}) / dy.  For each interface
// j' + 1/2 with psi = (mu_{j'+1} - mu_{j'}) / dy the gradients of its two
// reconstructions (weno5_grad) are scattered to rows j'-2 .. j'+3 times
// dg+-/du = (U_perp +- alpha_y) / 2 (alpha_y does not depend on u) through an
// accumulation window that slides down the column; a row is complete once the
// last interface touching it (j' = row + 2) is done.  A thread covers the
// interfaces j0 - 3 .. j0 + Q + 1 of its rows [j0, j0 + Q).
// ---------------------------------------------------------------------------
template <typename T>
struct YSweepTArgs {
    const T* u;              // stage state, physical [batch][ny][nx]
    const T* mu;             // cotangent of b, physical [batch][ny][nx]
    T* yT;                   // out [batch][ny][nx]
    const double* coef;      // [ny][3]: U_par, U_perp, d U_perp / dy
    const double* bmax;      // [n_bmax]
    int n_bmax, nx, ny, Q;
    long long inst_elems;
    T eps, inv_dy;
};

template <typename T>
__host__ __device__ constexpr size_t ysweepT_smem(int Q)
{
    // u rows j0-5 .. j0+Q+4, mu rows j0-3 .. j0+Q+2, per-row factors of the u rows
    return ((size_t)(Q + 10) * (YSWEEP_THREADS + 3) + (size_t)(Q + 6) * YSWEEP_THREADS) * sizeof(T);
}

template <typename T>
__global__ void __launch_bounds__(YSWEEP_THREADS) ysweepT_kernel(YSweepTArgs<T> a)
{
    extern __shared__ __align__(16) unsigned char yt_smem[];
    const int tid = threadIdx.x;
    const int k0 = blockIdx.x * YSWEEP_THREADS, k = k0 + tid;
    const int j0 = blockIdx.y * a.Q;
    const int ny = a.ny, nx = a.nx;
    const int Q = min(a.Q, ny - j0);
    const int Ru = Q + 10, Rm = Q + 6;
    T* tu = reinterpret_cast<T*>(yt_smem);      // [Ru][128]: rows j0-5 ..
    T* tm = tu + (size_t)Ru * YSWEEP_THREADS;   // [Rm][128]: rows j0-3 ..
    T* dgp = tm + (size_t)Rm * YSWEEP_THREADS;  // [Ru]: (U_perp + alpha_y) / 2
    T* dgm = dgp + Ru;                          // [Ru]: (U_perp - alpha_y) / 2
    T* dpr = dgm + Ru;                          // [Ru]: d U_perp / dy
    const double ay = bmax_all(a.bmax, a.n_bmax);
    const T* u = a.u + (long long)blockIdx.z * a.inst_elems;
    const T* mu = a.mu + (long long)blockIdx.z * a.inst_elems;
    for (int idx = tid; idx < Ru * YSWEEP_THREADS; idx += YSWEEP_THREADS) {
        const int r = idx / YSWEEP_THREADS, c = idx % YSWEEP_THREADS;
        const int row = (((j0 - 5 + r) % ny) + ny) % ny;
        tu[idx] = (k0 + c < nx) ? __ldg(u + (long long)row * nx + k0 + c) : T(0);
    }
    for (int idx = tid; idx < Rm * YSWEEP_THREADS; idx += YSWEEP_THREADS) {
        const int r = idx / YSWEEP_THREADS, c = idx % YSWEEP_THREADS;
        const int row = (((j0 - 3 + r) % ny) + ny) % ny;
        tm[idx] = (k0 + c < nx) ? __ldg(mu + (long long)row * nx + k0 + c) : T(0);
    }
    for (int r = tid; r < Ru; r += YSWEEP_THREADS) {
        const int row = (((j0 - 5 + r) % ny) + ny) % ny;
        const double up = __ldg(a.coef + 3 * row + 1);
        dgp[r] = (T)(0.5 * (up + ay));
        dgm[r] = (T)(0.5 * (up - ay));
        dpr[r] = (T)__ldg(a.coef + 3 * row + 2);
    }
    __syncthreads();
    if (k >= nx) return;
    T* out = a.yT + (long long)blockIdx.z * a.inst_elems + k;
    const T eps4 = T(4) * a.eps;
    const T inv_dy6 = a.inv_dy * (T(1) / T(6));
    auto U = [&](int row) { return tu[(row - (j0 - 5)) * YSWEEP_THREADS + tid]; };
    auto M = [&](int row) { return tm[(row - (j0 - 3)) * YSWEEP_THREADS + tid]; };
    // window slot s <-> row j' - 2 + s for interface j' + 1/2
    T gp[6], gm[6], fp[6], fm[6], acc[6];
    int jp = j0 - 3;
#pragma unroll
    for (int s = 0; s < 6; s++) {
        const int r = jp - 2 + s - (j0 - 5);
        const T v = U(jp - 2 + s);
        fp[s] = dgp[r];
        fm[s] = dgm[r];
        gp[s] = fp[s] * v;
        gm[s] = fm[s] * v;
        acc[s] = T(0);
    }
    for (; jp <= j0 + Q + 1; jp++) {
        const T psi6 = (M(jp + 1) - M(jp)) * inv_dy6;
        T gP[5], gM[5];
        weno5_grad<T>(gp[0], gp[1], gp[2], gp[3], gp[4], eps4, psi6, gP);
        weno5_grad<T>(gm[5], gm[4], gm[3], gm[2], gm[1], eps4, psi6, gM);
#pragma unroll
        for (int s = 0; s < 5; s++) acc[s] = fma(gP[s], fp[s], acc[s]);
#pragma unroll
        for (int s = 0; s < 5; s++) acc[5 - s] = fma(gM[s], fm[5 - s], acc[5 - s]);
        const int done = jp - 2;                       // its last interface
        if (done >= j0 && done < j0 + Q)
            out[(long long)done * nx] = fma(dpr[done - (j0 - 5)], M(done), acc[0]);
#pragma unroll
        for (int s = 0; s < 5; s++) {
            gp[s] = gp[s + 1]; gm[s] = gm[s + 1]; fp[s] = fp[s + 1]; fm[s] = fm[s + 1]; acc[s] = acc[s + 1];
        }
        if (jp + 4 <= j0 + Q + 4) {
            const int r = jp + 4 - (j0 - 5);
            const T v = U(jp + 4);
            fp[5] = dgp[r];
            fm[5] = dgm[r];
            gp[5] = fp[5] * v;
            gm[5] = fm[5] * v;
        }
        acc[5] = T(0);
    }
}

}  // namespace kzk
