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
        sincos(fma(a.a_sig[n], a.sigma, a.phase[n]), &s, &c);
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

}  // namespace kzk
