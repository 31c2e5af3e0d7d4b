// kzk_ysweep_pair.cuh -- the y part of the random medium's flux (Eq. 7, the
// U_perp u component, and the source -d_y U_perp u; Algorithm 1's field) for
// FP32 plans on column pairs.
//
// The same sweep as ysweep_kernel (kzk_medium.cuh): a CTA stages a block of
// rows (its Q rows and a halo of 4 above, 3 below, periodic in y) and each
// thread slides the WENO5 window down its columns, every interface once.
// Here a thread takes two neighbouring columns k, k + 1 as the two lanes of
// packed FP32 values (f2, as the row-pair kernels do), so one FADD2 / FMUL2 /
// FFMA2 does both columns' work; a CTA of YSWEEP_THREADS threads covers
// 2 YSWEEP_THREADS columns, and the rows are loaded and stored as float2.
#pragma once
#include "kzk_medium.cuh"
#include "kzk_rowpair.cuh"

namespace kzk {

// shared memory: Q + 7 rows of 2 YSWEEP_THREADS columns, and the split-flux
// factors and source coefficient of those rows
__host__ __device__ constexpr size_t ysweep_pair_smem(int Q)
{
    return (size_t)(Q + 7) * (2 * YSWEEP_THREADS + 3) * sizeof(float);
}

// nx even (every plan grid is: the real FFT packs nx / 2 pairs)
__global__ void __launch_bounds__(YSWEEP_THREADS) ysweep_pair_kernel(YSweepArgs<float> a)
{
    extern __shared__ __align__(16) unsigned char ysp_smem[];
    const int tid = threadIdx.x;
    const int k0 = blockIdx.x * 2 * YSWEEP_THREADS, k = k0 + 2 * tid;
    const int j0 = blockIdx.y * a.Q;
    const int ny = a.ny, nx = a.nx;
    const int Q = min(a.Q, ny - j0);
    const int R = Q + 7;                                 // rows j0 - 4 .. j0 + Q + 2
    float2* tile = reinterpret_cast<float2*>(ysp_smem);  // [R][YSWEEP_THREADS] column pairs
    float* cp = reinterpret_cast<float*>(tile + (size_t)R * YSWEEP_THREADS);   // [R]: 2 (U_perp + alpha_y)
    float* cm = cp + R;                                  // [R]: 2 (U_perp - alpha_y)
    float* dp = cm + R;                                  // [R]: d U_perp / dy
    const double ay = bmax_all(a.bmax, a.n_bmax);
    const float* u = a.u + (long long)blockIdx.z * a.inst_elems;
    // this thread's column pair of the CTA's rows (periodic in y), loads
    // issued in batches of 8 before they are stored
    const bool live = k < nx;
    for (int r0 = 0; r0 < R; r0 += 8) {
        float2 v[8];
#pragma unroll
        for (int q = 0; q < 8; q++) {
            const int r = r0 + q;
            const int row = (((j0 - 4 + r) % ny) + ny) % ny;
            v[q] = (live && r < R) ? __ldg(reinterpret_cast<const float2*>(u + (long long)row * nx + k))
                                   : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int q = 0; q < 8; q++)
            if (r0 + q < R) tile[(r0 + q) * YSWEEP_THREADS + tid] = v[q];
    }
    for (int r = tid; r < R; r += YSWEEP_THREADS) {
        const int row = (((j0 - 4 + r) % ny) + ny) % ny;
        const double up = __ldg(a.coef + 3 * row + 1);
        cp[r] = (float)(2.0 * (up + ay));
        cm[r] = (float)(2.0 * (up - ay));
        dp[r] = (float)__ldg(a.coef + 3 * row + 2);
    }
    __syncthreads();
    if (k >= nx) return;
    float* by = a.by + (long long)blockIdx.z * a.inst_elems + k;
    // split fluxes carried as 4 g+- = 2 (U_perp +- alpha_y) u, as ysweep_kernel
    const f2 scale(-a.inv_dy * (1.0f / 24.0f));
    const f2 eps4(64.0f * a.eps);
    auto load = [&](int jj, f2& p, f2& m) {
        const int r = jj - (j0 - 4);
        const f2 v(tile[r * YSWEEP_THREADS + tid]);
        p = v * f2(cp[r]);
        m = v * f2(cm[r]);
    };
    auto store = [&](int jj, f2 d) {
        const int r = jj - (j0 - 4);
        const f2 res = fma(f2(dp[r]), f2(tile[r * YSWEEP_THREADS + tid]), d);
        *reinterpret_cast<float2*>(by + (long long)jj * nx) = res.v;
    };
    weno_sweep<f2>(j0, Q, eps4, scale, load, store);
}

}  // namespace kzk
