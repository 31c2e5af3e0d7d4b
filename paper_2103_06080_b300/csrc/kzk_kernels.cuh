// kzk_kernels.cuh -- row (tau) and column (y) kernels of one ExpRK22 step.
//
// Spectral state layout (device, per instance): V[ny][nx/2] complex, row j
// holding the tau-spectrum of grid row j divided by nx, packed: slot 0 holds
// (F(u)[0], F(u)[nx/2]) / nx, both real for real rows.  Every array of the
// step (V, b1, V*, b2) uses this layout, so a tau-row is contiguous and a
// column tile is a strided band.
//
// One step (Algorithm 2, STEP 1-4) is four passes over HBM:
//   R(V -> b1):       tau-C2R into shared memory, WENO5, tau-R2C     (STEP 1)
//   C1(V, b1 -> V*):  y-FFT of both, V* = E V + dsigma Phi1 b1, y-IFFT (STEP 2)
//   R(V* -> b2):                                                      (STEP 3)
//   C2(V*, b1, b2 -> V): y-FFT of b2 - b1,
//                     V' = V* + IFFT(dsigma Phi2 (b2 - b1))           (STEP 4)
// The last line is STEP 4 rewritten with STEP 2:
//   E V + ds[(Phi1 - Phi2) b1 + Phi2 b2] = V* + ds Phi2 (b2 - b1),
// which needs neither E nor Phi1 again.  The 1/nx, 1/ny normalisations and
// dsigma are folded into the tables (powers of two: exact).
// FP64 plans also carry Sigma = FFT_y(V) / ny between steps (modes COL_FWD,
// COL_S1, COL_S2 below): C1 then transforms only b1 (X = ny E' Sigma + P1' B1,
// T = X - P2' B1 kept, V* = IFFT_y(X)) and C2 only b2 (Sigma' = T + P2' B2,
// V' = IFFT_y(Sigma')), four y-transforms per step instead of five.
#pragma once
#include "kzk_common.cuh"
#include "kzk_fft.cuh"
#include "kzk_weno.cuh"
#include <algorithm>

namespace kzk {

enum RowMode { ROW_RHS = 0, ROW_FWD = 1, ROW_INV = 2, ROW_RHS_MED = 3 };

template <typename T>
struct RowArgs {
    const cx<T>* in;        // ROW_RHS / ROW_INV: spectral rows; ROW_FWD: physical rows (as T)
    cx<T>* out;             // ROW_RHS / ROW_FWD: spectral rows; ROW_INV: physical rows (as T)
    const cx<T>* tw;        // exp(-2 pi i k / nx), k in [0, nx) (real-FFT pre/post-processing)
    const cx<T>* tws;       // staged twiddles of the length-nx/2 complex FFT
    double* diag_rows;      // [batch][ny][4] or nullptr
    int log2nx;
    int ny;
    long long inst_stride;  // complex elements per instance (ny * nx / 2)
    WenoCoef<T> wc;
    T cA;                   // nx * (A(sigma) - A): absorption-deviation term
    T kscale;               // 2 pi / (tau_max - tau_min)
    T out_scale;            // ROW_FWD: 1/nx; ROW_INV: scale of the result
    T* u_out;               // ROW_RHS: also store the physical row here ([batch][ny][nx]; nullable)
    // ROW_RHS_MED (random medium): b from the physical rows, with the tau-flux
    // -2 pi U_par u - B u^2/2, plus the y-flux difference and the source
    // d_y U_perp u computed by ysweep_kernel (Eq. 7 and the text after it)
    const T* uphys;         // physical rows [batch][ny][nx]
    const T* by;            // the y-flux difference and source of every point [batch][ny][nx] (ysweep_kernel)
    const double* med_coef; // [ny][3]: U_par, U_perp, d U_perp / dy at this sigma
    // nullable: this stage's sigma-dependent values from device memory,
    // {sigma, B(sigma), B(sigma) M, nx (A(sigma) - A)} (FP64), in place of
    // wc.B, wc.alpha and cA (launches replayed from a captured graph)
    const double* coef;
};

// The stage's WENO coefficients and absorption-deviation factor (from
// RowArgs::coef when it is set).
template <typename T>
__device__ __forceinline__ WenoCoef<T> stage_wc(const RowArgs<T>& a)
{
    WenoCoef<T> w = a.wc;
    if (a.coef) {
        w.B = (T)__ldg(a.coef + 1);
        w.alpha = (T)__ldg(a.coef + 2);
    }
    return w;
}
template <typename T>
__device__ __forceinline__ T stage_cA(const RowArgs<T>& a)
{
    return a.coef ? (T)__ldg(a.coef + 3) : a.cA;
}

// Block reduction of the four diagnostics (FP64 across threads, fixed
// order: deterministic).  blockDim.x must be a power of two; red holds
// 4 * blockDim.x doubles.
__device__ __forceinline__ void block_diag(double* red, double s1, double s2, double mx, double nf,
                                           double* dst)
{
    const int tid = threadIdx.x, nthr = blockDim.x;
    double* r0 = red;
    double* r1 = red + nthr;
    double* r2 = red + 2 * nthr;
    double* r3 = red + 3 * nthr;
    r0[tid] = s1; r1[tid] = s2; r2[tid] = mx; r3[tid] = nf;
    __syncthreads();
    for (int h = nthr >> 1; h > 0; h >>= 1) {
        if (tid < h) {
            r0[tid] += r0[tid + h];
            r1[tid] += r1[tid + h];
            r2[tid] = fmax(r2[tid], r2[tid + h]);
            r3[tid] += r3[tid + h];
        }
        __syncthreads();
    }
    if (tid == 0) { dst[0] = r0[0]; dst[1] = r1[0]; dst[2] = r2[0]; dst[3] = r3[0]; }
    __syncthreads();
}

// Block reduction of one row's statistics: within each warp in the working
// precision (shuffles, fixed order), across warps in FP64 by thread 0 (fixed
// order); red holds one double4 per warp.  Deterministic.
template <typename T>
__device__ __forceinline__ void block_diag_t(double* red, T s1, T s2, T mx, int nf, double* dst)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        nf += __shfl_xor_sync(0xffffffffu, nf, o);
    }
    if (lane == 0) {
        red[4 * warp] = (double)s1; red[4 * warp + 1] = (double)s2;
        red[4 * warp + 2] = (double)mx; red[4 * warp + 3] = (double)nf;
    }
    __syncthreads();
    if (tid == 0) {
        double a = 0, b = 0, c = 0, d = 0;
        for (int w = 0; w < nw; w++) {
            a += red[4 * w]; b += red[4 * w + 1]; c = fmax(c, red[4 * w + 2]); d += red[4 * w + 3];
        }
        dst[0] = a; dst[1] = b; dst[2] = c; dst[3] = d;
    }
}

// block_diag_t split at a barrier the caller has anyway: diag_partial before
// it (shuffles, lane 0 of each warp stores its partials), diag_final after it
// by threads 0..3 (component c summed over the warps in warp order, as
// block_diag_t's thread 0 does): the same results.
template <typename T>
__device__ __forceinline__ void diag_partial(double* red, T s1, T s2, T mx, int nf)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        nf += __shfl_xor_sync(0xffffffffu, nf, o);
    }
    if ((threadIdx.x & 31) == 0) {
        double* r = red + 4 * (threadIdx.x >> 5);
        r[0] = (double)s1; r[1] = (double)s2; r[2] = (double)mx; r[3] = (double)nf;
    }
}
__device__ __forceinline__ void diag_final(const double* red, double* dst)
{
    const int c = threadIdx.x, nw = (blockDim.x + 31) >> 5;
    double v = 0;
    for (int w = 0; w < nw; w++) v = c == 2 ? fmax(v, red[4 * w + c]) : v + red[4 * w + c];
    dst[c] = v;
}

// C2R pre-processing in place: packed half spectrum X (n = nx/2 slots) ->
// Z with IFFT_n(Z) = nx * (x_even + i x_odd), Z_k = (X_k + conj X_{n-k})
// + i conj(W^k) (X_k - conj X_{n-k}), W = exp(-2 pi i / nx).
template <typename T, bool PAD = false>
__device__ __forceinline__ void c2r_pre(cx<T>* X, int n, const cx<T>* __restrict__ tw, int tid, int nthr)
{
    for (int k = tid; k <= n / 2; k += nthr) {
        if (k == 0) {
            const T x0 = X[0].x, xn = X[0].y;
            X[0] = mk<T>(x0 + xn, x0 - xn);
        } else if (2 * k == n) {
            const cx<T> a = X[sidx<PAD>(k)];
            X[sidx<PAD>(k)] = mk<T>(T(2) * a.x, T(-2) * a.y);
        } else {
            const cx<T> a = X[sidx<PAD>(k)], b = X[sidx<PAD>(n - k)];
            const cx<T> w = tw[k];                      // W^k
            const cx<T> s = add<T>(a, conj<T>(b)), d = sub<T>(a, conj<T>(b));
            const cx<T> r = mul_si<T, 1>(mulc<T>(d, w));    // i conj(W^k) d
            // n - k: its s and d are conj(s) and -conj(d), and with
            // conj(W^{n-k}) = -W^k its r is -conj(r): Z_{n-k} = conj(s - r)
            X[sidx<PAD>(k)] = add<T>(s, r);
            X[sidx<PAD>(n - k)] = conj<T>(sub<T>(s, r));
        }
    }
}

// R2C post-processing: Z = FFT_n(x_even + i x_odd) -> packed X = FFT_nx(x),
// X_k = 1/2 [(Z_k + conj Z_{n-k}) - i W^k (Z_k - conj Z_{n-k})].
// Returns the pair (X_k, X_{n-k}) for 0 < k < n/2, handles k = 0 and n/2.
template <typename T, bool PAD = false>
__device__ __forceinline__ void r2c_post_pair_w(const cx<T>* Z, int n, int k, cx<T> wk, cx<T>& Xk, cx<T>& Xnk)
{
    const T h = T(0.5);
    if (k == 0) {
        const cx<T> z = Z[0];
        Xk = mk<T>(z.x + z.y, z.x - z.y);    // (X_0, X_{nx/2}) packed
        Xnk = Xk;
    } else if (2 * k == n) {
        Xk = conj<T>(Z[sidx<PAD>(k)]);
        Xnk = Xk;
    } else {
        const cx<T> a = Z[sidx<PAD>(k)], b = Z[sidx<PAD>(n - k)];
        const cx<T> s = add<T>(a, conj<T>(b)), d = sub<T>(a, conj<T>(b));
        // r = -i W^k d / 2 (the halving exact, on the twiddle): X_k = s/2 + r;
        // n - k: its s and d are conj(s) and -conj(d), and with
        // W^{n-k} = -conj(W^k) its r is -conj(r): X_{n-k} = conj(s/2 - r)
        const cx<T> r = mul_si<T, -1>(mul<T>(scale<T>(wk, h), d));
        Xk = mk<T>(fma(h, s.x, r.x), fma(h, s.y, r.y));
        Xnk = mk<T>(fma(h, s.x, -r.x), fma(-h, s.y, r.y));
    }
}
// the same with the twiddle W^k read from the table (0 <= k <= n/2)
template <typename T, bool PAD = false>
__device__ __forceinline__ void r2c_post_pair(const cx<T>* Z, int n, int k, const cx<T>* __restrict__ tw,
                                              cx<T>& Xk, cx<T>& Xnk)
{
    r2c_post_pair_w<T, PAD>(Z, n, k, tw[k], Xk, Xnk);
}

// Row of n complex values from global memory into a padded shared buffer:
// up to 8 loads per thread are issued before the shared stores, so each
// thread keeps several requests in flight.
template <typename T>
__device__ __forceinline__ void load_row(const cx<T>* __restrict__ src, cx<T>* dst, int n, int tid, int nthr)
{
    int i = tid;
    for (; i + 7 * nthr < n; i += 8 * nthr) {
        cx<T> v[8];
#pragma unroll
        for (int q = 0; q < 8; q++) v[q] = __ldcg(src + i + q * nthr);
#pragma unroll
        for (int q = 0; q < 8; q++) dst[padx(i + q * nthr)] = v[q];
    }
    for (; i < n; i += nthr) dst[padx(i)] = __ldcg(src + i);
}

// Padded length of one row buffer (n complex + one slot per 16).
__host__ __device__ constexpr int row_buf_len(int n) { return n + (n >> 4); }

// points per thread in the row FFTs (FP32: 16, radix-16 passes; FP64: 8,
// radix-8 passes, which keeps a double-complex butterfly in registers)
template <typename T> __host__ __device__ constexpr int row_ppt_of() { return 8; }
constexpr int ROW_MAX_THREADS = 512; // n / 8 for nx = 8192

// Row kernel.  One CTA per (row, instance), n / PPT threads (at least 32).
// Shared memory: two padded buffers of n complex (= nx reals) each, plus a
// reduction area of 4 doubles per thread.
// Body of one row task, run by all nthr = blockDim.x threads of a CTA
// (nthr may exceed n / PPT; extra threads idle through the barriers).
// State arrays are read with L2-coherent loads (__ldcg) so that the body is
// also correct inside one persistent launch, where they are rewritten by
// other CTAs between passes.
// LOG2N > 0 (ROW_RHS only): the body for rows of nx = 2^(LOG2N + 1) points run
// by 2^LOG2N / 8 threads (LOG2N >= 8): lengths, thread count, transform
// schedule and WENO chunks are compile-time constants.
template <typename T, int MODE, int LOG2N = 0>
__device__ __forceinline__ void row_body(const RowArgs<T>& a, int row, int inst, unsigned char* smem_raw)
{
    static_assert(LOG2N == 0 || (MODE == ROW_RHS && LOG2N >= 8), "length-specialised b passes only");
    constexpr bool CT = LOG2N > 0;
    const int tid = threadIdx.x, nthr = CT ? (1 << LOG2N) / 8 : blockDim.x;
    const int nx = CT ? 2 << LOG2N : 1 << a.log2nx, n = nx >> 1, log2n = CT ? LOG2N : a.log2nx - 1;
    cx<T>* X = reinterpret_cast<cx<T>*>(smem_raw);       // buffer U
    cx<T>* Y = X + row_buf_len(n);                         // buffer B
    double* red = reinterpret_cast<double*>(Y + row_buf_len(n));
    const long long base = (long long)inst * a.inst_stride + (long long)row * n;
    const Tw<T> tw{a.tws, nullptr, -1};
    constexpr int ROW_PPT = row_ppt_of<T>();

    if constexpr (MODE == ROW_FWD) {
        // physical row -> packed half spectrum / nx
        const cx<T>* src = a.in + base;                   // physical pairs (x_2i, x_2i+1)
        load_row<T>(src, Y, n, tid, nthr);
        __syncthreads();
        fft_batched<T, ROW_PPT, false, false, true>(Y, log2n, 0, 1, 0, tw, tid, nthr);
        for (int k = tid; k <= n / 2; k += nthr) {
            cx<T> xk, xnk;
            r2c_post_pair<T, true>(Y, n, k, a.tw, xk, xnk);
            a.out[base + k] = scale<T>(xk, a.out_scale);
            if (k != 0 && 2 * k != n) a.out[base + n - k] = scale<T>(xnk, a.out_scale);
        }
    } else {
        // U: the physical row (the WENO sweep's input), Bf: the sweep's output
        // and the forward transform's buffer.  The b passes run their
        // transforms out of place between the two (one barrier per pass), so
        // which buffer holds what depends on the number of passes.
        cx<T>* U = X;
        cx<T>* Bf = Y;
        if constexpr (MODE == ROW_RHS_MED) {
            // the physical row, written by the ROW_INV pass of this stage
            const T* urow = a.uphys + 2 * base;
            for (int i = tid; i < nx; i += nthr) st_real<T, true>(X, i, __ldcg(urow + i));
            __syncthreads();
        } else {
            // spectral row -> physical row
            load_row<T>(a.in + base, X, n, tid, nthr);
            __syncthreads();
            c2r_pre<T, true>(X, n, a.tw, tid, nthr);
            __syncthreads();
            if constexpr (CT) {
                U = fft_batched_pp_ct<T, ROW_PPT, false, true, true, false, LOG2N>(X, Y, tw, tid, nthr);
                Bf = U == X ? Y : X;
            } else if constexpr (MODE == ROW_RHS) {
                U = fft_batched_pp<T, ROW_PPT, false, true, true>(X, Y, log2n, 0, 1, 0, tw, tid, nthr);
                Bf = U == X ? Y : X;
            } else {
                fft_batched<T, ROW_PPT, false, true, true>(X, log2n, 0, 1, 0, tw, tid, nthr);
            }
        }

        T s1 = 0, s2 = 0, mx = 0;
        int nf = 0;
        if constexpr (MODE == ROW_INV) {
            T* dst = reinterpret_cast<T*>(a.out + base);
            for (int i = tid; i < nx; i += nthr) {
                const T v = ld_real<T, true>(X, i) * a.out_scale;
                dst[i] = v;
                if (isfinite(v)) { s1 += v; s2 = fma(v, v, s2); mx = fmax(mx, fabs(v)); } else { nf++; }
            }
            if (a.diag_rows) block_diag_t<T>(red, s1, s2, mx, nf, a.diag_rows + ((long long)inst * a.ny + row) * 4);
        } else {
            // ROW_RHS: WENO5 flux derivative into Y, then tau-R2C of Y
            if (a.u_out) {
                // the stage state in physical space, for the adjoint sweep
                T* dst = a.u_out + 2 * base;
                for (int i = tid; i < nx; i += nthr) dst[i] = ld_real<T, true>(U, i);
            }
            // chunks of at least 16 points (the sweep's pre-roll is 3 centres)
            const int Q = nx / nthr >= 16 ? nx / nthr : (nx >= 16 ? 16 : nx);
            const int k0 = tid * Q;
            if (k0 < nx) {
                WenoCoef<T> wc = stage_wc(a);
                if constexpr (MODE == ROW_RHS_MED) {
                    // this row's advection speed c = 2 pi U_par and LF speed |c| + B M
                    const double cj = 2.0 * 3.14159265358979323846 * __ldg(a.med_coef + 3 * row);
                    wc.alpha = (T)(fabs(cj) + (double)wc.alpha);
                    wc.c = (T)cj;
                    weno_row_chunk<T, true, true>(U, Bf, nx, k0, Q, wc);
                } else {
                    weno_row_chunk<T, true, false, true, CT>(U, Bf, nx, k0, Q, wc);
                }
                if (a.diag_rows) row_stats<T, true, CT>(U, k0, Q, s1, s2, mx, nf);
            }
            // the row statistics reduced across the barrier that ends the sweep
            if (a.diag_rows) diag_partial<T>(red, s1, s2, mx, nf);
            __syncthreads();
            if (a.diag_rows && tid < 4) diag_final(red, a.diag_rows + ((long long)inst * a.ny + row) * 4);
            if constexpr (MODE == ROW_RHS_MED) {
                // plus the y-flux difference and source of this row
                const T* byrow = a.by + 2 * base;
                for (int k = tid; k < nx; k += nthr) st_real<T, true>(Bf, k, ld_real<T, true>(Bf, k) + __ldcg(byrow + k));
                __syncthreads();
            }
            const cx<T>* Z;
            if constexpr (CT) Z = fft_batched_pp_ct<T, ROW_PPT, false, false, true, false, LOG2N>(Bf, U, tw, tid, nthr);
            else Z = fft_batched_pp<T, ROW_PPT, false, false, true>(Bf, U, log2n, 0, 1, 0, tw, tid, nthr);
            const cx<T>* vin = a.in + base;
            const T cA = stage_cA(a);
            // nx (A(sigma) - A) k_tau^2 = cA kscale^2 k^2, k^2 an exact integer
            const T cAk = cA * a.kscale * a.kscale;
            for (int k = tid; k <= n / 2; k += nthr) {
                cx<T> xk, xnk;
                r2c_post_pair<T, true>(Z, n, k, a.tw, xk, xnk);
                if (cA != T(0)) {
                    // b_hat -= nx (A(sigma) - A) k_tau^2 V   (V = F(u)/nx)
                    if (k == 0) {
                        xk.y -= cAk * T((long long)n * n) * __ldcg(vin).y;
                    } else {
                        const T f = cAk * T((long long)k * k);
                        const cx<T> v = __ldcg(vin + k);
                        xk.x = fma(-f, v.x, xk.x);
                        xk.y = fma(-f, v.y, xk.y);
                        if (2 * k != n) {
                            const T g = cAk * T((long long)(n - k) * (n - k));
                            const cx<T> w = __ldcg(vin + n - k);
                            xnk.x = fma(-g, w.x, xnk.x);
                            xnk.y = fma(-g, w.y, xnk.y);
                        }
                    }
                }
                a.out[base + k] = xk;
                if (k != 0 && 2 * k != n) a.out[base + n - k] = xnk;
            }
        }
    }
}

template <typename T, int MODE, int LOG2N = 0>
__global__ void __launch_bounds__(ROW_MAX_THREADS, sizeof(T) == 4 ? 2 : 1) row_kernel(RowArgs<T> a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    row_body<T, MODE, LOG2N>(a, blockIdx.x, blockIdx.y, smem_raw);
}

// Threads and dynamic shared memory of one row CTA.
template <typename T>
__host__ __forceinline__ int row_threads(int nx)
{
    return (nx / 2) / row_ppt_of<T>() > 32 ? (nx / 2) / row_ppt_of<T>() : 32;
}
template <typename T>
__host__ __forceinline__ size_t row_smem_bytes(int nx)
{
    return 2 * (size_t)row_buf_len(nx / 2) * sizeof(cx<T>) + 4 * (size_t)row_threads<T>(nx) * sizeof(double);
}

// STAGE1 / STAGE2: the two column passes of a step on the tau-spectral state
// V (five y-transforms per step).  FWD, S1, S2 (FP64 plans on the per-tile
// kernels): the same step with the state's normalised y-spectrum
// Sigma = FFT_y(V) / ny carried between steps, so stage 1 no longer
// transforms V (four y-transforms per step):
//   FWD: Sigma = FFT_y(V) / ny                      (once per loaded state)
//   S1:  B1 = FFT_y(b1);  X = ny E' Sigma + P1' B1;  T = X - P2' B1;
//        V* = IFFT_y(X), and T kept                 (STEP 2, Eq. 11)
//   S2:  B2 = FFT_y(b2);  Sigma' = T + P2' B2;  V' = IFFT_y(Sigma')
//                                                   (STEP 4: E V + ds[(Phi1 - Phi2) b1 + Phi2 b2])
enum ColMode { COL_STAGE1 = 0, COL_STAGE2 = 1, COL_FWD = 2, COL_S1 = 3, COL_S2 = 4 };

template <typename T>
struct ColArgs {
    const cx<T>* a;         // STAGE1: V;    STAGE2: b1
    const cx<T>* b;         // STAGE1: b1;   STAGE2: b2
    const cx<T>* c;         // STAGE1: -;    STAGE2: V*
    cx<T>* out;             // STAGE1: V*;   STAGE2: V'
    const cx<T>* Ta;        // STAGE1: E';   STAGE2: P2'
    const cx<T>* Ta_lo;     // STAGE1, FP32: lo part of E' (hi + lo = FP64 value)
    const cx<T>* Tb;        // STAGE1: P1';  STAGE2: -
    const cx<T>* tw;        // staged twiddles of the length-ny FFT
    const cx<T>* tw_lo;     // FP32: lo parts of tw
    int log2ny, log2n, log2tc;
    long long inst_stride;
    // diagnostics of the step (STAGE1, CTA x = 0 of each instance)
    const double* diag_rows;  // [batch][ny][4] or nullptr
    double* diag_hist;        // [batch][4] for this step
    double inv_count, cell;   // 1/(nx ny), dtau dy
    // compensated state (FP32 plans): the state is the pair hi + lo; STAGE1
    // takes lo of V (hi: a) and writes lo of V* (hi: out), with Ta = (E - 1)/ny
    // so that the transforms carry only the increment; STAGE2 takes lo of V*
    // (hi: c) and writes lo of V' (hi: out).  nullptr: plain state.
    const lo_t<T>* lo_in;
    lo_t<T>* lo_out;
    // y-spectral state (modes FWD, S1, S2): the second output (S1: T, S2:
    // Sigma'), S1's third table (P2'), and the power-of-two scale (FWD: 1/ny,
    // S1: ny)
    cx<T>* out2;
    const cx<T>* Tc;
    T yscale;
};

// Table entry at (l, m) applied to a column-FFT'd value z (zm: the value at
// row ny - l of the same column, used only by the packed column m = 0, which
// holds the tau-DC sequence in its real part and the tau-Nyquist one in its
// imaginary part; their spectra are separated through the pair (l, ny - l)
// and each is multiplied by its own real table entry).
template <typename T>
__device__ __forceinline__ cx<T> mult_entry(cx<T> M, cx<T> z, cx<T> zm, bool packed)
{
    if (!packed) return mul<T>(M, z);
    const T h = T(0.5) * (M.x + M.y), g = T(0.5) * (M.x - M.y);
    // explicit fused forms: every kernel that inlines this rounds alike
    return mk<T>(fma(h, z.x, g * zm.x), fma(h, z.y, -(g * zm.y)));
}

template <typename T> __host__ __device__ constexpr int col_ppt_of() { return 8; }
template <typename T> __host__ __device__ constexpr int col_max_threads() { return 512; }
// shared memory for the two tiles of stage 1: small enough that two CTAs
// (plus their twiddle copies) share an SM, so one CTA's loads overlap the
// other's transforms
constexpr size_t COL_TILE_BYTES = 64 * 1024;

// bytes of the tile area (or of the diagnostics reduction area, if larger)
template <typename T>
__host__ __device__ __forceinline__ size_t col_tile_area(int ny, int log2tc, int nthr)
{
    const size_t e = (size_t)ny << log2tc;
    const size_t tiles = 2 * (e + (e >> 4)) * sizeof(cx<T>);
    const size_t red = 4 * (size_t)nthr * sizeof(double);
    return tiles > red ? tiles : red;
}

constexpr int COL_MAX_THREADS = 1024;

// Column kernel.  One CTA per (tile of TC columns, instance).
//  STAGE1 (STEP 2): shared memory holds two tiles [ny][2 TC]: columns [0, TC)
//    the state V, [TC, 2 TC) b1.  FFT both along y (the state's transform
//    with two-float constants in FP32), combine E' V + P1' b1 into the state
//    half, inverse FFT it (two-float again) and store V*.  Compensated FP32
//    state (lo_out set): Ta = (E - 1)', and the result is the increment,
//    added to V = a + lo_in by TwoSum into V* = out + lo_out.
//  STAGE2 (STEP 4): one tile of b2 - b1, FFT, times P2', inverse FFT, plus V*.
// Body of one column-tile task (tile index `tile`), run by all nthr =
// blockDim.x threads of a CTA (nthr * PPT >= ny * TC).
template <typename T, int MODE>
__device__ __forceinline__ void col_body(const ColArgs<T>& a, int tile, int inst, unsigned char* smem_raw)
{
    cx<T>* S = reinterpret_cast<cx<T>*>(smem_raw);
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int ny = 1 << a.log2ny, n = 1 << a.log2n, TC = 1 << a.log2tc;
    const int m0 = tile * TC;
    const long long ibase = (long long)inst * a.inst_stride;
    const int total = ny << a.log2tc;                   // elements of one tile
    constexpr bool ACC = sizeof(T) == 4;
    constexpr int COL_PPT = col_ppt_of<T>();
    // y twiddles in shared memory after the tile area
    cx<T>* tws = reinterpret_cast<cx<T>*>(smem_raw + col_tile_area<T>(ny, a.log2tc, nthr));
    cx<T>* twl = tws + ny;
    for (int i = tid; i < ny; i += nthr) {
        tws[i] = a.tw[i];
        if constexpr (ACC) twl[i] = a.tw_lo[i];
    }
    const Tw<T> twp{tws, nullptr, -1};
    const Tw<T> twa{tws, twl, -1};

    auto gidx = [&](int e) -> long long {
        return ibase + (long long)(e >> a.log2tc) * n + m0 + (e & (TC - 1));
    };
    // tile element e = l * TC + c lives at padx(e) of its region (one padding
    // slot per 16 elements: conflict-free strided Stockham stores)
    cx<T>* SA = S;                                  // state / b2 - b1 tile
    cx<T>* SB = S + (total + (total >> 4));         // b1 tile (stage 1)

    if constexpr (MODE == COL_STAGE1) {
        // diagnostics of the state this step started from (rows written by R)
        if (tile == 0 && a.diag_rows && a.diag_hist) {
            double* red = reinterpret_cast<double*>(smem_raw);
            double s1 = 0, s2 = 0, mx = 0, nf = 0;
            const double* dr = a.diag_rows + (long long)inst * ny * 4;
            for (int r = tid; r < ny; r += nthr) {
                s1 += __ldcg(dr + 4 * r); s2 += __ldcg(dr + 4 * r + 1);
                mx = fmax(mx, __ldcg(dr + 4 * r + 2)); nf += __ldcg(dr + 4 * r + 3);
            }
            double tmp[4];
            block_diag(red, s1, s2, mx, nf, tmp);
            if (tid == 0) {
                double* d = a.diag_hist + inst * 4;
                d[0] = tmp[0] * a.inv_count;
                d[1] = tmp[1] * a.cell;
                d[2] = tmp[2];
                d[3] = tmp[3];
            }
        }
        {
            int e = tid;
            for (; e + 3 * nthr < total; e += 4 * nthr) {
                cx<T> va[4], vb[4];
#pragma unroll
                for (int q = 0; q < 4; q++) { va[q] = __ldcg(a.a + gidx(e + q * nthr)); vb[q] = __ldcg(a.b + gidx(e + q * nthr)); }
#pragma unroll
                for (int q = 0; q < 4; q++) { SA[padx(e + q * nthr)] = va[q]; SB[padx(e + q * nthr)] = vb[q]; }
            }
            for (; e < total; e += nthr) {
                const long long g = gidx(e);
                SA[padx(e)] = __ldcg(a.a + g);
                SB[padx(e)] = __ldcg(a.b + g);
            }
        }
        __syncthreads();
        // state tile: accurate transform; b1 tile: plain
        fft_batched<T, COL_PPT, true, false, true, ACC>(SA, a.log2ny, a.log2tc, TC, 1, twa, tid, nthr);
        fft_batched<T, COL_PPT, true, false, true, false>(SB, a.log2ny, a.log2tc, TC, 1, twp, tid, nthr);
        // V*_hat = E' V_hat + P1' b1_hat, in place in the state tile.  Every
        // element is combined by its owner; the packed column 0 (first tile
        // only) couples rows l and ny - l, so one thread owns each such pair.
        for (int e = tid; e < total; e += nthr) {
            const int l = e >> a.log2tc, c = e & (TC - 1), m = m0 + c;
            if (m == 0) continue;
            const int lf = l <= (ny >> 1) ? l : ny - l;
            const long long ti = (long long)lf * n + m;
            const cx<T> zv = SA[padx(e)], zb = SB[padx(e)];
            cx<T> r = mul<T>(a.Ta[ti], zv);
            if constexpr (ACC) {
                if (a.Ta_lo) r = fma_c<T>(a.Ta_lo[ti], zv, r);
            }
            SA[padx(e)] = fma_c<T>(a.Tb[ti], zb, r);
        }
        if (m0 == 0) {
            for (int l = tid; l <= (ny >> 1); l += nthr) {
                const int lm = (ny - l) & (ny - 1);
                const long long ti = (long long)l * n;        // l <= ny/2: folded row l
                const int e = padx(l << a.log2tc), em = padx(lm << a.log2tc);
                const cx<T> zv = SA[e], zvm = SA[em], zb = SB[e], zbm = SB[em];
                cx<T> r = mult_entry<T>(a.Ta[ti], zv, zvm, true);
                cx<T> rm = mult_entry<T>(a.Ta[ti], zvm, zv, true);
                if (ACC && a.Ta_lo) {
                    r = add<T>(r, mult_entry<T>(a.Ta_lo[ti], zv, zvm, true));
                    rm = add<T>(rm, mult_entry<T>(a.Ta_lo[ti], zvm, zv, true));
                }
                r = add<T>(r, mult_entry<T>(a.Tb[ti], zb, zbm, true));
                rm = add<T>(rm, mult_entry<T>(a.Tb[ti], zbm, zb, true));
                SA[e] = r;
                if (lm != l) SA[em] = rm;
            }
        }
        __syncthreads();
        fft_batched<T, COL_PPT, true, true, true, ACC>(SA, a.log2ny, a.log2tc, TC, 1, twa, tid, nthr);
        if (a.lo_out) {
            // the transforms carried the increment: V* = V + increment, compensated
            for (int e = tid; e < total; e += nthr) {
                const long long g = gidx(e);
                cx<T> h, l;
                comp_add<T>(__ldcg(a.a + g), lo_load<T>(a.lo_in + g), SA[padx(e)], h, l);
                a.out[g] = h;
                lo_store<T>(a.lo_out + g, l);
            }
        } else {
            for (int e = tid; e < total; e += nthr) a.out[gidx(e)] = SA[padx(e)];
        }
    } else if constexpr (MODE == COL_FWD) {
        // Sigma = FFT_y(V) / ny of a loaded state
        {
            int e = tid;
            for (; e + 3 * nthr < total; e += 4 * nthr) {
                cx<T> va[4];
#pragma unroll
                for (int q = 0; q < 4; q++) va[q] = __ldcg(a.a + gidx(e + q * nthr));
#pragma unroll
                for (int q = 0; q < 4; q++) SA[padx(e + q * nthr)] = va[q];
            }
            for (; e < total; e += nthr) SA[padx(e)] = __ldcg(a.a + gidx(e));
        }
        __syncthreads();
        fft_batched<T, COL_PPT, true, false, true, false>(SA, a.log2ny, a.log2tc, TC, 1, twp, tid, nthr);
        for (int e = tid; e < total; e += nthr) a.out[gidx(e)] = scale<T>(SA[padx(e)], a.yscale);
    } else if constexpr (MODE == COL_S1 || MODE == COL_S2) {
        if constexpr (MODE == COL_S1) {
            // diagnostics of the state this step started from (rows written by R)
            if (tile == 0 && a.diag_rows && a.diag_hist) {
                double* red = reinterpret_cast<double*>(smem_raw);
                double s1 = 0, s2 = 0, mx = 0, nf = 0;
                const double* dr = a.diag_rows + (long long)inst * ny * 4;
                for (int r = tid; r < ny; r += nthr) {
                    s1 += __ldcg(dr + 4 * r); s2 += __ldcg(dr + 4 * r + 1);
                    mx = fmax(mx, __ldcg(dr + 4 * r + 2)); nf += __ldcg(dr + 4 * r + 3);
                }
                double tmp[4];
                block_diag(red, s1, s2, mx, nf, tmp);
                if (tid == 0) {
                    double* d = a.diag_hist + inst * 4;
                    d[0] = tmp[0] * a.inv_count;
                    d[1] = tmp[1] * a.cell;
                    d[2] = tmp[2];
                    d[3] = tmp[3];
                }
            }
        }
        // SA: the y-spectral tile (S1: Sigma, S2: T); SB: the b tile
        {
            int e = tid;
            for (; e + 3 * nthr < total; e += 4 * nthr) {
                cx<T> va[4], vb[4];
#pragma unroll
                for (int q = 0; q < 4; q++) { va[q] = __ldcg(a.a + gidx(e + q * nthr)); vb[q] = __ldcg(a.b + gidx(e + q * nthr)); }
#pragma unroll
                for (int q = 0; q < 4; q++) { SA[padx(e + q * nthr)] = va[q]; SB[padx(e + q * nthr)] = vb[q]; }
            }
            for (; e < total; e += nthr) {
                const long long g = gidx(e);
                SA[padx(e)] = __ldcg(a.a + g);
                SB[padx(e)] = __ldcg(a.b + g);
            }
        }
        __syncthreads();
        fft_batched<T, COL_PPT, true, false, true, false>(SB, a.log2ny, a.log2tc, TC, 1, twp, tid, nthr);
        for (int e = tid; e < total; e += nthr) {
            const int l = e >> a.log2tc, c = e & (TC - 1), m = m0 + c;
            if (m == 0) continue;
            const int lf = l <= (ny >> 1) ? l : ny - l;
            const long long ti = (long long)lf * n + m;
            const cx<T> zs = SA[padx(e)], zb = SB[padx(e)];
            cx<T> r;
            if constexpr (MODE == COL_S1) {
                r = fma_c<T>(a.Tb[ti], zb, scale<T>(mul<T>(a.Ta[ti], zs), a.yscale));
                const cx<T> t = a.Tc[ti];
                a.out2[gidx(e)] = fma_c<T>(mk<T>(-t.x, -t.y), zb, r);
            } else {
                r = fma_c<T>(a.Ta[ti], zb, zs);
                a.out2[gidx(e)] = r;
            }
            SA[padx(e)] = r;
        }
        if (m0 == 0) {
            // the packed column 0 couples rows l and ny - l (see mult_entry)
            for (int l = tid; l <= (ny >> 1); l += nthr) {
                const int lm = (ny - l) & (ny - 1);
                const long long ti = (long long)l * n;
                const int e = padx(l << a.log2tc), em = padx(lm << a.log2tc);
                const cx<T> zs = SA[e], zsm = SA[em], zb = SB[e], zbm = SB[em];
                cx<T> r, rm;
                if constexpr (MODE == COL_S1) {
                    r = add<T>(scale<T>(mult_entry<T>(a.Ta[ti], zs, zsm, true), a.yscale),
                               mult_entry<T>(a.Tb[ti], zb, zbm, true));
                    rm = add<T>(scale<T>(mult_entry<T>(a.Ta[ti], zsm, zs, true), a.yscale),
                                mult_entry<T>(a.Tb[ti], zbm, zb, true));
                    a.out2[gidx(l << a.log2tc)] = sub<T>(r, mult_entry<T>(a.Tc[ti], zb, zbm, true));
                    if (lm != l) a.out2[gidx(lm << a.log2tc)] = sub<T>(rm, mult_entry<T>(a.Tc[ti], zbm, zb, true));
                } else {
                    r = add<T>(zs, mult_entry<T>(a.Ta[ti], zb, zbm, true));
                    rm = add<T>(zsm, mult_entry<T>(a.Ta[ti], zbm, zb, true));
                    a.out2[gidx(l << a.log2tc)] = r;
                    if (lm != l) a.out2[gidx(lm << a.log2tc)] = rm;
                }
                SA[e] = r;
                if (lm != l) SA[em] = rm;
            }
        }
        __syncthreads();
        fft_batched<T, COL_PPT, true, true, true, false>(SA, a.log2ny, a.log2tc, TC, 1, twp, tid, nthr);
        for (int e = tid; e < total; e += nthr) a.out[gidx(e)] = SA[padx(e)];
    } else {
        {
            int e = tid;
            for (; e + 3 * nthr < total; e += 4 * nthr) {
                cx<T> va[4], vb[4];
#pragma unroll
                for (int q = 0; q < 4; q++) { va[q] = __ldcg(a.a + gidx(e + q * nthr)); vb[q] = __ldcg(a.b + gidx(e + q * nthr)); }
#pragma unroll
                for (int q = 0; q < 4; q++) SA[padx(e + q * nthr)] = sub<T>(vb[q], va[q]);
            }
            for (; e < total; e += nthr) {
                const long long g = gidx(e);
                SA[padx(e)] = sub<T>(__ldcg(a.b + g), __ldcg(a.a + g));
            }
        }
        __syncthreads();
        fft_batched<T, COL_PPT, true, false, true, false>(SA, a.log2ny, a.log2tc, TC, 1, twp, tid, nthr);
        for (int e = tid; e < total; e += nthr) {
            const int l = e >> a.log2tc, c = e & (TC - 1), m = m0 + c;
            if (m == 0) continue;
            const int lf = l <= (ny >> 1) ? l : ny - l;
            SA[padx(e)] = mul<T>(a.Ta[(long long)lf * n + m], SA[padx(e)]);
        }
        if (m0 == 0) {
            for (int l = tid; l <= (ny >> 1); l += nthr) {
                const int lm = (ny - l) & (ny - 1);
                const cx<T> M = a.Ta[(long long)l * n];
                const int e = padx(l << a.log2tc), em = padx(lm << a.log2tc);
                const cx<T> z = SA[e], zm = SA[em];
                SA[e] = mult_entry<T>(M, z, zm, true);
                if (lm != l) SA[em] = mult_entry<T>(M, zm, z, true);
            }
        }
        __syncthreads();
        fft_batched<T, COL_PPT, true, true, true, false>(SA, a.log2ny, a.log2tc, TC, 1, twp, tid, nthr);
        if (a.lo_out) {
            for (int e = tid; e < total; e += nthr) {
                const long long g = gidx(e);
                cx<T> h, l;
                comp_add<T>(__ldcg(a.c + g), lo_load<T>(a.lo_in + g), SA[padx(e)], h, l);
                a.out[g] = h;
                lo_store<T>(a.lo_out + g, l);
            }
        } else {
            int e = tid;
            for (; e + 3 * nthr < total; e += 4 * nthr) {
                cx<T> vc[4];
#pragma unroll
                for (int q = 0; q < 4; q++) vc[q] = __ldcg(a.c + gidx(e + q * nthr));
#pragma unroll
                for (int q = 0; q < 4; q++) a.out[gidx(e + q * nthr)] = add<T>(vc[q], SA[padx(e + q * nthr)]);
            }
            for (; e < total; e += nthr) {
                const long long g = gidx(e);
                a.out[g] = add<T>(__ldcg(a.c + g), SA[padx(e)]);
            }
        }
    }
}

template <typename T, int MODE>
__global__ void __launch_bounds__(col_max_threads<T>(), (sizeof(T) == 4 && MODE == COL_STAGE2) ? 2 : 1)
    col_kernel(ColArgs<T> a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    col_body<T, MODE>(a, blockIdx.x, blockIdx.y, smem_raw);
}

// Column tile width (log2) and threads: STAGE1 holds two tiles of
// ny x TC complex in at most 128 KB, with TC * ny / COL_PPT <= 512 threads.
template <typename T>
__host__ __forceinline__ int col_log2tc(int nx, int ny)
{
    int tc = std::min(16, nx / 2);
    while (tc > 1 && (2 * (size_t)ny * tc * sizeof(cx<T>) > COL_TILE_BYTES ||
                      (long long)ny * tc / col_ppt_of<T>() > col_max_threads<T>()))
        tc >>= 1;
    int l = 0;
    while ((1 << l) < tc) ++l;
    return l;
}
template <typename T>
__host__ __forceinline__ int col_threads(int ny, int log2tc)
{
    const long long t = ((long long)ny << log2tc) / col_ppt_of<T>();
    return t > 32 ? (int)t : 32;
}
// tiles (or the diagnostics reduction area, if larger), then the y twiddles
// (hi, and lo for FP32) copied to shared memory
template <typename T>
__host__ __forceinline__ size_t col_smem_bytes(int ny, int log2tc)
{
    return col_tile_area<T>(ny, log2tc, col_threads<T>(ny, log2tc)) + (sizeof(T) == 4 ? 2 : 1) * (size_t)ny * sizeof(cx<T>);
}

// Final diagnostics of each instance from its per-row partials.
static __global__ void diag_reduce_kernel(const double* __restrict__ rows, int ny, double inv_count, double cell,
                                   double* __restrict__ out)
{
    __shared__ double red[4 * 256];
    const int tid = threadIdx.x, inst = blockIdx.x;
    double s1 = 0, s2 = 0, mx = 0, nf = 0;
    const double* dr = rows + (long long)inst * ny * 4;
    for (int r = tid; r < ny; r += blockDim.x) {
        s1 += dr[4 * r]; s2 += dr[4 * r + 1]; mx = fmax(mx, dr[4 * r + 2]); nf += dr[4 * r + 3];
    }
    red[tid] = s1; red[256 + tid] = s2; red[512 + tid] = mx; red[768 + tid] = nf;
    __syncthreads();
    for (int h = blockDim.x >> 1; h > 0; h >>= 1) {
        if (tid < h) {
            red[tid] += red[tid + h];
            red[256 + tid] += red[256 + tid + h];
            red[512 + tid] = fmax(red[512 + tid], red[512 + tid + h]);
            red[768 + tid] += red[768 + tid + h];
        }
        __syncthreads();
    }
    if (tid == 0) {
        out[inst * 4 + 0] = red[0] * inv_count;
        out[inst * 4 + 1] = red[256] * cell;
        out[inst * 4 + 2] = red[512];
        out[inst * 4 + 3] = red[768];
    }
}

}  // namespace kzk
