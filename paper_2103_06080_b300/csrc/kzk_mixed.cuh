// kzk_mixed.cuh -- the ExpRK22 step on grids whose sizes are not powers of
// two.  The paper's grids (Table 1) have 7 * 2^k points in retarded time and
// 1250 * 2^k = 2^(k+1) * 5^4 transverse points.
//
// Transforms of such lengths run in place in shared memory as mixed-radix
// Cooley-Tukey passes of radix 2, 3, 4, 5, 7 or 8:
//  * forward: decimation in frequency -- natural order in, digit-reversed
//    order out.  Pass q splits every sub-transform of span L into R groups of
//    m = L / R: the R elements j, j + m, .., j + (R - 1) m of a block go
//    through a DFT of size R and output s is multiplied by exp(-2 pi i j s / L);
//  * inverse: decimation in time, the same passes in reverse order, each the
//    conjugate transpose of its forward pass -- digit-reversed order in,
//    natural order out.
// Each pass combines disjoint groups of R elements where they lie, so the
// threads of a CTA loop over their groups with one barrier per pass and no
// second buffer.  The digit-reversed order never leaves shared memory: the tau
// rows apply the real-FFT pre-/post-processing and the y columns apply the
// diagonal propagators (indexed by frequency) directly in that order, through
// plan-time tables of the position of every frequency.
//
// The step itself is the one of kzk_kernels.cuh (four passes over the state,
// Algorithm 2), except that the first column pass is split in two: the y
// column of a 7 * 2^k x 10^4 grid no longer fits shared memory twice, so
//   MIX_C1B: W = P1' FFT_y(b1)                                   (scratch)
//   MIX_C1V: V* = IFFT_y(E' FFT_y(V) + W)
// and the second column pass is unchanged:
//   MIX_C2:  V' = V* + IFFT_y(P2' FFT_y(b2 - b1)).
// The transposed step (the adjoint) has its row pass (mix_adj_row_kernel)
// and column passes (mix_adj_col_kernel) on the same transforms; its
// two-output column pass is split the same way, through the same scratch.
#pragma once
#include "kzk_adjoint.cuh"
#include "kzk_kernels.cuh"

namespace kzk {

constexpr int MIX_MAX_PASSES = 16;

// Radix schedule of one transform length (forward pass order).
struct MixFFT {
    int n;                       // transform length
    int np;                      // passes
    int R[MIX_MAX_PASSES];       // radix of pass q
    int m[MIX_MAX_PASSES];       // distance between the R elements of a group (span L = m R)
    int ts[MIX_MAX_PASSES];      // exp(-2 pi i j s / L) = tw[j s ts] in the plan's twiddle table
};

// Host: radix schedule of length n (odd radices first, then radix 8, then one
// 4 or 2) for a twiddle table exp(-2 pi i k / (n tmul)).  False if n has a
// prime factor above 7 or needs too many passes.
inline bool mix_plan(int n, int tmul, MixFFT* f)
{
    f->n = n;
    f->np = 0;
    int rest = n, L = n;
    auto add = [&](int R) {
        if (f->np >= MIX_MAX_PASSES) return false;
        f->R[f->np] = R;
        f->m[f->np] = L / R;
        f->ts[f->np] = (n / L) * tmul;
        f->np++;
        L /= R;
        rest /= R;
        return true;
    };
    const int odd[3] = {7, 5, 3};
    for (int R : odd)
        while (rest % R == 0)
            if (!add(R)) return false;
    while (rest % 8 == 0)
        if (!add(8)) return false;
    if (rest % 4 == 0) {
        if (!add(4)) return false;
    } else if (rest % 2 == 0) {
        if (!add(2)) return false;
    }
    return rest == 1 && n >= 1;
}

// Host: position of frequency k in the output of the forward passes (the
// mixed-radix digit reversal): its digits k = s_0 + R_0 (s_1 + R_1 (...))
// select group s_q of pass q, at offset s_q m_q.
inline int mix_position(const MixFFT& f, int k)
{
    int p = 0;
    for (int q = 0; q < f.np; q++) {
        p += (k % f.R[q]) * f.m[q];
        k /= f.R[q];
    }
    return p;
}

// cos and sin of 2 pi q / R for the odd radices, q = 1 .. (R - 1) / 2
__host__ __device__ constexpr double cos_odd(int R, int q)
{
    return R == 3 ? -0.5
         : R == 5 ? (q == 1 ? 0.3090169943749474241023 : -0.8090169943749474241023)
                  : (q == 1 ? 0.6234898018587335305251 : q == 2 ? -0.2225209339563144042889 : -0.9009688679024191262361);
}
__host__ __device__ constexpr double sin_odd(int R, int q)
{
    return R == 3 ? 0.8660254037844386467637
         : R == 5 ? (q == 1 ? 0.9510565162951535721164 : 0.5877852522924731291687)
                  : (q == 1 ? 0.7818314824680298087084 : q == 2 ? 0.9749279121818236070181 : 0.4338837391175581204758);
}

// acc + x * C for a real constant C (ACC, float: C as a two-float hi + lo)
template <typename T, bool ACC>
__device__ __forceinline__ cx<T> fma_rc(cx<T> x, double C, cx<T> acc)
{
    const T hi = (T)C;
    if constexpr (ACC && sizeof(T) == 4) {
        const T lo = (T)(C - (double)hi);
        return mk<T>(fma(x.x, hi, fma(x.x, lo, acc.x)), fma(x.y, hi, fma(x.y, lo, acc.y)));
    } else {
        return mk<T>(fma(x.x, hi, acc.x), fma(x.y, hi, acc.y));
    }
}

// In-register DFT of odd prime size R, sign S, natural order in and out.
// With a_j = x_j + x_{R-j}, b_j = x_j - x_{R-j} (j = 1 .. (R-1)/2):
//   X_k     = C_k + S i D_k,   X_{R-k} = C_k - S i D_k,
//   C_k = x_0 + sum_j a_j cos(2 pi j k / R),  D_k = sum_j b_j sin(2 pi j k / R).
template <typename T, int R, int S, bool ACC>
__device__ __forceinline__ void odd_dft(cx<T>* v)
{
    constexpr int H = (R - 1) / 2;
    cx<T> a[H], b[H];
    cx<T> sum = v[0];
#pragma unroll
    for (int j = 1; j <= H; j++) {
        a[j - 1] = add<T>(v[j], v[R - j]);
        b[j - 1] = sub<T>(v[j], v[R - j]);
        sum = add<T>(sum, a[j - 1]);
    }
    const cx<T> x0 = v[0];
#pragma unroll
    for (int k = 1; k <= H; k++) {
        cx<T> C = x0, D = mk<T>(T(0), T(0));
#pragma unroll
        for (int j = 1; j <= H; j++) {
            const int q = (j * k) % R;
            const double c = q <= H ? cos_odd(R, q) : cos_odd(R, R - q);
            const double s = q <= H ? sin_odd(R, q) : -sin_odd(R, R - q);
            C = fma_rc<T, ACC>(a[j - 1], c, C);
            D = fma_rc<T, ACC>(b[j - 1], s, D);
        }
        const cx<T> iD = mul_si<T, S>(D);
        v[k] = add<T>(C, iD);
        v[R - k] = sub<T>(C, iD);
    }
    v[0] = sum;
}

template <typename T, int R, int S, bool ACC>
__device__ __forceinline__ void small_dft(cx<T>* v)
{
    if constexpr (R == 2 || R == 4 || R == 8) RegDFT<T, R, S, ACC>::run(v);
    else odd_dft<T, R, S, ACC>(v);
}

// One pass of radix R over a tile of 2^lc interleaved transforms (element i
// of transform c at buf[i 2^lc + c]).  Ends with a barrier.
template <typename T, int R, bool INV, bool ACC>
__device__ __forceinline__ void mix_pass(cx<T>* buf, int n, int lc, int m, int ts, const cx<T>* __restrict__ tw,
                                         const cx<T>* __restrict__ twl, int tid, int nthr)
{
    constexpr int S = INV ? 1 : -1;
    const int total = (n / R) << lc;
    const int cm = (1 << lc) - 1;
    const int step = m << lc;
    for (int u = tid; u < total; u += nthr) {
        const int c = u & cm, t = u >> lc;
        const int blk = t / m, j = t - blk * m;
        const int base = ((blk * m * R + j) << lc) + c;
        cx<T> v[R];
#pragma unroll
        for (int r = 0; r < R; r++) v[r] = buf[base + r * step];
        if constexpr (INV) {
#pragma unroll
            for (int s = 1; s < R; s++) {
                const int ti = j * s * ts;
                const cx<T> w = __ldg(tw + ti);
                if constexpr (ACC && sizeof(T) == 4) v[s] = fma_c<T>(v[s], conj<T>(__ldg(twl + ti)), mulc<T>(v[s], w));
                else v[s] = mulc<T>(v[s], w);
            }
            small_dft<T, R, S, ACC>(v);
        } else {
            small_dft<T, R, S, ACC>(v);
#pragma unroll
            for (int s = 1; s < R; s++) {
                const int ti = j * s * ts;
                const cx<T> w = __ldg(tw + ti);
                if constexpr (ACC && sizeof(T) == 4) v[s] = fma_c<T>(v[s], __ldg(twl + ti), mul<T>(v[s], w));
                else v[s] = mul<T>(v[s], w);
            }
        }
#pragma unroll
        for (int r = 0; r < R; r++) buf[base + r * step] = v[r];
    }
    __syncthreads();
}

template <typename T, bool INV, bool ACC>
__device__ __forceinline__ void mix_pass_any(cx<T>* buf, const MixFFT& f, int q, int lc, const cx<T>* tw,
                                             const cx<T>* twl, int tid, int nthr)
{
    switch (f.R[q]) {
    case 2: mix_pass<T, 2, INV, ACC>(buf, f.n, lc, f.m[q], f.ts[q], tw, twl, tid, nthr); break;
    case 3: mix_pass<T, 3, INV, ACC>(buf, f.n, lc, f.m[q], f.ts[q], tw, twl, tid, nthr); break;
    case 4: mix_pass<T, 4, INV, ACC>(buf, f.n, lc, f.m[q], f.ts[q], tw, twl, tid, nthr); break;
    case 5: mix_pass<T, 5, INV, ACC>(buf, f.n, lc, f.m[q], f.ts[q], tw, twl, tid, nthr); break;
    case 7: mix_pass<T, 7, INV, ACC>(buf, f.n, lc, f.m[q], f.ts[q], tw, twl, tid, nthr); break;
    default: mix_pass<T, 8, INV, ACC>(buf, f.n, lc, f.m[q], f.ts[q], tw, twl, tid, nthr); break;
    }
}

// Forward transform (natural -> digit-reversed) and inverse transform
// (digit-reversed -> natural) of a tile; the data must be in place (and a
// barrier passed) on entry; both end with a barrier.  Unnormalised.
template <typename T, bool ACC>
__device__ __forceinline__ void mix_forward(cx<T>* buf, const MixFFT& f, int lc, const cx<T>* tw, const cx<T>* twl,
                                         int tid, int nthr)
{
    for (int q = 0; q < f.np; q++) mix_pass_any<T, false, ACC>(buf, f, q, lc, tw, twl, tid, nthr);
}
template <typename T, bool ACC>
__device__ __forceinline__ void mix_inverse(cx<T>* buf, const MixFFT& f, int lc, const cx<T>* tw, const cx<T>* twl,
                                         int tid, int nthr)
{
    for (int q = f.np - 1; q >= 0; q--) mix_pass_any<T, true, ACC>(buf, f, q, lc, tw, twl, tid, nthr);
}

// ---------------------------------------------------------------------------
// Real-FFT packing of a tau row (the same formulas as c2r_pre / r2c_post_pair,
// on values): n = nx / 2 complex points, w = exp(-2 pi i k / nx).
// ---------------------------------------------------------------------------

// Packed half spectrum X_k, X_{n-k} -> Z_k, Z_{n-k} with IFFT_n(Z) the row's
// even / odd samples as real / imaginary parts.
template <typename T>
__device__ __forceinline__ void c2r_vals(cx<T> a, cx<T> b, cx<T> w, int k, int n, cx<T>& zk, cx<T>& znk)
{
    if (k == 0) {
        zk = mk<T>(a.x + a.y, a.x - a.y);
        znk = zk;
    } else if (2 * k == n) {
        zk = mk<T>(T(2) * a.x, T(-2) * a.y);
        znk = zk;
    } else {
        const cx<T> s = add<T>(a, conj<T>(b)), d = sub<T>(a, conj<T>(b));
        const cx<T> r = mul_si<T, 1>(mulc<T>(d, w));
        zk = add<T>(s, r);
        znk = conj<T>(sub<T>(s, r));              // n - k: conj(s - r), as in c2r_pre
    }
}

// Z_k, Z_{n-k} of FFT_n(even + i odd) -> packed X_k, X_{n-k}.
template <typename T>
__device__ __forceinline__ void r2c_vals(cx<T> a, cx<T> b, cx<T> w, int k, int n, cx<T>& xk, cx<T>& xnk)
{
    const T h = T(0.5);
    if (k == 0) {
        xk = mk<T>(a.x + a.y, a.x - a.y);
        xnk = xk;
    } else if (2 * k == n) {
        xk = conj<T>(a);
        xnk = xk;
    } else {
        const cx<T> s = add<T>(a, conj<T>(b)), d = sub<T>(a, conj<T>(b));
        const cx<T> r = mul_si<T, -1>(mul<T>(scale<T>(w, h), d));   // as in r2c_post_pair
        xk = mk<T>(fma(h, s.x, r.x), fma(h, s.y, r.y));
        xnk = mk<T>(fma(h, s.x, -r.x), fma(-h, s.y, r.y));
    }
}

// ---------------------------------------------------------------------------
// Row kernel (tau): one CTA per (row, instance); the modes of row_kernel.
// ---------------------------------------------------------------------------

template <typename T>
struct MixRowArgs {
    RowArgs<T> r;           // as for power-of-two rows (log2nx unused; tws unused)
    int nx;
    MixFFT f;               // length nx / 2 on the table r.tw = exp(-2 pi i k / nx) (stride 2)
    const int* pos;         // [nx / 2]: position of frequency k after the forward passes
};

constexpr int MIX_ROW_MAX_THREADS = 512;

// threads of one row CTA (a multiple of 32; about 16 tau points each)
__host__ __forceinline__ int mix_row_threads(int nx)
{
    int t = (nx / 16 + 31) / 32 * 32;
    return t < 64 ? 64 : (t > MIX_ROW_MAX_THREADS ? MIX_ROW_MAX_THREADS : t);
}
template <typename T>
__host__ __forceinline__ size_t mix_row_smem(int nx, int nthr)
{
    return 2 * (size_t)(nx / 2) * sizeof(cx<T>) + 4 * (size_t)((nthr + 31) / 32) * sizeof(double);
}

template <typename T, int MODE>
__global__ void __launch_bounds__(MIX_ROW_MAX_THREADS) mix_row_kernel(MixRowArgs<T> A)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const RowArgs<T>& a = A.r;
    const int row = blockIdx.x, inst = blockIdx.y;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int nx = A.nx, n = nx >> 1;
    cx<T>* X = reinterpret_cast<cx<T>*>(smem_raw);       // the row u (physical) / its transform
    cx<T>* Y = X + n;                                     // b
    double* red = reinterpret_cast<double*>(Y + n);
    const long long base = (long long)inst * a.inst_stride + (long long)row * n;
    const int* pos = A.pos;

    if constexpr (MODE == ROW_FWD) {
        const cx<T>* src = a.in + base;                   // physical pairs (x_2i, x_2i+1)
        for (int i = tid; i < n; i += nthr) X[i] = __ldcg(src + i);
        __syncthreads();
        mix_forward<T, false>(X, A.f, 0, a.tw, nullptr, tid, nthr);
        for (int k = tid; k <= n / 2; k += nthr) {
            const int kn = k == 0 ? 0 : n - k;
            cx<T> xk, xnk;
            r2c_vals<T>(X[__ldg(pos + k)], X[__ldg(pos + kn)], __ldg(a.tw + k), k, n, xk, xnk);
            a.out[base + k] = scale<T>(xk, a.out_scale);
            if (k != 0 && 2 * k != n) a.out[base + n - k] = scale<T>(xnk, a.out_scale);
        }
        return;
    }
    // The row loops below take this thread's indices in batches of RB, all
    // loads of a batch issued before the first is used (one load in flight
    // per thread left these passes waiting on latency).
    constexpr int RB = 4;
    if constexpr (MODE == ROW_RHS_MED) {
        const T* urow = a.uphys + 2 * base;
        for (int i0 = tid; i0 < nx; i0 += RB * nthr) {
            T v[RB];
#pragma unroll
            for (int q = 0; q < RB; q++) v[q] = i0 + q * nthr < nx ? __ldcg(urow + i0 + q * nthr) : T(0);
#pragma unroll
            for (int q = 0; q < RB; q++)
                if (i0 + q * nthr < nx) st_real<T, false>(X, i0 + q * nthr, v[q]);
        }
        __syncthreads();
    } else {
        // spectral row -> Z in digit-reversed order -> inverse passes
        const cx<T>* vin = a.in + base;
        for (int k0 = tid; k0 <= n / 2; k0 += RB * nthr) {
            cx<T> vk[RB], vn[RB];
#pragma unroll
            for (int q = 0; q < RB; q++) {
                const int k = k0 + q * nthr;
                if (k <= n / 2) {
                    vk[q] = __ldcg(vin + k);
                    vn[q] = __ldcg(vin + (k == 0 ? 0 : n - k));
                }
            }
#pragma unroll
            for (int q = 0; q < RB; q++) {
                const int k = k0 + q * nthr;
                if (k > n / 2) break;
                const int kn = k == 0 ? 0 : n - k;
                cx<T> zk, znk;
                c2r_vals<T>(vk[q], vn[q], __ldg(a.tw + k), k, n, zk, znk);
                X[__ldg(pos + k)] = zk;
                if (k != 0 && 2 * k != n) X[__ldg(pos + kn)] = znk;
            }
        }
        __syncthreads();
        mix_inverse<T, false>(X, A.f, 0, a.tw, nullptr, tid, nthr);
    }

    T s1 = 0, s2 = 0, mx = 0;
    int nf = 0;
    if constexpr (MODE == ROW_INV) {
        T* dst = reinterpret_cast<T*>(a.out + base);
        for (int i = tid; i < nx; i += nthr) {
            const T v = ld_real<T, false>(X, i) * a.out_scale;
            dst[i] = v;
            if (isfinite(v)) { s1 += v; s2 = fma(v, v, s2); mx = fmax(mx, fabs(v)); } else { nf++; }
        }
        if (a.diag_rows) block_diag_t<T>(red, s1, s2, mx, nf, a.diag_rows + ((long long)inst * a.ny + row) * 4);
        return;
    }
    // ROW_RHS / ROW_RHS_MED: WENO5 into Y, forward passes, packed spectrum out
    if (MODE == ROW_RHS && a.u_out) {
        T* dst = a.u_out + 2 * base;
        for (int i = tid; i < nx; i += nthr) dst[i] = ld_real<T, false>(X, i);
    }
    const int Q = (nx + nthr - 1) / nthr;
    const int k0 = tid * Q;
    if (k0 < nx) {
        const int Qt = min(Q, nx - k0);
        WenoCoef<T> wc = stage_wc(a);
        if constexpr (MODE == ROW_RHS_MED) {
            const double cj = 2.0 * 3.14159265358979323846 * __ldg(a.med_coef + 3 * row);
            wc.alpha = (T)(fabs(cj) + (double)wc.alpha);
            wc.c = (T)cj;
            weno_row_chunk<T, false, true, false>(X, Y, nx, k0, Qt, wc);
        } else {
            weno_row_chunk<T, false, false, false>(X, Y, nx, k0, Qt, wc);
        }
        if (a.diag_rows) row_stats<T, false>(X, k0, Qt, s1, s2, mx, nf);
    }
    __syncthreads();
    if constexpr (MODE == ROW_RHS_MED) {
        const T* byrow = a.by + 2 * base;
        for (int i0 = tid; i0 < nx; i0 += RB * nthr) {
            T v[RB];
#pragma unroll
            for (int q = 0; q < RB; q++) v[q] = i0 + q * nthr < nx ? __ldcg(byrow + i0 + q * nthr) : T(0);
#pragma unroll
            for (int q = 0; q < RB; q++) {
                const int k = i0 + q * nthr;
                if (k < nx) st_real<T, false>(Y, k, ld_real<T, false>(Y, k) + v[q]);
            }
        }
        __syncthreads();
    }
    mix_forward<T, false>(Y, A.f, 0, a.tw, nullptr, tid, nthr);
    const cx<T>* vin = a.in + base;
    const T cA = stage_cA(a);
    for (int k0 = tid; k0 <= n / 2; k0 += RB * nthr) {
        cx<T> vk[RB], vn[RB];
        if (cA != T(0)) {
#pragma unroll
            for (int q = 0; q < RB; q++) {
                const int k = k0 + q * nthr;
                if (k <= n / 2) {
                    vk[q] = __ldcg(vin + k);
                    vn[q] = __ldcg(vin + (k == 0 ? 0 : n - k));
                }
            }
        }
#pragma unroll
        for (int q = 0; q < RB; q++) {
            const int k = k0 + q * nthr;
            if (k > n / 2) break;
            const int kn = k == 0 ? 0 : n - k;
            cx<T> xk, xnk;
            r2c_vals<T>(Y[__ldg(pos + k)], Y[__ldg(pos + kn)], __ldg(a.tw + k), k, n, xk, xnk);
            if (cA != T(0)) {
                // b_hat -= nx (A(sigma) - A) k_tau^2 V   (V = F(u)/nx)
                if (k == 0) {
                    const T kN = a.kscale * T(n);
                    xk.y -= cA * kN * kN * vk[q].y;
                } else {
                    const T kt = a.kscale * T(k);
                    xk.x -= cA * kt * kt * vk[q].x;
                    xk.y -= cA * kt * kt * vk[q].y;
                    if (2 * k != n) {
                        const T kt2 = a.kscale * T(n - k);
                        xnk.x -= cA * kt2 * kt2 * vn[q].x;
                        xnk.y -= cA * kt2 * kt2 * vn[q].y;
                    }
                }
            }
            a.out[base + k] = xk;
            if (k != 0 && 2 * k != n) a.out[base + n - k] = xnk;
        }
    }
    if (a.diag_rows) block_diag_t<T>(red, s1, s2, mx, nf, a.diag_rows + ((long long)inst * a.ny + row) * 4);
}

// ---------------------------------------------------------------------------
// Column kernels (y): one CTA per (tile of 2^lc columns, instance).
// ---------------------------------------------------------------------------

enum MixColMode { MIX_C1B = 0, MIX_C1V = 1, MIX_C2 = 2 };

template <typename T>
struct MixColArgs {
    ColArgs<T> c;           // a, b, c, out, Ta, Ta_lo, Tb, diagnostics as for col_kernel;
                            // tw / tw_lo: exp(-2 pi i k / ny) (hi / lo), k in [0, ny)
    cx<T>* w;               // scratch [batch][ny][nx/2]: P1' FFT_y(b1) in transformed order
    int ny, n, lc;          // column length, columns (nx / 2), log2 of the tile width
    MixFFT f;               // length ny on the table c.tw (stride 1)
    const int* pos;         // [ny]: position of frequency l after the forward passes
    const int* ipos;        // [ny]: frequency at position p
};

constexpr int MIX_COL_THREADS = 512;
// FP32 tiles that hold one CTA per SM (columns of ~10^4 points) run with 1024
// threads: the latency of the strided loads is what bounds them, and their
// registers (<= 64) allow it
template <typename T> __host__ __device__ constexpr int mix_col_max_threads() { return sizeof(T) == 4 ? 1024 : 512; }

// INC: the FP32 compensated state, whose transforms carry only the stage
// increment (R12): plain FP32 constants suffice there, the two-float ones are
// for the transform of a plain FP32 state.
template <typename T, int MODE, bool INC = false>
__global__ void __launch_bounds__(mix_col_max_threads<T>()) mix_col_kernel(MixColArgs<T> A)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cx<T>* S = reinterpret_cast<cx<T>*>(smem_raw);
    const ColArgs<T>& a = A.c;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int ny = A.ny, n = A.n, lc = A.lc, TC = 1 << lc;
    const int tile = blockIdx.x, inst = blockIdx.y;
    const int m0 = tile * TC;
    const long long ibase = (long long)inst * a.inst_stride;
    const int total = ny << lc;
    constexpr bool ACC = (MODE == MIX_C1V) && sizeof(T) == 4 && !INC;
    auto gidx = [&](int e) -> long long { return ibase + (long long)(e >> lc) * n + m0 + (e & (TC - 1)); };

    if (MODE == MIX_C1V && tile == 0 && a.diag_rows && a.diag_hist) {
        // diagnostics of the state this step started from (rows written by R)
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
    // The element loops below take this thread's elements e = tid + i nthr in
    // batches of MU, every load of a batch issued before the first is used:
    // the row segments of a tile are 8- or 16-byte pieces at the pitch of a
    // row, so these passes wait on the latency of their loads, and one load
    // in flight per thread left them there (FP32: ~0.8 TB/s).
    constexpr int MU = sizeof(T) == 4 ? 8 : 4;
    for (int e0 = tid; e0 < total; e0 += MU * nthr) {
        cx<T> v[MU], w[MU];
#pragma unroll
        for (int q = 0; q < MU; q++) {
            const int e = e0 + q * nthr;
            if (e < total) {
                const long long g = gidx(e);
                if (MODE == MIX_C1B) v[q] = __ldcg(a.b + g);
                else if (MODE == MIX_C1V) v[q] = __ldcg(a.a + g);
                else { v[q] = __ldcg(a.b + g); w[q] = __ldcg(a.a + g); }
            }
        }
#pragma unroll
        for (int q = 0; q < MU; q++) {
            const int e = e0 + q * nthr;
            if (e < total) S[e] = MODE == MIX_C2 ? sub<T>(v[q], w[q]) : v[q];
        }
    }
    __syncthreads();
    mix_forward<T, ACC>(S, A.f, lc, a.tw, a.tw_lo, tid, nthr);

    // the diagonal propagator at the frequency of each position; the packed
    // column 0 (first tile only) couples frequencies l and ny - l, so one
    // thread owns each such pair
    for (int e0 = tid; e0 < total; e0 += MU * nthr) {
        // frequency positions, then the table entries (and W) of the batch
        int lq[MU];
#pragma unroll
        for (int q = 0; q < MU; q++) {
            const int e = e0 + q * nthr;
            lq[q] = e < total ? __ldg(A.ipos + (e >> lc)) : 0;
        }
        cx<T> tq[MU], tl[MU], wq[MU];
#pragma unroll
        for (int q = 0; q < MU; q++) {
            const int e = e0 + q * nthr, m = m0 + (e & (TC - 1));
            if (e < total && m != 0) {
                const int l = lq[q];
                const int lf = l <= (ny >> 1) ? l : ny - l;
                const long long ti = (long long)lf * n + m;
                tq[q] = __ldg((MODE == MIX_C1B ? a.Tb : a.Ta) + ti);
                if constexpr (ACC) {
                    if (a.Ta_lo) tl[q] = __ldg(a.Ta_lo + ti);
                }
                if constexpr (MODE == MIX_C1V) wq[q] = __ldcg(A.w + gidx(e));
            }
        }
#pragma unroll
        for (int q = 0; q < MU; q++) {
            const int e = e0 + q * nthr, m = m0 + (e & (TC - 1));
            if (e >= total || m == 0) continue;
            const cx<T> z = S[e];
            if constexpr (MODE == MIX_C1B) {
                A.w[gidx(e)] = mul<T>(tq[q], z);
            } else if constexpr (MODE == MIX_C1V) {
                cx<T> r = mul<T>(tq[q], z);
                if constexpr (ACC) {
                    if (a.Ta_lo) r = fma_c<T>(tl[q], z, r);
                }
                S[e] = add<T>(r, wq[q]);
            } else {
                S[e] = mul<T>(tq[q], z);
            }
        }
    }
    if (m0 == 0) {
        for (int l = tid; l <= (ny >> 1); l += nthr) {
            const int lm = l == 0 ? 0 : ny - l;
            const int e = __ldg(A.pos + l) << lc, em = __ldg(A.pos + lm) << lc;
            const long long ti = (long long)l * n;
            const cx<T> z = S[e], zm = S[em];
            if constexpr (MODE == MIX_C1B) {
                const cx<T> M = __ldg(a.Tb + ti);
                A.w[gidx(e)] = mult_entry<T>(M, z, zm, true);
                if (lm != l) A.w[gidx(em)] = mult_entry<T>(M, zm, z, true);
            } else if constexpr (MODE == MIX_C1V) {
                const cx<T> M = __ldg(a.Ta + ti);
                cx<T> r = mult_entry<T>(M, z, zm, true), rm = mult_entry<T>(M, zm, z, true);
                if (ACC && a.Ta_lo) {
                    const cx<T> Ml = __ldg(a.Ta_lo + ti);
                    r = add<T>(r, mult_entry<T>(Ml, z, zm, true));
                    rm = add<T>(rm, mult_entry<T>(Ml, zm, z, true));
                }
                S[e] = add<T>(r, __ldcg(A.w + gidx(e)));
                if (lm != l) S[em] = add<T>(rm, __ldcg(A.w + gidx(em)));
            } else {
                const cx<T> M = __ldg(a.Ta + ti);
                S[e] = mult_entry<T>(M, z, zm, true);
                if (lm != l) S[em] = mult_entry<T>(M, zm, z, true);
            }
        }
    }
    if constexpr (MODE == MIX_C1B) return;
    __syncthreads();
    mix_inverse<T, ACC>(S, A.f, lc, a.tw, a.tw_lo, tid, nthr);
    for (int e0 = tid; e0 < total; e0 += MU * nthr) {
        // the state hi (and lo) the result is added to, for the batch
        cx<T> hq[MU], lq[MU];
        if (a.lo_out || MODE == MIX_C2) {
#pragma unroll
            for (int q = 0; q < MU; q++) {
                const int e = e0 + q * nthr;
                if (e < total) {
                    const long long g = gidx(e);
                    hq[q] = __ldcg((MODE == MIX_C1V ? a.a : a.c) + g);
                    if (a.lo_out) lq[q] = lo_load<T>(a.lo_in + g);
                }
            }
        }
#pragma unroll
        for (int q = 0; q < MU; q++) {
            const int e = e0 + q * nthr;
            if (e >= total) continue;
            const long long g = gidx(e);
            if (a.lo_out) {
                // compensated state: the transforms carried the increment
                cx<T> h, l;
                comp_add<T>(hq[q], lq[q], S[e], h, l);
                a.out[g] = h;
                lo_store<T>(a.lo_out + g, l);
            } else {
                a.out[g] = MODE == MIX_C1V ? S[e] : add<T>(hq[q], S[e]);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Transposed step (adjoint) on mixed-radix grids: the row pass of
// adj_row_kernel and the column passes of adj_col_kernel.
// ---------------------------------------------------------------------------

template <typename T>
struct MixAdjRowArgs {
    AdjRowArgs<T> r;        // as for power-of-two rows (log2nx and tws unused)
    int nx, Q;              // row length; points per WENO chunk (Q divides nx)
    MixFFT f;               // length nx / 2 on r.tw (stride 2)
    const int* pos;         // [nx / 2]
};

template <typename T>
__host__ __forceinline__ size_t mix_adj_row_smem(int nx, int nthr)
{
    return 3 * (size_t)(nx / 2) * sizeof(cx<T>) + 5 * (size_t)nthr * sizeof(T);
}

// One row of J_G^T (see adj_row_kernel): the physical state row, the C2R of
// the cotangent row, the WENO5 transpose over chunks of Q points (chunk
// boundaries exchange their spilled sums), the transposed y part, R2C.
template <typename T, int MODE>
__global__ void __launch_bounds__(MIX_ROW_MAX_THREADS) mix_adj_row_kernel(MixAdjRowArgs<T> A)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const AdjRowArgs<T>& a = A.r;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int nx = A.nx, n = nx >> 1;
    const int row = blockIdx.x, inst = blockIdx.y;
    cx<T>* U = reinterpret_cast<cx<T>*>(smem_raw);
    cx<T>* M = U + n;
    cx<T>* G = M + n;
    T* spl = reinterpret_cast<T*>(G + n);
    T* spr = spl + 2 * nthr;
    const long long base = (long long)inst * a.inst_stride + (long long)row * n;
    const int* pos = A.pos;

    const T* urow = a.u + 2 * base;
    for (int i = tid; i < nx; i += nthr) st_real<T, false>(U, i, __ldcg(urow + i));
    for (int k = tid; k <= n / 2; k += nthr) {
        const int kn = k == 0 ? 0 : n - k;
        cx<T> zk, znk;
        c2r_vals<T>(__ldcg(a.m + base + k), __ldcg(a.m + base + kn), __ldg(a.tw + k), k, n, zk, znk);
        M[__ldg(pos + k)] = zk;
        if (k != 0 && 2 * k != n) M[__ldg(pos + kn)] = znk;
    }
    __syncthreads();
    mix_inverse<T, false>(M, A.f, 0, a.tw, nullptr, tid, nthr);

    const int Q = A.Q, nact = nx / Q, k0 = tid * Q;
    WenoCoef<T> wc = a.wc;
    if (a.med_coef) {
        const double cj = 2.0 * 3.14159265358979323846 * __ldg(a.med_coef + 3 * row);
        wc.c = (T)cj;
        wc.alpha = (T)(fabs(cj) + (double)a.wc.alpha);
    }
    if (tid < nact) weno_row_chunk_T<T, false, false>(U, M, G, spl + 2 * tid, spr + 3 * tid, nx, k0, Q, wc);
    __syncthreads();
    if (tid < nact) {
        const int left = (tid + nact - 1) % nact, right = (tid + 1) % nact;
        for (int s = 0; s < 3; s++) st_real<T, false>(G, k0 + s, ld_real<T, false>(G, k0 + s) + spr[3 * left + s]);
        st_real<T, false>(G, k0 + Q - 2, ld_real<T, false>(G, k0 + Q - 2) + spl[2 * right + 0]);
        st_real<T, false>(G, k0 + Q - 1, ld_real<T, false>(G, k0 + Q - 1) + spl[2 * right + 1]);
    }
    __syncthreads();
    if (a.yT) {
        const T* yrow = a.yT + 2 * base;
        for (int k = tid; k < nx; k += nthr) st_real<T, false>(G, k, ld_real<T, false>(G, k) + __ldcg(yrow + k));
        __syncthreads();
    }
    mix_forward<T, false>(G, A.f, 0, a.tw, nullptr, tid, nthr);
    for (int k = tid; k <= n / 2; k += nthr) {
        const int kn = k == 0 ? 0 : n - k;
        cx<T> xk, xnk;
        r2c_vals<T>(G[__ldg(pos + k)], G[__ldg(pos + kn)], __ldg(a.tw + k), k, n, xk, xnk);
        xk = scale<T>(xk, a.inv_nx);
        xnk = scale<T>(xnk, a.inv_nx);
        const cx<T> mk0 = __ldcg(a.m + base + k);
        const cx<T> lk = __ldcg(a.l + base + k);
        if (k == 0) {
            const T kN = a.kscale * T(n);
            xk.y -= a.dA * kN * kN * mk0.y;
            a.out[base] = add<T>(lk, xk);
        } else {
            const T kt = a.kscale * T(k);
            xk.x -= a.dA * kt * kt * mk0.x;
            xk.y -= a.dA * kt * kt * mk0.y;
            a.out[base + k] = add<T>(lk, xk);
            if (2 * k != n) {
                const T kt2 = a.kscale * T(n - k);
                const cx<T> mk2 = __ldcg(a.m + base + n - k);
                xnk.x -= a.dA * kt2 * kt2 * mk2.x;
                xnk.y -= a.dA * kt2 * kt2 * mk2.y;
                a.out[base + n - k] = add<T>(__ldcg(a.l + base + n - k), xnk);
            }
        }
    }
}

// Transposed column passes: MIX_ADJ_C2: out = IFFT(sa conj(Ta) FFT(a));
// MIX_ADJ_C1A: z = FFT(a) (kept in the scratch w, transformed order),
// out = IFFT(sa conj(Ta) z); MIX_ADJ_C1B: out2 = IFFT(sb conj(Tb) z) - b.
// (out may alias a: z is saved before out is written.)
enum MixAdjColMode { MIX_ADJ_C2 = 0, MIX_ADJ_C1A = 1, MIX_ADJ_C1B = 2 };

template <typename T>
struct MixAdjColArgs {
    AdjColArgs<T> c;        // a, b, out, out2, Ta, Tb, sa, sb, inst_stride (tw: full y table)
    cx<T>* w;               // scratch [batch][ny][nx/2]
    int ny, n, lc;
    MixFFT f;
    const int* pos;
    const int* ipos;
};

template <typename T, int MODE>
__global__ void __launch_bounds__(MIX_COL_THREADS) mix_adj_col_kernel(MixAdjColArgs<T> A)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cx<T>* S = reinterpret_cast<cx<T>*>(smem_raw);
    const AdjColArgs<T>& a = A.c;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int ny = A.ny, n = A.n, lc = A.lc, TC = 1 << lc;
    const int m0 = blockIdx.x * TC, inst = blockIdx.y;
    const long long ibase = (long long)inst * a.inst_stride;
    const int total = ny << lc;
    auto gidx = [&](int e) -> long long { return ibase + (long long)(e >> lc) * n + m0 + (e & (TC - 1)); };

    if constexpr (MODE == MIX_ADJ_C1B) {
        for (int e = tid; e < total; e += nthr) S[e] = __ldcg(A.w + gidx(e));
        __syncthreads();
    } else {
        for (int e = tid; e < total; e += nthr) S[e] = __ldcg(a.a + gidx(e));
        __syncthreads();
        mix_forward<T, false>(S, A.f, lc, a.tw, nullptr, tid, nthr);
        if constexpr (MODE == MIX_ADJ_C1A) {
            for (int e = tid; e < total; e += nthr) A.w[gidx(e)] = S[e];
            __syncthreads();    // the packed column's pairs are rewritten below
        }
    }
    const cx<T>* Tm = MODE == MIX_ADJ_C1B ? a.Tb : a.Ta;
    const T sm = MODE == MIX_ADJ_C1B ? a.sb : a.sa;
    for (int e = tid; e < total; e += nthr) {
        const int c = e & (TC - 1), m = m0 + c;
        if (m == 0) continue;
        const int l = __ldg(A.ipos + (e >> lc));
        const int lf = l <= (ny >> 1) ? l : ny - l;
        S[e] = mulc<T>(S[e], scale<T>(__ldg(Tm + (long long)lf * n + m), sm));
    }
    if (m0 == 0) {
        for (int l = tid; l <= (ny >> 1); l += nthr) {
            const int lm = l == 0 ? 0 : ny - l;
            const int e = __ldg(A.pos + l) << lc, em = __ldg(A.pos + lm) << lc;
            const cx<T> M = scale<T>(__ldg(Tm + (long long)l * n), sm);
            const cx<T> z = S[e], zm = S[em];
            S[e] = conj_mult_entry<T>(M, z, zm, true);
            if (lm != l) S[em] = conj_mult_entry<T>(M, zm, z, true);
        }
    }
    __syncthreads();
    mix_inverse<T, false>(S, A.f, lc, a.tw, nullptr, tid, nthr);
    for (int e = tid; e < total; e += nthr) {
        const long long g = gidx(e);
        if constexpr (MODE == MIX_ADJ_C1B) a.out2[g] = sub<T>(S[e], __ldcg(a.b + g));
        else a.out[g] = S[e];
    }
}

}  // namespace kzk
