// kzk_fft.cuh -- shared-memory Stockham FFTs (power-of-two lengths).
//
// A batch of nb independent complex transforms of length n = 2^log2n lives in
// shared memory; element i of transform b sits at buf[idx(b * sb + i * si)],
// where idx() is the identity or, with PAD, i + i/16 (one padding slot per
// 16 elements, which removes the bank conflicts of the first pass's strided
// stores and of the WENO sweep over the same buffer).  Each stage is an
// autosort (Stockham) pass of radix R in {2, 4, 8, 16}: a thread loads R
// points with stride n/R into registers, applies the inter-stage twiddles,
// runs an in-register DFT of size R and writes the results to their sorted
// positions, so the output is in natural order with no bit reversal.
// Twiddles come from a plan-time staged table (see Tw), built in long double
// on the host.
//
// ACC (float only): every multiplication by a fixed constant -- table
// twiddles and the DFT's own roots of unity -- uses a two-float (hi + lo)
// representation of the constant.  A transform applied to the propagated
// state once per step then carries no systematic rounding of its constants,
// which would otherwise compound linearly over thousands of steps.
//
// Forward transforms use exp(-2 pi i ...), inverse ones exp(+2 pi i ...); no
// transform is normalised (the 1/N factors are folded into the tables).
#pragma once
#include "kzk_common.cuh"

namespace kzk {

// cos(2 pi j / 16), exact to double rounding
__host__ __device__ constexpr double cos16(int j)
{
    switch (j & 15) {
    case 0: return 1.0;
    case 1: return 0.92387953251128675613;
    case 2: return 0.70710678118654752440;
    case 3: return 0.38268343236508977173;
    case 4: return 0.0;
    case 5: return -0.38268343236508977173;
    case 6: return -0.70710678118654752440;
    case 7: return -0.92387953251128675613;
    case 8: return -1.0;
    case 9: return -0.92387953251128675613;
    case 10: return -0.70710678118654752440;
    case 11: return -0.38268343236508977173;
    case 12: return 0.0;
    case 13: return 0.38268343236508977173;
    case 14: return 0.70710678118654752440;
    default: return 0.92387953251128675613;
    }
}
__host__ __device__ constexpr double sin16(int j) { return cos16(j - 4); }

__device__ __forceinline__ int padx(int i) { return i + (i >> 4); }
template <bool PAD> __device__ __forceinline__ int sidx(int i) { return PAD ? padx(i) : i; }

// x * exp(S 2 pi i k / R) for compile-time R | 16, k; trivial factors are exact.
template <typename T, int R, int K, int S, bool ACC>
__device__ __forceinline__ cx<T> rot(cx<T> x)
{
    constexpr int j = (K * (16 / R)) & 15;          // angle 2 pi j / 16
    if constexpr (j == 0) return x;
    else if constexpr (j == 4) return mul_si<T, S>(x);
    else if constexpr (j == 8) return mk<T>(-x.x, -x.y);
    else if constexpr (j == 12) return mul_si<T, -S>(x);
    else {
        constexpr T c = (T)cos16(j);
        constexpr T s = (T)(S * sin16(j));
        if constexpr (ACC && sizeof(T) == 4) {
            constexpr T cl = (T)(cos16(j) - (double)c);
            constexpr T sl = (T)(S * sin16(j) - (double)s);
            const T re = fma(x.x, c, fma(x.x, cl, -fma(x.y, s, x.y * sl)));
            const T im = fma(x.x, s, fma(x.x, sl, fma(x.y, c, x.y * cl)));
            return mk<T>(re, im);
        } else {
            return mk<T>(fma(x.x, c, -x.y * s), fma(x.x, s, x.y * c));
        }
    }
}

// In-register DFT of size R (natural order in and out), sign S.
template <typename T, int R, int S, bool ACC> struct RegDFT {
    template <int K>
    static __device__ __forceinline__ void combine(cx<T>* v, const cx<T>* e, const cx<T>* o)
    {
        if constexpr (K < R / 2) {
            constexpr int j = (K * (16 / R)) & 15;   // the root's angle 2 pi j / 16
            if constexpr (!ACC && (j & 3) == 2) {
                // |cos| = |sin| = h: o_K times the root is h (A + i B) with A, B
                // sums of +-o_K's parts, and e_K +- h (A + i B) are fused
                // multiply-adds (six operations instead of eight)
                constexpr bool cp = cos16(j) > 0, sp = S * sin16(j) > 0;
                constexpr T h = (T)cos16(2), mh = (T)(-cos16(2));
                const cx<T> x = o[K];
                const T A = (cp ? x.x : -x.x) - (sp ? x.y : -x.y);
                const T B = (sp ? x.x : -x.x) + (cp ? x.y : -x.y);
                v[K] = mk<T>(fma(h, A, e[K].x), fma(h, B, e[K].y));
                v[K + R / 2] = mk<T>(fma(mh, A, e[K].x), fma(mh, B, e[K].y));
            } else {
                cx<T> t = rot<T, R, K, S, ACC>(o[K]);
                v[K] = add<T>(e[K], t);
                v[K + R / 2] = sub<T>(e[K], t);
            }
            combine<K + 1>(v, e, o);
        }
    }
    static __device__ __forceinline__ void run(cx<T>* v)
    {
        if constexpr (R == 1) {
            return;
        } else if constexpr (R == 2) {
            cx<T> a = v[0], b = v[1];
            v[0] = add<T>(a, b);
            v[1] = sub<T>(a, b);
        } else if constexpr (R == 4) {
            cx<T> a0 = add<T>(v[0], v[2]), a1 = sub<T>(v[0], v[2]);
            cx<T> a2 = add<T>(v[1], v[3]), a3 = mul_si<T, S>(sub<T>(v[1], v[3]));
            v[0] = add<T>(a0, a2);
            v[2] = sub<T>(a0, a2);
            v[1] = add<T>(a1, a3);
            v[3] = sub<T>(a1, a3);
        } else {
            cx<T> e[R / 2], o[R / 2];
#pragma unroll
            for (int i = 0; i < R / 2; i++) { e[i] = v[2 * i]; o[i] = v[2 * i + 1]; }
            RegDFT<T, R / 2, S, ACC>::run(e);
            RegDFT<T, R / 2, S, ACC>::run(o);
            combine<0>(v, e, o);
        }
    }
};

// Twiddle tables: hi part and, for ACC, the lo correction (lo == nullptr
// otherwise), as a per-pass ("staged") table for the transform length and
// radix schedule: pass p with Ns_p, R_p occupies (R_p - 1) * Ns_p entries,
// entry (r - 1) * Ns_p + k = exp(-2 pi i r k / (Ns_p R_p)), so the lanes of a
// warp (consecutive k) read consecutive entries.  (log2 is unused: -1.)
template <typename T>
struct Tw {
    const cx<T>* __restrict__ hi;
    const cx<T>* __restrict__ lo;
    int log2;
};

// One Stockham pass of radix R over a batch.  PPT = points each thread holds
// (PPT / R butterflies per pass).  COLS: consecutive threads take consecutive
// transforms (column tiles, transform index fastest in memory); otherwise
// consecutive threads take consecutive butterflies of one transform.
// In place (src == dst, OOP false): a barrier between the loads and the
// stores; out of place (OOP): none.  Both end with a __syncthreads().
template <typename T, int R, int PPT, bool COLS, bool INV, bool PAD, bool ACC, bool OOP = false>
__device__ __forceinline__ void fft_pass(const cx<T>* src, cx<T>* dst, int log2n, int log2nb, int si, int sb,
                                         int log2Ns, const Tw<T>& tw, int stage_off, int tid, int nthr)
{
    constexpr int NB = PPT / R;
    constexpr int LR = (R == 2) ? 1 : (R == 4) ? 2 : (R == 8) ? 3 : 4;
    constexpr int S = INV ? 1 : -1;
    const int log2nbf = log2n - LR;                 // butterflies per transform = n / R
    const int total = 1 << (log2nb + log2nbf);
    const int Ns = 1 << log2Ns;
    cx<T> v[NB][R];
    int obase[NB];
#pragma unroll
    for (int q = 0; q < NB; q++) {
        int t = tid + q * nthr;
        obase[q] = -1;
        if (t < total) {
            int b, j;
            if (COLS) { b = t & ((1 << log2nb) - 1); j = t >> log2nb; }
            else { b = t >> log2nbf; j = t & ((1 << log2nbf) - 1); }
            const int k = j & (Ns - 1);
            const int ib = b * sb + j * si;
            const int stride = (1 << log2nbf) * si;
            if (!PAD || (stride & 15) == 0) {
                // padded index of ib + r * stride is padx(ib) + r * padded stride
                const int pb = sidx<PAD>(ib), ps = PAD ? stride + (stride >> 4) : stride;
#pragma unroll
                for (int r = 0; r < R; r++) v[q][r] = src[pb + r * ps];
            } else {
#pragma unroll
                for (int r = 0; r < R; r++) v[q][r] = src[sidx<PAD>(ib + r * stride)];
            }
            if (log2Ns > 0) {
#pragma unroll
                for (int r = 1; r < R; r++) {
                    const int ti = stage_off + (r - 1) * Ns + k;
                    const cx<T> w = tw.hi[ti];
                    if constexpr (ACC && sizeof(T) == 4) {
                        const cx<T> wl = tw.lo[ti];
                        const cx<T> x = v[q][r];
                        v[q][r] = INV ? fma_c<T>(x, conj<T>(wl), mulc<T>(x, w)) : fma_c<T>(x, wl, mul<T>(x, w));
                    } else {
                        v[q][r] = INV ? mulc<T>(v[q][r], w) : mul<T>(v[q][r], w);
                    }
                }
            }
            RegDFT<T, R, S, ACC>::run(v[q]);
            obase[q] = b * sb + (((j - k) << LR) + k) * si;
        }
    }
    if constexpr (!OOP) __syncthreads();
    const int ostride = Ns * si;
#pragma unroll
    for (int q = 0; q < NB; q++) {
        if (obase[q] >= 0) {
            if (!PAD || (ostride & 15) == 0) {
                const int pb = sidx<PAD>(obase[q]), ps = PAD ? ostride + (ostride >> 4) : ostride;
#pragma unroll
                for (int r = 0; r < R; r++) dst[pb + r * ps] = v[q][r];
            } else {
#pragma unroll
                for (int r = 0; r < R; r++) dst[sidx<PAD>(obase[q] + r * ostride)] = v[q][r];
            }
        }
    }
    __syncthreads();
}
template <typename T, int R, int PPT, bool COLS, bool INV, bool PAD, bool ACC>
__device__ __forceinline__ void fft_pass(cx<T>* buf, int log2n, int log2nb, int si, int sb, int log2Ns,
                                         const Tw<T>& tw, int stage_off, int tid, int nthr)
{
    fft_pass<T, R, PPT, COLS, INV, PAD, ACC, false>(buf, buf, log2n, log2nb, si, sb, log2Ns, tw, stage_off, tid, nthr);
}

// Full transform: radix-16 passes while possible, then one smaller pass.
// Requires nthr * PPT >= nb * n.  Ends with a __syncthreads().
template <typename T, int PPT, bool COLS, bool INV, bool PAD = false, bool ACC = false>
__device__ __forceinline__ void fft_batched(cx<T>* buf, int log2n, int log2nb, int si, int sb, const Tw<T>& tw,
                                            int tid, int nthr)
{
    int done = 0, off = 0;
    while (done < log2n) {
        const int rem = log2n - done;
        if (PPT >= 16 && rem >= 4) {
            fft_pass<T, (PPT >= 16 ? 16 : 2), PPT, COLS, INV, PAD, ACC>(buf, log2n, log2nb, si, sb, done, tw, off, tid, nthr);
            off += (done > 0 ? ((PPT >= 16 ? 16 : 2) - 1) << done : 0);
            done += (PPT >= 16 ? 4 : 1);
        } else if (PPT >= 8 && rem >= 3) {
            fft_pass<T, (PPT >= 8 ? 8 : 2), PPT, COLS, INV, PAD, ACC>(buf, log2n, log2nb, si, sb, done, tw, off, tid, nthr);
            off += (done > 0 ? ((PPT >= 8 ? 8 : 2) - 1) << done : 0);
            done += (PPT >= 8 ? 3 : 1);
        } else if (PPT >= 4 && rem >= 2) {
            fft_pass<T, (PPT >= 4 ? 4 : 2), PPT, COLS, INV, PAD, ACC>(buf, log2n, log2nb, si, sb, done, tw, off, tid, nthr);
            off += (done > 0 ? ((PPT >= 4 ? 4 : 2) - 1) << done : 0);
            done += (PPT >= 4 ? 2 : 1);
        } else {
            fft_pass<T, 2, PPT, COLS, INV, PAD, ACC>(buf, log2n, log2nb, si, sb, done, tw, off, tid, nthr);
            off += (done > 0 ? 1 << done : 0);
            done += 1;
        }
    }
}

// The same schedule out of place, passes alternating between buffers a (the
// input) and b; returns the buffer holding the result.  One barrier per pass.
template <typename T, int PPT, bool COLS, bool INV, bool PAD = false, bool ACC = false>
__device__ __forceinline__ cx<T>* fft_batched_pp(cx<T>* a, cx<T>* b, int log2n, int log2nb, int si, int sb,
                                                 const Tw<T>& tw, int tid, int nthr)
{
    int done = 0, off = 0;
    cx<T>* s = a;
    cx<T>* d = b;
    while (done < log2n) {
        const int rem = log2n - done;
        if (PPT >= 16 && rem >= 4) {
            fft_pass<T, (PPT >= 16 ? 16 : 2), PPT, COLS, INV, PAD, ACC, true>(s, d, log2n, log2nb, si, sb, done, tw,
                                                                             off, tid, nthr);
            off += (done > 0 ? ((PPT >= 16 ? 16 : 2) - 1) << done : 0);
            done += (PPT >= 16 ? 4 : 1);
        } else if (PPT >= 8 && rem >= 3) {
            fft_pass<T, (PPT >= 8 ? 8 : 2), PPT, COLS, INV, PAD, ACC, true>(s, d, log2n, log2nb, si, sb, done, tw,
                                                                           off, tid, nthr);
            off += (done > 0 ? ((PPT >= 8 ? 8 : 2) - 1) << done : 0);
            done += (PPT >= 8 ? 3 : 1);
        } else if (PPT >= 4 && rem >= 2) {
            fft_pass<T, (PPT >= 4 ? 4 : 2), PPT, COLS, INV, PAD, ACC, true>(s, d, log2n, log2nb, si, sb, done, tw,
                                                                           off, tid, nthr);
            off += (done > 0 ? ((PPT >= 4 ? 4 : 2) - 1) << done : 0);
            done += (PPT >= 4 ? 2 : 1);
        } else {
            fft_pass<T, 2, PPT, COLS, INV, PAD, ACC, true>(s, d, log2n, log2nb, si, sb, done, tw, off, tid, nthr);
            off += (done > 0 ? 1 << done : 0);
            done += 1;
        }
        cx<T>* t = s;
        s = d;
        d = t;
    }
    return s;
}

// fft_batched / fft_batched_pp with the length 2^LOG2N known at compile
// time: the same passes in the same order (the schedule unrolled by template
// recursion), so every stride, twiddle offset and trip count is a constant.
template <int PPT, int REM>
__host__ __device__ constexpr int ct_log2_radix()
{
    return (PPT >= 16 && REM >= 4) ? 4 : (PPT >= 8 && REM >= 3) ? 3 : (PPT >= 4 && REM >= 2) ? 2 : 1;
}
template <typename T, int PPT, bool COLS, bool INV, bool PAD, bool ACC, int LOG2N, int DONE = 0, int OFF = 0>
__device__ __forceinline__ void fft_batched_ct(cx<T>* buf, const Tw<T>& tw, int tid, int nthr)
{
    if constexpr (DONE < LOG2N) {
        constexpr int LR = ct_log2_radix<PPT, LOG2N - DONE>();
        constexpr int R = 1 << LR;
        fft_pass<T, R, PPT, COLS, INV, PAD, ACC>(buf, LOG2N, 0, 1, 0, DONE, tw, OFF, tid, nthr);
        fft_batched_ct<T, PPT, COLS, INV, PAD, ACC, LOG2N, DONE + LR, OFF + (DONE > 0 ? (R - 1) << DONE : 0)>(
            buf, tw, tid, nthr);
    }
}
template <typename T, int PPT, bool COLS, bool INV, bool PAD, bool ACC, int LOG2N, int DONE = 0, int OFF = 0>
__device__ __forceinline__ cx<T>* fft_batched_pp_ct(cx<T>* a, cx<T>* b, const Tw<T>& tw, int tid, int nthr)
{
    if constexpr (DONE >= LOG2N) {
        return a;
    } else {
        constexpr int LR = ct_log2_radix<PPT, LOG2N - DONE>();
        constexpr int R = 1 << LR;
        fft_pass<T, R, PPT, COLS, INV, PAD, ACC, true>(a, b, LOG2N, 0, 1, 0, DONE, tw, OFF, tid, nthr);
        return fft_batched_pp_ct<T, PPT, COLS, INV, PAD, ACC, LOG2N, DONE + LR,
                                 OFF + (DONE > 0 ? (R - 1) << DONE : 0)>(b, a, tw, tid, nthr);
    }
}

// Radix schedule of fft_batched for a length 2^log2n with PPT points
// per thread, as (log2 R, log2 Ns) pairs.
__host__ __device__ inline int fft_schedule(int log2n, int ppt, int* lr, int* lns)
{
    int done = 0, p = 0;
    while (done < log2n) {
        const int rem = log2n - done;
        int l = 1;
        if (ppt >= 16 && rem >= 4) l = 4;
        else if (ppt >= 8 && rem >= 3) l = 3;
        else if (ppt >= 4 && rem >= 2) l = 2;
        lr[p] = l;
        lns[p] = done;
        done += l;
        p++;
    }
    return p;
}

}  // namespace kzk
