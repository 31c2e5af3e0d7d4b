// kzk_colpipe.cuh -- column kernels (Algorithm 2, STEP 2 and STEP 4) whose
// tiles are staged by the tensor memory accelerator.
//
// One CTA per column tile, two CTAs per SM (64 registers per thread, about
// 100 KB of shared memory each), so that one CTA's copies run under the other
// CTA's transforms.  One thread issues the tile's TMA copies
// (cp.async.bulk.tensor) from HBM into shared memory, each group completing
// on its own mbarrier:
//   STAGE1: V and b1 (the two dense tiles);
//   STAGE2: b1, b2 and the P2' slice, then V* once b2 has been consumed.
// The first forward pass reads the dense tiles and writes the padded work
// tiles over them; the phi-multiply is applied while the last forward pass
// stores (STAGE1 reads E', E'_lo, P1' from L2 -- with the compensated FP32
// state (E - 1)' and P1' -- the multiply needs each table entry twice, for rows
// l and ny - l); the last inverse pass writes HBM directly (with the
// compensated state: adds the increment to hi + lo by TwoSum).  The CTA also prefetches into L2 the copies of the tile a CTA one
// wave later will take.  Arithmetic and rounding are those of col_body
// (kzk_kernels.cuh): the same passes, twiddles and products in the same order.
//
// Every wait on a copy is bounded (timeout_ns): a CTA whose copy has not
// arrived in time sets FLAG_TIMEOUT and leaves the kernel.
#pragma once
#include <cuda.h>

#include "kzk_kernels.cuh"

namespace kzk {

__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* b, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(b)), "r"(count) : "memory");
}
// make the initialised barriers visible to the async (TMA) proxy
__device__ __forceinline__ void mbar_fence_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// one arrival that also announces `bytes` of copies completing on the barrier
__device__ __forceinline__ void mbar_expect(unsigned long long* b, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(b)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try(unsigned long long* b, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
// wait for the phase of the given parity; false once timeout_ns has passed
__device__ __forceinline__ bool mbar_wait(unsigned long long* b, unsigned parity, long long timeout_ns)
{
    if (mbar_try(b, parity)) return true;
    const long long t0 = global_ns();
    while (!mbar_try(b, parity))
        if (global_ns() - t0 > timeout_ns) return false;
    return true;
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* m, int x, int y, unsigned long long* b)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_addr(dst)),
        "l"(reinterpret_cast<unsigned long long>(m)), "r"(x), "r"(y), "r"(smem_addr(b))
        : "memory");
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* m, int x, int y, int z,
                                            unsigned long long* b)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<unsigned long long>(m)), "r"(x), "r"(y), "r"(z), "r"(smem_addr(b))
        : "memory");
}

// contiguous copy global -> shared (16-byte aligned, size a multiple of 16),
// completing on mbarrier b
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes, unsigned long long* b)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(reinterpret_cast<unsigned long long>(src)), "r"(bytes), "r"(smem_addr(b))
        : "memory");
}

// ---------------------------------------------------------------------------
// Stockham passes over a column tile with pluggable loads and stores.
// Element i = l * TC + c is row l of column c.  A loader fills v[0..R) with
// the elements i0 + r s; a storer writes v[0..R) to i0 + r s.
// ---------------------------------------------------------------------------

// padded work tile: element i at padx(i)
template <typename T>
struct PadIO {
    cx<T>* W;
    template <int R>
    __device__ __forceinline__ void ld(int i0, int s, cx<T>* v) const
    {
        if ((s & 15) == 0) {
            const int pb = padx(i0), ps = s + (s >> 4);
#pragma unroll
            for (int r = 0; r < R; r++) v[r] = W[pb + r * ps];
        } else {
#pragma unroll
            for (int r = 0; r < R; r++) v[r] = W[padx(i0 + r * s)];
        }
    }
    template <int R>
    __device__ __forceinline__ void st(int i0, int s, const cx<T>* v) const
    {
        if ((s & 15) == 0) {
            const int pb = padx(i0), ps = s + (s >> 4);
#pragma unroll
            for (int r = 0; r < R; r++) W[pb + r * ps] = v[r];
        } else {
#pragma unroll
            for (int r = 0; r < R; r++) W[padx(i0 + r * s)] = v[r];
        }
    }
};

// dense staging tile (as written by TMA)
template <typename T>
struct DenseLd {
    const cx<T>* S;
    template <int R>
    __device__ __forceinline__ void ld(int i0, int s, cx<T>* v) const
    {
#pragma unroll
        for (int r = 0; r < R; r++) v[r] = S[i0 + r * s];
    }
};

// B - A from two dense staging tiles (STAGE2: b2 - b1)
template <typename T>
struct DiffLd {
    const cx<T>* A;
    const cx<T>* B;
    template <int R>
    __device__ __forceinline__ void ld(int i0, int s, cx<T>* v) const
    {
#pragma unroll
        for (int r = 0; r < R; r++) v[r] = sub<T>(B[i0 + r * s], A[i0 + r * s]);
    }
};

// Folded table row of tile row l (tables are even in k_y).
__device__ __forceinline__ int fold_row(int l, int ny) { return l <= (ny >> 1) ? l : ny - l; }

// STAGE2 multiply as the last forward pass stores: P2' (b2 - b1)_hat.
template <typename T>
struct Mul2St {
    cx<T>* WA;
    const cx<T>* P2;
    int log2tc, ny, m0;
    template <int R>
    __device__ __forceinline__ void st(int i0, int s, const cx<T>* v) const
    {
        const int c = i0 & ((1 << log2tc) - 1);
        const bool packed = m0 + c == 0;
#pragma unroll
        for (int r = 0; r < R; r++) {
            const int i = i0 + r * s, pi = padx(i);
            if (packed) {
                WA[pi] = v[r];
                continue;
            }
            WA[pi] = mul<T>(P2[(fold_row(i >> log2tc, ny) << log2tc) + c], v[r]);
        }
    }
};

// last inverse pass: results straight to HBM (STAGE2: plus V* from staging)
template <typename T, bool ADD, bool COMP = false>
struct OutSt {
    cx<T>* out;
    const cx<T>* C;
    long long ibase;
    int log2tc, log2n, m0;
    // COMP (compensated state): out = hi + v with hi from C (ADD) or from
    // hi_g (the state the stage started from), lo in lo_in / lo_out
    const cx<T>* hi_g;
    const lo_t<T>* lo_in;
    lo_t<T>* lo_out;
    template <int R>
    __device__ __forceinline__ void st(int i0, int s, const cx<T>* v) const
    {
        const int c = i0 & ((1 << log2tc) - 1);
        const long long o0 = ibase + m0 + c;
#pragma unroll
        for (int r = 0; r < R; r++) {
            const int i = i0 + r * s;
            const long long g = o0 + ((long long)(i >> log2tc) << log2n);
            if constexpr (COMP) {
                cx<T> h, l;
                comp_add<T>(ADD ? C[i] : __ldcg(hi_g + g), lo_load<T>(lo_in + g), v[r], h, l);
                out[g] = h;
                lo_store<T>(lo_out + g, l);
            } else {
                out[g] = ADD ? add<T>(C[i], v[r]) : v[r];
            }
        }
    }
};

// One Stockham pass of radix R (8 points per thread) over the TC transforms of
// a tile, pass input stride n/R, output stride Ns (staged twiddles, offset
// stage_off).  Loads, __syncthreads, stores, __syncthreads.
template <typename T, int R, bool INV, bool ACC, class LD, class ST>
__device__ __forceinline__ void tile_pass(int log2n, int log2tc, int log2Ns, const Tw<T>& tw, int stage_off, int tid,
                                          int nthr, LD ld, ST st)
{
    constexpr int NB = 8 / R;
    constexpr int LR = (R == 2) ? 1 : (R == 4) ? 2 : 3;
    constexpr int S = INV ? 1 : -1;
    const int log2nbf = log2n - LR;
    const int total = 1 << (log2tc + log2nbf);
    const int Ns = 1 << log2Ns;
    const int istride = 1 << (log2nbf + log2tc);
    cx<T> v[NB][R];
    int obase[NB];
#pragma unroll
    for (int q = 0; q < NB; q++) {
        const int t = tid + q * nthr;
        obase[q] = -1;
        if (t < total) {
            const int b = t & ((1 << log2tc) - 1), j = t >> log2tc, k = j & (Ns - 1);
            ld.template ld<R>(t, istride, v[q]);           // element b + j TC = t
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
            obase[q] = b + ((((j - k) << LR) + k) << log2tc);
        }
    }
    __syncthreads();
    const int ostride = Ns << log2tc;
#pragma unroll
    for (int q = 0; q < NB; q++)
        if (obase[q] >= 0) st.template st<R>(obase[q], ostride, v[q]);
    __syncthreads();
}

// The radix schedule of a length-2^log2n transform (log2n >= 4): radix 8 up to
// the last pass, which is 8, 4 or 2 -- the schedule of fft_batched with 8
// points per thread, whose staged twiddle table this reads.
template <typename T, bool INV, bool ACC, class LD>
__device__ __forceinline__ void tile_first(int log2n, int log2tc, const Tw<T>& tw, int tid, int nthr, LD ld,
                                           cx<T>* W)
{
    tile_pass<T, 8, INV, ACC>(log2n, log2tc, 0, tw, 0, tid, nthr, ld, PadIO<T>{W});
}
template <typename T, bool INV, bool ACC>
__device__ __forceinline__ void tile_middle(int log2n, int log2tc, const Tw<T>& tw, int tid, int nthr, cx<T>* W)
{
    const PadIO<T> io{W};
    int off = 0;
    for (int done = 3; done + 3 < log2n; done += 3) {
        tile_pass<T, 8, INV, ACC>(log2n, log2tc, done, tw, off, tid, nthr, io, io);
        off += 7 << done;
    }
}
template <typename T, bool INV, bool ACC, class ST>
__device__ __forceinline__ void tile_last(int log2n, int log2tc, const Tw<T>& tw, int tid, int nthr, cx<T>* W,
                                          ST st)
{
    const PadIO<T> io{W};
    int off = 0, done = 3;
    for (; done + 3 < log2n; done += 3) off += 7 << done;
    const int lr = log2n - done;
    if (lr == 3) tile_pass<T, 8, INV, ACC>(log2n, log2tc, done, tw, off, tid, nthr, io, st);
    else if (lr == 2) tile_pass<T, 4, INV, ACC>(log2n, log2tc, done, tw, off, tid, nthr, io, st);
    else tile_pass<T, 2, INV, ACC>(log2n, log2tc, done, tw, off, tid, nthr, io, st);
}

// ---------------------------------------------------------------------------
// Paired passes (STAGE1 forward): the state tile A (two-float constants in
// FP32 with the plain state) and the b1 tile B go through the same butterflies between one pair of
// barriers, so a thread holds both spectra at the same positions when the last
// pass stores -- the multiply then reads b1_hat from registers.
// ---------------------------------------------------------------------------
template <typename T>
struct PadIO2 {
    cx<T>* WA;
    cx<T>* WB;
    template <int R>
    __device__ __forceinline__ void st(int i0, int s, const cx<T>* va, const cx<T>* vb) const
    {
        PadIO<T>{WA}.template st<R>(i0, s, va);
        PadIO<T>{WB}.template st<R>(i0, s, vb);
    }
};

// V*_hat = E' V_hat (+ E'_lo V_hat in FP32; the compensated state passes
// (E - 1)' and no lo part) + P1' b1_hat, tables read from
// global memory (L2); the packed column m = 0 keeps both spectra untouched for
// the row-pair combination
template <typename T, bool ACC>
struct Mul1St2 {
    cx<T>* WA;
    cx<T>* WB;
    const cx<T>* E;
    const cx<T>* El;
    const cx<T>* P1;
    int log2tc, log2n, ny, m0;
    template <int R>
    __device__ __forceinline__ void st(int i0, int s, const cx<T>* va, const cx<T>* vb) const
    {
        const int c = i0 & ((1 << log2tc) - 1);
        if (m0 + c == 0) {
            PadIO<T>{WA}.template st<R>(i0, s, va);
            PadIO<T>{WB}.template st<R>(i0, s, vb);
            return;
        }
        cx<T> te[R], tl[R], tp[R];
#pragma unroll
        for (int r = 0; r < R; r++) {
            const long long ti = ((long long)fold_row((i0 + r * s) >> log2tc, ny) << log2n) + m0 + c;
            te[r] = __ldg(E + ti);
            if constexpr (ACC) tl[r] = __ldg(El + ti);
            tp[r] = __ldg(P1 + ti);
        }
        const bool fast = (s & 15) == 0;
        const int pb = padx(i0), ps = s + (s >> 4);
#pragma unroll
        for (int r = 0; r < R; r++) {
            cx<T> o = mul<T>(te[r], va[r]);
            if constexpr (ACC) o = fma_c<T>(tl[r], va[r], o);
            WA[fast ? pb + r * ps : padx(i0 + r * s)] = fma_c<T>(tp[r], vb[r], o);
        }
    }
};

template <typename T, int R, bool INV, bool ACC>
__device__ __forceinline__ void apply_twiddles(cx<T>* v, const Tw<T>& tw, int stage_off, int Ns, int k)
{
#pragma unroll
    for (int r = 1; r < R; r++) {
        const int ti = stage_off + (r - 1) * Ns + k;
        const cx<T> w = tw.hi[ti];
        if constexpr (ACC && sizeof(T) == 4) {
            const cx<T> wl = tw.lo[ti];
            const cx<T> x = v[r];
            v[r] = INV ? fma_c<T>(x, conj<T>(wl), mulc<T>(x, w)) : fma_c<T>(x, wl, mul<T>(x, w));
        } else {
            v[r] = INV ? mulc<T>(v[r], w) : mul<T>(v[r], w);
        }
    }
}

// forward pass over tiles A (ACC constants) and B (plain) together
template <typename T, int R, bool ACC, class LDA, class LDB, class ST2>
__device__ __forceinline__ void tile_pass2(int log2n, int log2tc, int log2Ns, const Tw<T>& twa, const Tw<T>& twp,
                                           int stage_off, int tid, int nthr, LDA lda, LDB ldb, ST2 st)
{
    constexpr int NB = 8 / R;
    constexpr int LR = (R == 2) ? 1 : (R == 4) ? 2 : 3;
    const int log2nbf = log2n - LR;
    const int total = 1 << (log2tc + log2nbf);
    const int Ns = 1 << log2Ns;
    const int istride = 1 << (log2nbf + log2tc);
    cx<T> va[NB][R], vb[NB][R];
    int obase[NB];
#pragma unroll
    for (int q = 0; q < NB; q++) {
        const int t = tid + q * nthr;
        obase[q] = -1;
        if (t < total) {
            const int b = t & ((1 << log2tc) - 1), j = t >> log2tc, k = j & (Ns - 1);
            lda.template ld<R>(t, istride, va[q]);
            ldb.template ld<R>(t, istride, vb[q]);
            if (log2Ns > 0) {
                apply_twiddles<T, R, false, ACC>(va[q], twa, stage_off, Ns, k);
                apply_twiddles<T, R, false, false>(vb[q], twp, stage_off, Ns, k);
            }
            RegDFT<T, R, -1, ACC>::run(va[q]);
            RegDFT<T, R, -1, false>::run(vb[q]);
            obase[q] = b + ((((j - k) << LR) + k) << log2tc);
        }
    }
    __syncthreads();
    const int ostride = Ns << log2tc;
#pragma unroll
    for (int q = 0; q < NB; q++)
        if (obase[q] >= 0) st.template st<R>(obase[q], ostride, va[q], vb[q]);
    __syncthreads();
}

template <typename T, bool ACC, class LDA, class LDB>
__device__ __forceinline__ void tile2_first(int log2n, int log2tc, const Tw<T>& twa, const Tw<T>& twp, int tid,
                                            int nthr, LDA lda, LDB ldb, cx<T>* WA, cx<T>* WB)
{
    tile_pass2<T, 8, ACC>(log2n, log2tc, 0, twa, twp, 0, tid, nthr, lda, ldb, PadIO2<T>{WA, WB});
}
template <typename T, bool ACC>
__device__ __forceinline__ void tile2_middle(int log2n, int log2tc, const Tw<T>& twa, const Tw<T>& twp, int tid,
                                             int nthr, cx<T>* WA, cx<T>* WB)
{
    int off = 0;
    for (int done = 3; done + 3 < log2n; done += 3) {
        tile_pass2<T, 8, ACC>(log2n, log2tc, done, twa, twp, off, tid, nthr, PadIO<T>{WA}, PadIO<T>{WB},
                              PadIO2<T>{WA, WB});
        off += 7 << done;
    }
}
template <typename T, bool ACC, class ST2>
__device__ __forceinline__ void tile2_last(int log2n, int log2tc, const Tw<T>& twa, const Tw<T>& twp, int tid,
                                           int nthr, cx<T>* WA, cx<T>* WB, ST2 st)
{
    int off = 0, done = 3;
    for (; done + 3 < log2n; done += 3) off += 7 << done;
    const int lr = log2n - done;
    const PadIO<T> ia{WA}, ib{WB};
    if (lr == 3) tile_pass2<T, 8, ACC>(log2n, log2tc, done, twa, twp, off, tid, nthr, ia, ib, st);
    else if (lr == 2) tile_pass2<T, 4, ACC>(log2n, log2tc, done, twa, twp, off, tid, nthr, ia, ib, st);
    else tile_pass2<T, 2, ACC>(log2n, log2tc, done, twa, twp, off, tid, nthr, ia, ib, st);
}

// ---------------------------------------------------------------------------
// Kernel arguments and shared-memory layout
// ---------------------------------------------------------------------------
template <typename T>
struct ColPipeArgs {
    ColArgs<T> c;                  // pointers and sizes, as for col_kernel
    CUtensorMap ma, mb, mc;        // state arrays, {2 n, ny, batch} of T, box {2 TC, by, 1}
    CUtensorMap mt0;               // STAGE2: P2', {2 n, ny/2 + 1} of T, box {2 TC, bt}
    int by, nby;                   // rows per state box, boxes per tile column
    int bt, nbt;                   // rows per table box, boxes per table slice
    int n_tiles, total;            // tiles per instance, tiles of all instances
    int ahead;                     // CTA q prefetches tile q + ahead into L2 (0: none)
    int* flag;                     // FLAG_TIMEOUT on a wait that ran out
    long long timeout_ns;
};

constexpr int COLP_THREADS = 512;

__host__ __device__ constexpr unsigned up128(unsigned v) { return (v + 127u) & ~127u; }

struct ColPipeLayout {
    unsigned red, ra, rb, t0, tw, twl, total;
    unsigned stage_bytes, table_bytes;
};

// mbarriers (128 B); diagnostics scratch; region A: dense tile (V | b1), then the padded work tile;
// region B: dense tile (b1 | b2), then the padded b1 work tile (STAGE1) or the
// dense V* tile (STAGE2); the P2' slice (STAGE2); the y twiddles (+ lo parts,
// STAGE1 FP32).
template <typename T, int MODE>
__host__ __device__ __forceinline__ ColPipeLayout colp_layout(int ny, int log2tc, int bt, int nbt)
{
    constexpr bool ACC = sizeof(T) == 4;
    const unsigned es = sizeof(cx<T>);
    const unsigned tile = (unsigned)ny << log2tc;
    ColPipeLayout L;
    L.stage_bytes = tile * es;
    L.table_bytes = ((unsigned)(bt * nbt) << log2tc) * es;
    const unsigned region = up128((tile + (tile >> 4)) * es);   // padded tile >= dense tile
    unsigned off = 128;
    L.red = off; off += 4 * sizeof(double) * (COLP_THREADS / 32);
    L.ra = off; off += region;
    L.rb = off; off += region;
    L.t0 = off; if (MODE == COL_STAGE2) off += up128(L.table_bytes);
    L.tw = off; off += up128(ny * es);
    L.twl = off; if (MODE == COL_STAGE1 && ACC) off += up128(ny * es);
    L.total = off;
    return L;
}

// Copies of tile q into region A / B (barrier 0: inputs; STAGE2 also the P2'
// slice) and of V* into region B (barrier 1, STAGE2).  Issued by one thread.
template <typename T, int MODE>
__device__ __forceinline__ void colp_issue_in(const ColPipeArgs<T>& P, unsigned char* smem, const ColPipeLayout& L, int q)
{
    unsigned long long* bar = reinterpret_cast<unsigned long long*>(smem);
    const int inst = q / P.n_tiles, x = (2 * (q - inst * P.n_tiles)) << P.c.log2tc;
    const unsigned box = L.stage_bytes / P.nby;
    mbar_expect(bar, 2 * L.stage_bytes + (MODE == COL_STAGE2 ? L.table_bytes : 0u));
    for (int k = 0; k < P.nby; k++) {
        tma_load_3d(smem + L.ra + k * box, &P.ma, x, k * P.by, inst, bar);
        tma_load_3d(smem + L.rb + k * box, &P.mb, x, k * P.by, inst, bar);
    }
    if (MODE == COL_STAGE2) {
        const unsigned tbox = L.table_bytes / P.nbt;
        for (int k = 0; k < P.nbt; k++) tma_load_2d(smem + L.t0 + k * tbox, &P.mt0, x, k * P.bt, bar);
    }
}
template <typename T>
__device__ __forceinline__ void colp_issue_c(const ColPipeArgs<T>& P, unsigned char* smem, const ColPipeLayout& L, int q)
{
    unsigned long long* bar = reinterpret_cast<unsigned long long*>(smem) + 1;
    const int inst = q / P.n_tiles, x = (2 * (q - inst * P.n_tiles)) << P.c.log2tc;
    const unsigned box = L.stage_bytes / P.nby;
    mbar_expect(bar, L.stage_bytes);
    for (int k = 0; k < P.nby; k++) tma_load_3d(smem + L.rb + k * box, &P.mc, x, k * P.by, inst, bar);
}

// L2 prefetch of tile q's inputs (for the CTA that will take it)
__device__ __forceinline__ void tma_prefetch_2d(const CUtensorMap* m, int x, int y)
{
    asm volatile("cp.async.bulk.prefetch.tensor.2d.L2.global [%0, {%1, %2}];" ::"l"(
                     reinterpret_cast<unsigned long long>(m)),
                 "r"(x), "r"(y)
                 : "memory");
}
__device__ __forceinline__ void tma_prefetch_3d(const CUtensorMap* m, int x, int y, int z)
{
    asm volatile("cp.async.bulk.prefetch.tensor.3d.L2.global [%0, {%1, %2, %3}];" ::"l"(
                     reinterpret_cast<unsigned long long>(m)),
                 "r"(x), "r"(y), "r"(z)
                 : "memory");
}
template <typename T, int MODE>
__device__ __forceinline__ void colp_prefetch(const ColPipeArgs<T>& P, int q)
{
    const int inst = q / P.n_tiles, x = (2 * (q - inst * P.n_tiles)) << P.c.log2tc;
    for (int k = 0; k < P.nby; k++) {
        tma_prefetch_3d(&P.ma, x, k * P.by, inst);
        tma_prefetch_3d(&P.mb, x, k * P.by, inst);
        if (MODE == COL_STAGE2) tma_prefetch_3d(&P.mc, x, k * P.by, inst);
    }
    if (MODE == COL_STAGE2)
        for (int k = 0; k < P.nbt; k++) tma_prefetch_2d(&P.mt0, x, k * P.bt);
}

// every thread waits on barrier i; a timeout anywhere ends the CTA uniformly.
// pending: the barriers whose copies may still be in flight at this point
// (bit j: barrier j; 0 selects barrier i alone).  On a timeout thread 0 gives
// each of them a second bounded wait before it leaves, so that no copy is
// still writing into the CTA's shared memory once the CTA has ended.
__device__ __forceinline__ bool colp_wait(unsigned char* smem, int i, unsigned ph, long long timeout_ns, int* flag,
                                          unsigned pending = 0u)
{
    unsigned long long* bar = reinterpret_cast<unsigned long long*>(smem);
    const bool ok = mbar_wait(bar + i, ph, timeout_ns);
    if (__syncthreads_or(!ok)) {
        if (threadIdx.x == 0) {
            atomicOr(flag, FLAG_TIMEOUT);
            const unsigned m = pending ? pending : 1u << i;
            for (int j = 0; j < 8; j++)
                if (m & (1u << j)) mbar_wait(bar + j, ph, timeout_ns);
        }
        return false;
    }
    return true;
}

// diagnostics of the state the step started from (per-row partials written
// by the row pass), reduced in FP64 in a fixed order: within warps by
// shuffles, across warps by thread 0; red: 4 doubles per warp.  Ends with a
// __syncthreads().
__device__ __noinline__ void colp_diag(const double* dr, int ny, double inv_count, double cell, double* out,
                                       double* red)
{
    const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31, warp = tid >> 5;
    double s1 = 0, s2 = 0, mx = 0, nf = 0;
    for (int r = tid; r < ny; r += nthr) {
        s1 += __ldcg(dr + 4 * r); s2 += __ldcg(dr + 4 * r + 1);
        mx = fmax(mx, __ldcg(dr + 4 * r + 2)); nf += __ldcg(dr + 4 * r + 3);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        nf += __shfl_xor_sync(0xffffffffu, nf, o);
    }
    if (lane == 0) {
        red[4 * warp] = s1; red[4 * warp + 1] = s2; red[4 * warp + 2] = mx; red[4 * warp + 3] = nf;
    }
    __syncthreads();
    if (tid == 0) {
        double a = 0, b = 0, c = 0, d = 0;
        for (int w = 0; w < (nthr >> 5); w++) {
            a += red[4 * w]; b += red[4 * w + 1]; c = fmax(c, red[4 * w + 2]); d += red[4 * w + 3];
        }
        out[0] = a * inv_count;
        out[1] = b * cell;
        out[2] = c;
        out[3] = d;
    }
    __syncthreads();
}

// packed column 0 of the first tile: the tau-DC (re) and tau-Nyquist (im)
// sequences are separated through the row pair (l, ny - l)
template <typename T, int MODE>
__device__ __noinline__ void colp_packed(const ColArgs<T>& a, unsigned char* smem, const ColPipeLayout& L)
{
    constexpr bool ACC = sizeof(T) == 4;
    const int ny = 1 << a.log2ny, log2tc = a.log2tc;
    cx<T>* WA = reinterpret_cast<cx<T>*>(smem + L.ra);
    const cx<T>* WB = reinterpret_cast<const cx<T>*>(smem + L.rb);
    const cx<T>* P2 = reinterpret_cast<const cx<T>*>(smem + L.t0);
    for (int l = threadIdx.x; l <= (ny >> 1); l += blockDim.x) {
        const int lm = (ny - l) & (ny - 1);
        const int e = padx(l << log2tc), em = padx(lm << log2tc);
        if constexpr (MODE == COL_STAGE1) {
            const long long ti = (long long)l << a.log2n;   // folded row l, column 0
            const cx<T> E = __ldg(a.Ta + ti), P1 = __ldg(a.Tb + ti);
            const cx<T> zv = WA[e], zvm = WA[em], zb = WB[e], zbm = WB[em];
            cx<T> r = mult_entry<T>(E, zv, zvm, true);
            cx<T> rm = mult_entry<T>(E, zvm, zv, true);
            if (ACC && a.Ta_lo) {
                const cx<T> El = __ldg(a.Ta_lo + ti);
                r = add<T>(r, mult_entry<T>(El, zv, zvm, true));
                rm = add<T>(rm, mult_entry<T>(El, zvm, zv, true));
            }
            r = add<T>(r, mult_entry<T>(P1, zb, zbm, true));
            rm = add<T>(rm, mult_entry<T>(P1, zbm, zb, true));
            WA[e] = r;
            if (lm != l) WA[em] = rm;
        } else {
            const cx<T> M = P2[l << log2tc];
            const cx<T> z = WA[e], zm = WA[em];
            WA[e] = mult_entry<T>(M, z, zm, true);
            if (lm != l) WA[em] = mult_entry<T>(M, zm, z, true);
        }
    }
    __syncthreads();
}

// One column tile (CTA q = tile q).  COMP: the compensated FP32 state (the
// transforms carry increments only, so their constants need no lo parts).
template <typename T, int MODE, bool COMP = false>
__global__ void __launch_bounds__(COLP_THREADS, 2) colp_kernel(const __grid_constant__ ColPipeArgs<T> P)
{
    extern __shared__ __align__(128) unsigned char colp_smem[];
    unsigned char* smem = colp_smem;
    constexpr bool ACC = sizeof(T) == 4 && !COMP;
    const ColArgs<T>& a = P.c;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int log2ny = a.log2ny, log2tc = a.log2tc, ny = 1 << log2ny;
    const int q = blockIdx.x;
    if (q >= P.total) return;
    if (smem_addr(smem) & 127u) {   // tensor copies land on 128-byte boundaries
        if (tid == 0) atomicOr(P.flag, FLAG_BAD_LAUNCH);
        return;
    }
    const ColPipeLayout L = colp_layout<T, MODE>(ny, log2tc, P.bt, P.nbt);
    if (tid == 0) {
        unsigned long long* bar = reinterpret_cast<unsigned long long*>(smem);
        mbar_init(bar, 1);
        mbar_init(bar + 1, 1);
        mbar_fence_init();
        colp_issue_in<T, MODE>(P, smem, L, q);
        if (P.ahead > 0 && q + P.ahead < P.total) colp_prefetch<T, MODE>(P, q + P.ahead);
    }
    cx<T>* tws = reinterpret_cast<cx<T>*>(smem + L.tw);
    cx<T>* twl = reinterpret_cast<cx<T>*>(smem + L.twl);
    for (int i = tid; i < ny; i += nthr) {
        tws[i] = a.tw[i];
        if constexpr (MODE == COL_STAGE1 && ACC) twl[i] = a.tw_lo[i];
    }
    const int inst = q / P.n_tiles, m0 = (q - inst * P.n_tiles) << log2tc;
    if (MODE == COL_STAGE1 && m0 == 0 && a.diag_rows && a.diag_hist)
        colp_diag(a.diag_rows + (long long)inst * ny * 4, ny, a.inv_count, a.cell, a.diag_hist + inst * 4,
                  reinterpret_cast<double*>(smem + L.red));
    __syncthreads();
    const Tw<T> twp{tws, nullptr, -1};
    const Tw<T> twa{tws, twl, -1};
    cx<T>* WA = reinterpret_cast<cx<T>*>(smem + L.ra);
    cx<T>* WB = reinterpret_cast<cx<T>*>(smem + L.rb);
    if (!colp_wait(smem, 0, 0u, P.timeout_ns, P.flag)) return;
    // forward: dense tiles -> padded work tiles (all loads precede all stores
    // in a pass, so the work tiles may overwrite the dense ones)
    if constexpr (MODE == COL_STAGE1) {
        tile2_first<T, ACC>(log2ny, log2tc, twa, twp, tid, nthr, DenseLd<T>{WA}, DenseLd<T>{WB}, WA, WB);
        tile2_middle<T, ACC>(log2ny, log2tc, twa, twp, tid, nthr, WA, WB);
        tile2_last<T, ACC>(log2ny, log2tc, twa, twp, tid, nthr, WA, WB,
                           Mul1St2<T, ACC>{WA, WB, a.Ta, a.Ta_lo, a.Tb, log2tc, a.log2n, ny, m0});
    } else {
        cx<T>* SB = WB;
        tile_first<T, false, false>(log2ny, log2tc, twp, tid, nthr, DiffLd<T>{WA, SB}, WA);
        // b2 consumed: bring V* into region B
        if (tid == 0) colp_issue_c<T>(P, smem, L, q);
        tile_middle<T, false, false>(log2ny, log2tc, twp, tid, nthr, WA);
        tile_last<T, false, false>(log2ny, log2tc, twp, tid, nthr, WA,
                                   Mul2St<T>{WA, reinterpret_cast<const cx<T>*>(smem + L.t0), log2tc, ny, m0});
    }
    if (m0 == 0) colp_packed<T, MODE>(a, smem, L);
    // inverse -> HBM
    const long long ibase = (long long)inst * a.inst_stride;
    if constexpr (MODE == COL_STAGE1) {
        tile_first<T, true, ACC>(log2ny, log2tc, twa, tid, nthr, PadIO<T>{WA}, WA);
        tile_middle<T, true, ACC>(log2ny, log2tc, twa, tid, nthr, WA);
        tile_last<T, true, ACC>(log2ny, log2tc, twa, tid, nthr, WA,
                                OutSt<T, false, COMP>{a.out, nullptr, ibase, log2tc, a.log2n, m0, a.a, a.lo_in, a.lo_out});
    } else {
        tile_first<T, true, false>(log2ny, log2tc, twp, tid, nthr, PadIO<T>{WA}, WA);
        tile_middle<T, true, false>(log2ny, log2tc, twp, tid, nthr, WA);
        if (!colp_wait(smem, 1, 0u, P.timeout_ns, P.flag)) return;
        tile_last<T, true, false>(log2ny, log2tc, twp, tid, nthr, WA,
                                  OutSt<T, true, COMP>{a.out, WB, ibase, log2tc, a.log2n, m0, nullptr, a.lo_in, a.lo_out});
    }
}

}  // namespace kzk
