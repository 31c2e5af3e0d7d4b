// kzk_colpair.cuh -- FP32 column passes (Algorithm 2, STEP 2 and STEP 4) on
// column pairs, with in-place transforms whose middle passes stay in a warp.
//
// A CTA takes the two columns m0, m0 + 1 of one instance (ny rows) and carries
// them as the two lanes of packed FP32 values (f2 / c2, as the row-pair
// kernels do), so one FADD2 / FMUL2 / FFMA2 does the work of both columns.
// The y transforms run in place in shared memory:
//   forward: decimation in frequency, natural order in, digit-reversed out;
//   inverse: decimation in time, the conjugate transpose of the forward
//            passes in reverse order, digit-reversed in, natural order out.
// Each pass combines disjoint groups of elements where they lie, so a pass
// needs no second buffer and no barrier between its loads and stores.  With
// ny = 2^L the schedule (PairSched) is: "block" passes at strides >= 256
// (their groups span warps: a __syncthreads after each), then three "warp"
// passes (radix 8 at stride 32, radix 8 at stride 4, radix 4 at stride 1)
// that stay within the aligned 256-element block a warp owns (__syncwarp
// only).  A tile therefore sees two or three block-wide barriers per stage
// instead of two per Stockham pass, and each warp runs its middle passes at
// its own pace.
//
// The propagator multiply happens in registers between the last forward pass
// and the first inverse pass (both radix 4 at stride 1, same groups): the
// folded tables arrive in shared memory with the state tiles, each slice one
// bulk copy (the plan stores them pair-major, as lane pairs, with their rows
// permuted by pair_tab_row so that the digit-reversed row indices the warps
// read hit distinct banks).  The state tiles (16-byte rows, one per y) come by
// TMA; the tensor engine takes them at about one row per cycle, so the
// copies are ordered for overlap (STAGE1: b1 first, transformed while V and
// the tables arrive; V again into the freed b1 region for the last pass; V*
// out by a tensor store) and nothing else goes through it (no L2 prefetch of
// later tiles: that doubled the rows it had to process and made both passes
// slower; STAGE2 takes b2 - b1 from the row pass, two tiles in).  Elements of
// the work tiles sit at psw(i) = i ^ ((i >> 3) & 7) (16-byte slots), which
// makes every pass's shared-memory accesses conflict-free.  The packed column
// m = 0 (its row l is coupled with row ny - l) takes a separate pass between
// the transforms, in the one CTA per instance that holds it.
//
// Only the compensated FP32 state is handled here (the transforms carry the
// stage increment; the last pass adds it to hi + lo by TwoSum), for
// 256 <= ny <= 4096; other FP32 plans use the Stockham tile kernels.
#pragma once
#include "kzk_colpipe.cuh"
#include "kzk_rowpair.cuh"

namespace kzk {

template <int L>
struct PairSched {
    static constexpr int N = 1 << L;
    static constexpr int T = N / 8;                 // threads: 8 elements each per pass
    static constexpr int NBP = (L - 8 + 2) / 3;     // block passes
    static constexpr int NP = NBP + 3;              // all passes
    __host__ __device__ static constexpr int radix(int i)
    {
        return i < NBP ? (i < (L - 8) / 3 ? 8 : 1 << ((L - 8) % 3)) : (i < NP - 1 ? 8 : 4);
    }
    __host__ __device__ static constexpr int stride(int i)
    {
        int s = N;
        for (int j = 0; j <= i; j++) s /= radix(j);
        return s;
    }
    // frequency at position p after the forward passes, and its inverse
    __host__ __device__ static constexpr int freq(int p)
    {
        int k = 0, m = 1;
        for (int i = 0; i < NP; i++) {
            k += ((p / stride(i)) % radix(i)) * m;
            m *= radix(i);
        }
        return k;
    }
    __host__ __device__ static constexpr int pos(int k)
    {
        int p = 0;
        for (int i = 0; i < NP; i++) {
            p += (k % radix(i)) * stride(i);
            k /= radix(i);
        }
        return p;
    }
    // twiddles of pass i: (R - 1) s entries, entry (r - 1) s + q = w_{R s}^{q r}
    __host__ __device__ static constexpr int tw_off(int i)
    {
        int o = 0;
        for (int j = 0; j < i; j++) o += (radix(j) - 1) * stride(j);
        return o;
    }
    static constexpr int TW = tw_off(NP - 1);       // the stride-1 pass needs none
};

// work-tile slot of element i (16-byte slots)
__host__ __device__ __forceinline__ int psw(int i) { return i ^ ((i >> 3) & 7); }

// Shared-memory row of folded table row r: r with its low three bits XORed by
// three bits of r >> 3, chosen per length so that the rows a warp reads in the
// fused multiply fall in distinct banks (rows stay within their group of 8).
template <int L>
__host__ __device__ constexpr int pair_tab_row(int r)
{
    constexpr int a = L == 8 ? 4 : L == 9 ? 2 : L == 10 ? 3 : L == 11 ? 0 : 1;
    constexpr int b = L == 8 ? 1 : L == 9 ? 2 : L == 10 ? 4 : L == 11 ? 4 : 5;
    constexpr int c = L == 8 ? 2 : L == 9 ? 3 : L == 10 ? 3 : L == 11 ? 5 : 6;
    const int m = r >> 3;
    return r ^ (((m >> a) & 1) | (((m >> b) & 1) << 1) | (((m >> c) & 1) << 2));
}
// rows of a pair table: ny/2 + 1 folded rows, rounded up to whole groups of 8
__host__ __device__ constexpr int pair_tab_rows(int ny) { return ny / 2 + 8; }

// dense tile row (re_m0, im_m0, re_m0+1, im_m0+1) <-> lane pair
__device__ __forceinline__ c2 pair_of(float4 f) { return c2{f2(f.x, f.z), f2(f.y, f.w)}; }
__device__ __forceinline__ float4 row_of(c2 z) { return make_float4(z.x.v.x, z.y.v.x, z.x.v.y, z.y.v.y); }

// Plan time: folded table T [(ny/2 + 1)][n] -> pair table [n/2][pair_tab_rows]
// (pair-major: the slice of column pair m is one contiguous run; lane 0:
// column 2m, lane 1: column 2m + 1), row r stored at pair_tab_row(r).
template <int L>
__global__ void pair_table_kernel(const float2* __restrict__ T, c2* __restrict__ PT, int n)
{
    const int half = n / 2;
    const long long count = (long long)((1 << L) / 2 + 1) * half;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const int r = (int)(i / half), m = (int)(i - (long long)r * half);
    const float2 x = T[(long long)r * n + 2 * m], y = T[(long long)r * n + 2 * m + 1];
    PT[(long long)m * pair_tab_rows(1 << L) + pair_tab_row<L>(r)] = pack2(x, y);
}

// The lo part of the compensated state is stored pair-major for these
// kernels: the bf16 pairs of column pair m (both columns of a row side by
// side) form one contiguous run of ny rows, [batch][n/2][ny][2].
struct ColPairArgs {
    ColArgs<float> c;          // pointers and sizes, as for col_kernel (tables unused; lo pair-major)
    CUtensorMap ma, mb, mc;    // state arrays {2 n, ny, batch} floats, box {4, by, 1}
    CUtensorMap mo;            // the output state array, same shape and box
    const c2* tab0;            // pair tables [n/2][pair_tab_rows]: STAGE1 (E - 1)', STAGE2 P2'
    const c2* tab1;            // STAGE1 P1'
    const c2* tw;              // twiddles of the schedule as lane pairs
    int by, nby;               // rows per state box, boxes per tile column
    int n_tiles, total;        // column pairs per instance, CTAs
    int* flag;
    long long timeout_ns;
};

struct PairLayout {
    unsigned red, ra, rb, t0, t1, total, tile_bytes, table_bytes;
};

// mbarriers (128 B: STAGE1 b1 | V and tables | V again; STAGE2 inputs | V*);
// diagnostics scratch; region A: dense tile (V | b1), then
// the work tile; region B: dense tile (b1 | b2), then (STAGE1) the b1 work
// tile or (STAGE2) the dense V* tile; the table slice(s).
template <int L, int MODE>
__host__ __device__ constexpr PairLayout pair_layout()
{
    constexpr int N = 1 << L;
    PairLayout y{};
    y.tile_bytes = (unsigned)N * 16u;
    y.table_bytes = (unsigned)pair_tab_rows(N) * 16u;
    unsigned off = 128;
    y.red = off;
    off += up128(4 * sizeof(double) * (PairSched<L>::T / 32));
    y.ra = off;
    off += y.tile_bytes;
    y.rb = off;
    off += y.tile_bytes;
    y.t0 = off;
    off += up128(y.table_bytes);
    y.t1 = off;
    if (MODE == COL_STAGE1) off += up128(y.table_bytes);
    y.total = off;
    return y;
}

// Group u of thread tid in pass I: base element and q (offset within the stride).
template <int L, int I>
__host__ __device__ __forceinline__ void pair_group(int tid, int u, int& base, int& qq)
{
    using S = PairSched<L>;
    constexpr int R = S::radix(I), s = S::stride(I);
    if constexpr (I < S::NBP) {
        const int g = tid + S::T * u;
        qq = g & (s - 1);
        base = (g - qq) * R + qq;
    } else {
        const int w = tid >> 5, l = tid & 31;
        if constexpr (s == 32) {
            qq = l;
            base = 256 * w + l;
        } else if constexpr (s == 4) {
            qq = l & 3;
            base = 256 * w + 32 * (l >> 2) + qq;
        } else {
            qq = 0;
            base = 256 * w + 8 * l + 4 * u;
        }
    }
}

// loaders / storers of element i
struct SwzIO {
    c2* W;
    static constexpr bool DENSE = false;
    __device__ __forceinline__ c2 ld(int i) const { return W[psw(i)]; }
    __device__ __forceinline__ void st(int i, c2 v) const { W[psw(i)] = v; }
};
struct DenseIn {   // the copied tile (rows of two complex values)
    const c2* D;
    static constexpr bool DENSE = true;
    __device__ __forceinline__ c2 ld(int i) const { return pair_of(reinterpret_cast<const float4*>(D)[i]); }
};
struct DiffIn {    // STAGE2: b2 - b1 from the two copied tiles
    const c2* A;
    const c2* B;
    static constexpr bool DENSE = true;
    __device__ __forceinline__ c2 ld(int i) const
    {
        const c2 x = pair_of(reinterpret_cast<const float4*>(B)[i]);
        const c2 y = pair_of(reinterpret_cast<const float4*>(A)[i]);
        return c2{x.x - y.x, x.y - y.y};
    }
};

// One pass I, forward (DIF: butterfly, then twiddles) or inverse (conjugate
// twiddles, then butterfly), every group of the thread.  A dense input (the
// first pass) is rewritten into the permuted slots of the same 8-element
// groups, which other lanes of the same warp read: __syncwarp in between.
template <int L, int I, bool FWD, class LD, class ST>
__device__ __forceinline__ void pair_pass(const c2* __restrict__ tw, int tid, LD ld, ST st)
{
    using S = PairSched<L>;
    constexpr int R = S::radix(I), s = S::stride(I), G = 8 / R, off = S::tw_off(I);
    c2 v[G][R];
    int bs[G];
#pragma unroll
    for (int u = 0; u < G; u++) {
        int base, qq;
        pair_group<L, I>(tid, u, base, qq);
        bs[u] = base;
#pragma unroll
        for (int j = 0; j < R; j++) v[u][j] = ld.ld(base + s * j);
        if constexpr (FWD) {
            RegDFT<f2, R, -1, false>::run(v[u]);
            if constexpr (s > 1) {
#pragma unroll
                for (int r = 1; r < R; r++) v[u][r] = mul<f2>(v[u][r], tw[off + (r - 1) * s + qq]);
            }
        } else {
            if constexpr (s > 1) {
#pragma unroll
                for (int r = 1; r < R; r++) v[u][r] = mulc<f2>(v[u][r], tw[off + (r - 1) * s + qq]);
            }
            RegDFT<f2, R, 1, false>::run(v[u]);
        }
    }
    if constexpr (LD::DENSE) __syncwarp();
#pragma unroll
    for (int u = 0; u < G; u++)
#pragma unroll
        for (int j = 0; j < R; j++) st.st(bs[u] + s * j, v[u][j]);
}

// Forward transform of region W up to (not including) the last pass; the
// first pass reads `in`.  Ends with a __syncwarp (the last pass stays in the warp).
template <int L, class IN>
__device__ __forceinline__ void pair_forward_head(c2* W, IN in, const c2* tw, int tid)
{
    using S = PairSched<L>;
    const SwzIO io{W};
    pair_pass<L, 0, true>(tw, tid, in, io);
    if constexpr (S::NBP >= 1) __syncthreads(); else __syncwarp();
    if constexpr (S::NBP >= 2) {
        pair_pass<L, 1, true>(tw, tid, io, io);
        __syncthreads();
    }
    if constexpr (S::NBP > 0) {   // the first warp pass, unless it was pass 0
        pair_pass<L, S::NBP, true>(tw, tid, io, io);
        __syncwarp();
    }
    pair_pass<L, S::NP - 2, true>(tw, tid, io, io);
    __syncwarp();
}

// Last forward pass, the propagator multiply and the first inverse pass of a
// non-packed tile, in registers (radix 4 at stride 1: positions 8 lane + 4 u + j).
// STAGE1: X = (E - 1)' V_hat + P1' b1_hat (b1_hat in B, written by this lane);
// STAGE2: X = P2' (b2 - b1)_hat.
template <int L, int MODE>
__device__ __forceinline__ void pair_fused(c2* A, const c2* B, const c2* T0, const c2* T1, int tid)
{
    using S = PairSched<L>;
    constexpr int N = S::N;
    c2 v[2][4];
    int bs[2];
#pragma unroll
    for (int u = 0; u < 2; u++) {
        int qq;
        pair_group<L, S::NP - 1>(tid, u, bs[u], qq);
#pragma unroll
        for (int j = 0; j < 4; j++) v[u][j] = A[psw(bs[u] + j)];
        RegDFT<f2, 4, -1, false>::run(v[u]);
#pragma unroll
        for (int r = 0; r < 4; r++) {
            const int p = bs[u] + r, k = S::freq(p);
            const int tr = pair_tab_row<L>(k <= N / 2 ? k : N - k);
            if constexpr (MODE == COL_STAGE1) {
                const c2 o = mul<f2>(T0[tr], v[u][r]);
                v[u][r] = fma_c<f2>(T1[tr], B[psw(p)], o);
            } else {
                v[u][r] = mul<f2>(T0[tr], v[u][r]);
            }
        }
        RegDFT<f2, 4, 1, false>::run(v[u]);
    }
#pragma unroll
    for (int u = 0; u < 2; u++)
#pragma unroll
        for (int j = 0; j < 4; j++) A[psw(bs[u] + j)] = v[u][j];
}

// The packed tile (m0 = 0): multiply with column 0 separated through the row
// pair (l, ny - l), after the forward transforms are complete in A (and B).
template <int L, int MODE>
__device__ __noinline__ void pair_fixup(c2* A, const c2* B, const c2* T0, const c2* T1)
{
    using S = PairSched<L>;
    constexpr int N = S::N;
    for (int l = threadIdx.x; l <= N / 2; l += blockDim.x) {
        const int pa = psw(S::pos(l)), pb = psw(S::pos((N - l) & (N - 1)));
        const int tr = pair_tab_row<L>(l);
        const c2 z = A[pa], zm = A[pb];
        float2 r0, rm0, r1, rm1;
        if constexpr (MODE == COL_STAGE1) {
            const c2 zb = B[pa], zbm = B[pb], E = T0[tr], P1 = T1[tr];
            r0 = add<float>(mult_entry<float>(lane0(E), lane0(z), lane0(zm), true),
                            mult_entry<float>(lane0(P1), lane0(zb), lane0(zbm), true));
            rm0 = add<float>(mult_entry<float>(lane0(E), lane0(zm), lane0(z), true),
                             mult_entry<float>(lane0(P1), lane0(zbm), lane0(zb), true));
            r1 = fma_c<float>(lane1(P1), lane1(zb), mul<float>(lane1(E), lane1(z)));
            rm1 = fma_c<float>(lane1(P1), lane1(zbm), mul<float>(lane1(E), lane1(zm)));
        } else {
            const c2 M = T0[tr];
            r0 = mult_entry<float>(lane0(M), lane0(z), lane0(zm), true);
            rm0 = mult_entry<float>(lane0(M), lane0(zm), lane0(z), true);
            r1 = mul<float>(lane1(M), lane1(z));
            rm1 = mul<float>(lane1(M), lane1(zm));
        }
        A[pa] = pack2(r0, r1);
        if (pb != pa) A[pb] = pack2(rm0, rm1);
    }
}

// Copies of CTA q.  STAGE1: the b1 tile into B (barrier 0), then the table
// slices (one contiguous run each) and the V tile into A (barrier 1), so the
// transform of b1 runs while the rest arrives.  STAGE2: the table slice and
// both tiles (barrier 0); D2 (the row pass stored b2 - b1): that tile into A
// and the table (barrier 0), V* into B at once (barrier 1).
template <int MODE, bool D2>
__device__ __forceinline__ void pair_issue_in(const ColPairArgs& P, unsigned char* smem, const PairLayout& y, int q)
{
    unsigned long long* bar = reinterpret_cast<unsigned long long*>(smem);
    const int inst = q / P.n_tiles, m = q - inst * P.n_tiles, x = 4 * m;
    const unsigned box = y.tile_bytes / P.nby;
    const long long toff = (long long)m * (y.table_bytes / 16);
    if (MODE == COL_STAGE1) {
        mbar_expect(bar, y.tile_bytes);
        for (int k = 0; k < P.nby; k++) tma_load_3d(smem + y.rb + k * box, &P.mb, x, k * P.by, inst, bar);
        mbar_expect(bar + 1, y.tile_bytes + 2 * y.table_bytes);
        bulk_load(smem + y.t0, P.tab0 + toff, y.table_bytes, bar + 1);
        bulk_load(smem + y.t1, P.tab1 + toff, y.table_bytes, bar + 1);
        for (int k = 0; k < P.nby; k++) tma_load_3d(smem + y.ra + k * box, &P.ma, x, k * P.by, inst, bar + 1);
    } else if (D2) {
        mbar_expect(bar, y.tile_bytes + y.table_bytes);
        for (int k = 0; k < P.nby; k++) tma_load_3d(smem + y.ra + k * box, &P.mb, x, k * P.by, inst, bar);
        bulk_load(smem + y.t0, P.tab0 + toff, y.table_bytes, bar);
        mbar_expect(bar + 1, y.tile_bytes);
        for (int k = 0; k < P.nby; k++) tma_load_3d(smem + y.rb + k * box, &P.mc, x, k * P.by, inst, bar + 1);
    } else {
        mbar_expect(bar, 2 * y.tile_bytes + y.table_bytes);
        bulk_load(smem + y.t0, P.tab0 + toff, y.table_bytes, bar);
        for (int k = 0; k < P.nby; k++) {
            tma_load_3d(smem + y.ra + k * box, &P.ma, x, k * P.by, inst, bar);
            tma_load_3d(smem + y.rb + k * box, &P.mb, x, k * P.by, inst, bar);
        }
    }
}
// The state hi the increment is added to, into B once B is free (STAGE1: V
// on barrier 2; STAGE2: V* on barrier 1)
template <int MODE>
__device__ __forceinline__ void pair_issue_c(const ColPairArgs& P, unsigned char* smem, const PairLayout& y, int q)
{
    unsigned long long* bar = reinterpret_cast<unsigned long long*>(smem) + (MODE == COL_STAGE1 ? 2 : 1);
    const CUtensorMap* m = MODE == COL_STAGE1 ? &P.ma : &P.mc;
    const int inst = q / P.n_tiles, x = 4 * (q - inst * P.n_tiles);
    const unsigned box = y.tile_bytes / P.nby;
    mbar_expect(bar, y.tile_bytes);
    for (int k = 0; k < P.nby; k++) tma_load_3d(smem + y.rb + k * box, m, x, k * P.by, inst, bar);
}

// tensor store of a shared-memory box, its bulk group, and the wait for its
// reads of shared memory
__device__ __forceinline__ void tma_store_3d(const CUtensorMap* m, const void* src, int x, int y, int z)
{
    asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%2, %3, %4}], [%1];" ::"l"(
                     reinterpret_cast<unsigned long long>(m)),
                 "r"(smem_addr(src)), "r"(x), "r"(y), "r"(z)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
// Last inverse pass (pass 0): the increment v is added to the state hi + lo
// by TwoSum, hi from the copy in B (STAGE1: V, STAGE2: V*), lo from HBM
// (loaded before the wait for that copy, which is also the barrier the pass
// needs); the lo rows (pair-major: coalesced) are stored directly.  STAGE1
// writes the new hi rows over A in row order and sends them by a tensor store
// (C1 then loads 3 tiles and stores 1 through the tensor engine); STAGE2,
// whose engine already takes 3 tiles in, stores its rows from the threads.
template <int L, int MODE>
__device__ __forceinline__ bool pair_last(const ColPairArgs& P, unsigned char* smem, c2* A, const c2* B,
                                          long long gbase, long long lbase, int inst, int m, int tid)
{
    constexpr bool TOUT = MODE == COL_STAGE1;
    using S = PairSched<L>;
    constexpr int R = S::radix(0), s = S::stride(0), G = 8 / R, off = S::tw_off(0);
    const ColArgs<float>& a = P.c;
    int bs[G], qs[G];
    uint2 lo[G][R];
#pragma unroll
    for (int u = 0; u < G; u++) {
        pair_group<L, 0>(tid, u, bs[u], qs[u]);
#pragma unroll
        for (int j = 0; j < R; j++)
            lo[u][j] = __ldcg(reinterpret_cast<const uint2*>(a.lo_in + lbase + 2 * (bs[u] + s * j)));
    }
    if (!colp_wait(smem, MODE == COL_STAGE1 ? 2 : 1, 0u, P.timeout_ns, P.flag)) return false;
    c2 v[G][R];
#pragma unroll
    for (int u = 0; u < G; u++) {
#pragma unroll
        for (int r = 0; r < R; r++) v[u][r] = A[psw(bs[u] + s * r)];
        if constexpr (s > 1) {
#pragma unroll
            for (int r = 1; r < R; r++) v[u][r] = mulc<f2>(v[u][r], P.tw[off + (r - 1) * s + qs[u]]);
        }
        RegDFT<f2, R, 1, false>::run(v[u]);
    }
    if constexpr (TOUT) __syncwarp();   // row e's slot held element psw(e), read above by a lane of this warp
    float4* out = reinterpret_cast<float4*>(A);
#pragma unroll
    for (int u = 0; u < G; u++)
#pragma unroll
        for (int j = 0; j < R; j++) {
            const int row = bs[u] + s * j;
            __nv_bfloat162 l0, l1;
            memcpy(&l0, &lo[u][j].x, 4);
            memcpy(&l1, &lo[u][j].y, 4);
            const c2 lc = pack2(__bfloat1622float2(l0), __bfloat1622float2(l1));
            c2 sh, sl;
            comp_add<f2>(pair_of(reinterpret_cast<const float4*>(B)[row]), lc, v[u][j], sh, sl);
            if constexpr (TOUT) out[row] = row_of(sh);
            else *reinterpret_cast<float4*>(a.out + gbase + ((long long)row << a.log2n)) = row_of(sh);
            const __nv_bfloat162 o0 = __float22bfloat162_rn(lane0(sl)), o1 = __float22bfloat162_rn(lane1(sl));
            uint2 w;
            memcpy(&w.x, &o0, 4);
            memcpy(&w.y, &o1, 4);
            *reinterpret_cast<uint2*>(a.lo_out + lbase + 2 * row) = w;
        }
    if constexpr (!TOUT) return true;
    fence_async_smem();
    __syncthreads();
    if (tid == 0) {
        const unsigned box = S::N * 16u / P.nby;
        for (int k = 0; k < P.nby; k++)
            tma_store_3d(&P.mo, reinterpret_cast<const unsigned char*>(A) + k * box, 4 * m, k * P.by, inst);
        bulk_commit();
        bulk_wait_read();
    }
    return true;
}

// One column pair (CTA q = pair q), compensated FP32 state.  D2 (STAGE2): the
// input array b holds b2 - b1 (written so by the row-pair pass).
template <int L, int MODE, bool D2 = false>
__global__ void __launch_bounds__(PairSched<L>::T, 512 / PairSched<L>::T) colpair_kernel(
    const __grid_constant__ ColPairArgs P)
{
    using S = PairSched<L>;
    constexpr int N = S::N;
    extern __shared__ __align__(128) unsigned char cpair_smem[];
    unsigned char* smem = cpair_smem;
    const ColArgs<float>& a = P.c;
    const int tid = threadIdx.x;
    const int q = blockIdx.x;
    if (q >= P.total) return;
    if (smem_addr(smem) & 127u) {
        if (tid == 0) atomicOr(P.flag, FLAG_BAD_LAUNCH);
        return;
    }
    const PairLayout y = pair_layout<L, MODE>();
    if (tid == 0) {
        unsigned long long* bar = reinterpret_cast<unsigned long long*>(smem);
        mbar_init(bar, 1);
        mbar_init(bar + 1, 1);
        mbar_init(bar + 2, 1);
        mbar_fence_init();
        pair_issue_in<MODE, D2>(P, smem, y, q);
    }
    const int inst = q / P.n_tiles, m0 = 2 * (q - inst * P.n_tiles);
    if (MODE == COL_STAGE1 && m0 == 0 && a.diag_rows && a.diag_hist)
        colp_diag(a.diag_rows + (long long)inst * N * 4, N, a.inv_count, a.cell, a.diag_hist + inst * 4,
                  reinterpret_cast<double*>(smem + y.red));
    __syncthreads();   // barrier initialisation visible to every waiting thread
    c2* A = reinterpret_cast<c2*>(smem + y.ra);
    c2* B = reinterpret_cast<c2*>(smem + y.rb);
    const c2* T0 = reinterpret_cast<const c2*>(smem + y.t0);
    const c2* T1 = reinterpret_cast<const c2*>(smem + y.t1);
    const c2* tw = P.tw;
    // copies in flight: STAGE1 and D2 issued barriers 0 and 1 up front
    if (!colp_wait(smem, 0, 0u, P.timeout_ns, P.flag, MODE == COL_STAGE1 || D2 ? 3u : 1u)) return;
    const SwzIO ia{A};
    if constexpr (MODE == COL_STAGE1) {
        pair_forward_head<L>(B, DenseIn{B}, tw, tid);
        pair_pass<L, S::NP - 1, true>(tw, tid, SwzIO{B}, SwzIO{B});   // b1_hat, read back by the same lane
        if (!colp_wait(smem, 1, 0u, P.timeout_ns, P.flag)) return;
        pair_forward_head<L>(A, DenseIn{A}, tw, tid);
    } else if constexpr (D2) {
        pair_forward_head<L>(A, DenseIn{A}, tw, tid);
    } else {
        pair_forward_head<L>(A, DiffIn{A, B}, tw, tid);
    }
    // STAGE2: b2 is consumed once every warp has passed its first pass (a
    // block-wide barrier follows pass 0 when it spans warps; one warp otherwise)
    if constexpr (MODE == COL_STAGE2 && !D2) {
        if constexpr (S::NBP == 0) __syncthreads();
        if (tid == 0) pair_issue_c<MODE>(P, smem, y, q);
    }
    if (m0 != 0) {
        pair_fused<L, MODE>(A, B, T0, T1, tid);
    } else {
        pair_pass<L, S::NP - 1, true>(tw, tid, ia, ia);
        __syncthreads();
        pair_fixup<L, MODE>(A, B, T0, T1);
        __syncthreads();
        pair_pass<L, S::NP - 1, false>(tw, tid, ia, ia);
    }
    // STAGE1: b1_hat consumed by every warp; bring V into B for the last pass
    if constexpr (MODE == COL_STAGE1) {
        __syncthreads();
        if (tid == 0) pair_issue_c<MODE>(P, smem, y, q);
    }
    __syncwarp();
    // inverse: the remaining warp passes, then the block passes; pass 0 to HBM
    if constexpr (S::NP - 2 > 0) {
        pair_pass<L, S::NP - 2, false>(tw, tid, ia, ia);
        __syncwarp();
    }
    if constexpr (S::NP - 3 > 0) {
        pair_pass<L, S::NP - 3, false>(tw, tid, ia, ia);
        __syncwarp();
    }
    if constexpr (S::NBP >= 2) {
        __syncthreads();
        pair_pass<L, 1, false>(tw, tid, ia, ia);
    }
    pair_last<L, MODE>(P, smem, A, B, (long long)inst * a.inst_stride + m0,
                       (long long)inst * a.inst_stride + (long long)m0 * N, inst, m0 / 2, tid);
}

}  // namespace kzk
