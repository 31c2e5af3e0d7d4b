// kzk_api.cu -- plan management and the C ABI of include/kzk.h.
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/kzk.h"
#include "kzk_adjoint.cuh"
#include "kzk_batched.cuh"
#include "kzk_colpipe.cuh"
#include "kzk_kernels.cuh"
#include "kzk_medium.cuh"
#include "kzk_mixed.cuh"
#include "kzk_rowpair.cuh"
#include "kzk_tables.cuh"
// after the FP64 headers: the pair type's overloads (kzk_rowpair.cuh) would hide
// the scalar math functions they call inside namespace kzk
#include "kzk_colpair.cuh"
#include "kzk_copyrate.cuh"
#include "kzk_ysweep_pair.cuh"

using namespace kzk;

namespace {

thread_local char g_err[512] = "";
std::atomic<long long> g_launches{0};

kzk_status fail(kzk_status s, const char* fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return s;
}

#define KZK_CUDA(call)                                                                         \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            return fail(e_ == cudaErrorMemoryAllocation ? KZK_ERR_OOM : KZK_ERR_CUDA,          \
                        "%s:%d %s: %s", __FILE__, __LINE__, #call, cudaGetErrorString(e_));    \
    } while (0)

#define KZK_LAUNCHED()                                                                         \
    do {                                                                                       \
        g_launches.fetch_add(1, std::memory_order_relaxed);                                    \
        cudaError_t e_ = cudaGetLastError();                                                   \
        if (e_ != cudaSuccess)                                                                 \
            return fail(KZK_ERR_CUDA, "%s:%d launch: %s", __FILE__, __LINE__,                  \
                        cudaGetErrorString(e_));                                               \
    } while (0)

#define KZK_TRY(expr)                                                                          \
    do {                                                                                       \
        kzk_status s_ = (expr);                                                                \
        if (s_ != KZK_OK) return s_;                                                           \
    } while (0)

bool is_pow2(long long v) { return v > 0 && (v & (v - 1)) == 0; }

double horner(const double* c, double s) { return ((c[3] * s + c[2]) * s + c[1]) * s + c[0]; }

}  // namespace

struct kzk_plan_s {
    kzk_grid g;
    kzk_coeffs c;
    kzk_options opt;            // the choices requested at creation (KZK_AUTO where left open)
    double dt;
    int batch;
    int prec;
    int nx, ny, n, log2nx, log2ny;
    size_t csz;
    long long inst_stride;      // complex elements per instance: ny * nx / 2
    void *V, *b1, *vs, *b2;     // spectral work arrays [batch][ny][nx/2]
    void *E, *P1, *P2;          // folded, scaled tables [(ny/2+1)][nx/2]
    void* E_lo;                 // FP32 plans: lo part of E' (two-float E')
    void *twr, *twc;            // twiddles, exp(-2 pi i k / nx), exp(-2 pi i k / ny)
    void* twc_lo;               // FP32 plans: lo part of the staged y twiddles
    void* tws_row;              // staged twiddles of the row (length nx/2) FFT
    void* twc_full;             // full y twiddle table exp(-2 pi i k / ny) (adjoint kernels)
    double* diag_rows;          // [batch][ny][4]
    double* diag_hist;          // [hist_cap][batch][4]
    double* diag_final;         // [batch][4]
    long long hist_cap;
    long long hist_steps;
    int row_thr, col_thr, log2tc, adj_row_thr;
    size_t row_smem, col_smem, adj_smem;
    // TMA-staged Stockham column kernels (kzk_colpipe.cuh): colp_ok = the plan
    // fits them (configuration colp_l2 ...); colp_log2tc < 0: not in use
    int colp_ok, colp_l2;
    int colp_log2tc, colp_thr, colp_by, colp_nby, colp_bt, colp_nbt, sm_count;
    size_t colp_smem1, colp_smem2;
    int* colp_flag;             // device: FLAG_TIMEOUT from a copy wait that ran out
    // random medium of Algorithm 1 (kzk_plan_set_medium); med_n = 0: homogeneous
    int med_n, med_nb;          // modes; CTAs of the coefficient kernel (= entries of each bmax)
    void* med_Ty;               // device [N][ny] double2: exp(i |K_n| lambda sin(theta_n) y_j)
    double* med_mode;           // device [5][N]: a_sig, phase, w0, w1, w2 (see kzk_medium.cuh)
    double* med_coef;           // device [2][ny][3]: U_par, U_perp, dU_perp/dy of stages 1 and 2
    double* med_bmax;           // device [2][med_nb]
    void* uphys;                // device [batch][ny][nx]: physical rows of the current stage
    void* by;                   // device [batch][ny][nx]: y-flux difference + source of the current stage
    // adjoint workspace (allocated on first use)
    void *lam, *mu, *nu, *ls;   // spectral adjoint arrays
    void* seg;                  // segment store: physical u^n, u*^n of k steps, [(2 k)][batch][ny][nx]
    void* ckpt;                 // checkpoints  [n_ckpt][batch][ny][nx/2]
    long long seg_cap, ckpt_cap; // in arrays
    long long ck_steps;         // forward run whose checkpoints are stored (0: none)
    double ck_sigma0;
    int ck_every;
    // batched plans (kzk_plan_create_batched): one sub-plan per instance
    int batched;
    std::vector<kzk_plan_s*>* subs;
    void* binst;                // device BatchInst<T>[n]
    int* row_prefix;            // device [n + 1]
    int* col_prefix;            // device [n + 1]
    void* coef;                 // device [coef_cap steps][n][6]
    long long coef_cap;
    unsigned* bar;              // device: count, generation, flag
    int grid_ctas;
    size_t batch_smem;
    int tile_cap;               // autotuned cap on log2 of the column tile width
    long long graph_steps;      // steps the cached graph advances
    cudaGraphExec_t graph;
    unsigned test_extra_blocks; // testing hook: barrier waits for this many extra CTAs
    long long timeout_ns;
    cudaStream_t cap_stream;    // capturable stream for building the graph
    // streams mode (the default): the graph advances every instance on its own stream
    int batch_streams;
    double graph_sigma0;
    std::vector<void*>* graph_u;        // state pointers the cached graph was captured with
    std::vector<cudaStream_t>* side;    // one captured stream per instance
    std::vector<cudaEvent_t>* evs;      // fork event, then one join event per instance
    // grids whose sizes are not powers of two (kzk_mixed.cuh)
    int mixed;
    MixFFT mrow, mcol;          // radix schedules of the tau (length nx/2) and y transforms
    int *mpos_row, *mpos_col;   // device: position of each frequency after the forward passes
    int* mipos_col;             // device: frequency at each position (y)
    void* wsc;                  // device [batch][ny][nx/2]: P1' FFT_y(b1) between the two C1 launches
    int mrow_thr, mcol_lc, mcol_thr;
    size_t mrow_smem, mcol_smem;
    int madj_thr, madj_Q;       // transposed row pass: threads, WENO chunk length (0: not available)
    size_t madj_smem;
    // FP32 plans: compensated state (the spectral state as hi + lo; the column
    // passes transform increments, with the table (E - 1)/ny)
    int comp;
    void *Vlo, *vslo;           // lo parts of V and V*
    void* Em1;                  // (E - 1)/ny, folded as E'
    // FP32 plans: row passes on row pairs in packed FP32 (kzk_rowpair.cuh);
    // rowpair_ok = the plan fits them, rowpair = in use
    int rowpair_ok, rowpair;
    size_t rowpair_smem, rowpair_ct_smem;   // the length-specialised b passes also hold the row twiddles
    int rowpair_ct_ok;                      // ... and fit the device's shared memory
    void *twr2, *tws2;          // the tau twiddle tables with every entry as a lane pair
    // FP32 plans with the compensated state: column passes on column pairs
    // (kzk_colpair.cuh); colpair_ok = the plan fits them, colpair = in use
    int colpair_ok, colpair, cpair_by, cpair_nby;
    int cpair_diff;             // row pairs store b2 - b1 for the column-pair STAGE2 (both kernels in use)
    size_t cpair_smem1, cpair_smem2;
    void *Em1p, *P1p, *P2p;     // (E - 1)', P1', P2' as pair tables [nx/4][pair_tab_rows(ny)]
    void* twcp;                 // twiddles of the pair schedule, as lane pairs
    // FP64 plans on the per-tile column kernels: the state's normalised
    // y-spectrum Sigma = FFT_y(V) / ny carried between steps (column modes
    // FWD / S1 / S2, four y-transforms per step); ysig_ok = the plan has the
    // arrays, the path is in use while the per-tile kernels are
    int ysig_ok;
    void *ysig, *ytmp;          // Sigma and the stage-1 intermediate T, [batch][ny][nx/2]
    // kzk_advance from captured graphs: gx[0] advances GRAPH_CHUNK steps,
    // gx[1] one step, both on the plan's arrays; the sigma-dependent values of
    // the steps a replay covers come from dcoef ([GRAPH_CHUNK][2][4]: sigma,
    // B, B M, nx (A - A0) of each stage), written before each replay; the
    // replays write their diagnostics to dhist, copied to diag_hist after each
    cudaGraphExec_t gx[2];
    long long gx_kernels[2];    // kernels in each (counted by kzk_launch_count at every replay)
    double* dcoef;
    double* dhist;
};

namespace {

double B_of(const kzk_plan* p, double s) { return p->c.has_profile ? p->c.B * horner(p->c.B_prof, s) : p->c.B; }
double dA_of(const kzk_plan* p, double s)
{
    return p->c.has_profile ? p->c.A * horner(p->c.A_prof, s) - p->c.A : 0.0;
}

template <typename T> constexpr int row_ppt() { return 8; }
template <typename T> size_t adj_row_smem(const kzk_plan* p) { return adj_row_smem_bytes<T>(p->n, p->adj_row_thr); }

template <typename T, int MODE>
kzk_status set_row_attr(size_t smem)
{
    KZK_CUDA(cudaFuncSetAttribute(row_kernel<T, MODE>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    return KZK_OK;
}
template <typename T, int MODE>
kzk_status set_col_attr(size_t smem)
{
    KZK_CUDA(cudaFuncSetAttribute(col_kernel<T, MODE>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    return KZK_OK;
}
template <typename T, int MODE>
kzk_status set_adj_row_attr(size_t smem)
{
    KZK_CUDA(cudaFuncSetAttribute(adj_row_kernel<T, row_ppt<T>(), MODE>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    if constexpr (sizeof(T) == 8)
        KZK_CUDA(cudaFuncSetAttribute(adj_row_kernel<T, row_ppt<T>(), MODE, 128, 3>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    return KZK_OK;
}
template <typename T, int MODE>
kzk_status set_adj_col_attr(size_t smem)
{
    KZK_CUDA(cudaFuncSetAttribute(adj_col_kernel<T, col_ppt_of<T>(), MODE>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    return KZK_OK;
}

// cuTensorMapEncodeTiled from the driver, looked up once through the runtime
// (no link-time dependency on libcuda)
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled()
{
    static const EncodeTiledFn fn = []() -> EncodeTiledFn {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return nullptr;
        return reinterpret_cast<EncodeTiledFn>(f);
    }();
    return fn;
}

// Table slices are copied in nbt boxes of bt rows (bt a multiple of 128 bytes
// / row bytes, so that every box lands 128-byte aligned; rows past ny/2 + 1
// are filled with zeros by the copy and never read).
void table_boxes(int nl, int row_bytes, int* bt, int* nbt)
{
    const int ra = row_bytes >= 128 ? 1 : 128 / row_bytes;
    *nbt = (nl + 255) / 256;
    const int per = (nl + *nbt - 1) / *nbt;
    *bt = (per + ra - 1) / ra * ra;
}

// Widest column tile (TC <= 16 columns) of the TMA-staged column kernels:
// ny TC / 8 threads (at most COLP_THREADS, at least one warp), rows of at
// least 16 bytes (TMA's innermost extent and coordinate alignment), and both
// stages' shared memory within the device limit.  Sets colp_ok and the
// configuration; whether the kernels are used is select_kernels' choice.
template <typename T>
void colp_configure(kzk_plan* p, int optin)
{
    p->colp_ok = 0;
    p->colp_log2tc = -1;
    if (p->log2ny < 4 || !encode_tiled()) return;
    for (int l2 = 4; l2 >= 0; l2--) {
        const int TC = 1 << l2;
        if (TC > p->n || TC * (int)sizeof(cx<T>) < 16) continue;
        const long long thr = ((long long)p->ny << l2) / 8;
        if (thr > COLP_THREADS || thr < 32) continue;
        int bt = 0, nbt = 0;
        table_boxes(p->ny / 2 + 1, TC * (int)sizeof(cx<T>), &bt, &nbt);
        const size_t s1 = colp_layout<T, COL_STAGE1>(p->ny, l2, bt, nbt).total;
        const size_t s2 = colp_layout<T, COL_STAGE2>(p->ny, l2, bt, nbt).total;
        if (std::max(s1, s2) > (size_t)optin) continue;
        p->colp_ok = 1;
        p->colp_l2 = l2;
        p->colp_thr = (int)thr;
        p->colp_bt = bt;
        p->colp_nbt = nbt;
        p->colp_by = std::min(p->ny, 256);
        p->colp_nby = p->ny / p->colp_by;
        p->colp_smem1 = s1;
        p->colp_smem2 = s2;
        return;
    }
}

// Column-pair kernels (kzk_colpair.cuh): FP32 plans with the compensated
// state, 256 <= ny <= 4096; sets colpair_ok when the plan fits them.
template <int L>
kzk_status cpair_attr(kzk_plan* p, int optin)
{
    const size_t s1 = pair_layout<L, COL_STAGE1>().total;
    const size_t s2 = pair_layout<L, COL_STAGE2>().total;
    if (std::max(s1, s2) > (size_t)optin) return KZK_OK;
    KZK_CUDA(cudaFuncSetAttribute(colpair_kernel<L, COL_STAGE1>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
    KZK_CUDA(cudaFuncSetAttribute(colpair_kernel<L, COL_STAGE2>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
    KZK_CUDA(cudaFuncSetAttribute(colpair_kernel<L, COL_STAGE2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  optin));
    int per_sm = 0;
    KZK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, colpair_kernel<L, COL_STAGE1>, PairSched<L>::T,
                                                           s1));
    if (per_sm < 1) return KZK_OK;
    p->cpair_smem1 = s1;
    p->cpair_smem2 = s2;
    p->colpair_ok = 1;
    return KZK_OK;
}
template <typename T>
kzk_status cpair_configure(kzk_plan* p, int optin)
{
    p->colpair_ok = 0;
    p->colpair = 0;
    if (sizeof(T) != 4 || !p->comp || p->mixed) return KZK_OK;
    if (p->log2ny < 8 || p->log2ny > 12 || p->n < 2 || !encode_tiled()) return KZK_OK;
    p->cpair_by = std::min(p->ny, 256);
    p->cpair_nby = p->ny / p->cpair_by;
    switch (p->log2ny) {
    case 8: return cpair_attr<8>(p, optin);
    case 9: return cpair_attr<9>(p, optin);
    case 10: return cpair_attr<10>(p, optin);
    case 11: return cpair_attr<11>(p, optin);
    default: return cpair_attr<12>(p, optin);
    }
}

void drop_step_graphs(kzk_plan* p)
{
    for (cudaGraphExec_t& g : p->gx)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
}

// Put a row / column kernel choice (KZK_ROW_*, KZK_COL_*; both eligible) in use.
void select_kernels(kzk_plan* p, int row, int col)
{
    drop_step_graphs(p);   // captured with the previous kernels
    p->rowpair = row == KZK_ROW_PAIR ? 1 : 0;
    p->colpair = col == KZK_COL_PAIR ? 1 : 0;
    p->colp_log2tc = col == KZK_COL_TMA ? p->colp_l2 : -1;
    // row pairs storing b2 - b1 feed the column-pair STAGE2 directly
    p->cpair_diff = p->colpair && p->rowpair;
}

// The row / column kernels in use, as KZK_ROW_* / KZK_COL_* values.
int row_choice(const kzk_plan* p) { return p->rowpair ? KZK_ROW_PAIR : KZK_ROW_SINGLE; }
int col_choice(const kzk_plan* p)
{
    return p->colpair ? KZK_COL_PAIR : p->colp_log2tc >= 0 ? KZK_COL_TMA : KZK_COL_TILE;
}

// Mixed-radix plans: one row per CTA; column tiles of the widest power of two
// (at most 16) dividing nx/2 whose tile fits 96 KB (two CTAs per SM), else
// single columns up to the device's shared-memory limit.
template <typename T>
kzk_status configure_mixed(kzk_plan* p)
{
    if (!mix_plan(p->n, 2, &p->mrow) || !mix_plan(p->ny, 1, &p->mcol))
        return fail(KZK_ERR_SIZE, "nx/2 = %d and ny = %d must have no prime factor above 7", p->n, p->ny);
    int dev = 0, optin = 0;
    KZK_CUDA(cudaGetDevice(&dev));
    KZK_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    KZK_CUDA(cudaDeviceGetAttribute(&p->sm_count, cudaDevAttrMultiProcessorCount, dev));
    p->mrow_thr = mix_row_threads(p->nx);
    p->mrow_smem = mix_row_smem<T>(p->nx, p->mrow_thr);
    int lc = 0;
    // widest tile within 96 KB (two CTAs per SM) that still leaves tiles for
    // three quarters of the SMs (measured on the paper's grids: 28 tiles of
    // eight columns lose to narrower ones; 112 of four beat 224 of two)
    while (lc < 4 && p->n % (2 << lc) == 0 && (size_t)p->ny * (2 << lc) * sizeof(cx<T>) <= 96 * 1024 &&
           4 * (p->n >> (lc + 1)) * p->batch >= 3 * p->sm_count)
        lc++;
    // FP32 columns too long for two per tile at two CTAs per SM still take two (one CTA per SM) where
    // they fit: the 8-byte rows of a single column use a quarter of each 32-byte sector
    if (sizeof(T) == 4 && lc == 0 && p->n % 2 == 0 && (size_t)p->ny * 2 * sizeof(cx<T>) > 96 * 1024 &&
        (size_t)p->ny * 2 * sizeof(cx<T>) <= (size_t)optin)
        lc = 1;
    p->mcol_lc = lc;
    // threads of the forward column passes: 512 (two CTAs per SM), or the
    // FP32 maximum where one tile takes more than half of the SM
    p->mcol_thr = ((size_t)p->ny << lc) * sizeof(cx<T>) > 96 * 1024 ? mix_col_max_threads<T>() : MIX_COL_THREADS;
    p->mcol_smem = std::max(((size_t)p->ny << lc) * sizeof(cx<T>), 4 * (size_t)mix_col_max_threads<T>() * sizeof(double));
    if (p->mrow_smem > (size_t)optin || p->mcol_smem > (size_t)optin)
        return fail(KZK_ERR_SIZE, "grid %d x %d needs more shared memory than the device offers", p->nx, p->ny);
    p->colp_log2tc = -1;
    // transposed row pass: chunks of Q points (the largest divisor of nx in
    // [4, 16]), one thread per chunk
    p->madj_Q = 0;
    for (int q = 16; q >= 4; q--)
        if (p->nx % q == 0 && p->nx / q <= MIX_ROW_MAX_THREADS) { p->madj_Q = q; break; }
    if (p->madj_Q) {
        p->madj_thr = std::max(64, (p->nx / p->madj_Q + 31) / 32 * 32);
        p->madj_smem = mix_adj_row_smem<T>(p->nx, p->madj_thr);
        if (p->madj_smem > (size_t)optin) p->madj_Q = 0;
    }
    KZK_CUDA(cudaFuncSetAttribute(mix_adj_row_kernel<T, ADJ_ROW_1>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
    KZK_CUDA(cudaFuncSetAttribute(mix_adj_row_kernel<T, ADJ_ROW_2>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
    KZK_CUDA(cudaFuncSetAttribute(mix_adj_col_kernel<T, MIX_ADJ_C2>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
    KZK_CUDA(cudaFuncSetAttribute(mix_adj_col_kernel<T, MIX_ADJ_C1A>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
    KZK_CUDA(cudaFuncSetAttribute(mix_adj_col_kernel<T, MIX_ADJ_C1B>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
    KZK_CUDA(cudaFuncSetAttribute(ysweepT_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
    KZK_CUDA(cudaFuncSetAttribute(mix_row_kernel<T, ROW_RHS>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
    KZK_CUDA(cudaFuncSetAttribute(mix_row_kernel<T, ROW_FWD>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
    KZK_CUDA(cudaFuncSetAttribute(mix_row_kernel<T, ROW_INV>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
    KZK_CUDA(cudaFuncSetAttribute(mix_row_kernel<T, ROW_RHS_MED>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
    KZK_CUDA(cudaFuncSetAttribute(mix_col_kernel<T, MIX_C1B>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
    KZK_CUDA(cudaFuncSetAttribute(mix_col_kernel<T, MIX_C1V>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
    KZK_CUDA(cudaFuncSetAttribute(mix_col_kernel<T, MIX_C1V, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
    KZK_CUDA(cudaFuncSetAttribute(mix_col_kernel<T, MIX_C2>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
    KZK_CUDA(cudaFuncSetAttribute(ysweep_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
    if constexpr (sizeof(T) == 4)
        KZK_CUDA(cudaFuncSetAttribute(ysweep_pair_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
    return KZK_OK;
}

template <typename T>
kzk_status configure(kzk_plan* p)
{
    if (p->mixed) return configure_mixed<T>(p);
    p->row_thr = row_threads<T>(p->nx);
    if (p->row_thr > ROW_MAX_THREADS) return fail(KZK_ERR_SIZE, "nx = %d too large for one row per CTA", p->nx);
    p->row_smem = row_smem_bytes<T>(p->nx);
    p->adj_row_thr = std::max(32, p->n / row_ppt<T>());
    p->log2tc = col_log2tc<T>(p->nx, p->ny);
    p->col_thr = col_threads<T>(p->ny, p->log2tc);
    if (p->col_thr > col_max_threads<T>())
        return fail(KZK_ERR_SIZE, "ny = %d too large for a shared-memory column tile", p->ny);
    p->col_smem = col_smem_bytes<T>(p->ny, p->log2tc);
    // Every kernel may use up to the device's opt-in maximum; the launch's own
    // dynamic size decides occupancy.  (Setting the plan's size here would
    // shrink the limit for plans created earlier.)
    int dev = 0, optin = 0;
    KZK_CUDA(cudaGetDevice(&dev));
    KZK_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    if (p->row_smem > (size_t)optin || adj_row_smem<T>(p) > (size_t)optin || p->col_smem > (size_t)optin)
        return fail(KZK_ERR_SIZE, "grid %d x %d needs more shared memory than the device offers", p->nx, p->ny);
    const size_t sm = (size_t)optin;
    KZK_TRY((set_row_attr<T, ROW_RHS>(sm)));
    if (sizeof(T) == 8) {
        const void* ct[] = {(const void*)row_kernel<T, ROW_RHS, 9>, (const void*)row_kernel<T, ROW_RHS, 10>,
                            (const void*)row_kernel<T, ROW_RHS, 11>, (const void*)row_kernel<T, ROW_RHS, 12>};
        for (const void* f : ct) KZK_CUDA(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    }
    KZK_TRY((set_row_attr<T, ROW_FWD>(sm)));
    KZK_TRY((set_row_attr<T, ROW_INV>(sm)));
    KZK_TRY((set_row_attr<T, ROW_RHS_MED>(sm)));
    KZK_CUDA(cudaFuncSetAttribute(ysweep_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    if constexpr (sizeof(T) == 4)
        KZK_CUDA(cudaFuncSetAttribute(ysweep_pair_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    KZK_CUDA(cudaFuncSetAttribute(ysweepT_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    KZK_TRY((set_col_attr<T, COL_STAGE1>(sm)));
    KZK_TRY((set_col_attr<T, COL_STAGE2>(sm)));
    p->ysig_ok = 0;
    if (sizeof(T) == 8 && p->c.method == KZK_EXPRK22) {
        KZK_TRY((set_col_attr<T, COL_FWD>(sm)));
        KZK_TRY((set_col_attr<T, COL_S1>(sm)));
        KZK_TRY((set_col_attr<T, COL_S2>(sm)));
        p->ysig_ok = 1;
    }
    KZK_TRY((set_adj_row_attr<T, ADJ_ROW_2>(sm)));
    KZK_TRY((set_adj_row_attr<T, ADJ_ROW_1>(sm)));
    KZK_TRY((set_adj_col_attr<T, ADJ_COL_2>(sm)));
    KZK_TRY((set_adj_col_attr<T, ADJ_COL_1>(sm)));
    KZK_CUDA(cudaDeviceGetAttribute(&p->sm_count, cudaDevAttrMultiProcessorCount, dev));
    // FP32: row pairs in packed FP32 (even ny, the pair row fits)
    p->rowpair = 0;
    p->rowpair_ok = 0;
    if (sizeof(T) == 4 && p->ny % 2 == 0 && rowpair_smem_bytes(p->nx) <= (size_t)optin) {
        p->rowpair_ok = 1;
        p->rowpair_smem = rowpair_smem_bytes(p->nx);
        p->rowpair_ct_smem = rowpair_ct_smem_bytes(p->nx);
        p->rowpair_ct_ok = p->rowpair_ct_smem <= (size_t)optin;
        KZK_CUDA(cudaFuncSetAttribute(rowpair_kernel<ROW_RHS>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
        KZK_CUDA(cudaFuncSetAttribute(rowpair_kernel<ROW_FWD>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
        KZK_CUDA(cudaFuncSetAttribute(rowpair_kernel<ROW_INV>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
        KZK_CUDA(cudaFuncSetAttribute(rowpair_kernel<ROW_RHS_MED>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
        KZK_CUDA(cudaFuncSetAttribute(rowpair_kernel<ROW_RHS, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
        KZK_CUDA(cudaFuncSetAttribute(rowpair_kernel<ROW_RHS_MED, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      optin));
        const void* ct[] = {(const void*)rowpair_kernel<ROW_RHS, false, 9>, (const void*)rowpair_kernel<ROW_RHS, true, 9>,
                            (const void*)rowpair_kernel<ROW_RHS, false, 10>, (const void*)rowpair_kernel<ROW_RHS, true, 10>,
                            (const void*)rowpair_kernel<ROW_RHS, false, 11>, (const void*)rowpair_kernel<ROW_RHS, true, 11>,
                            (const void*)rowpair_kernel<ROW_RHS, false, 12>, (const void*)rowpair_kernel<ROW_RHS, true, 12>};
        for (const void* f : ct) KZK_CUDA(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
    }
    colp_configure<T>(p, optin);
    KZK_TRY(cpair_configure<T>(p, optin));
    p->cpair_diff = 0;
    if (p->colp_ok) {
        KZK_CUDA(cudaFuncSetAttribute(colp_kernel<T, COL_STAGE1, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
        KZK_CUDA(cudaFuncSetAttribute(colp_kernel<T, COL_STAGE2, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
        KZK_CUDA(cudaFuncSetAttribute(colp_kernel<T, COL_STAGE1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
        KZK_CUDA(cudaFuncSetAttribute(colp_kernel<T, COL_STAGE2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
    }
    return KZK_OK;
}

// twiddle table exp(-2 pi i k / N), k in [0, N), evaluated in long double;
// with lo != nullptr also the lo parts (value - hi) for a two-float table
template <typename T>
std::vector<cx<T>> twiddles(int N, std::vector<cx<T>>* lo = nullptr)
{
    std::vector<cx<T>> w(N);
    if (lo) lo->resize(N);
    const long double two_pi = 6.283185307179586476925286766559005768L;
    for (int k = 0; k < N; k++) {
        // reduce to the first octant by symmetry for exact 0 / +-1 entries
        long double a = two_pi * (long double)k / (long double)N;
        long double c = cosl(a), s = -sinl(a);
        if (4 * k == N) { c = 0; s = -1; }
        if (2 * k == N) { c = -1; s = 0; }
        if (4 * k == 3 * N) { c = 0; s = 1; }
        w[k] = mk<T>((T)(double)c, (T)(double)s);
        if (lo) (*lo)[k] = mk<T>((T)(double)(c - (long double)w[k].x), (T)(double)(s - (long double)w[k].y));
    }
    return w;
}

// staged twiddles of fft_batched for length 2^log2n with ppt points per
// thread (see Tw in kzk_fft.cuh), evaluated in long double; lo parts too when
// lo != nullptr
template <typename T>
std::vector<cx<T>> staged_twiddles(int log2n, int ppt, std::vector<cx<T>>* lo = nullptr)
{
    int lr[32], lns[32];
    const int P = fft_schedule(log2n, ppt, lr, lns);
    std::vector<cx<T>> w;
    if (lo) lo->clear();
    const long double two_pi = 6.283185307179586476925286766559005768L;
    for (int pidx = 0; pidx < P; pidx++) {
        if (lns[pidx] == 0) continue;
        const long long Ns = 1LL << lns[pidx], R = 1LL << lr[pidx];
        for (long long r = 1; r < R; r++)
            for (long long k = 0; k < Ns; k++) {
                const long long num = r * k, den = Ns * R;
                long double c, sn;
                if (4 * num == den) { c = 0; sn = -1; }
                else if (2 * num == den) { c = -1; sn = 0; }
                else if (4 * num == 3 * den) { c = 0; sn = 1; }
                else {
                    const long double a = two_pi * (long double)num / (long double)den;
                    c = cosl(a); sn = -sinl(a);
                }
                const cx<T> h = mk<T>((T)(double)c, (T)(double)sn);
                w.push_back(h);
                if (lo) lo->push_back(mk<T>((T)(double)(c - (long double)h.x), (T)(double)(sn - (long double)h.y)));
            }
    }
    if (w.empty()) w.push_back(mk<T>((T)1, (T)0));
    if (lo && lo->empty()) lo->push_back(mk<T>((T)0, (T)0));
    return w;
}

template <typename T>
RowArgs<T> row_args(const kzk_plan* p, const void* in, void* out, double sigma, double* diag_rows)
{
    RowArgs<T> a{};
    a.in = (const cx<T>*)in;
    a.out = (cx<T>*)out;
    a.tw = (const cx<T>*)p->twr;
    a.tws = (const cx<T>*)p->tws_row;
    a.diag_rows = diag_rows;
    a.log2nx = p->log2nx;
    a.ny = p->ny;
    a.inst_stride = p->inst_stride;
    const double Bs = B_of(p, sigma);
    a.wc.B = (T)Bs;
    a.wc.alpha = (T)(Bs * p->c.lf_umax);
    a.wc.eps = (T)p->c.weno_eps;
    a.wc.inv_dtau = (T)(p->nx / (p->g.tau_max - p->g.tau_min));
    a.cA = (T)(p->nx * dA_of(p, sigma));
    a.kscale = (T)(2.0 * M_PI / (p->g.tau_max - p->g.tau_min));
    a.out_scale = (T)1;
    a.u_out = nullptr;
    return a;
}

// sub (nullable, row pairs only): spectral rows subtracted from the result
template <typename T, int MODE>
kzk_status launch_row(const kzk_plan* p, const RowArgs<T>& a, cudaStream_t st, const void* sub = nullptr)
{
    if constexpr (std::is_same<T, float>::value) {
        if (p->rowpair) {
            RowPairArgs P{};
            P.r = a;
            P.tw2 = (const c2*)p->twr2;
            P.tws2 = (const c2*)p->tws2;
            P.sub = (const float2*)sub;
            P.flag = p->colp_flag;
            P.timeout_ns = 2000000000LL;
            const dim3 grid(p->ny / 2, p->batch);
            if constexpr (MODE == ROW_RHS) {
                // the length-specialised b passes for nx = 1024 ... 8192
                switch (p->rowpair_ct_ok ? p->log2nx - 1 : 0) {
#define KZK_ROWPAIR_CT(L)                                                                              \
    case L:                                                                                            \
        if (sub) rowpair_kernel<ROW_RHS, true, L><<<grid, p->row_thr, p->rowpair_ct_smem, st>>>(P);   \
        else rowpair_kernel<ROW_RHS, false, L><<<grid, p->row_thr, p->rowpair_ct_smem, st>>>(P);      \
        KZK_LAUNCHED();                                                                                \
        return KZK_OK;
                    KZK_ROWPAIR_CT(9)
                    KZK_ROWPAIR_CT(10)
                    KZK_ROWPAIR_CT(11)
                    KZK_ROWPAIR_CT(12)
#undef KZK_ROWPAIR_CT
                default: break;
                }
            }
            if constexpr (MODE == ROW_RHS || MODE == ROW_RHS_MED) {
                if (sub) {
                    rowpair_kernel<MODE, true><<<grid, p->row_thr, p->rowpair_smem, st>>>(P);
                    KZK_LAUNCHED();
                    return KZK_OK;
                }
            }
            rowpair_kernel<MODE><<<grid, p->row_thr, p->rowpair_smem, st>>>(P);
            KZK_LAUNCHED();
            return KZK_OK;
        }
    }
    if (p->mixed) {
        MixRowArgs<T> m{};
        m.r = a;
        m.nx = p->nx;
        m.f = p->mrow;
        m.pos = p->mpos_row;
        mix_row_kernel<T, MODE><<<dim3(p->ny, p->batch), p->mrow_thr, p->mrow_smem, st>>>(m);
        KZK_LAUNCHED();
        return KZK_OK;
    }
    if constexpr (MODE == ROW_RHS && std::is_same<T, double>::value) {
        // the length-specialised FP64 b passes for nx = 1024 ... 8192
        switch (p->log2nx - 1) {
#define KZK_ROW_CT(L)                                                                                  \
    case L:                                                                                            \
        row_kernel<T, ROW_RHS, L><<<dim3(p->ny, p->batch), p->row_thr, p->row_smem, st>>>(a);          \
        KZK_LAUNCHED();                                                                                \
        return KZK_OK;
            KZK_ROW_CT(9)
            KZK_ROW_CT(10)
            KZK_ROW_CT(11)
            KZK_ROW_CT(12)
#undef KZK_ROW_CT
        default: break;
        }
    }
    row_kernel<T, MODE><<<dim3(p->ny, p->batch), p->row_thr, p->row_smem, st>>>(a);
    KZK_LAUNCHED();
    return KZK_OK;
}

template <typename T>
kzk_status encode_map(CUtensorMap* m, int rank, const void* base, const cuuint64_t* dims, const cuuint64_t* strides,
                      const cuuint32_t* box)
{
    if (!base || ((uintptr_t)base & 15)) return fail(KZK_ERR_ARG, "tensor copy base %p not 16-byte aligned", base);
    const cuuint32_t es[3] = {1u, 1u, 1u};
    const CUresult r = encode_tiled()(m, sizeof(T) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64,
                                      (cuuint32_t)rank, const_cast<void*>(base), dims, strides, box, es,
                                      CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                      CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(KZK_ERR_CUDA, "cuTensorMapEncodeTiled: error %d", (int)r);
    return KZK_OK;
}
// state array [batch][ny][n] complex as {2 n, ny, batch} reals; box = one tile column block of colp_by rows
template <typename T>
kzk_status encode_state(CUtensorMap* m, const void* base, const kzk_plan* p)
{
    const cuuint64_t dims[3] = {2ull * p->n, (cuuint64_t)p->ny, (cuuint64_t)p->batch};
    const cuuint64_t strides[2] = {2ull * p->n * sizeof(T), 2ull * p->n * p->ny * sizeof(T)};
    const cuuint32_t box[3] = {2u << p->colp_log2tc, (cuuint32_t)p->colp_by, 1u};
    return encode_map<T>(m, 3, base, dims, strides, box);
}
// folded table [ny/2 + 1][n] complex as {2 n, ny/2 + 1} reals; box of colp_bt rows
template <typename T>
kzk_status encode_table(CUtensorMap* m, const void* base, const kzk_plan* p)
{
    const cuuint64_t dims[2] = {2ull * p->n, (cuuint64_t)(p->ny / 2 + 1)};
    const cuuint64_t strides[1] = {2ull * p->n * sizeof(T)};
    const cuuint32_t box[2] = {2u << p->colp_log2tc, (cuuint32_t)p->colp_bt};
    return encode_map<T>(m, 2, base, dims, strides, box);
}

// TMA-staged column kernel: one CTA per tile, each prefetching into L2 the tile
// taken one wave (two CTAs per SM) later.
template <typename T, int MODE>
kzk_status launch_colp(const kzk_plan* p, const ColArgs<T>& a, cudaStream_t st)
{
    ColPipeArgs<T> P;
    memset(&P, 0, sizeof(P));
    P.c = a;
    P.c.log2tc = p->colp_log2tc;
    KZK_TRY(encode_state<T>(&P.ma, a.a, p));
    KZK_TRY(encode_state<T>(&P.mb, a.b, p));
    if (MODE == COL_STAGE2) KZK_TRY(encode_state<T>(&P.mc, a.c, p));
    if (MODE == COL_STAGE2) KZK_TRY(encode_table<T>(&P.mt0, a.Ta, p));
    P.by = p->colp_by;
    P.nby = p->colp_nby;
    P.bt = p->colp_bt;
    P.nbt = p->colp_nbt;
    P.n_tiles = p->n >> p->colp_log2tc;
    P.total = P.n_tiles * p->batch;
    P.flag = p->colp_flag;
    P.timeout_ns = 2000000000LL;
    P.ahead = 2 * p->sm_count;   // two CTAs per SM: one wave ahead
    const int grid = P.total;
    const size_t smem = MODE == COL_STAGE1 ? p->colp_smem1 : p->colp_smem2;
    if (p->comp) colp_kernel<T, MODE, true><<<grid, p->colp_thr, smem, st>>>(P);
    else colp_kernel<T, MODE, false><<<grid, p->colp_thr, smem, st>>>(P);
    KZK_LAUNCHED();
    return KZK_OK;
}

// Column-pair kernels: state tiles {2 n, ny, batch} floats in boxes {4, by, 1};
// pair tables by bulk copies; the lo parts of the state pair-major.
template <int L, int MODE>
kzk_status launch_colpair_l(const kzk_plan* p, const ColArgs<float>& a, cudaStream_t st)
{
    ColPairArgs P;
    memset(&P, 0, sizeof(P));
    P.c = a;
    const cuuint64_t sdims[3] = {2ull * p->n, (cuuint64_t)p->ny, (cuuint64_t)p->batch};
    const cuuint64_t sstr[2] = {2ull * p->n * sizeof(float), 2ull * p->n * p->ny * sizeof(float)};
    const cuuint32_t sbox[3] = {4u, (cuuint32_t)p->cpair_by, 1u};
    KZK_TRY(encode_map<float>(&P.ma, 3, a.a, sdims, sstr, sbox));
    KZK_TRY(encode_map<float>(&P.mb, 3, a.b, sdims, sstr, sbox));
    KZK_TRY(encode_map<float>(&P.mo, 3, a.out, sdims, sstr, sbox));
    if (MODE == COL_STAGE1) {
        P.tab0 = (const c2*)p->Em1p;
        P.tab1 = (const c2*)p->P1p;
    } else {
        KZK_TRY(encode_map<float>(&P.mc, 3, a.c, sdims, sstr, sbox));
        P.tab0 = (const c2*)p->P2p;
    }
    P.tw = (const c2*)p->twcp;
    P.by = p->cpair_by;
    P.nby = p->cpair_nby;
    P.n_tiles = p->n / 2;
    P.total = P.n_tiles * p->batch;
    P.flag = p->colp_flag;
    P.timeout_ns = 2000000000LL;
    const size_t smem = MODE == COL_STAGE1 ? p->cpair_smem1 : p->cpair_smem2;
    if (MODE == COL_STAGE2 && p->cpair_diff) colpair_kernel<L, MODE, true><<<P.total, PairSched<L>::T, smem, st>>>(P);
    else colpair_kernel<L, MODE><<<P.total, PairSched<L>::T, smem, st>>>(P);
    KZK_LAUNCHED();
    return KZK_OK;
}
template <int MODE>
kzk_status launch_colpair(const kzk_plan* p, const ColArgs<float>& a, cudaStream_t st)
{
    switch (p->log2ny) {
    case 8: return launch_colpair_l<8, MODE>(p, a, st);
    case 9: return launch_colpair_l<9, MODE>(p, a, st);
    case 10: return launch_colpair_l<10, MODE>(p, a, st);
    case 11: return launch_colpair_l<11, MODE>(p, a, st);
    default: return launch_colpair_l<12, MODE>(p, a, st);
    }
}

// Mixed-radix plans: STAGE1 as two launches (P1' FFT_y(b1) into the scratch
// array, then the state's transform, propagator and inverse), STAGE2 as one.
template <typename T, int MODE>
kzk_status launch_mix_col(const kzk_plan* p, const ColArgs<T>& a, cudaStream_t st)
{
    MixColArgs<T> m{};
    m.c = a;
    m.c.tw = (const cx<T>*)p->twc;
    m.c.tw_lo = (const cx<T>*)p->twc_lo;
    m.w = (cx<T>*)p->wsc;
    m.ny = p->ny;
    m.n = p->n;
    m.lc = p->mcol_lc;
    m.f = p->mcol;
    m.pos = p->mpos_col;
    m.ipos = p->mipos_col;
    const dim3 grid(p->n >> p->mcol_lc, p->batch);
    if (MODE == COL_STAGE1) {
        mix_col_kernel<T, MIX_C1B><<<grid, p->mcol_thr, p->mcol_smem, st>>>(m);
        KZK_LAUNCHED();
        if (sizeof(T) == 4 && a.lo_out) mix_col_kernel<T, MIX_C1V, true><<<grid, p->mcol_thr, p->mcol_smem, st>>>(m);
        else mix_col_kernel<T, MIX_C1V><<<grid, p->mcol_thr, p->mcol_smem, st>>>(m);
        KZK_LAUNCHED();
    } else {
        mix_col_kernel<T, MIX_C2><<<grid, p->mcol_thr, p->mcol_smem, st>>>(m);
        KZK_LAUNCHED();
    }
    return KZK_OK;
}

template <typename T, int MODE>
kzk_status launch_col(const kzk_plan* p, const ColArgs<T>& a, cudaStream_t st)
{
    if (p->mixed) return launch_mix_col<T, MODE>(p, a, st);
    if constexpr (std::is_same<T, float>::value)
        if (p->colpair) return launch_colpair<MODE>(p, a, st);
    if (p->colp_log2tc >= 0) return launch_colp<T, MODE>(p, a, st);
    col_kernel<T, MODE><<<dim3(p->n >> p->log2tc, p->batch), p->col_thr, p->col_smem, st>>>(a);
    KZK_LAUNCHED();
    return KZK_OK;
}

template <typename T>
ColArgs<T> col_args(const kzk_plan* p)
{
    ColArgs<T> a{};
    memset(&a, 0, sizeof(a));
    a.tw = (const cx<T>*)p->twc;
    a.tw_lo = (const cx<T>*)p->twc_lo;
    a.Ta_lo = nullptr;
    a.log2ny = p->log2ny;
    a.log2n = p->log2nx - 1;
    a.log2tc = p->log2tc;
    a.inst_stride = p->inst_stride;
    a.inv_count = 1.0 / ((double)p->nx * p->ny);
    a.cell = (p->g.tau_max - p->g.tau_min) / p->nx * (p->g.y_max - p->g.y_min) / p->ny;
    return a;
}

// The y-spectral state path (column modes FWD / S1 / S2) is in use: FP64
// ExpRK22 plans while the per-tile column kernels are selected.
bool ysig_on(const kzk_plan* p) { return p->ysig_ok && !p->mixed && !p->colpair && p->colp_log2tc < 0; }

template <typename T, int MODE>
kzk_status launch_col_tile(const kzk_plan* p, const ColArgs<T>& a, cudaStream_t st)
{
    col_kernel<T, MODE><<<dim3(p->n >> p->log2tc, p->batch), p->col_thr, p->col_smem, st>>>(a);
    KZK_LAUNCHED();
    return KZK_OK;
}

// Sigma = FFT_y(V) / ny of a state just loaded into V (y-spectral path).
template <typename T>
kzk_status col_fwd(const kzk_plan* p, const void* V, cudaStream_t st)
{
    ColArgs<T> a = col_args<T>(p);
    a.a = (const cx<T>*)V;
    a.out = (cx<T>*)p->ysig;
    a.yscale = (T)(1.0 / p->ny);
    return launch_col_tile<T, COL_FWD>(p, a, st);
}

// Random-medium coefficients at sigma into stage buffer `stage` (0 or 1).
kzk_status launch_medium(kzk_plan* p, double sigma, int stage, cudaStream_t st, const double* dsig = nullptr)
{
    MedArgs m{};
    m.sig = dsig;
    m.Ty = (const double2*)p->med_Ty;
    m.a_sig = p->med_mode;
    m.phase = p->med_mode + p->med_n;
    m.w = p->med_mode + 2 * p->med_n;
    m.n_modes = p->med_n;
    m.ny = p->ny;
    m.sigma = sigma;
    m.coef = p->med_coef + (size_t)stage * 3 * p->ny;
    m.bmax = p->med_bmax + (size_t)stage * p->med_nb;
    medium_kernel<<<p->med_nb, MED_ROWS * MED_GROUPS, 0, st>>>(m);
    KZK_LAUNCHED();
    return KZK_OK;
}

// STEP 1 / STEP 3 of Algorithm 2: the row pass(es) computing the tau-spectrum
// of b(sigma, u) from the spectral state Vin.  Homogeneous / stratified
// medium: one pass (C2R, WENO5 along tau, R2C).  Random medium: the
// coefficient kernel, a C2R pass to the physical rows (with the row
// statistics), then the b pass with the y-flux and source terms.
// diag_rows, u_out: nullable (u_out: where the physical rows are kept).
template <typename T>
kzk_status rhs_stage(kzk_plan* p, double sigma, const void* Vin, void* bout, double* diag_rows, void* u_out,
                     int stage, cudaStream_t st, const double* dcoef = nullptr)
{
    // dcoef (nullable): this stage's {sigma, B, B M, nx (A - A0)} in device
    // memory, used in place of sigma (launches captured into a graph)
    if (p->med_n > 0) {
        // the physical stage state: into u_out when the adjoint sweep keeps it
        void* phys = u_out ? u_out : p->uphys;
        KZK_TRY(launch_medium(p, sigma, stage, st, dcoef));
        RowArgs<T> ri = row_args<T>(p, Vin, phys, 0.0, diag_rows);
        KZK_TRY((launch_row<T, ROW_INV>(p, ri, st)));
        YSweepArgs<T> y{};
        y.u = (const T*)phys;
        y.by = (T*)p->by;
        y.coef = p->med_coef + (size_t)stage * 3 * p->ny;
        y.bmax = p->med_bmax + (size_t)stage * p->med_nb;
        y.n_bmax = p->med_nb;
        y.nx = p->nx;
        y.ny = p->ny;
        y.inst_elems = (long long)p->nx * p->ny;
        y.eps = (T)p->c.weno_eps;
        y.inv_dy = (T)(p->ny / (p->g.y_max - p->g.y_min));
        // rows per CTA: 64 (FP64) / 32 (FP32), halved down to 16 while the
        // grid would leave SMs without two CTAs (short, narrow grids)
        const int xb = sizeof(T) == 4 ? (p->nx + 2 * YSWEEP_THREADS - 1) / (2 * YSWEEP_THREADS)
                                      : (p->nx + YSWEEP_THREADS - 1) / YSWEEP_THREADS;
        int q = sizeof(T) == 4 ? 32 : 64;
        while (q > 16 && (long long)xb * ((p->ny + q - 1) / q) * p->batch < 2LL * p->sm_count) q >>= 1;
        y.Q = std::min(p->ny, q);
        const dim3 yg(xb, (p->ny + y.Q - 1) / y.Q, p->batch);
        if constexpr (sizeof(T) == 4) {
            // FP32: column pairs in packed FP32 (kzk_ysweep_pair.cuh)
            ysweep_pair_kernel<<<yg, YSWEEP_THREADS, ysweep_pair_smem(y.Q), st>>>(y);
        } else {
            ysweep_kernel<T><<<yg, YSWEEP_THREADS, ysweep_smem<T>(y.Q), st>>>(y);
        }
        KZK_LAUNCHED();
        RowArgs<T> r = row_args<T>(p, Vin, bout, sigma, nullptr);
        r.coef = dcoef;
        r.uphys = (const T*)phys;
        r.by = (const T*)p->by;
        r.med_coef = p->med_coef + (size_t)stage * 3 * p->ny;
        return launch_row<T, ROW_RHS_MED>(p, r, st, stage == 1 && p->cpair_diff ? p->b1 : nullptr);
    }
    RowArgs<T> r = row_args<T>(p, Vin, bout, sigma, diag_rows);
    r.coef = dcoef;
    r.u_out = (T*)u_out;
    // column-pair plans on row pairs: the second stage stores b2 - b1 (C2's
    // input), the subtraction done once per element in the row pass
    return launch_row<T, ROW_RHS>(p, r, st, stage == 1 && p->cpair_diff ? p->b1 : nullptr);
}

// Stage-1 table and state pointers: the plain state takes E' (+ E'_lo in
// FP32); the compensated state (FP32 plans) takes (E - 1)/ny and the lo
// arrays, V* = V + increment (exponential Euler: V' in place of V).
template <typename T>
void stage1_tables(const kzk_plan* p, ColArgs<T>& c1, bool euler)
{
    if (p->comp) {
        c1.Ta = (const cx<T>*)p->Em1;
        c1.Ta_lo = nullptr;
        c1.lo_in = (const lo_t<T>*)p->Vlo;
        c1.lo_out = (lo_t<T>*)(euler ? p->Vlo : p->vslo);
    } else {
        c1.Ta = (const cx<T>*)p->E;
        c1.Ta_lo = (const cx<T>*)p->E_lo;
    }
}
template <typename T>
void stage2_lo(const kzk_plan* p, ColArgs<T>& c2)
{
    if (p->comp) {
        c2.lo_in = (const lo_t<T>*)p->vslo;
        c2.lo_out = (lo_t<T>*)p->Vlo;
    }
}

kzk_status reset_lo(kzk_plan* p, cudaStream_t st);

// One ExpRK22 step on the spectral state p->V (Algorithm 2, STEP 1-4).
// diag_hist_step: where C1 writes this step's diagnostics (nullable).
// vs_out / b1_out / b2_out: destinations (default: plan workspace).
// ev (nullable): five events recorded around the four passes (R1, C1, R2, C2).
// On the y-spectral path p->ysig must hold FFT_y(V) / ny on entry; it leaves
// FFT_y(V_out) / ny there.
template <typename T>
kzk_status step(kzk_plan* p, double sigma, cudaStream_t st, double* diag_hist_step, void* V, void* vs,
                void* V_out = nullptr, void* u_n = nullptr, void* u_s = nullptr, cudaEvent_t* ev = nullptr,
                const double* dcoef = nullptr)
{
    // dcoef (nullable): the step's sigma-dependent values in device memory
    // ([2][4], stage 1 then stage 2: see rhs_stage), used in place of sigma
    // V is read-only; the result goes to V_out (default: in place).  u_n, u_s
    // (nullable): where the row passes also store the physical u^n and u*.
    if (!V_out) V_out = V;
    const bool euler = p->c.method == KZK_EXPEULER;
    auto mark = [&](int i) -> kzk_status {
        if (ev) KZK_CUDA(cudaEventRecord(ev[i], st));
        return KZK_OK;
    };
    KZK_TRY(mark(0));
    KZK_TRY(rhs_stage<T>(p, sigma, V, p->b1, diag_hist_step ? p->diag_rows : nullptr, u_n, 0, st, dcoef));
    KZK_TRY(mark(1));
    if (ysig_on(p) && !euler) {
        // STEP 2: V* = IFFT_y(X), X = ny E' Sigma + P1' FFT_y(b1); T = X - P2' FFT_y(b1)
        ColArgs<T> c1 = col_args<T>(p);
        c1.a = (const cx<T>*)p->ysig;
        c1.b = (const cx<T>*)p->b1;
        c1.out = (cx<T>*)vs;
        c1.out2 = (cx<T>*)p->ytmp;
        c1.Ta = (const cx<T>*)p->E;
        c1.Tb = (const cx<T>*)p->P1;
        c1.Tc = (const cx<T>*)p->P2;
        c1.yscale = (T)p->ny;
        c1.diag_rows = diag_hist_step ? p->diag_rows : nullptr;
        c1.diag_hist = diag_hist_step;
        KZK_TRY((launch_col_tile<T, COL_S1>(p, c1, st)));
        KZK_TRY(mark(2));
        KZK_TRY(rhs_stage<T>(p, sigma + p->dt, vs, p->b2, nullptr, u_s, 1, st, dcoef ? dcoef + 4 : nullptr));
        KZK_TRY(mark(3));
        // STEP 4: Sigma' = T + P2' FFT_y(b2), V' = IFFT_y(Sigma')
        ColArgs<T> c2 = col_args<T>(p);
        c2.a = (const cx<T>*)p->ytmp;
        c2.b = (const cx<T>*)p->b2;
        c2.out = (cx<T>*)V_out;
        c2.out2 = (cx<T>*)p->ysig;
        c2.Ta = (const cx<T>*)p->P2;
        KZK_TRY((launch_col_tile<T, COL_S2>(p, c2, st)));
        return mark(4);
    }
    ColArgs<T> c1 = col_args<T>(p);
    c1.a = (const cx<T>*)V;
    c1.b = (const cx<T>*)p->b1;
    // exponential Euler: the first stage is the step (every column tile is
    // read whole before it is written, so V_out may alias V)
    c1.out = (cx<T>*)(euler ? V_out : vs);
    stage1_tables<T>(p, c1, euler);
    c1.Tb = (const cx<T>*)p->P1;
    c1.diag_rows = diag_hist_step ? p->diag_rows : nullptr;
    c1.diag_hist = diag_hist_step;
    KZK_TRY((launch_col<T, COL_STAGE1>(p, c1, st)));
    KZK_TRY(mark(2));
    if (euler) {
        KZK_TRY(mark(3));
        return mark(4);
    }
    KZK_TRY(rhs_stage<T>(p, sigma + p->dt, vs, p->b2, nullptr, u_s, 1, st, dcoef ? dcoef + 4 : nullptr));
    KZK_TRY(mark(3));
    ColArgs<T> c2 = col_args<T>(p);
    c2.a = (const cx<T>*)p->b1;
    c2.b = (const cx<T>*)p->b2;
    c2.c = (const cx<T>*)vs;
    c2.out = (cx<T>*)V_out;
    c2.Ta = (const cx<T>*)p->P2;
    stage2_lo<T>(p, c2);
    KZK_TRY((launch_col<T, COL_STAGE2>(p, c2, st)));
    return mark(4);
}

// zero lo part after a state is (re)loaded into p->V in spectral form
kzk_status reset_lo(kzk_plan* p, cudaStream_t st)
{
    if (p->comp)
        KZK_CUDA(cudaMemsetAsync(p->Vlo, 0, (size_t)p->batch * p->inst_stride * sizeof(__nv_bfloat162), st));
    return KZK_OK;
}

template <typename T>
kzk_status to_spectral(kzk_plan* p, const void* u, void* V, cudaStream_t st)
{
    RowArgs<T> a = row_args<T>(p, u, V, 0.0, nullptr);
    a.out_scale = (T)(1.0 / p->nx);
    KZK_TRY((launch_row<T, ROW_FWD>(p, a, st)));
    if (V != p->V) return KZK_OK;
    // a state loaded into the plan's state array starts with a zero lo part,
    // and on the y-spectral path with its y-spectrum
    KZK_TRY(reset_lo(p, st));
    return ysig_on(p) ? col_fwd<T>(p, V, st) : KZK_OK;
}

template <typename T>
kzk_status to_physical(kzk_plan* p, const void* V, void* u, double scale, double* diag_rows, cudaStream_t st)
{
    RowArgs<T> a = row_args<T>(p, V, u, 0.0, diag_rows);
    a.out_scale = (T)scale;
    return launch_row<T, ROW_INV>(p, a, st);
}

kzk_status ensure_hist(kzk_plan* p, long long steps)
{
    if (steps <= p->hist_cap) return KZK_OK;
    long long cap = std::max(steps, 2 * p->hist_cap);
    if (p->diag_hist) KZK_CUDA(cudaFree(p->diag_hist));
    p->diag_hist = nullptr;
    KZK_CUDA(cudaMalloc(&p->diag_hist, (size_t)cap * p->batch * 4 * sizeof(double)));
    p->hist_cap = cap;
    return KZK_OK;
}

kzk_status finish_diag(kzk_plan* p, long long n_steps, cudaStream_t st, kzk_diag* out)
{
    KZK_CUDA(cudaStreamSynchronize(st));
    if (p->colp_flag) {
        int f = 0;
        KZK_CUDA(cudaMemcpy(&f, p->colp_flag, sizeof(int), cudaMemcpyDeviceToHost));
        if (f) {
            KZK_CUDA(cudaMemset(p->colp_flag, 0, sizeof(int)));
            if (f & FLAG_BAD_LAUNCH) return fail(KZK_ERR_CUDA, "column kernel: shared memory not 128-byte aligned");
            return fail(KZK_ERR_TIMEOUT, "a column-tile copy did not arrive within its time limit");
        }
    }
    std::vector<double> hist((size_t)n_steps * p->batch * 4), fin((size_t)p->batch * 4);
    if (n_steps > 0)
        KZK_CUDA(cudaMemcpy(hist.data(), p->diag_hist, hist.size() * sizeof(double), cudaMemcpyDeviceToHost));
    KZK_CUDA(cudaMemcpy(fin.data(), p->diag_final, fin.size() * sizeof(double), cudaMemcpyDeviceToHost));
    bool nonfinite = false, cfl = false;
    for (int b = 0; b < p->batch; b++) {
        kzk_diag d;
        d.mean = fin[4 * b];
        d.energy = fin[4 * b + 1];
        d.max_abs = fin[4 * b + 2];
        d.nonfinite = fin[4 * b + 3];
        d.run_max_abs = d.max_abs;
        d.run_nonfinite = d.nonfinite;
        for (long long s = 0; s < n_steps; s++) {
            const double* h = &hist[((size_t)s * p->batch + b) * 4];
            d.run_max_abs = std::max(d.run_max_abs, h[2]);
            d.run_nonfinite += h[3];
        }
        out[b] = d;
        if (d.run_nonfinite > 0 || !std::isfinite(d.run_max_abs)) nonfinite = true;
        if (d.run_max_abs > p->c.lf_umax) cfl = true;
    }
    if (nonfinite) return fail(KZK_ERR_NONFINITE, "non-finite values in the state");
    if (cfl) return fail(KZK_ERR_CFL, "max|u| exceeded lf_umax = %g", p->c.lf_umax);
    return KZK_OK;
}

// Stage values of GRAPH_CHUNK-step replays: for local step s of a replay
// starting at global step s0, stage 1 at sigma = sigma0 + (s0 + s) dt and
// stage 2 at sigma + dt, each {sigma, B(sigma), B(sigma) M, nx (A(sigma) - A)}
// -- the host's expressions of B_of / dA_of / row_args, evaluated in FP64 with
// every product and sum rounded on its own (as the host computes them), so a
// replay uses bit for bit the values a direct launch would.
constexpr int GRAPH_CHUNK = 16;
struct StepCoefArgs {
    double* out;
    int count;
    long long s0;
    double sigma0, dt, B, A, M, nx;
    double Bp[4], Ap[4];
    int has_profile;
};
__global__ void step_coef_kernel(StepCoefArgs a)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= a.count) return;
    auto horner = [](const double* c, double x) {
        return __dadd_rn(__dmul_rn(__dadd_rn(__dmul_rn(__dadd_rn(__dmul_rn(c[3], x), c[2]), x), c[1]), x), c[0]);
    };
    const double s1 = __dadd_rn(a.sigma0, __dmul_rn((double)(a.s0 + s), a.dt));
    const double sg[2] = {s1, __dadd_rn(s1, a.dt)};
    for (int k = 0; k < 2; k++) {
        const double B = a.has_profile ? __dmul_rn(a.B, horner(a.Bp, sg[k])) : a.B;
        const double dA = a.has_profile ? __dadd_rn(__dmul_rn(a.A, horner(a.Ap, sg[k])), -a.A) : 0.0;
        double* o = a.out + 8 * s + 4 * k;
        o[0] = sg[k];
        o[1] = B;
        o[2] = __dmul_rn(B, a.M);
        o[3] = __dmul_rn(a.nx, dA);
    }
}

kzk_status launch_step_coef(kzk_plan* p, int count, long long s0, double sigma0, cudaStream_t st)
{
    StepCoefArgs a{};
    a.out = p->dcoef;
    a.count = count;
    a.s0 = s0;
    a.sigma0 = sigma0;
    a.dt = p->dt;
    a.B = p->c.B;
    a.A = p->c.A;
    a.M = p->c.lf_umax;
    a.nx = (double)p->nx;
    memcpy(a.Bp, p->c.B_prof, sizeof(a.Bp));
    memcpy(a.Ap, p->c.A_prof, sizeof(a.Ap));
    a.has_profile = p->c.has_profile;
    step_coef_kernel<<<1, GRAPH_CHUNK, 0, st>>>(a);
    KZK_LAUNCHED();
    return KZK_OK;
}

// Capture the step graphs of the plan (GRAPH_CHUNK steps and one step) on its
// own stream; the launches read their sigma values from p->dcoef and write
// their diagnostics to p->dhist.
template <typename T>
kzk_status capture_step_graphs(kzk_plan* p)
{
    if (!p->dcoef) KZK_CUDA(cudaMalloc(&p->dcoef, (size_t)GRAPH_CHUNK * 8 * sizeof(double)));
    if (!p->dhist) KZK_CUDA(cudaMalloc(&p->dhist, (size_t)GRAPH_CHUNK * p->batch * 4 * sizeof(double)));
    if (!p->cap_stream) KZK_CUDA(cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking));
    const int counts[2] = {GRAPH_CHUNK, 1};
    for (int g = 0; g < 2; g++) {
        if (p->gx[g]) continue;
        cudaGraph_t graph = nullptr;
        KZK_CUDA(cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeThreadLocal));
        kzk_status s = KZK_OK;
        // captured launches run at replays: count them there, not here
        const long long n0 = g_launches.load();
        for (int i = 0; i < counts[g] && s == KZK_OK; i++)
            s = step<T>(p, 0.0, p->cap_stream, p->dhist + (size_t)i * p->batch * 4, p->V, p->vs, nullptr, nullptr,
                        nullptr, nullptr, p->dcoef + 8 * i);
        const cudaError_t e = cudaStreamEndCapture(p->cap_stream, &graph);
        p->gx_kernels[g] = g_launches.load() - n0;
        g_launches.fetch_sub(p->gx_kernels[g]);
        if (s != KZK_OK || e != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            if (s != KZK_OK) return s;
            return fail(KZK_ERR_CUDA, "capture of the step graph: %s", cudaGetErrorString(e));
        }
        const cudaError_t ei = cudaGraphInstantiate(&p->gx[g], graph, 0);
        cudaGraphDestroy(graph);
        if (ei != cudaSuccess) {
            p->gx[g] = nullptr;
            return fail(KZK_ERR_CUDA, "step graph instantiate: %s", cudaGetErrorString(ei));
        }
    }
    return KZK_OK;
}

// direct: launch every kernel (no step graphs), as inside another capture
template <typename T>
kzk_status advance_impl(kzk_plan* p, void* u, long long n_steps, double sigma0, cudaStream_t st, kzk_diag* dout,
                        bool direct = false)
{
    KZK_TRY(ensure_hist(p, std::max(1LL, n_steps)));
    KZK_TRY(to_spectral<T>(p, u, p->V, st));
    if (!direct && p->opt.graph != KZK_GRAPH_OFF && n_steps > 0) {
        KZK_TRY(capture_step_graphs<T>(p));
        for (long long s = 0; s < n_steps;) {
            const int count = n_steps - s >= GRAPH_CHUNK ? GRAPH_CHUNK : 1;
            KZK_TRY(launch_step_coef(p, count, s, sigma0, st));
            const int g = count == GRAPH_CHUNK ? 0 : 1;
            KZK_CUDA(cudaGraphLaunch(p->gx[g], st));
            g_launches.fetch_add(p->gx_kernels[g], std::memory_order_relaxed);
            KZK_CUDA(cudaMemcpyAsync(p->diag_hist + (size_t)s * p->batch * 4, p->dhist,
                                     (size_t)count * p->batch * 4 * sizeof(double), cudaMemcpyDeviceToDevice, st));
            s += count;
        }
    } else {
        for (long long s = 0; s < n_steps; s++) {
            const double sigma = sigma0 + (double)s * p->dt;
            KZK_TRY(step<T>(p, sigma, st, p->diag_hist + (size_t)s * p->batch * 4, p->V, p->vs));
        }
    }
    KZK_TRY(to_physical<T>(p, p->V, u, 1.0, p->diag_rows, st));
    diag_reduce_kernel<<<p->batch, 256, 0, st>>>(p->diag_rows, p->ny, 1.0 / ((double)p->nx * p->ny),
                                                 (p->g.tau_max - p->g.tau_min) / p->nx *
                                                     (p->g.y_max - p->g.y_min) / p->ny,
                                                 p->diag_final);
    KZK_LAUNCHED();
    p->hist_steps = n_steps;
    if (dout) return finish_diag(p, n_steps, st, dout);
    return KZK_OK;
}

// Pair tables and twiddles of the column-pair kernels, from the folded FP32
// tables and the full y twiddle table w (exp(-2 pi i k / ny)).
template <int L, typename W>
kzk_status build_pair_tables(kzk_plan* p, const std::vector<W>& w, cudaStream_t st)
{
    using S = PairSched<L>;
    const size_t ptab = (size_t)pair_tab_rows(p->ny) * p->n * sizeof(float2);
    const void* src[3] = {p->Em1, p->P1, p->P2};
    void* dst[3] = {p->Em1p, p->P1p, p->P2p};
    const long long count = (long long)(p->ny / 2 + 1) * (p->n / 2);
    for (int i = 0; i < 3; i++) {
        KZK_CUDA(cudaMemsetAsync(dst[i], 0, ptab, st));
        pair_table_kernel<L><<<(unsigned)((count + 255) / 256), 256, 0, st>>>((const float2*)src[i], (c2*)dst[i],
                                                                            p->n);
        KZK_LAUNCHED();
    }
    std::vector<float4> t(S::TW > 0 ? S::TW : 1);
    for (int i = 0; i < S::NP - 1; i++) {
        const int R = S::radix(i), s = S::stride(i), step = S::N / (R * s);
        for (int r = 1; r < R; r++)
            for (int q = 0; q < s; q++) {
                const W z = w[(size_t)((long long)q * r * step % S::N)];
                t[S::tw_off(i) + (r - 1) * s + q] = make_float4((float)z.x, (float)z.x, (float)z.y, (float)z.y);
            }
    }
    KZK_CUDA(cudaMemcpy(p->twcp, t.data(), t.size() * sizeof(float4), cudaMemcpyHostToDevice));
    return KZK_OK;
}

template <typename T>
kzk_status build_tables(kzk_plan* p, cudaStream_t st)
{
    TabArgs a{};
    a.nx = p->nx;
    a.ny = p->ny;
    a.dt = p->dt;
    a.A = p->c.A;
    a.diffraction = p->c.diffraction;
    a.reg_eps = p->c.reg_eps;
    a.kts = 2.0 * M_PI / (p->g.tau_max - p->g.tau_min);
    a.kys = 2.0 * M_PI / (p->g.y_max - p->g.y_min);
    a.E = p->E;
    a.P1 = p->P1;
    a.P2 = p->P2;
    a.E_lo = p->E_lo;
    a.Em1 = p->Em1;
    a.n_relax = p->c.n_relax;
    for (int r = 0; r < 2; r++) {
        a.relax_C[r] = r < p->c.n_relax ? p->c.relax_C[r] : 0.0;
        a.relax_theta[r] = r < p->c.n_relax ? p->c.relax_theta[r] : 1.0;
    }
    const long long count = (long long)(p->ny / 2 + 1) * p->n;
    tables_kernel<T><<<(unsigned)((count + 255) / 256), 256, 0, st>>>(a);
    KZK_LAUNCHED();
    auto tr = twiddles<T>(p->nx);
    auto tcf = twiddles<T>(p->ny);
    if (p->mixed) {
        // full y table (hi and, FP32, lo) and the digit-reversal positions
        std::vector<cx<T>> tcl;
        auto tch = twiddles<T>(p->ny, &tcl);
        std::vector<int> pr(p->n), pc(p->ny), ipc(p->ny);
        for (int k = 0; k < p->n; k++) pr[k] = mix_position(p->mrow, k);
        for (int l = 0; l < p->ny; l++) {
            pc[l] = mix_position(p->mcol, l);
            ipc[pc[l]] = l;
        }
        KZK_CUDA(cudaMemcpy(p->twr, tr.data(), tr.size() * sizeof(cx<T>), cudaMemcpyHostToDevice));
        KZK_CUDA(cudaMemcpy(p->twc_full, tcf.data(), tcf.size() * sizeof(cx<T>), cudaMemcpyHostToDevice));
        KZK_CUDA(cudaMemcpy(p->twc, tch.data(), tch.size() * sizeof(cx<T>), cudaMemcpyHostToDevice));
        if (p->twc_lo)
            KZK_CUDA(cudaMemcpy(p->twc_lo, tcl.data(), tcl.size() * sizeof(cx<T>), cudaMemcpyHostToDevice));
        KZK_CUDA(cudaMemcpy(p->mpos_row, pr.data(), pr.size() * sizeof(int), cudaMemcpyHostToDevice));
        KZK_CUDA(cudaMemcpy(p->mpos_col, pc.data(), pc.size() * sizeof(int), cudaMemcpyHostToDevice));
        KZK_CUDA(cudaMemcpy(p->mipos_col, ipc.data(), ipc.size() * sizeof(int), cudaMemcpyHostToDevice));
        KZK_CUDA(cudaStreamSynchronize(st));
        return KZK_OK;
    }
    auto trs = staged_twiddles<T>(p->log2nx - 1, row_ppt_of<T>());
    std::vector<cx<T>> tcl;
    auto tcs = staged_twiddles<T>(p->log2ny, col_ppt_of<T>(), &tcl);
    if ((long long)trs.size() > p->n || (long long)tcs.size() > p->ny)
        return fail(KZK_ERR_SIZE, "staged twiddle table larger than its transform");
    KZK_CUDA(cudaMemcpy(p->twr, tr.data(), tr.size() * sizeof(cx<T>), cudaMemcpyHostToDevice));
    KZK_CUDA(cudaMemcpy(p->twc_full, tcf.data(), tcf.size() * sizeof(cx<T>), cudaMemcpyHostToDevice));
    KZK_CUDA(cudaMemcpy(p->tws_row, trs.data(), trs.size() * sizeof(cx<T>), cudaMemcpyHostToDevice));
    KZK_CUDA(cudaMemcpy(p->twc, tcs.data(), tcs.size() * sizeof(cx<T>), cudaMemcpyHostToDevice));
    if (p->twc_lo)
        KZK_CUDA(cudaMemcpy(p->twc_lo, tcl.data(), tcl.size() * sizeof(cx<T>), cudaMemcpyHostToDevice));
    if (p->twr2) {
        // every FP32 entry (wr, wi) as ((wr, wr), (wi, wi))
        auto pairs = [](const std::vector<cx<T>>& w) {
            std::vector<float4> q(w.size());
            for (size_t i = 0; i < w.size(); i++)
                q[i] = make_float4((float)w[i].x, (float)w[i].x, (float)w[i].y, (float)w[i].y);
            return q;
        };
        const auto r2 = pairs(tr), s2 = pairs(trs);
        KZK_CUDA(cudaMemcpy(p->twr2, r2.data(), r2.size() * sizeof(float4), cudaMemcpyHostToDevice));
        KZK_CUDA(cudaMemcpy(p->tws2, s2.data(), s2.size() * sizeof(float4), cudaMemcpyHostToDevice));
    }
    if (p->Em1p) {
        switch (p->log2ny) {
        case 8: KZK_TRY(build_pair_tables<8>(p, tcf, st)); break;
        case 9: KZK_TRY(build_pair_tables<9>(p, tcf, st)); break;
        case 10: KZK_TRY(build_pair_tables<10>(p, tcf, st)); break;
        case 11: KZK_TRY(build_pair_tables<11>(p, tcf, st)); break;
        default: KZK_TRY(build_pair_tables<12>(p, tcf, st)); break;
        }
    }
    KZK_CUDA(cudaStreamSynchronize(st));
    return KZK_OK;
}

void plan_free(kzk_plan* p)
{
    if (!p) return;
    if (p->subs) {
        for (kzk_plan* q : *p->subs) plan_free(q);
        delete p->subs;
        p->subs = nullptr;
    }
    if (p->graph) cudaGraphExecDestroy(p->graph);
    for (cudaGraphExec_t& g : p->gx)
        if (g) cudaGraphExecDestroy(g);
    if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
    if (p->side) {
        for (cudaStream_t q : *p->side) cudaStreamDestroy(q);
        delete p->side;
    }
    if (p->evs) {
        for (cudaEvent_t q : *p->evs) cudaEventDestroy(q);
        delete p->evs;
    }
    delete p->graph_u;
    void* bptrs[] = {p->binst, p->row_prefix, p->col_prefix, p->coef, p->bar};
    for (void* q : bptrs)
        if (q) cudaFree(q);
    void* ptrs[] = {p->V, p->b1, p->vs, p->b2, p->E, p->P1, p->P2, p->E_lo, p->twr, p->twc, p->twc_lo,
                    p->tws_row, p->twc_full,
                    p->diag_rows, p->diag_hist, p->diag_final, p->lam, p->mu, p->nu, p->ls,
                    p->seg, p->ckpt, p->colp_flag, p->med_Ty, p->med_mode, p->med_coef, p->med_bmax,
                    p->uphys, p->by, p->mpos_row, p->mpos_col, p->mipos_col, p->wsc, p->twr2, p->tws2,
                    p->Vlo, p->vslo, p->Em1, p->Em1p, p->P1p, p->P2p, p->twcp, p->ysig, p->ytmp, p->dcoef, p->dhist};
    for (void* q : ptrs)
        if (q) cudaFree(q);
    delete p;
}

}  // namespace

// ---------------------------------------------------------------------------
// Adjoint driver (kernels in kzk_adjoint.cuh)
// ---------------------------------------------------------------------------
namespace {

kzk_status ensure_buf(void** ptr, long long* cap, long long need, size_t unit)
{
    if (need <= *cap) return KZK_OK;
    if (*ptr) KZK_CUDA(cudaFree(*ptr));
    *ptr = nullptr;
    *cap = 0;
    KZK_CUDA(cudaMalloc(ptr, (size_t)need * unit));
    *cap = need;
    return KZK_OK;
}

template <typename T>
AdjRowArgs<T> adj_row_args(const kzk_plan* p, const void* m, const void* u, const void* l, void* out, double sigma)
{
    AdjRowArgs<T> a{};
    a.m = (const cx<T>*)m;
    a.u = (const T*)u;
    a.l = (const cx<T>*)l;
    a.out = (cx<T>*)out;
    a.tw = (const cx<T>*)p->twr;
    a.tws = (const cx<T>*)p->tws_row;
    a.log2nx = p->log2nx;
    a.inst_stride = p->inst_stride;
    const double Bs = B_of(p, sigma);
    a.wc.B = (T)Bs;
    a.wc.alpha = (T)(Bs * p->c.lf_umax);
    a.wc.eps = (T)p->c.weno_eps;
    a.wc.inv_dtau = (T)(p->nx / (p->g.tau_max - p->g.tau_min));
    a.dA = (T)dA_of(p, sigma);
    a.kscale = (T)(2.0 * M_PI / (p->g.tau_max - p->g.tau_min));
    a.inv_nx = (T)(1.0 / p->nx);
    return a;
}

template <typename T>
AdjColArgs<T> adj_col_args(const kzk_plan* p)
{
    AdjColArgs<T> a{};
    memset(&a, 0, sizeof(a));
    a.tw = (const cx<T>*)p->twc;
    a.log2ny = p->log2ny;
    a.log2n = p->log2nx - 1;
    a.log2tc = p->log2tc;
    a.inst_stride = p->inst_stride;
    return a;
}

// Transposed step on the plan's cotangent p->lam (packed spectral), given the
// step's stage states V^n and V* (packed spectral).
// One transposed row pass: out = l + F(J_{G_sigma}(u)^T C2R(m)) / nx, u the
// physical stage state.  With a random medium: the coefficients at sigma, the
// cotangent in physical space (p->uphys) and the transposed y part (p->by)
// first.
template <typename T, int MODE>
kzk_status adj_row_stage(kzk_plan* p, const void* m, const void* u, const void* l, void* out, double sigma,
                         int slot, cudaStream_t st)
{
    AdjRowArgs<T> r = adj_row_args<T>(p, m, u, l, out, sigma);
    if (p->med_n > 0) {
        KZK_TRY(launch_medium(p, sigma, slot, st));
        KZK_TRY(to_physical<T>(p, m, p->uphys, 1.0, nullptr, st));
        YSweepTArgs<T> y{};
        y.u = (const T*)u;
        y.mu = (const T*)p->uphys;
        y.yT = (T*)p->by;
        y.coef = p->med_coef + (size_t)slot * 3 * p->ny;
        y.bmax = p->med_bmax + (size_t)slot * p->med_nb;
        y.n_bmax = p->med_nb;
        y.nx = p->nx;
        y.ny = p->ny;
        y.Q = std::min(p->ny, 32);
        y.inst_elems = (long long)p->nx * p->ny;
        y.eps = (T)p->c.weno_eps;
        y.inv_dy = (T)(p->ny / (p->g.y_max - p->g.y_min));
        const dim3 yg((p->nx + YSWEEP_THREADS - 1) / YSWEEP_THREADS, (p->ny + y.Q - 1) / y.Q, p->batch);
        ysweepT_kernel<T><<<yg, YSWEEP_THREADS, ysweepT_smem<T>(y.Q), st>>>(y);
        KZK_LAUNCHED();
        r.med_coef = y.coef;
        r.yT = (const T*)p->by;
    }
    const dim3 rgrid(p->ny, p->batch);
    if (p->mixed) {
        MixAdjRowArgs<T> m{};
        m.r = r;
        m.nx = p->nx;
        m.Q = p->madj_Q;
        m.f = p->mrow;
        m.pos = p->mpos_row;
        mix_adj_row_kernel<T, MODE><<<rgrid, p->madj_thr, p->madj_smem, st>>>(m);
        KZK_LAUNCHED();
        return KZK_OK;
    }
    if constexpr (sizeof(T) == 8) {
        if (p->adj_row_thr <= 128) {
            adj_row_kernel<T, row_ppt<T>(), MODE, 128, 3><<<rgrid, p->adj_row_thr, adj_row_smem<T>(p), st>>>(r);
            KZK_LAUNCHED();
            return KZK_OK;
        }
    }
    adj_row_kernel<T, row_ppt<T>(), MODE><<<rgrid, p->adj_row_thr, adj_row_smem<T>(p), st>>>(r);
    KZK_LAUNCHED();
    return KZK_OK;
}

// Transposed column pass (adj_col_kernel, or on mixed-radix grids the
// mix_adj_col_kernel launches: ADJ_COL_1 as two, through the scratch array).
template <typename T, int MODE>
kzk_status launch_adj_col(const kzk_plan* p, const AdjColArgs<T>& c, cudaStream_t st)
{
    if (p->mixed) {
        MixAdjColArgs<T> m{};
        m.c = c;
        m.c.tw = (const cx<T>*)p->twc;
        m.w = (cx<T>*)p->wsc;
        m.ny = p->ny;
        m.n = p->n;
        m.lc = p->mcol_lc;
        m.f = p->mcol;
        m.pos = p->mpos_col;
        m.ipos = p->mipos_col;
        const dim3 grid(p->n >> p->mcol_lc, p->batch);
        if (MODE == ADJ_COL_2) {
            mix_adj_col_kernel<T, MIX_ADJ_C2><<<grid, MIX_COL_THREADS, p->mcol_smem, st>>>(m);
            KZK_LAUNCHED();
        } else {
            mix_adj_col_kernel<T, MIX_ADJ_C1A><<<grid, MIX_COL_THREADS, p->mcol_smem, st>>>(m);
            KZK_LAUNCHED();
            mix_adj_col_kernel<T, MIX_ADJ_C1B><<<grid, MIX_COL_THREADS, p->mcol_smem, st>>>(m);
            KZK_LAUNCHED();
        }
        return KZK_OK;
    }
    const dim3 cgrid(p->n >> p->log2tc, p->batch);
    adj_col_kernel<T, col_ppt_of<T>(), MODE><<<cgrid, p->col_thr, p->col_smem, st>>>(c);
    KZK_LAUNCHED();
    return KZK_OK;
}

template <typename T>
kzk_status adjoint_step(kzk_plan* p, double sigma, const void* un, const void* us, cudaStream_t st)
{
    if (p->c.method == KZK_EXPEULER) {
        // transpose of u' = P_E u + P_{ds Phi1} G_n(u): with mu2 = 0 the
        // stage-1 column pass gives lam_lin = P_{conj E} lam', nu1 =
        // P_{conj(ds Phi1)} lam', then lam = lam_lin + J_{G_n}(u)^T nu1
        const size_t arr = (size_t)p->batch * p->inst_stride * p->csz;
        KZK_CUDA(cudaMemsetAsync(p->mu, 0, arr, st));
        AdjColArgs<T> c1 = adj_col_args<T>(p);
        c1.a = (const cx<T>*)p->lam;
        c1.b = (const cx<T>*)p->mu;
        c1.out = (cx<T>*)p->ls;
        c1.out2 = (cx<T>*)p->nu;
        c1.Ta = (const cx<T>*)p->E;
        c1.sa = (T)1;
        c1.Tb = (const cx<T>*)p->P1;
        c1.sb = (T)p->nx;
        KZK_TRY((launch_adj_col<T, ADJ_COL_1>(p, c1, st)));
        return adj_row_stage<T, ADJ_ROW_1>(p, p->nu, un, p->ls, p->lam, sigma, 0, st);
    }
    // mu2 = P_{conj(ds Phi2)} lam'
    AdjColArgs<T> c2 = adj_col_args<T>(p);
    c2.a = (const cx<T>*)p->lam;
    c2.out = (cx<T>*)p->mu;
    c2.Ta = (const cx<T>*)p->P2;
    c2.sa = (T)p->nx;
    KZK_TRY((launch_adj_col<T, ADJ_COL_2>(p, c2, st)));
    // lam* = lam' + J_{G_{n+1}}(u*)^T mu2
    KZK_TRY((adj_row_stage<T, ADJ_ROW_2>(p, p->mu, us, p->lam, p->ls, sigma + p->dt, 1, st)));
    // lam_lin = P_{conj E} lam*,  nu1 = P_{conj(ds Phi1)} lam* - mu2
    AdjColArgs<T> c1 = adj_col_args<T>(p);
    c1.a = (const cx<T>*)p->ls;
    c1.b = (const cx<T>*)p->mu;
    c1.out = (cx<T>*)p->ls;
    c1.out2 = (cx<T>*)p->nu;
    c1.Ta = (const cx<T>*)p->E;
    c1.sa = (T)1;
    c1.Tb = (const cx<T>*)p->P1;
    c1.sb = (T)p->nx;
    KZK_TRY((launch_adj_col<T, ADJ_COL_1>(p, c1, st)));
    // lam = lam_lin + J_{G_n}(u)^T nu1
    return adj_row_stage<T, ADJ_ROW_1>(p, p->nu, un, p->ls, p->lam, sigma, 0, st);
}

template <typename T>
kzk_status adjoint_buffers(kzk_plan* p, long long n_steps, int k)
{
    const size_t arr = (size_t)p->batch * p->inst_stride * p->csz;
    if (!p->lam) {
        KZK_CUDA(cudaMalloc(&p->lam, arr));
        KZK_CUDA(cudaMalloc(&p->mu, arr));
        KZK_CUDA(cudaMalloc(&p->nu, arr));
        KZK_CUDA(cudaMalloc(&p->ls, arr));
    }
    const long long n_ckpt = (n_steps + k - 1) / k;
    KZK_TRY(ensure_buf(&p->ckpt, &p->ckpt_cap, std::max(1LL, n_ckpt), arr));
    // segment store: the physical u^n and u*^n of every step of a segment
    // (a physical array has the bytes of a spectral one)
    KZK_TRY(ensure_buf(&p->seg, &p->seg_cap, 2 * std::min((long long)k, std::max(1LL, n_steps)), arr));
    return KZK_OK;
}

// Forward sweep from the physical u0 keeping the spectral state at steps
// 0, k, 2k, ... in p->ckpt; the final state is left in p->V.
template <typename T>
kzk_status forward_ckpt(kzk_plan* p, const void* u0, long long n_steps, double sigma0, int k, cudaStream_t st)
{
    KZK_TRY(adjoint_buffers<T>(p, n_steps, k));
    const size_t arr = (size_t)p->batch * p->inst_stride * p->csz;
    KZK_TRY(to_spectral<T>(p, u0, p->V, st));
    for (long long s = 0; s < n_steps; s++) {
        if (s % k == 0)
            KZK_CUDA(cudaMemcpyAsync((char*)p->ckpt + (size_t)(s / k) * arr, p->V, arr, cudaMemcpyDeviceToDevice, st));
        KZK_TRY(step<T>(p, sigma0 + (double)s * p->dt, st, nullptr, p->V, p->vs));
    }
    p->ck_steps = n_steps;
    p->ck_sigma0 = sigma0;
    p->ck_every = k;
    return KZK_OK;
}

// Reverse sweep over the stored checkpoints: per segment, recompute the steps
// from the checkpoint (the spectral state advancing in place in p->V), the
// row passes storing the physical stage states u^n, u*^n into the segment
// store, then apply the transposed steps in reverse order.
template <typename T>
kzk_status reverse_sweep(kzk_plan* p, const void* g_end, void* g0, cudaStream_t st)
{
    const long long n_steps = p->ck_steps, k = p->ck_every;
    const double sigma0 = p->ck_sigma0;
    const long long n_ckpt = (n_steps + k - 1) / k;
    const size_t arr = (size_t)p->batch * p->inst_stride * p->csz;
    auto arr_at = [&](void* base, long long i) { return (void*)((char*)base + (size_t)i * arr); };
    KZK_TRY(to_spectral<T>(p, g_end, p->lam, st));
    for (long long c = n_ckpt - 1; c >= 0; c--) {
        const long long s0 = c * k, s1 = std::min(n_steps, s0 + k);
        for (long long s = s0; s < s1; s++) {
            const long long i = s - s0;
            void* Vn = i == 0 ? arr_at(p->ckpt, c) : p->V;
            if (i == 0) {
                KZK_TRY(reset_lo(p, st));     // checkpoints keep the hi part
                if (ysig_on(p)) KZK_TRY(col_fwd<T>(p, Vn, st));
            }
            KZK_TRY(step<T>(p, sigma0 + (double)s * p->dt, st, nullptr, Vn, p->vs, p->V, arr_at(p->seg, 2 * i),
                            arr_at(p->seg, 2 * i + 1)));
        }
        for (long long s = s1 - 1; s >= s0; s--) {
            const long long i = s - s0;
            KZK_TRY(adjoint_step<T>(p, sigma0 + (double)s * p->dt, arr_at(p->seg, 2 * i), arr_at(p->seg, 2 * i + 1),
                                    st));
        }
    }
    return to_physical<T>(p, p->lam, g0, 1.0, nullptr, st);
}

template <typename T>
kzk_status adjoint_impl(kzk_plan* p, const void* u0, const void* g_end, void* g0, long long n_steps,
                        double sigma0, int ckpt_every, cudaStream_t st)
{
    KZK_TRY(forward_ckpt<T>(p, u0, n_steps, sigma0, ckpt_every, st));
    return reverse_sweep<T>(p, g_end, g0, st);
}

}  // namespace

namespace kzk_internal {
// error reporting for the other translation unit (kzk_noalloc.cu)
kzk_status set_error(kzk_status s, const char* msg) { return fail(s, "%s", msg); }
}  // namespace kzk_internal

// ---------------------------------------------------------------------------
// Batched plans: one persistent cooperative launch for all instances
// ---------------------------------------------------------------------------
namespace {

template <typename T>
size_t batch_smem_for(const kzk_plan* q, int log2tc)
{
    const size_t row = 2 * (size_t)row_buf_len(q->n) * sizeof(cx<T>) + 4 * (BATCH_THREADS / 32) * sizeof(double);
    const size_t col = col_tile_area<T>(q->ny, log2tc, BATCH_THREADS) +
                       (sizeof(T) == 4 ? 2 : 1) * (size_t)q->ny * sizeof(cx<T>);
    const size_t fin = 4 * (size_t)BATCH_THREADS * sizeof(double);
    return std::max(std::max(row, col), fin);
}

// Descriptors of all instances (column tiles capped at 2^tile_cap) and the
// task prefix sums; returns the dynamic shared memory the launch needs.
template <typename T>
kzk_status batch_upload(kzk_plan* p, void* const* u, int tile_cap, size_t* smem_out, cudaStream_t st,
                        long long n_steps = 1)
{
    const int n = (int)p->subs->size();
    // the history buffers must exist (at their final size) before their
    // addresses go into the descriptors
    for (kzk_plan* q : *p->subs) KZK_TRY(ensure_hist(q, std::max(1LL, n_steps)));
    std::vector<BatchInst<T>> bi(n);
    std::vector<int> rp(n + 1, 0), cp(n + 1, 0);
    size_t smem = 0;
    for (int i = 0; i < n; i++) {
        kzk_plan* q = (*p->subs)[i];
        const int l2tc = std::min(q->log2tc, tile_cap);
        BatchInst<T>& I = bi[i];
        memset(&I, 0, sizeof(I));
        I.row = row_args<T>(q, nullptr, nullptr, 0.0, nullptr);
        I.col = col_args<T>(q);
        I.col.log2tc = l2tc;
        I.V = (cx<T>*)q->V; I.b1 = (cx<T>*)q->b1; I.vs = (cx<T>*)q->vs; I.b2 = (cx<T>*)q->b2;
        I.u = u ? (cx<T>*)u[i] : nullptr;
        I.E = (const cx<T>*)q->E; I.E_lo = (const cx<T>*)q->E_lo;
        I.P1 = (const cx<T>*)q->P1; I.P2 = (const cx<T>*)q->P2;
        if (q->comp) {
            I.Em1 = (const cx<T>*)q->Em1;
            I.Vlo = (lo_t<T>*)q->Vlo;
            I.vslo = (lo_t<T>*)q->vslo;
            if (!I.Em1 || !I.Vlo || !I.vslo) return fail(KZK_ERR_STATE, "instance %d: missing lo arrays", i);
        }
        I.diag_rows = q->diag_rows; I.diag_hist = q->diag_hist; I.diag_final = q->diag_final;
        I.ny = q->ny;
        I.n_tiles = q->n >> l2tc;
        I.inv_count = 1.0 / ((double)q->nx * q->ny);
        I.cell = (q->g.tau_max - q->g.tau_min) / q->nx * (q->g.y_max - q->g.y_min) / q->ny;
        rp[i + 1] = rp[i] + q->ny;
        cp[i + 1] = cp[i] + I.n_tiles;
        // every buffer a launch touches must exist before it is described
        const void* need[] = {I.V, I.b1, I.vs, I.b2, I.E, I.P1, I.P2, I.diag_rows, I.diag_hist, I.diag_final,
                              I.row.tw, I.row.tws, I.col.tw};
        for (const void* ptr : need)
            if (!ptr) return fail(KZK_ERR_STATE, "instance %d: missing device buffer", i);
        if (sizeof(T) == 4 && (!I.E_lo || !I.col.tw_lo)) return fail(KZK_ERR_STATE, "instance %d: missing lo tables", i);
        if (u && !I.u) return fail(KZK_ERR_ARG, "u[%d] is NULL", i);
        if (col_threads<T>(q->ny, l2tc) > BATCH_THREADS || row_threads<T>(q->nx) > BATCH_THREADS)
            return fail(KZK_ERR_SIZE, "instance %d does not fit a %d-thread task", i, BATCH_THREADS);
        smem = std::max(smem, batch_smem_for<T>(q, l2tc));
    }
    KZK_CUDA(cudaMemcpyAsync(p->binst, bi.data(), n * sizeof(BatchInst<T>), cudaMemcpyHostToDevice, st));
    KZK_CUDA(cudaMemcpyAsync(p->row_prefix, rp.data(), (n + 1) * sizeof(int), cudaMemcpyHostToDevice, st));
    KZK_CUDA(cudaMemcpyAsync(p->col_prefix, cp.data(), (n + 1) * sizeof(int), cudaMemcpyHostToDevice, st));
    KZK_CUDA(cudaStreamSynchronize(st));     // host vectors go out of scope
    *smem_out = smem;
    return KZK_OK;
}

// per-step coefficients of every instance: B, alpha, nx dA at sigma_s and sigma_s + dt
template <typename T>
kzk_status batch_coefs(kzk_plan* p, long long n_steps, double sigma0, cudaStream_t st)
{
    const int n = (int)p->subs->size();
    if (n_steps > p->coef_cap) {
        if (p->coef) KZK_CUDA(cudaFree(p->coef));
        p->coef = nullptr;
        p->coef_cap = 0;
        KZK_CUDA(cudaMalloc(&p->coef, (size_t)n_steps * n * 6 * sizeof(T)));
        p->coef_cap = n_steps;
    }
    std::vector<T> c((size_t)n_steps * n * 6);
    for (long long s = 0; s < n_steps; s++)
        for (int i = 0; i < n; i++) {
            kzk_plan* q = (*p->subs)[i];
            const double s1 = sigma0 + (double)s * q->dt, s2 = s1 + q->dt;
            T* o = &c[((size_t)s * n + i) * 6];
            const double B1 = B_of(q, s1), B2 = B_of(q, s2);
            o[0] = (T)B1; o[1] = (T)(B1 * q->c.lf_umax); o[2] = (T)(q->nx * dA_of(q, s1));
            o[3] = (T)B2; o[4] = (T)(B2 * q->c.lf_umax); o[5] = (T)(q->nx * dA_of(q, s2));
        }
    KZK_CUDA(cudaMemcpyAsync(p->coef, c.data(), c.size() * sizeof(T), cudaMemcpyHostToDevice, st));
    KZK_CUDA(cudaStreamSynchronize(st));
    return KZK_OK;
}

template <typename T>
kzk_status batch_launch(kzk_plan* p, long long n_steps, cudaStream_t st, bool use_graph)
{
    BatchArgs<T> B{};
    B.inst = (const BatchInst<T>*)p->binst;
    B.row_prefix = p->row_prefix;
    B.col_prefix = p->col_prefix;
    B.coef = (const T*)p->coef;
    B.n_inst = (int)p->subs->size();
    B.n_steps = (int)n_steps;
    B.bar_count = p->bar;
    B.bar_gen = p->bar + 1;
    B.flag = (int*)(p->bar + 2);
    B.expected_blocks = (unsigned)p->grid_ctas + p->test_extra_blocks;
    B.timeout_ns = p->timeout_ns;
    void* args[] = {&B};
    auto enqueue = [&](cudaStream_t on) -> cudaError_t {
        cudaError_t e = cudaMemsetAsync(p->bar, 0, 4 * sizeof(unsigned), on);
        if (e != cudaSuccess) return e;
        // every launch loads its states afresh: the compensated lo parts start at zero
        for (kzk_plan* q : *p->subs)
            if (q->comp) {
                e = cudaMemsetAsync(q->Vlo, 0, (size_t)q->batch * q->inst_stride * sizeof(__nv_bfloat162), on);
                if (e != cudaSuccess) return e;
            }
        return cudaLaunchCooperativeKernel((const void*)batched_kernel<T>, dim3(p->grid_ctas), dim3(BATCH_THREADS),
                                           args, p->batch_smem, on);
    };
    if (!use_graph || p->test_extra_blocks) {
        KZK_CUDA(enqueue(st));
        KZK_LAUNCHED();
        return KZK_OK;
    }
    if (!p->graph || p->graph_steps != n_steps) {
        if (p->graph) { cudaGraphExecDestroy(p->graph); p->graph = nullptr; }
        // capture on the plan's own stream (the caller's may be the legacy
        // default stream, which cannot be captured); the graph is then
        // launched on the caller's stream
        if (!p->cap_stream) KZK_CUDA(cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking));
        cudaGraph_t g = nullptr;
        KZK_CUDA(cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeThreadLocal));
        cudaError_t e = enqueue(p->cap_stream);
        cudaError_t e2 = cudaStreamEndCapture(p->cap_stream, &g);
        if (e != cudaSuccess || e2 != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return fail(KZK_ERR_CUDA, "graph capture of the batched launch: %s",
                        cudaGetErrorString(e != cudaSuccess ? e : e2));
        }
        e = cudaGraphInstantiate(&p->graph, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) { p->graph = nullptr; return fail(KZK_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e)); }
        p->graph_steps = n_steps;
    }
    KZK_CUDA(cudaGraphLaunch(p->graph, st));
    KZK_LAUNCHED();
    return KZK_OK;
}

template <typename T>
kzk_status batch_configure(kzk_plan* p, int tile_cap, cudaStream_t st)
{
    size_t smem = 0;
    KZK_TRY(batch_upload<T>(p, nullptr, tile_cap, &smem, st));
    int dev = 0, sms = 0, optin = 0, nb = 0;
    KZK_CUDA(cudaGetDevice(&dev));
    KZK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    KZK_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    cudaFuncAttributes fa;
    KZK_CUDA(cudaFuncGetAttributes(&fa, batched_kernel<T>));
    const size_t dyn_max = (size_t)optin - fa.sharedSizeBytes;
    if (smem > dyn_max) return fail(KZK_ERR_SIZE, "batched launch needs %zu B of shared memory", smem);
    KZK_CUDA(cudaFuncSetAttribute(batched_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn_max));
    KZK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batched_kernel<T>, BATCH_THREADS, smem));
    if (nb < 1) return fail(KZK_ERR_SIZE, "batched kernel cannot be resident (shared memory %zu B)", smem);
    p->grid_ctas = nb * sms;
    p->batch_smem = smem;
    p->tile_cap = tile_cap;
    if (p->graph) { cudaGraphExecDestroy(p->graph); p->graph = nullptr; }
    return KZK_OK;
}

// Autotuner: time two steps from zero states for each cap on the column tile
// width and keep the fastest.
template <typename T>
kzk_status batch_autotune(kzk_plan* p, cudaStream_t st)
{
    const int n = (int)p->subs->size();
    std::vector<void*> tmp(n, nullptr);
    kzk_status status = KZK_OK;
    for (int i = 0; i < n && status == KZK_OK; i++) {
        kzk_plan* q = (*p->subs)[i];
        if (cudaMalloc(&tmp[i], (size_t)q->nx * q->ny * sizeof(T)) != cudaSuccess) status = fail(KZK_ERR_OOM, "autotune buffers");
        else if (cudaMemsetAsync(tmp[i], 0, (size_t)q->nx * q->ny * sizeof(T), st) != cudaSuccess) status = KZK_ERR_CUDA;
    }
    int best_cap = 4;
    float best = 1e30f;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (status == KZK_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
        status = fail(KZK_ERR_CUDA, "autotune events");
    for (int cap = 0; cap <= 3 && status == KZK_OK; cap++) {
        if ((status = batch_configure<T>(p, cap, st)) != KZK_OK) { status = KZK_OK; continue; }
        size_t smem = 0;
        if ((status = batch_upload<T>(p, tmp.data(), cap, &smem, st, 2)) != KZK_OK) break;
        if ((status = batch_coefs<T>(p, 2, 0.0, st)) != KZK_OK) break;
        if ((status = batch_launch<T>(p, 2, st, false)) != KZK_OK) break;   // warm-up
        cudaEventRecord(e0, st);
        if ((status = batch_launch<T>(p, 2, st, false)) != KZK_OK) break;
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) { best = ms; best_cap = cap; }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    for (void* q : tmp)
        if (q) cudaFree(q);
    if (status != KZK_OK) return status;
    return batch_configure<T>(p, best_cap, st);
}

// Autotuner of a single plan: every eligible (row, column) kernel combination
// the options leave open advances a zero state of the plan's shape for one
// untimed and two timed steps (CUDA events on st); the fastest is kept.
template <typename T>
kzk_status plan_autotune(kzk_plan* p, cudaStream_t st)
{
    std::vector<int> rows, cols;
    if (p->opt.row_kernel != KZK_AUTO) rows.push_back(p->opt.row_kernel);
    else {
        if (p->rowpair_ok) rows.push_back(KZK_ROW_PAIR);
        rows.push_back(KZK_ROW_SINGLE);
    }
    if (p->opt.col_kernel != KZK_AUTO) cols.push_back(p->opt.col_kernel);
    else {
        if (p->colpair_ok) cols.push_back(KZK_COL_PAIR);
        if (p->colp_ok) cols.push_back(KZK_COL_TMA);
        cols.push_back(KZK_COL_TILE);
    }
    if (rows.size() * cols.size() < 2) return KZK_OK;
    const int row0 = row_choice(p), col0 = col_choice(p);
    const size_t bytes = (size_t)p->batch * p->nx * p->ny * sizeof(T);
    void* u = nullptr;
    KZK_CUDA(cudaMalloc(&u, bytes));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    kzk_status status = KZK_OK;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        status = fail(KZK_ERR_CUDA, "autotune events");
    int best_row = row0, best_col = col0;
    float best = 1e30f;
    for (int r : rows)
        for (int c : cols) {
            if (status != KZK_OK) break;
            select_kernels(p, r, c);
            if (cudaMemsetAsync(u, 0, bytes, st) != cudaSuccess) { status = fail(KZK_ERR_CUDA, "autotune memset"); break; }
            if ((status = advance_impl<T>(p, u, 1, 0.0, st, nullptr, true)) != KZK_OK) break;   // warm-up
            cudaEventRecord(e0, st);
            if ((status = advance_impl<T>(p, u, 2, 0.0, st, nullptr, true)) != KZK_OK) break;
            cudaEventRecord(e1, st);
            if (cudaEventSynchronize(e1) != cudaSuccess) { status = fail(KZK_ERR_CUDA, "autotune timing"); break; }
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best) { best = ms; best_row = r; best_col = c; }
        }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(u);
    select_kernels(p, best_row, best_col);
    p->hist_steps = 0;
    return status;
}

template <typename T>
kzk_status advance_batched_impl(kzk_plan* p, void* const* u, long long n_steps, double sigma0, cudaStream_t st,
                                kzk_diag* dout)
{
    size_t smem = 0;
    KZK_TRY(batch_upload<T>(p, u, p->tile_cap, &smem, st, n_steps));
    KZK_TRY(batch_coefs<T>(p, n_steps, sigma0, st));
    KZK_CUDA(cudaMemsetAsync(p->bar + 2, 0, sizeof(unsigned), st));
    KZK_TRY(batch_launch<T>(p, n_steps, st, true));
    for (kzk_plan* q : *p->subs) q->hist_steps = n_steps;
    unsigned flag = 0;
    if (dout || p->test_extra_blocks) {
        KZK_CUDA(cudaStreamSynchronize(st));
        KZK_CUDA(cudaMemcpy(&flag, p->bar + 2, sizeof(unsigned), cudaMemcpyDeviceToHost));
    }
    if (flag & FLAG_TIMEOUT) return fail(KZK_ERR_TIMEOUT, "a grid barrier of the batched launch timed out");
    if (dout) {
        kzk_status worst = KZK_OK;
        for (size_t i = 0; i < p->subs->size(); i++) {
            kzk_status s = finish_diag((*p->subs)[i], n_steps, st, &dout[i]);
            if (s == KZK_ERR_NONFINITE || (s == KZK_ERR_CFL && worst == KZK_OK)) worst = s;
            else if (s != KZK_OK && s != KZK_ERR_CFL && s != KZK_ERR_NONFINITE) return s;
        }
        return worst;
    }
    return KZK_OK;
}

// Streams mode: one CUDA graph per (n_steps, sigma0, state pointers) in
// which every instance runs kzk_advance's launches on its own captured
// stream, forked from and joined back into one origin stream, so the
// instances' kernels run concurrently; replayed on the caller's stream.
template <typename T>
kzk_status advance_streams_impl(kzk_plan* p, void* const* u, long long n_steps, double sigma0, cudaStream_t st,
                                kzk_diag* dout)
{
    const int n = (int)p->subs->size();
    // every buffer the launches touch exists before capture (no allocation
    // may happen while capturing)
    for (kzk_plan* q : *p->subs) KZK_TRY(ensure_hist(q, std::max(1LL, n_steps)));
    std::vector<void*> us(u, u + n);
    const bool cached = p->graph && p->graph_steps == n_steps && p->graph_sigma0 == sigma0 && p->graph_u &&
                        *p->graph_u == us;
    if (!cached) {
        if (p->graph) { cudaGraphExecDestroy(p->graph); p->graph = nullptr; }
        if (!p->cap_stream) KZK_CUDA(cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking));
        if (!p->side) {
            p->side = new (std::nothrow) std::vector<cudaStream_t>();
            p->evs = new (std::nothrow) std::vector<cudaEvent_t>();
            if (!p->side || !p->evs) return fail(KZK_ERR_OOM, "host allocation failed");
            for (int i = 0; i < n; i++) {
                cudaStream_t q = nullptr;
                KZK_CUDA(cudaStreamCreateWithFlags(&q, cudaStreamNonBlocking));
                p->side->push_back(q);
            }
            for (int i = 0; i <= n; i++) {
                cudaEvent_t e = nullptr;
                KZK_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
                p->evs->push_back(e);
            }
        }
        cudaGraph_t g = nullptr;
        KZK_CUDA(cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeThreadLocal));
        kzk_status s = KZK_OK;
        cudaError_t e = cudaEventRecord((*p->evs)[0], p->cap_stream);
        for (int i = 0; i < n && e == cudaSuccess && s == KZK_OK; i++) {
            cudaStream_t q = (*p->side)[i];
            e = cudaStreamWaitEvent(q, (*p->evs)[0], 0);
            if (e == cudaSuccess) s = advance_impl<T>((*p->subs)[i], u[i], n_steps, sigma0, q, nullptr, true);
            if (e == cudaSuccess && s == KZK_OK) e = cudaEventRecord((*p->evs)[i + 1], q);
            if (e == cudaSuccess && s == KZK_OK) e = cudaStreamWaitEvent(p->cap_stream, (*p->evs)[i + 1], 0);
        }
        cudaError_t e2 = cudaStreamEndCapture(p->cap_stream, &g);
        if (s != KZK_OK || e != cudaSuccess || e2 != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            if (s != KZK_OK) return s;
            return fail(KZK_ERR_CUDA, "graph capture of the batched streams: %s",
                        cudaGetErrorString(e != cudaSuccess ? e : e2));
        }
        e = cudaGraphInstantiate(&p->graph, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) { p->graph = nullptr; return fail(KZK_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e)); }
        p->graph_steps = n_steps;
        p->graph_sigma0 = sigma0;
        if (!p->graph_u) p->graph_u = new (std::nothrow) std::vector<void*>();
        if (!p->graph_u) return fail(KZK_ERR_OOM, "host allocation failed");
        *p->graph_u = us;
    }
    KZK_CUDA(cudaGraphLaunch(p->graph, st));
    KZK_LAUNCHED();
    for (kzk_plan* q : *p->subs) q->hist_steps = n_steps;
    if (dout) {
        kzk_status worst = KZK_OK;
        for (size_t i = 0; i < p->subs->size(); i++) {
            kzk_status s = finish_diag((*p->subs)[i], n_steps, st, &dout[i]);
            if (s == KZK_ERR_NONFINITE || (s == KZK_ERR_CFL && worst == KZK_OK)) worst = s;
            else if (s != KZK_OK && s != KZK_ERR_CFL && s != KZK_ERR_NONFINITE) return s;
        }
        return worst;
    }
    return KZK_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// Measurement helpers
// ---------------------------------------------------------------------------
namespace {

// 8 independent FMA chains per thread, `iters` rounds; the result is stored
// only if it is impossible so the chains stay live.
template <typename T>
__global__ void fma_chain_kernel(T* sink, int iters, T a, T b)
{
    T x[8];
#pragma unroll
    for (int c = 0; c < 8; c++) x[c] = (T)(threadIdx.x + c);
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int c = 0; c < 8; c++) x[c] = fma(x[c], a, b);
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < 8; c++) s += x[c];
    if (s == (T)-1.2345) sink[0] = s;
}

// The same on packed FP32 pairs (FFMA2: two FMAs per instruction).
__global__ void fma_chain_pair_kernel(float* sink, int iters, float a, float b)
{
    f2 x[8];
#pragma unroll
    for (int c = 0; c < 8; c++) x[c] = f2((float)(threadIdx.x + c), (float)(threadIdx.x + 2 * c));
    const f2 va(a), vb(b);
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int c = 0; c < 8; c++) x[c] = fma(x[c], va, vb);
    }
    float s = 0;
#pragma unroll
    for (int c = 0; c < 8; c++) s += x[c].v.x + x[c].v.y;
    if (s == -1.2345f) sink[0] = s;
}

// FP32: the faster of scalar FFMA and packed FFMA2 chains (FLOPs per second)
template <typename T>
kzk_status alu_peak_impl(cudaStream_t st, double* out)
{
    int dev = 0, sms = 0;
    KZK_CUDA(cudaGetDevice(&dev));
    KZK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    T* sink = nullptr;
    KZK_CUDA(cudaMalloc(&sink, sizeof(T)));
    const int threads = 256, blocks = sms * 8;
    const int iters = sizeof(T) == 8 ? 2048 : 65536;
    cudaEvent_t e0, e1;
    KZK_CUDA(cudaEventCreate(&e0));
    KZK_CUDA(cudaEventCreate(&e1));
    // the fastest of 7 timed launches after one untimed one (clocks settle)
    float best = 1e30f;
    for (int rep = 0; rep < 8; rep++) {
        KZK_CUDA(cudaEventRecord(e0, st));
        fma_chain_kernel<T><<<blocks, threads, 0, st>>>(sink, iters, (T)0.999999, (T)1e-7);
        KZK_LAUNCHED();
        KZK_CUDA(cudaEventRecord(e1, st));
        KZK_CUDA(cudaEventSynchronize(e1));
        float ms = 0;
        KZK_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        if (rep > 0) best = std::min(best, ms);
    }
    double flops = 2.0 * 8.0 * iters * (double)threads * blocks / (best * 1e-3);
    if (sizeof(T) == 4) {
        float bestp = 1e30f;
        for (int rep = 0; rep < 8; rep++) {
            KZK_CUDA(cudaEventRecord(e0, st));
            fma_chain_pair_kernel<<<blocks, threads, 0, st>>>((float*)sink, iters, 0.999999f, 1e-7f);
            KZK_LAUNCHED();
            KZK_CUDA(cudaEventRecord(e1, st));
            KZK_CUDA(cudaEventSynchronize(e1));
            float ms = 0;
            KZK_CUDA(cudaEventElapsedTime(&ms, e0, e1));
            if (rep > 0) bestp = std::min(bestp, ms);
        }
        flops = std::max(flops, 4.0 * 8.0 * iters * (double)threads * blocks / (bestp * 1e-3));
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    *out = flops;
    return KZK_OK;
}

template <typename T>
kzk_status kernel_times_impl(kzk_plan* p, void* u, long long n_steps, double sigma0, cudaStream_t st, double* ms)
{
    // five events per step, all recorded before one synchronisation at the
    // end: no host wait between steps, so no launch latency lands inside an
    // interval
    std::vector<cudaEvent_t> ev((size_t)std::max(0LL, n_steps) * 5, nullptr);
    kzk_status status = KZK_OK;
    for (auto& e : ev)
        if (cudaEventCreate(&e) != cudaSuccess) { status = fail(KZK_ERR_CUDA, "event creation"); break; }
    double acc[4] = {0, 0, 0, 0};
    if (status == KZK_OK) status = ensure_hist(p, std::max(1LL, n_steps));
    if (status == KZK_OK) status = to_spectral<T>(p, u, p->V, st);
    for (long long s = 0; s < n_steps && status == KZK_OK; s++) {
        const double sigma = sigma0 + (double)s * p->dt;
        status = step<T>(p, sigma, st, p->diag_hist + (size_t)s * p->batch * 4, p->V, p->vs, nullptr, nullptr,
                         nullptr, &ev[(size_t)s * 5]);
    }
    if (status == KZK_OK) status = to_physical<T>(p, p->V, u, 1.0, nullptr, st);
    if (status == KZK_OK && cudaStreamSynchronize(st) != cudaSuccess) status = fail(KZK_ERR_CUDA, "synchronise");
    for (long long s = 0; s < n_steps && status == KZK_OK; s++)
        for (int k = 0; k < 4; k++) {
            float t = 0;
            if (cudaEventElapsedTime(&t, ev[(size_t)s * 5 + k], ev[(size_t)s * 5 + k + 1]) != cudaSuccess) {
                status = fail(KZK_ERR_CUDA, "event timing");
                break;
            }
            acc[k] += t;
        }
    for (auto& e : ev)
        if (e) cudaEventDestroy(e);
    if (status != KZK_OK) return status;
    for (int k = 0; k < 4; k++) ms[k] = n_steps > 0 ? acc[k] / (double)n_steps : 0.0;
    return KZK_OK;
}

// Copy-rate ceiling of the FP32 column-pair tiles (bytes per second): the
// fastest of 7 timed launches of tile_copy_kernel after one untimed one, the
// L2 cache overwritten before each.  Owns its buffers (freed on every path).
struct CopyRateScratch {
    unsigned char* a = nullptr;
    unsigned char* b = nullptr;
    unsigned char* flush = nullptr;
    int* flag = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    ~CopyRateScratch()
    {
        cudaFree(a);
        cudaFree(b);
        cudaFree(flush);
        cudaFree(flag);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    }
};

size_t pair_stage1_smem(int log2ny)
{
    switch (log2ny) {
    case 8: return pair_layout<8, COL_STAGE1>().total;
    case 9: return pair_layout<9, COL_STAGE1>().total;
    case 10: return pair_layout<10, COL_STAGE1>().total;
    case 11: return pair_layout<11, COL_STAGE1>().total;
    default: return pair_layout<12, COL_STAGE1>().total;
    }
}

kzk_status tile_copy_rate_impl(int n, int ny, int contiguous, cudaStream_t st, double* out)
{
    CopyRateScratch m;
    const size_t arr = (size_t)n * ny * 2 * sizeof(float);
    const size_t flush_bytes = 256ull << 20;   // twice the L2 cache
    KZK_CUDA(cudaMalloc(&m.a, arr));
    KZK_CUDA(cudaMalloc(&m.b, arr));
    KZK_CUDA(cudaMalloc(&m.flush, flush_bytes));
    KZK_CUDA(cudaMalloc(&m.flag, sizeof(int)));
    KZK_CUDA(cudaMemsetAsync(m.a, 0, arr, st));
    KZK_CUDA(cudaMemsetAsync(m.b, 0, arr, st));
    KZK_CUDA(cudaMemsetAsync(m.flag, 0, sizeof(int), st));
    TileCopyArgs P;
    memset(&P, 0, sizeof(P));
    P.by = std::min(ny, 256);
    P.nby = ny / P.by;
    P.total = n / 2;
    P.contiguous = contiguous;
    P.tile_bytes = (unsigned)ny * 16u;
    P.a = m.a;
    P.b = m.b;
    P.flag = m.flag;
    P.timeout_ns = 2000000000LL;
    const cuuint64_t dims[3] = {2ull * n, (cuuint64_t)ny, 1ull};
    const cuuint64_t str[2] = {2ull * n * sizeof(float), 2ull * n * ny * sizeof(float)};
    const cuuint32_t box[3] = {4u, (cuuint32_t)P.by, 1u};
    KZK_TRY(encode_map<float>(&P.ma, 3, m.a, dims, str, box));
    KZK_TRY(encode_map<float>(&P.mb, 3, m.b, dims, str, box));
    int log2ny = 0;
    while ((1 << log2ny) < ny) log2ny++;
    const size_t smem = std::max<size_t>(pair_stage1_smem(log2ny), 128 + 2 * (size_t)P.tile_bytes);
    KZK_CUDA(cudaFuncSetAttribute(tile_copy_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    KZK_CUDA(cudaEventCreate(&m.e0));
    KZK_CUDA(cudaEventCreate(&m.e1));
    float best = 1e30f;
    for (int rep = 0; rep < 8; rep++) {
        KZK_CUDA(cudaMemsetAsync(m.flush, rep, flush_bytes, st));
        KZK_CUDA(cudaEventRecord(m.e0, st));
        tile_copy_kernel<<<P.total, 256, smem, st>>>(P);
        KZK_LAUNCHED();
        KZK_CUDA(cudaEventRecord(m.e1, st));
        KZK_CUDA(cudaEventSynchronize(m.e1));
        float ms = 0;
        KZK_CUDA(cudaEventElapsedTime(&ms, m.e0, m.e1));
        if (rep > 0) best = std::min(best, ms);
    }
    int flag = 0;
    KZK_CUDA(cudaMemcpy(&flag, m.flag, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag & FLAG_TIMEOUT) return fail(KZK_ERR_TIMEOUT, "tile copy: a bounded wait ran out");
    if (flag) return fail(KZK_ERR_CUDA, "tile copy: bad launch (flag %d)", flag);
    *out = 2.0 * (double)arr / (best * 1e-3);
    return KZK_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

kzk_status kzk_kernel_times(kzk_plan* p, void* u, int64_t n_steps, double sigma0, void* stream, double* ms)
{
    if (!p || !u || !ms) return fail(KZK_ERR_ARG, "NULL argument");
    if (n_steps < 0) return fail(KZK_ERR_ARG, "n_steps < 0");
    cudaStream_t st = (cudaStream_t)stream;
    return p->prec == KZK_FP64 ? kernel_times_impl<double>(p, u, n_steps, sigma0, st, ms)
                               : kernel_times_impl<float>(p, u, n_steps, sigma0, st, ms);
}

kzk_status kzk_alu_peak(int32_t prec, void* stream, double* flops)
{
    if (!flops || (prec != KZK_FP64 && prec != KZK_FP32)) return fail(KZK_ERR_ARG, "bad argument");
    cudaStream_t st = (cudaStream_t)stream;
    return prec == KZK_FP64 ? alu_peak_impl<double>(st, flops) : alu_peak_impl<float>(st, flops);
}


kzk_status kzk_tile_copy_rate(int32_t n, int32_t ny, int32_t pattern, void* stream, double* bytes_per_s)
{
    if (!bytes_per_s) return fail(KZK_ERR_ARG, "bytes_per_s is NULL");
    if (pattern != KZK_COPY_STRIP && pattern != KZK_COPY_CONTIGUOUS) return fail(KZK_ERR_ARG, "bad pattern %d", pattern);
    if (n < 2 || (n & 1) || ny < 256 || ny > 4096 || !is_pow2(ny) || (long long)n * ny > (1ll << 28))
        return fail(KZK_ERR_SIZE, "tile copy: n = %d, ny = %d (n even, ny a power of two in [256, 4096])", n, ny);
    return tile_copy_rate_impl(n, ny, pattern == KZK_COPY_CONTIGUOUS, (cudaStream_t)stream, bytes_per_s);
}

const char* kzk_status_string(kzk_status s)
{
    switch (s) {
    case KZK_OK: return "ok";
    case KZK_ERR_ARG: return "invalid argument";
    case KZK_ERR_SIZE: return "unsupported grid size";
    case KZK_ERR_CFL: return "max|u| exceeded the Lax-Friedrichs bound lf_umax";
    case KZK_ERR_NONFINITE: return "non-finite value in the state";
    case KZK_ERR_CUDA: return "CUDA error";
    case KZK_ERR_TIMEOUT: return "bounded device wait timed out";
    case KZK_ERR_OOM: return "device out of memory";
    case KZK_ERR_STATE: return "call not valid for this plan";
    }
    return "unknown status";
}

const char* kzk_last_error(void) { return g_err; }

int64_t kzk_launch_count(void) { return (int64_t)g_launches.load(); }

kzk_status kzk_plan_create_ex(const kzk_grid* grid, const kzk_coeffs* coeffs, double dt, int32_t batch,
                              const kzk_options* opts, kzk_plan** out)
{
    if (!out) return fail(KZK_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!grid || !coeffs) return fail(KZK_ERR_ARG, "grid or coeffs is NULL");
    if (grid->prec != KZK_FP64 && grid->prec != KZK_FP32) return fail(KZK_ERR_ARG, "bad precision %d", grid->prec);
    kzk_options o{};
    if (opts) o = *opts;
    if (o.row_kernel < KZK_AUTO || o.row_kernel > KZK_ROW_SINGLE || o.col_kernel < KZK_AUTO ||
        o.col_kernel > KZK_COL_TILE || o.fp32_state < KZK_AUTO || o.fp32_state > KZK_STATE_PLAIN ||
        o.transforms < KZK_AUTO || o.transforms > KZK_TRANSFORMS_MIXED || o.graph < KZK_AUTO ||
        o.graph > KZK_GRAPH_OFF)
        return fail(KZK_ERR_ARG, "unknown option value");
    // powers of two: the radix-8/16 kernels; other even sizes with no prime
    // factor above 7 (the paper's 7 * 2^k x 1250 * 2^k grids), or
    // KZK_TRANSFORMS_MIXED: the mixed-radix kernels
    const bool mixed = !(is_pow2(grid->nx) && is_pow2(grid->ny)) || o.transforms == KZK_TRANSFORMS_MIXED;
    if (!mixed && (grid->nx < 8 || grid->nx > 8192 || grid->ny < 2 || grid->ny > 4096))
        return fail(KZK_ERR_SIZE, "nx = %d, ny = %d: powers of two in [8, 8192] x [2, 4096] required",
                    grid->nx, grid->ny);
    if (mixed && (grid->nx < 8 || grid->nx > 16384 || (grid->nx & 1) || grid->ny < 2 || grid->ny > 32768 ||
                  (grid->ny & 1)))
        return fail(KZK_ERR_SIZE, "nx = %d, ny = %d: even sizes in [8, 16384] x [2, 32768] required",
                    grid->nx, grid->ny);
    if (mixed && (o.row_kernel == KZK_ROW_PAIR || o.col_kernel != KZK_AUTO))
        return fail(KZK_ERR_SIZE, "mixed-radix plans run single rows and the mixed-radix column kernels only");
    if (!(grid->tau_max > grid->tau_min) || !(grid->y_max > grid->y_min))
        return fail(KZK_ERR_ARG, "empty domain");
    if (!(dt > 0) || !std::isfinite(dt)) return fail(KZK_ERR_ARG, "dt must be positive and finite");
    if (!(coeffs->B > 0) || !(coeffs->A >= 0) || !(coeffs->lf_umax > 0))
        return fail(KZK_ERR_ARG, "need B > 0, A >= 0, lf_umax > 0");
    if (coeffs->method != KZK_EXPRK22 && coeffs->method != KZK_EXPEULER)
        return fail(KZK_ERR_ARG, "unknown method %d", coeffs->method);
    if (coeffs->n_relax < 0 || coeffs->n_relax > KZK_MAX_RELAX)
        return fail(KZK_ERR_ARG, "n_relax = %d outside [0, %d]", coeffs->n_relax, KZK_MAX_RELAX);
    for (int r = 0; r < coeffs->n_relax; r++)
        if (!(coeffs->relax_C[r] >= 0) || !std::isfinite(coeffs->relax_C[r]) || !(coeffs->relax_theta[r] > 0) ||
            !std::isfinite(coeffs->relax_theta[r]))
            return fail(KZK_ERR_ARG, "relaxation process %d: need C >= 0 and theta > 0 (finite)", r);
    if (batch < 1) return fail(KZK_ERR_ARG, "batch must be >= 1");

    kzk_plan* p = new (std::nothrow) kzk_plan_s();
    if (!p) return fail(KZK_ERR_OOM, "host allocation failed");
    memset(p, 0, sizeof(*p));
    p->g = *grid;
    p->c = *coeffs;
    p->opt = o;
    if (!(p->c.diffraction > 0)) p->c.diffraction = 1.0 / (4.0 * M_PI);
    // epsilon of the precision the multiplier is evaluated in: the tables are
    // generated in FP64 for both plan precisions
    if (!(p->c.reg_eps > 0)) p->c.reg_eps = std::ldexp(1.0, -53);
    if (!(p->c.weno_eps > 0)) p->c.weno_eps = 1e-6;
    if (!p->c.has_profile) {
        const double one[4] = {1, 0, 0, 0};
        memcpy(p->c.B_prof, one, sizeof(one));
        memcpy(p->c.A_prof, one, sizeof(one));
    }
    p->dt = dt;
    p->batch = batch;
    p->prec = grid->prec;
    p->nx = grid->nx;
    p->ny = grid->ny;
    p->n = grid->nx / 2;
    p->log2nx = ilog2(grid->nx);
    p->log2ny = ilog2(grid->ny);
    p->csz = p->prec == KZK_FP64 ? sizeof(double2) : sizeof(float2);
    p->inst_stride = (long long)p->ny * p->n;
    p->mixed = mixed ? 1 : 0;
    // FP32: compensated spectral state unless a plain one is asked for
    p->comp = (p->prec == KZK_FP32 && o.fp32_state != KZK_STATE_PLAIN) ? 1 : 0;

    kzk_status s = p->prec == KZK_FP64 ? configure<double>(p) : configure<float>(p);
    if (s != KZK_OK) { plan_free(p); return s; }

    // kernel choices: explicit ones must fit; open ones take the defaults (row
    // and column pairs where they fit, else TMA Stockham tiles for FP32, else
    // per-tile kernels), or with autotune every fitting candidate is kept
    // available and timed below
    int row = KZK_ROW_SINGLE, col = KZK_COL_TILE;
    bool keep_rowpair = false, keep_colpair = false;
    if (!mixed) {
        if (o.row_kernel == KZK_ROW_PAIR && !p->rowpair_ok) {
            plan_free(p);
            return fail(KZK_ERR_SIZE, "row pairs need an FP32 plan with even ny whose row pair fits shared memory");
        }
        if (o.col_kernel == KZK_COL_PAIR && !p->colpair_ok) {
            plan_free(p);
            return fail(KZK_ERR_SIZE, "column pairs need an FP32 plan with the compensated state and 256 <= ny <= 4096");
        }
        if (o.col_kernel == KZK_COL_TMA && !p->colp_ok) {
            plan_free(p);
            return fail(KZK_ERR_SIZE, "the TMA-staged column tiles do not fit ny = %d", p->ny);
        }
        row = o.row_kernel != KZK_AUTO ? o.row_kernel : (p->rowpair_ok ? KZK_ROW_PAIR : KZK_ROW_SINGLE);
        col = o.col_kernel != KZK_AUTO ? o.col_kernel
                                        : (p->colpair_ok ? KZK_COL_PAIR
                                                         : (p->colp_ok && p->prec == KZK_FP32 ? KZK_COL_TMA : KZK_COL_TILE));
        keep_rowpair = p->rowpair_ok && (row == KZK_ROW_PAIR || (o.autotune && o.row_kernel == KZK_AUTO));
        keep_colpair = p->colpair_ok && (col == KZK_COL_PAIR || (o.autotune && o.col_kernel == KZK_AUTO));
    }

    const size_t arr = (size_t)batch * p->inst_stride * p->csz;
    const size_t tab = (size_t)(p->ny / 2 + 1) * p->n * p->csz;
    cudaError_t e = cudaSuccess;
    void** bufs[] = {&p->V, &p->b1, &p->vs, &p->b2};
    for (void** b : bufs)
        if (e == cudaSuccess) e = cudaMalloc(b, arr);
    void** tabs[] = {&p->E, &p->P1, &p->P2};
    for (void** t : tabs)
        if (e == cudaSuccess) e = cudaMalloc(t, tab);
    if (e == cudaSuccess && p->prec == KZK_FP32) e = cudaMalloc(&p->E_lo, tab);
    if (e == cudaSuccess && p->prec == KZK_FP32) e = cudaMalloc(&p->twc_lo, (size_t)p->ny * p->csz);
    if (e == cudaSuccess) e = cudaMalloc(&p->twr, (size_t)p->nx * p->csz);
    if (e == cudaSuccess) e = cudaMalloc(&p->tws_row, (size_t)p->n * p->csz);
    if (e == cudaSuccess) e = cudaMalloc(&p->twc_full, (size_t)p->ny * p->csz);
    if (e == cudaSuccess) e = cudaMalloc(&p->twc, (size_t)p->ny * p->csz);
    if (e == cudaSuccess) e = cudaMalloc(&p->diag_rows, (size_t)batch * p->ny * 4 * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&p->diag_final, (size_t)batch * 4 * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&p->colp_flag, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(p->colp_flag, 0, sizeof(int));
    if (p->comp) {
        // lo parts: one bf16 pair per complex value
        const size_t lo_arr = (size_t)batch * p->inst_stride * sizeof(__nv_bfloat162);
        if (e == cudaSuccess) e = cudaMalloc(&p->Vlo, lo_arr);
        if (e == cudaSuccess) e = cudaMalloc(&p->vslo, lo_arr);
        if (e == cudaSuccess) e = cudaMalloc(&p->Em1, tab);
    }
    if (p->ysig_ok) {
        if (e == cudaSuccess) e = cudaMalloc(&p->ysig, arr);
        if (e == cudaSuccess) e = cudaMalloc(&p->ytmp, arr);
    }
    if (keep_colpair) {
        const size_t ptab = (size_t)pair_tab_rows(p->ny) * p->n * sizeof(float2);
        void** ptabs[] = {&p->Em1p, &p->P1p, &p->P2p};
        for (void** t : ptabs)
            if (e == cudaSuccess) e = cudaMalloc(t, ptab);
        if (e == cudaSuccess) e = cudaMalloc(&p->twcp, (size_t)p->ny * sizeof(float4));
    }
    if (keep_rowpair) {
        if (e == cudaSuccess) e = cudaMalloc(&p->twr2, (size_t)p->nx * sizeof(float4));
        if (e == cudaSuccess) e = cudaMalloc(&p->tws2, (size_t)p->n * sizeof(float4));
    }
    if (p->mixed) {
        if (e == cudaSuccess) e = cudaMalloc(&p->mpos_row, (size_t)p->n * sizeof(int));
        if (e == cudaSuccess) e = cudaMalloc(&p->mpos_col, (size_t)p->ny * sizeof(int));
        if (e == cudaSuccess) e = cudaMalloc(&p->mipos_col, (size_t)p->ny * sizeof(int));
        if (e == cudaSuccess) e = cudaMalloc(&p->wsc, arr);
    }
    if (e != cudaSuccess) {
        plan_free(p);
        return fail(e == cudaErrorMemoryAllocation ? KZK_ERR_OOM : KZK_ERR_CUDA, "plan allocation: %s",
                    cudaGetErrorString(e));
    }
    select_kernels(p, row, col);
    s = p->prec == KZK_FP64 ? build_tables<double>(p, 0) : build_tables<float>(p, 0);
    if (s == KZK_OK && o.autotune && !mixed)
        s = p->prec == KZK_FP64 ? plan_autotune<double>(p, 0) : plan_autotune<float>(p, 0);
    if (s != KZK_OK) { plan_free(p); return s; }
    *out = p;
    return KZK_OK;
}

kzk_status kzk_plan_create(const kzk_grid* grid, const kzk_coeffs* coeffs, double dt, int32_t batch,
                           kzk_plan** out)
{
    return kzk_plan_create_ex(grid, coeffs, dt, batch, nullptr, out);
}

kzk_status kzk_plan_info(kzk_plan* p, kzk_options* out)
{
    if (!p || !out) return fail(KZK_ERR_ARG, "NULL argument");
    if (p->batched) return fail(KZK_ERR_STATE, "batched plan");
    kzk_options o{};
    o.row_kernel = row_choice(p);
    o.col_kernel = p->mixed ? KZK_AUTO : col_choice(p);
    o.fp32_state = p->prec == KZK_FP32 ? (p->comp ? KZK_STATE_COMPENSATED : KZK_STATE_PLAIN) : KZK_AUTO;
    o.transforms = p->mixed ? KZK_TRANSFORMS_MIXED : KZK_AUTO;
    o.autotune = p->opt.autotune;
    o.graph = p->opt.graph == KZK_GRAPH_OFF ? KZK_GRAPH_OFF : KZK_GRAPH_ON;
    *out = o;
    return KZK_OK;
}

kzk_status kzk_plan_set_medium(kzk_plan* p, const kzk_medium* m)
{
    if (!p || !m) return fail(KZK_ERR_ARG, "plan or medium is NULL");
    if (p->batched) return fail(KZK_ERR_STATE, "batched plans take no medium");
    const int N = m->n_modes;
    if (N < 0 || N > KZK_MAX_MODES) return fail(KZK_ERR_ARG, "n_modes = %d outside [0, %d]", N, KZK_MAX_MODES);
    if (N > 0 && (!m->klam || !m->theta || !m->phase || !m->amp))
        return fail(KZK_ERR_ARG, "mode arrays are NULL");
    for (int n = 0; n < N; n++)
        if (!std::isfinite(m->klam[n]) || !std::isfinite(m->theta[n]) || !std::isfinite(m->phase[n]) ||
            !std::isfinite(m->amp[n]))
            return fail(KZK_ERR_ARG, "mode %d: non-finite value", n);
    drop_step_graphs(p);   // captured without (or with another) medium
    void* old[] = {p->med_Ty, p->med_mode, p->med_coef, p->med_bmax, p->uphys, p->by};
    for (void* q : old)
        if (q) KZK_CUDA(cudaFree(q));
    p->med_Ty = nullptr; p->med_mode = nullptr; p->med_coef = nullptr; p->med_bmax = nullptr; p->uphys = nullptr;
    p->by = nullptr;
    p->med_n = 0;
    if (N == 0) return KZK_OK;
    const int ny = p->ny;
    const int nb = (ny + MED_ROWS - 1) / MED_ROWS;
    std::vector<double> mode(5 * (size_t)N), Ty(2 * (size_t)N * ny);
    const double dy = (p->g.y_max - p->g.y_min) / ny;
    for (int n = 0; n < N; n++) {
        const double st = std::sin(m->theta[n]), ct = std::cos(m->theta[n]);
        const double c_n = m->klam[n] * st;                 // d(arg)/dy
        mode[n] = m->klam[n] * ct;                          // d(arg)/dsigma
        mode[N + n] = m->phase[n];
        mode[2 * N + n] = -m->amp[n] * st;                  // U_par weight
        mode[3 * N + n] = m->amp[n] * ct;                   // U_perp weight
        mode[4 * N + n] = -m->amp[n] * ct * c_n;            // d U_perp / dy weight (of Im P)
        for (int j = 0; j < ny; j++) {
            const double y = p->g.y_min + j * dy;
            Ty[2 * ((size_t)n * ny + j)] = std::cos(c_n * y);
            Ty[2 * ((size_t)n * ny + j) + 1] = std::sin(c_n * y);
        }
    }
    cudaError_t e = cudaMalloc(&p->med_Ty, Ty.size() * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc((void**)&p->med_mode, mode.size() * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc((void**)&p->med_coef, 2 * 3 * (size_t)ny * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc((void**)&p->med_bmax, 2 * (size_t)nb * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&p->uphys, (size_t)p->batch * p->inst_stride * p->csz);
    if (e == cudaSuccess) e = cudaMalloc(&p->by, (size_t)p->batch * p->inst_stride * p->csz);
    if (e == cudaSuccess) e = cudaMemcpy(p->med_Ty, Ty.data(), Ty.size() * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(p->med_mode, mode.data(), mode.size() * sizeof(double), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        void* got[] = {p->med_Ty, p->med_mode, p->med_coef, p->med_bmax, p->uphys, p->by};
        for (void* q : got)
            if (q) cudaFree(q);
        p->med_Ty = nullptr; p->med_mode = nullptr; p->med_coef = nullptr; p->med_bmax = nullptr; p->uphys = nullptr;
        p->by = nullptr;
        return fail(e == cudaErrorMemoryAllocation ? KZK_ERR_OOM : KZK_ERR_CUDA, "medium set-up: %s",
                    cudaGetErrorString(e));
    }
    p->med_n = N;
    p->med_nb = nb;
    p->ck_steps = 0;      // stored adjoint checkpoints belong to the old medium
    return KZK_OK;
}

kzk_status kzk_medium_eval(kzk_plan* p, double sigma, double* out, double* max_uperp, void* stream)
{
    if (!p || !out) return fail(KZK_ERR_ARG, "NULL argument");
    if (p->med_n < 1) return fail(KZK_ERR_STATE, "no medium set");
    cudaStream_t st = (cudaStream_t)stream;
    KZK_TRY(launch_medium(p, sigma, 0, st));
    KZK_CUDA(cudaMemcpyAsync(out, p->med_coef, 3 * (size_t)p->ny * sizeof(double), cudaMemcpyDeviceToHost, st));
    std::vector<double> bm(p->med_nb);
    KZK_CUDA(cudaMemcpyAsync(bm.data(), p->med_bmax, bm.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    KZK_CUDA(cudaStreamSynchronize(st));
    if (max_uperp) {
        double mx = 0.0;
        for (double v : bm) mx = std::max(mx, v);
        *max_uperp = mx;
    }
    return KZK_OK;
}

kzk_status kzk_plan_create_batched_ex(const kzk_grid* grids, const kzk_coeffs* coeffs, const double* dts, int32_t n,
                                      int32_t flags, const kzk_options* opts, kzk_plan** out)
{
    if (!out) return fail(KZK_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!grids || !coeffs || !dts || n < 1) return fail(KZK_ERR_ARG, "need grids, coeffs, dts and n >= 1");
    if ((flags & KZK_BATCH_STREAMS) && (flags & KZK_BATCH_PERSISTENT))
        return fail(KZK_ERR_ARG, "KZK_BATCH_STREAMS and KZK_BATCH_PERSISTENT are exclusive");
    if (flags & ~(KZK_BATCH_AUTOTUNE | KZK_BATCH_STREAMS | KZK_BATCH_PERSISTENT))
        return fail(KZK_ERR_ARG, "unknown batched-plan flag");
    const bool persistent = (flags & KZK_BATCH_PERSISTENT) != 0;
    for (int i = 1; i < n; i++)
        if (grids[i].prec != grids[0].prec) return fail(KZK_ERR_ARG, "all instances must share one precision");
    // instance plans: streams mode runs their own kernels (autotuned with
    // KZK_BATCH_AUTOTUNE); the persistent kernel has its own bodies, so its
    // instances take the single-row / per-tile choices, which allocate nothing
    // for the pair kernels
    kzk_options io{};
    if (opts) io = *opts;
    if (persistent) {
        io.row_kernel = KZK_ROW_SINGLE;
        io.col_kernel = KZK_COL_TILE;
        io.autotune = 0;
    } else if (flags & KZK_BATCH_AUTOTUNE) {
        io.autotune = 1;
    }
    kzk_plan* p = new (std::nothrow) kzk_plan_s();
    if (!p) return fail(KZK_ERR_OOM, "host allocation failed");
    memset(p, 0, sizeof(*p));
    p->batched = 1;
    p->prec = grids[0].prec;
    p->batch = n;
    p->timeout_ns = 2000000000LL;
    p->subs = new (std::nothrow) std::vector<kzk_plan_s*>();
    if (!p->subs) { delete p; return fail(KZK_ERR_OOM, "host allocation failed"); }
    for (int i = 0; i < n; i++) {
        kzk_plan* q = nullptr;
        kzk_status s = kzk_plan_create_ex(&grids[i], &coeffs[i], dts[i], 1, &io, &q);
        if (s != KZK_OK) { plan_free(p); return s; }
        p->subs->push_back(q);
        if (persistent && (q->nx > 8192 || q->mixed)) {
            plan_free(p);
            return fail(KZK_ERR_SIZE, "instance %d: the persistent batched kernel needs power-of-two grids, nx <= 8192", i);
        }
    }
    cudaError_t e = cudaMalloc(&p->binst, (size_t)n * std::max(sizeof(BatchInst<float>), sizeof(BatchInst<double>)));
    if (e == cudaSuccess) e = cudaMalloc(&p->row_prefix, (n + 1) * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&p->col_prefix, (n + 1) * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&p->bar, 4 * sizeof(unsigned));
    if (e != cudaSuccess) { plan_free(p); return fail(KZK_ERR_OOM, "batched plan allocation: %s", cudaGetErrorString(e)); }
    kzk_status s;
    if (!persistent) {
        p->batch_streams = 1;
        *out = p;
        return KZK_OK;
    }
    if (flags & KZK_BATCH_AUTOTUNE)
        s = p->prec == KZK_FP64 ? batch_autotune<double>(p, 0) : batch_autotune<float>(p, 0);
    else
        s = p->prec == KZK_FP64 ? batch_configure<double>(p, 4, 0) : batch_configure<float>(p, 4, 0);
    if (s != KZK_OK) { plan_free(p); return s; }
    *out = p;
    return KZK_OK;
}

kzk_status kzk_plan_create_batched(const kzk_grid* grids, const kzk_coeffs* coeffs, const double* dts, int32_t n,
                                   int32_t flags, kzk_plan** out)
{
    return kzk_plan_create_batched_ex(grids, coeffs, dts, n, flags, nullptr, out);
}

kzk_status kzk_advance_batched(kzk_plan* p, void* const* u, int64_t n_steps, double sigma0, void* stream,
                               kzk_diag* diag_out)
{
    if (!p || !u) return fail(KZK_ERR_ARG, "plan or u is NULL");
    if (!p->batched) return fail(KZK_ERR_STATE, "not a batched plan");
    if (n_steps < 0 || n_steps > (1LL << 30)) return fail(KZK_ERR_ARG, "bad n_steps");
    for (int i = 0; i < p->batch; i++)
        if (!u[i]) return fail(KZK_ERR_ARG, "u[%d] is NULL", i);
    if (n_steps == 0 && !diag_out) return KZK_OK;
    cudaStream_t st = (cudaStream_t)stream;
    if (p->batch_streams)
        return p->prec == KZK_FP64 ? advance_streams_impl<double>(p, u, n_steps, sigma0, st, diag_out)
                                   : advance_streams_impl<float>(p, u, n_steps, sigma0, st, diag_out);
    return p->prec == KZK_FP64 ? advance_batched_impl<double>(p, u, n_steps, sigma0, st, diag_out)
                               : advance_batched_impl<float>(p, u, n_steps, sigma0, st, diag_out);
}

kzk_status kzk_batch_info(kzk_plan* p, int32_t* grid_ctas, int32_t* tile_cap, int64_t* smem_bytes)
{
    if (!p || !p->batched) return fail(KZK_ERR_STATE, "not a batched plan");
    if (grid_ctas) *grid_ctas = p->grid_ctas;
    if (tile_cap) *tile_cap = p->tile_cap;
    if (smem_bytes) *smem_bytes = (int64_t)p->batch_smem;
    return KZK_OK;
}

kzk_status kzk_batch_test_barrier(kzk_plan* p, int32_t extra_blocks, int64_t timeout_ms)
{
    if (!p || !p->batched) return fail(KZK_ERR_STATE, "not a batched plan");
    if (p->batch_streams) return fail(KZK_ERR_STATE, "a batched plan in streams mode has no grid barrier");
    if (extra_blocks < 0 || timeout_ms < 1 || timeout_ms > 60000) return fail(KZK_ERR_ARG, "bad barrier test values");
    p->test_extra_blocks = (unsigned)extra_blocks;
    p->timeout_ns = timeout_ms * 1000000LL;
    return KZK_OK;
}

kzk_status kzk_plan_destroy(kzk_plan* plan)
{
    plan_free(plan);
    return KZK_OK;
}

kzk_status kzk_advance(kzk_plan* p, void* u, int64_t n_steps, double sigma0, void* stream, kzk_diag* diag_out)
{
    if (!p || !u) return fail(KZK_ERR_ARG, "plan or u is NULL");
    if (p->batched) return fail(KZK_ERR_STATE, "batched plan: use kzk_advance_batched");
    if (n_steps < 0) return fail(KZK_ERR_ARG, "n_steps < 0");
    if (n_steps == 0 && !diag_out) return KZK_OK;
    cudaStream_t st = (cudaStream_t)stream;
    return p->prec == KZK_FP64 ? advance_impl<double>(p, u, n_steps, sigma0, st, diag_out)
                               : advance_impl<float>(p, u, n_steps, sigma0, st, diag_out);
}

kzk_status kzk_diag_history(kzk_plan* p, double* hist, int64_t n, void* stream)
{
    if (!p || !hist) return fail(KZK_ERR_ARG, "plan or hist is NULL");
    const long long m = std::min<long long>(n, p->hist_steps);
    KZK_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    if (m > 0)
        KZK_CUDA(cudaMemcpy(hist, p->diag_hist, (size_t)m * p->batch * 4 * sizeof(double), cudaMemcpyDeviceToHost));
    return KZK_OK;
}

kzk_status kzk_rhs(kzk_plan* p, const void* u, void* b, double sigma, void* stream)
{
    if (!p || !u || !b) return fail(KZK_ERR_ARG, "NULL argument");
    if (u == b) return fail(KZK_ERR_ARG, "b may not alias u");
    cudaStream_t st = (cudaStream_t)stream;
    if (p->prec == KZK_FP64) {
        KZK_TRY(to_spectral<double>(p, u, p->V, st));
        KZK_TRY(rhs_stage<double>(p, sigma, p->V, p->b1, nullptr, nullptr, 0, st));
        return to_physical<double>(p, p->b1, b, 1.0 / p->nx, nullptr, st);
    }
    KZK_TRY(to_spectral<float>(p, u, p->V, st));
    KZK_TRY(rhs_stage<float>(p, sigma, p->V, p->b1, nullptr, nullptr, 0, st));
    return to_physical<float>(p, p->b1, b, 1.0 / p->nx, nullptr, st);
}

kzk_status kzk_step_stages(kzk_plan* p, const void* u, void* u_star, void* u_next, double sigma0, void* stream)
{
    if (!p || !u || !u_star || !u_next) return fail(KZK_ERR_ARG, "NULL argument");
    cudaStream_t st = (cudaStream_t)stream;
    // exponential Euler: the step is its first stage, u_star = u_next
    const bool euler = p->c.method == KZK_EXPEULER;
    if (p->prec == KZK_FP64) {
        KZK_TRY(to_spectral<double>(p, u, p->V, st));
        KZK_TRY(step<double>(p, sigma0, st, nullptr, p->V, p->vs));
        KZK_TRY(to_physical<double>(p, euler ? p->V : p->vs, u_star, 1.0, nullptr, st));
        return to_physical<double>(p, p->V, u_next, 1.0, nullptr, st);
    }
    KZK_TRY(to_spectral<float>(p, u, p->V, st));
    KZK_TRY(step<float>(p, sigma0, st, nullptr, p->V, p->vs));
    KZK_TRY(to_physical<float>(p, euler ? p->V : p->vs, u_star, 1.0, nullptr, st));
    return to_physical<float>(p, p->V, u_next, 1.0, nullptr, st);
}

kzk_status kzk_tau_fft(kzk_plan* p, const void* in, void* out, int32_t dir, void* stream)
{
    if (!p || !in || !out) return fail(KZK_ERR_ARG, "NULL argument");
    if (in == out) return fail(KZK_ERR_ARG, "in and out may not alias");
    if (dir != -1 && dir != 1) return fail(KZK_ERR_ARG, "dir must be -1 or +1");
    cudaStream_t st = (cudaStream_t)stream;
    if (p->prec == KZK_FP64)
        return dir < 0 ? to_spectral<double>(p, in, out, st) : to_physical<double>(p, in, out, 1.0, nullptr, st);
    return dir < 0 ? to_spectral<float>(p, in, out, st) : to_physical<float>(p, in, out, 1.0, nullptr, st);
}

kzk_status kzk_get_tables(kzk_plan* p, double* E, double* Phi1, double* Phi2)
{
    if (!p || !E || !Phi1 || !Phi2) return fail(KZK_ERR_ARG, "NULL argument");
    KZK_CUDA(cudaDeviceSynchronize());
    const int nl = p->ny / 2 + 1, n = p->n;
    const size_t cnt = (size_t)nl * n;
    std::vector<double> raw(cnt * 2);
    void* src[3] = {p->E, p->P1, p->P2};
    double* dst[3] = {E, Phi1, Phi2};
    const double unscale[3] = {(double)p->ny, (double)p->nx * p->ny / p->dt, (double)p->nx * p->ny / p->dt};
    for (int t = 0; t < 3; t++) {
        if (p->prec == KZK_FP64) {
            KZK_CUDA(cudaMemcpy(raw.data(), src[t], cnt * sizeof(double2), cudaMemcpyDeviceToHost));
        } else {
            std::vector<float> f(cnt * 2);
            KZK_CUDA(cudaMemcpy(f.data(), src[t], cnt * sizeof(float2), cudaMemcpyDeviceToHost));
            for (size_t i = 0; i < f.size(); i++) raw[i] = f[i];
        }
        const int w = n + 1;
        for (int l = 0; l < nl; l++) {
            for (int m = 0; m < n; m++) {
                const double re = raw[2 * ((size_t)l * n + m)] * unscale[t];
                const double im = raw[2 * ((size_t)l * n + m) + 1] * unscale[t];
                if (m == 0) {
                    dst[t][2 * ((size_t)l * w + 0)] = re;
                    dst[t][2 * ((size_t)l * w + 0) + 1] = 0.0;
                    dst[t][2 * ((size_t)l * w + n)] = im;
                    dst[t][2 * ((size_t)l * w + n) + 1] = 0.0;
                } else {
                    dst[t][2 * ((size_t)l * w + m)] = re;
                    dst[t][2 * ((size_t)l * w + m) + 1] = im;
                }
            }
        }
    }
    return KZK_OK;
}

kzk_status kzk_advance_checkpointed(kzk_plan* p, void* u, int64_t n_steps, double sigma0, int32_t ckpt_every,
                                    void* stream)
{
    if (!p || !u) return fail(KZK_ERR_ARG, "plan or u is NULL");
    if (p->batched) return fail(KZK_ERR_STATE, "batched plan");
    if (n_steps < 1 || ckpt_every < 1) return fail(KZK_ERR_ARG, "need n_steps >= 1 and ckpt_every >= 1");
    if (p->mixed && !p->madj_Q) return fail(KZK_ERR_SIZE, "nx = %d: no transposed row pass for this length", p->nx);
    cudaStream_t st = (cudaStream_t)stream;
    p->ck_steps = 0;
    if (p->prec == KZK_FP64) {
        KZK_TRY(forward_ckpt<double>(p, u, n_steps, sigma0, ckpt_every, st));
        return to_physical<double>(p, p->V, u, 1.0, nullptr, st);
    }
    KZK_TRY(forward_ckpt<float>(p, u, n_steps, sigma0, ckpt_every, st));
    return to_physical<float>(p, p->V, u, 1.0, nullptr, st);
}

kzk_status kzk_adjoint_checkpointed(kzk_plan* p, const void* g_end, void* g0, void* stream)
{
    if (!p || !g_end || !g0) return fail(KZK_ERR_ARG, "NULL argument");
    if (p->batched) return fail(KZK_ERR_STATE, "batched plan");
    if (p->ck_steps < 1) return fail(KZK_ERR_STATE, "no checkpointed forward run stored in this plan");
    cudaStream_t st = (cudaStream_t)stream;
    return p->prec == KZK_FP64 ? reverse_sweep<double>(p, g_end, g0, st) : reverse_sweep<float>(p, g_end, g0, st);
}

kzk_status kzk_adjoint(kzk_plan* p, const void* u0, const void* g_end, void* g0, int64_t n_steps, double sigma0,
                       int32_t ckpt_every, void* stream)
{
    if (!p || !u0 || !g_end || !g0) return fail(KZK_ERR_ARG, "NULL argument");
    if (n_steps < 0 || ckpt_every < 1) return fail(KZK_ERR_ARG, "need n_steps >= 0 and ckpt_every >= 1");
    if (p->mixed && !p->madj_Q) return fail(KZK_ERR_SIZE, "nx = %d: no transposed row pass for this length", p->nx);
    cudaStream_t st = (cudaStream_t)stream;
    if (n_steps == 0) {
        if (g0 != g_end)
            KZK_CUDA(cudaMemcpyAsync(g0, g_end, (size_t)p->batch * p->ny * p->nx * (p->csz / 2),
                                     cudaMemcpyDeviceToDevice, st));
        return KZK_OK;
    }
    return p->prec == KZK_FP64 ? adjoint_impl<double>(p, u0, g_end, g0, n_steps, sigma0, ckpt_every, st)
                               : adjoint_impl<float>(p, u0, g_end, g0, n_steps, sigma0, ckpt_every, st);
}

}  // extern "C"
