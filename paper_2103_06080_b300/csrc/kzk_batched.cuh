// kzk_batched.cuh -- many independent propagations (different grids, pulse
// shapes, atmosphere profiles and steps dsigma) advanced by ONE persistent
// cooperative launch.
//
// The launch walks the passes of every step for all instances together:
//   FWD (physical -> spectral), then per step R1, C1, R2, C2
//   (Algorithm 2, STEP 1-4), then INV (spectral -> physical) and the final
//   diagnostics.
// FP32 instances carry the compensated state of their plans (the column
// bodies transform increments and add them to hi + lo; the lo parts start at
// zero with every launch).
// Each pass is a list of tasks -- rows of every instance for the row passes,
// column tiles of every instance for the column passes -- handed out round
// robin over the CTAs; a grid barrier separates the passes.  The barrier's
// wait is bounded: after timeout_ns a CTA sets FLAG_TIMEOUT and every CTA
// leaves the kernel at its next barrier, so a bad launch cannot hang.
#pragma once
#include "kzk_kernels.cuh"

namespace kzk {

template <typename T>
struct BatchInst {
    RowArgs<T> row;          // constant fields; in/out/coefficients set per pass
    ColArgs<T> col;          // constant fields; arrays set per pass
    cx<T>* V;
    cx<T>* b1;
    cx<T>* vs;
    cx<T>* b2;
    cx<T>* u;                // caller's physical state (as complex pairs)
    const cx<T>* E;
    const cx<T>* E_lo;
    const cx<T>* P1;
    const cx<T>* P2;
    // FP32 plans with the compensated state (hi + lo, lo in row layout here):
    // (E - 1)', and the lo parts of V and V*; nullptr for the plain state
    const cx<T>* Em1;
    lo_t<T>* Vlo;
    lo_t<T>* vslo;
    double* diag_rows;       // [ny][4]
    double* diag_hist;       // [hist_cap][4]
    double* diag_final;      // [4]
    int ny, n_tiles;
    double inv_count, cell;
};

template <typename T>
struct BatchArgs {
    const BatchInst<T>* inst;    // [n_inst]
    const int* row_prefix;       // [n_inst + 1]: cumulative rows
    const int* col_prefix;       // [n_inst + 1]: cumulative column tiles
    const T* coef;               // [n_steps][n_inst][6]: B, alpha, nx dA at sigma_s and at sigma_s + dt
    int n_inst, n_steps;
    unsigned* bar_count;
    unsigned* bar_gen;
    int* flag;
    unsigned expected_blocks;    // CTAs the barrier waits for
    long long timeout_ns;
};

// Grid-wide barrier with a bounded wait.  Returns false once any CTA has
// timed out (the caller then leaves the kernel).
template <typename T>
__device__ __forceinline__ bool grid_sync(const BatchArgs<T>& B, int* sflag)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned* genp = B.bar_gen;
        const unsigned g = *genp;
        __threadfence();
        const unsigned arrived = atomicAdd(B.bar_count, 1u) + 1u;
        if (arrived == B.expected_blocks) {
            atomicExch(B.bar_count, 0u);
            __threadfence();
            atomicAdd(B.bar_gen, 1u);
        } else {
            const long long t0 = global_ns();
            while (*genp == g) {
                if (*(volatile int*)B.flag & FLAG_TIMEOUT) break;
                if (global_ns() - t0 > B.timeout_ns) {
                    atomicOr(B.flag, FLAG_TIMEOUT);
                    break;
                }
                __nanosleep(100);
            }
        }
        __threadfence();
        *sflag = *(volatile int*)B.flag;
    }
    __syncthreads();
    return (*sflag & FLAG_TIMEOUT) == 0;
}

__device__ __forceinline__ int find_inst(const int* prefix, int n, int item)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(prefix + mid) <= item) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// The arguments of the current task are staged in shared memory (one copy
// per CTA), so the inlined bodies read them like the standalone kernels read
// their constant-bank parameters instead of holding them in registers.
template <typename T>
union TaskArgs {
    RowArgs<T> row;
    ColArgs<T> col;
};

template <typename T, int MODE>
__device__ __forceinline__ void batched_rows(const BatchArgs<T>& B, int step, unsigned char* smem, TaskArgs<T>* targs)
{
    const int total = __ldg(B.row_prefix + B.n_inst);
    for (int item = blockIdx.x; item < total; item += gridDim.x) {
        const int i = find_inst(B.row_prefix, B.n_inst, item);
        const int row = item - __ldg(B.row_prefix + i);
        if (threadIdx.x == 0) {
        const BatchInst<T>& I = B.inst[i];
        RowArgs<T> a = I.row;
        if (MODE == ROW_FWD) {
            a.in = I.u; a.out = I.V; a.diag_rows = nullptr;
            a.out_scale = T(1) / T(1 << a.log2nx);            // V = F(u) / nx
        } else if (MODE == ROW_INV) {
            a.in = I.V; a.out = I.u; a.diag_rows = I.diag_rows; a.out_scale = (T)1;
        } else {
            const int stage = step < 0 ? 0 : (step & 1);          // encoded: 2 s + stage
            const int s = step >> 1;
            const T* c = B.coef + ((size_t)s * B.n_inst + i) * 6 + 3 * stage;
            a.wc.B = c[0]; a.wc.alpha = c[1]; a.cA = c[2];
            a.in = stage == 0 ? I.V : I.vs;
            a.out = stage == 0 ? I.b1 : I.b2;
            a.diag_rows = stage == 0 ? I.diag_rows : nullptr;
        }
        targs->row = a;
        }
        __syncthreads();
        row_body<T, MODE>(targs->row, row, 0, smem);
        __syncthreads();
    }
}

template <typename T, int MODE>
__device__ __forceinline__ void batched_cols(const BatchArgs<T>& B, int s, unsigned char* smem, TaskArgs<T>* targs)
{
    const int total = __ldg(B.col_prefix + B.n_inst);
    for (int item = blockIdx.x; item < total; item += gridDim.x) {
        const int i = find_inst(B.col_prefix, B.n_inst, item);
        const int tile = item - __ldg(B.col_prefix + i);
        if (threadIdx.x == 0) {
        const BatchInst<T>& I = B.inst[i];
        ColArgs<T> a = I.col;
        if (MODE == COL_STAGE1) {
            a.a = I.V; a.b = I.b1; a.out = I.vs;
            a.Ta = I.E; a.Ta_lo = I.E_lo; a.Tb = I.P1;
            a.diag_rows = I.diag_rows;
            a.diag_hist = I.diag_hist + (size_t)s * 4;
            if (I.Vlo) { a.Ta = I.Em1; a.Ta_lo = nullptr; a.lo_in = I.Vlo; a.lo_out = I.vslo; }
        } else {
            a.a = I.b1; a.b = I.b2; a.c = I.vs; a.out = I.V;
            a.Ta = I.P2;
            a.diag_rows = nullptr;
            if (I.Vlo) { a.lo_in = I.vslo; a.lo_out = I.Vlo; }
        }
        targs->col = a;
        }
        __syncthreads();
        col_body<T, MODE>(targs->col, tile, 0, smem);
        __syncthreads();
    }
}

// One call per pass: the task loop and its body are register-allocated on
// their own (like a standalone kernel) instead of as part of one function
// holding every body.
template <typename T, int MODE>
__device__ __noinline__ void pass_rows(const BatchArgs<T>* B, int step, unsigned char* smem, TaskArgs<T>* targs)
{
    batched_rows<T, MODE>(*B, step, smem, targs);
}
template <typename T, int MODE>
__device__ __noinline__ void pass_cols(const BatchArgs<T>* B, int s, unsigned char* smem, TaskArgs<T>* targs)
{
    batched_cols<T, MODE>(*B, s, smem, targs);
}

constexpr int BATCH_THREADS = 512;

template <typename T>
__global__ void __launch_bounds__(BATCH_THREADS, 1) batched_kernel(BatchArgs<T> B)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int sflag;
    __shared__ TaskArgs<T> targs;
    pass_rows<T, ROW_FWD>(&B, -1, smem, &targs);
    if (!grid_sync(B, &sflag)) return;
    for (int s = 0; s < B.n_steps; s++) {
        pass_rows<T, ROW_RHS>(&B, 2 * s, smem, &targs);
        if (!grid_sync(B, &sflag)) return;
        pass_cols<T, COL_STAGE1>(&B, s, smem, &targs);
        if (!grid_sync(B, &sflag)) return;
        pass_rows<T, ROW_RHS>(&B, 2 * s + 1, smem, &targs);
        if (!grid_sync(B, &sflag)) return;
        pass_cols<T, COL_STAGE2>(&B, s, smem, &targs);
        if (!grid_sync(B, &sflag)) return;
    }
    pass_rows<T, ROW_INV>(&B, -1, smem, &targs);
    if (!grid_sync(B, &sflag)) return;
    // final diagnostics: CTA i reduces the rows of instance i (fixed order)
    for (int i = blockIdx.x; i < B.n_inst; i += gridDim.x) {
        const BatchInst<T>& I = B.inst[i];
        double* red = reinterpret_cast<double*>(smem);
        double s1 = 0, s2 = 0, mx = 0, nf = 0;
        for (int r = threadIdx.x; r < I.ny; r += blockDim.x) {
            s1 += __ldcg(I.diag_rows + 4 * r); s2 += __ldcg(I.diag_rows + 4 * r + 1);
            mx = fmax(mx, __ldcg(I.diag_rows + 4 * r + 2)); nf += __ldcg(I.diag_rows + 4 * r + 3);
        }
        double tmp[4];
        block_diag(red, s1, s2, mx, nf, tmp);
        if (threadIdx.x == 0) {
            I.diag_final[0] = tmp[0] * I.inv_count;
            I.diag_final[1] = tmp[1] * I.cell;
            I.diag_final[2] = tmp[2];
            I.diag_final[3] = tmp[3];
        }
    }
}

}  // namespace kzk
