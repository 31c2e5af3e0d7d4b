// kzk_noalloc.cu -- kzk_rhs_noalloc: the nonlinear term b(sigma, u) without
// any device allocation.
//
// Some callers cannot let this library call cudaMalloc: a host application
// that hands all device memory to its own pool allocator up front (a
// cudaMalloc from a library would then fail, or bypass the pool's
// accounting), or code on a latency-critical path where cudaMalloc's
// implicit device-wide synchronisation is not acceptable.  A plan
// (kzk_plan_create) allocates its tables and workspace, so such callers get
// this entry point instead: it needs no plan, the caller passes the input u
// and the output b, and the two spectral intermediates plus the twiddle table
// live in the file-scope array below, which every GPU that loads the library
// holds until the process exits.
//
// Scratch contents are not cleared between calls: every element a call reads
// is written earlier in the same call, except the twiddle tables, which a call
// leaves in place for the next call with the same nx and precision on the
// same context.  All calls share the one array, so calls whose GPU work
// overlaps (different streams, or different host threads) race on it;
// serialise them (one stream, or explicit ordering).
//
// Per-device set-up (the array's device address, the kernels' shared-memory
// limit, which twiddle tables the array holds) is cached under the id of the
// device's current CUDA context: if that context is destroyed and re-created
// (cudaDeviceReset), the module is loaded afresh, and the next call sees a new
// id and repeats the set-up.
#include <cuda.h>
#include <mutex>

#include "../../include/kzk.h"
#include "kzk_kernels.cuh"

using namespace kzk;

namespace {

// Largest problem: batch * nx * ny <= KZK_NOALLOC_MAX_POINTS, nx <= 8192.
constexpr long long kMaxPoints = KZK_NOALLOC_MAX_POINTS;
constexpr int kMaxNx = 8192;
// two packed spectral arrays of kMaxPoints FP64 points (8 bytes per point
// each) and one FP64 twiddle table of kMaxNx entries
constexpr size_t kSpecBytes = (size_t)kMaxPoints * 8;
constexpr size_t kScratchBytes = 2 * kSpecBytes + (size_t)kMaxNx * 16 + (size_t)(kMaxNx / 2) * 16;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Set-up per device, valid for the context whose id it records.
constexpr int kMaxDevices = 64;
struct DevSetup {
    unsigned long long ctx_id;  // cuCtxGetId of the context the entries below belong to (0: none)
    void* scratch;              // device address of g_noalloc_scratch in that context
    int tw_nx;                  // nx and precision of the twiddle tables in the array (0: none)
    int tw_prec;
};
std::mutex g_mu;
DevSetup g_dev[kMaxDevices] = {};

// cuCtxGetCurrent / cuCtxGetId from the driver, looked up once through the
// runtime (no link-time dependency on libcuda)
typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);
template <typename F>
F driver_fn(const char* name)
{
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion(name, &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
        return nullptr;
    return reinterpret_cast<F>(f);
}

// id of the calling thread's current context; with none current, device
// dev's primary context is made current first (cudaSetDevice, which creates
// it if needed); 0 on failure
unsigned long long current_ctx_id(int dev)
{
    static const CtxGetCurrentFn get_cur = driver_fn<CtxGetCurrentFn>("cuCtxGetCurrent");
    static const CtxGetIdFn get_id = driver_fn<CtxGetIdFn>("cuCtxGetId");
    if (!get_cur || !get_id) return 0;
    CUcontext c = nullptr;
    if (get_cur(&c) != CUDA_SUCCESS) return 0;
    if (!c && (cudaSetDevice(dev) != cudaSuccess || get_cur(&c) != CUDA_SUCCESS || !c)) return 0;
    unsigned long long id = 0;
    if (get_id(c, &id) != CUDA_SUCCESS) return 0;
    return id;
}

template <typename T>
__global__ void noalloc_twiddles(cx<T>* tw, int nx)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nx) return;
    double s, c;
    sincospi(2.0 * (double)k / (double)nx, &s, &c);   // exp(-2 pi i k / nx)
    tw[k] = mk<T>((T)c, (T)(-s));
}

// staged twiddles of the row FFT (length 2^log2n, ppt points per thread),
// one thread per table entry
template <typename T>
__global__ void noalloc_staged_twiddles(cx<T>* tws, int log2n, int ppt)
{
    int lr[32], lns[32];
    const int P = fft_schedule(log2n, ppt, lr, lns);
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    for (int p = 0; p < P; p++) {
        if (lns[p] == 0) continue;
        const int Ns = 1 << lns[p], R = 1 << lr[p], cnt = (R - 1) * Ns;
        if (e < cnt) {
            const int r = 1 + e / Ns, k = e % Ns;
            double s, c;
            sincospi(2.0 * (double)(r * k) / (double)(Ns * R), &s, &c);
            tws[blockIdx.x * blockDim.x + threadIdx.x] = mk<T>((T)c, (T)(-s));
            return;
        }
        e -= cnt;
    }
}

double horner4(const double* c, double s) { return ((c[3] * s + c[2]) * s + c[1]) * s + c[0]; }

template <typename T>
kzk_status run(void* scratch, bool tables_valid, const kzk_grid* g, const kzk_coeffs* c, int batch, const void* u,
               void* b, double sigma, cudaStream_t st)
{
    const int nx = g->nx, ny = g->ny, n = nx / 2;
    const int log2nx = ilog2((unsigned)nx);
    unsigned char* base = (unsigned char*)scratch;
    cx<T>* V = (cx<T>*)base;
    cx<T>* Bh = (cx<T>*)(base + kSpecBytes);
    cx<T>* tw = (cx<T>*)(base + 2 * kSpecBytes);
    cx<T>* tws = (cx<T>*)(base + 2 * kSpecBytes + (size_t)kMaxNx * 16);
    const int thr = row_threads<T>(nx);
    const size_t smem = row_smem_bytes<T>(nx);
    if (!tables_valid) {
        noalloc_twiddles<T><<<(nx + 255) / 256, 256, 0, st>>>(tw, nx);
        noalloc_staged_twiddles<T><<<(n + 255) / 256, 256, 0, st>>>(tws, log2nx - 1, row_ppt_of<T>());
    }

    RowArgs<T> a{};
    a.tw = tw;
    a.tws = tws;
    a.diag_rows = nullptr;
    a.log2nx = log2nx;
    a.ny = ny;
    a.inst_stride = (long long)ny * n;
    const double Bs = c->has_profile ? c->B * horner4(c->B_prof, sigma) : c->B;
    const double dA = c->has_profile ? c->A * horner4(c->A_prof, sigma) - c->A : 0.0;
    a.wc.B = (T)Bs;
    a.wc.alpha = (T)(Bs * c->lf_umax);
    a.wc.eps = (T)(c->weno_eps > 0 ? c->weno_eps : 1e-6);
    a.wc.inv_dtau = (T)(nx / (g->tau_max - g->tau_min));
    a.cA = (T)(nx * dA);
    a.kscale = (T)(2.0 * M_PI / (g->tau_max - g->tau_min));
    const dim3 grid(ny, batch);
    // physical u -> packed spectrum / nx
    a.in = (const cx<T>*)u;
    a.out = V;
    a.out_scale = (T)(1.0 / nx);
    row_kernel<T, ROW_FWD><<<grid, thr, smem, st>>>(a);
    // WENO5 flux derivative and absorption deviation, spectral
    a.in = V;
    a.out = Bh;
    a.out_scale = (T)1;
    row_kernel<T, ROW_RHS><<<grid, thr, smem, st>>>(a);
    // back to physical space (the spectrum carries a factor nx)
    a.in = Bh;
    a.out = (cx<T>*)b;
    a.out_scale = (T)(1.0 / nx);
    row_kernel<T, ROW_INV><<<grid, thr, smem, st>>>(a);
    return cudaGetLastError() == cudaSuccess ? KZK_OK : KZK_ERR_CUDA;
}

}  // namespace

namespace kzk_internal {
kzk_status set_error(kzk_status s, const char* msg);   // kzk_api.cu: feeds kzk_last_error()
}

extern "C" kzk_status kzk_rhs_noalloc(const kzk_grid* grid, const kzk_coeffs* coeffs, int32_t batch,
                                      const void* u, void* b, double sigma, void* stream)
{
    using kzk_internal::set_error;
    if (!grid || !coeffs || !u || !b) return set_error(KZK_ERR_ARG, "kzk_rhs_noalloc: NULL argument");
    if (u == b) return set_error(KZK_ERR_ARG, "kzk_rhs_noalloc: b may not alias u");
    if (batch < 1) return set_error(KZK_ERR_ARG, "kzk_rhs_noalloc: batch must be >= 1");
    if (grid->prec != KZK_FP64 && grid->prec != KZK_FP32)
        return set_error(KZK_ERR_ARG, "kzk_rhs_noalloc: bad precision");
    const long long nx = grid->nx, ny = grid->ny;
    if (nx < 8 || nx > kMaxNx || (nx & (nx - 1)) || ny < 1 || (ny & (ny - 1)))
        return set_error(KZK_ERR_SIZE, "kzk_rhs_noalloc: nx must be a power of two in [8, 8192], ny a power of two");
    if ((long long)batch * nx * ny > kMaxPoints)
        return set_error(KZK_ERR_SIZE, "kzk_rhs_noalloc: batch * nx * ny exceeds KZK_NOALLOC_MAX_POINTS (262144)");
    if (!(grid->tau_max > grid->tau_min) || !(coeffs->B > 0) || !(coeffs->lf_umax > 0) || !(coeffs->A >= 0))
        return set_error(KZK_ERR_ARG, "kzk_rhs_noalloc: need tau_max > tau_min, B > 0, A >= 0, lf_umax > 0");
    // an error left pending by the caller's earlier work would be read back
    // as a failure of this call's launches: refuse to run, and leave it pending
    const cudaError_t pending = cudaPeekAtLastError();
    if (pending != cudaSuccess)
        return set_error(KZK_ERR_CUDA, "kzk_rhs_noalloc: a CUDA error from earlier work was pending before the call "
                                       "(left pending, nothing launched)");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return set_error(KZK_ERR_CUDA, "kzk_rhs_noalloc: no usable current device");
    const unsigned long long ctx = current_ctx_id(dev);
    if (!ctx) return set_error(KZK_ERR_CUDA, "kzk_rhs_noalloc: could not identify the current CUDA context");
    const int prec = grid->prec == KZK_FP64 ? 8 : 4;
    void* scratch = nullptr;
    bool tables_valid = false;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        DevSetup& d = g_dev[dev];
        if (d.ctx_id != ctx) {
            // set-up, once per device and context, with that device current:
            // the array's name is only a host-side stand-in; its device address
            // comes from the runtime
            d = DevSetup{};
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p)
                return set_error(KZK_ERR_CUDA, "kzk_rhs_noalloc: cudaGetSymbolAddress of the scratch array failed");
            // lift the dynamic shared-memory limit of the row kernels (an
            // attribute, not an allocation)
            int optin = 0;
            if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
                return set_error(KZK_ERR_CUDA, "kzk_rhs_noalloc: device attribute query failed");
            for (cudaError_t e : {cudaFuncSetAttribute(row_kernel<double, ROW_FWD>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin),
                                  cudaFuncSetAttribute(row_kernel<double, ROW_RHS>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin),
                                  cudaFuncSetAttribute(row_kernel<double, ROW_INV>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin),
                                  cudaFuncSetAttribute(row_kernel<float, ROW_FWD>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin),
                                  cudaFuncSetAttribute(row_kernel<float, ROW_RHS>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin),
                                  cudaFuncSetAttribute(row_kernel<float, ROW_INV>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin)})
                if (e != cudaSuccess)
                    return set_error(KZK_ERR_CUDA, "kzk_rhs_noalloc: setting the kernels' shared-memory limit failed");
            d.scratch = p;
            d.ctx_id = ctx;
        }
        scratch = d.scratch;
        tables_valid = d.tw_nx == grid->nx && d.tw_prec == prec;
        // the tables this call leaves in the array (its launches write them
        // first when they are not there)
        d.tw_nx = grid->nx;
        d.tw_prec = prec;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const kzk_status s = grid->prec == KZK_FP64
                             ? run<double>(scratch, tables_valid, grid, coeffs, batch, u, b, sigma, st)
                             : run<float>(scratch, tables_valid, grid, coeffs, batch, u, b, sigma, st);
    return s == KZK_OK ? s : set_error(s, "kzk_rhs_noalloc: CUDA launch or attribute call failed");
}
