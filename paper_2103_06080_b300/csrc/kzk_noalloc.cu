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
// is written earlier in the same call.  All calls share the one array, so
// calls whose GPU work overlaps (different streams, or different host
// threads) race on it; serialise them (one stream, or explicit ordering).
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

// Device address of g_noalloc_scratch per device, found once per device.
constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {nullptr};
bool g_attr_done[kMaxDevices] = {false};

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
kzk_status run(void* scratch, const kzk_grid* g, const kzk_coeffs* c, int batch, const void* u, void* b,
               double sigma, cudaStream_t st, int dev)
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
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_attr_done[dev]) {
            // lift the dynamic shared-memory limit of the three row kernels once
            // per device (an attribute, not an allocation)
            int optin = 0;
            if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
                return KZK_ERR_CUDA;
            for (cudaError_t e : {cudaFuncSetAttribute(row_kernel<double, ROW_FWD>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin),
                                  cudaFuncSetAttribute(row_kernel<double, ROW_RHS>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin),
                                  cudaFuncSetAttribute(row_kernel<double, ROW_INV>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin),
                                  cudaFuncSetAttribute(row_kernel<float, ROW_FWD>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin),
                                  cudaFuncSetAttribute(row_kernel<float, ROW_RHS>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin),
                                  cudaFuncSetAttribute(row_kernel<float, ROW_INV>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin)})
                if (e != cudaSuccess) return KZK_ERR_CUDA;
            g_attr_done[dev] = true;
        }
    }
    noalloc_twiddles<T><<<(nx + 255) / 256, 256, 0, st>>>(tw, nx);
    noalloc_staged_twiddles<T><<<(n + 255) / 256, 256, 0, st>>>(tws, log2nx - 1, row_ppt_of<T>());

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
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return set_error(KZK_ERR_CUDA, "kzk_rhs_noalloc: no usable current device");
    void* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_scratch_ptr[dev]) {
            // set-up, once per device, with that device current: the array's
            // name is only a host-side stand-in; its device address comes from
            // the runtime
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p)
                return set_error(KZK_ERR_CUDA, "kzk_rhs_noalloc: cudaGetSymbolAddress of the scratch array failed");
            g_scratch_ptr[dev] = p;
        }
        scratch = g_scratch_ptr[dev];
    }
    cudaStream_t st = (cudaStream_t)stream;
    const kzk_status s = grid->prec == KZK_FP64
                             ? run<double>(scratch, grid, coeffs, batch, u, b, sigma, st, dev)
                             : run<float>(scratch, grid, coeffs, batch, u, b, sigma, st, dev);
    return s == KZK_OK ? s : set_error(s, "kzk_rhs_noalloc: CUDA launch or attribute call failed");
}
