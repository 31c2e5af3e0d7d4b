// kzk_common.cuh -- complex arithmetic and small helpers shared by the kernels.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace kzk {

template <typename T> struct cplx_of;
template <> struct cplx_of<float> { using type = float2; };
template <> struct cplx_of<double> { using type = double2; };
template <typename T> using cx = typename cplx_of<T>::type;

template <typename T> __host__ __device__ __forceinline__ cx<T> mk(T r, T i) { cx<T> c; c.x = r; c.y = i; return c; }
template <typename T> __device__ __forceinline__ cx<T> add(cx<T> a, cx<T> b) { return mk<T>(a.x + b.x, a.y + b.y); }
template <typename T> __device__ __forceinline__ cx<T> sub(cx<T> a, cx<T> b) { return mk<T>(a.x - b.x, a.y - b.y); }
template <typename T> __device__ __forceinline__ cx<T> conj(cx<T> a) { return mk<T>(a.x, -a.y); }
template <typename T> __device__ __forceinline__ cx<T> scale(cx<T> a, T s) { return mk<T>(a.x * s, a.y * s); }
template <typename T> __device__ __forceinline__ cx<T> mul(cx<T> a, cx<T> b)
{
    return mk<T>(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
// a * conj(b)
template <typename T> __device__ __forceinline__ cx<T> mulc(cx<T> a, cx<T> b)
{
    return mk<T>(fma(a.x, b.x, a.y * b.y), fma(a.y, b.x, -a.x * b.y));
}
// a * (s i) with s = +1 / -1 (exact)
template <typename T, int S> __device__ __forceinline__ cx<T> mul_si(cx<T> a)
{
    return S > 0 ? mk<T>(-a.y, a.x) : mk<T>(a.y, -a.x);
}
// acc + a * b
template <typename T> __device__ __forceinline__ cx<T> fma_c(cx<T> a, cx<T> b, cx<T> acc)
{
    return mk<T>(fma(a.x, b.x, fma(-a.y, b.y, acc.x)), fma(a.x, b.y, fma(a.y, b.x, acc.y)));
}

// Compensated state update: the value hi + lo plus an increment d, returned as
// a new pair (s_hi, s_lo) with s_hi + s_lo = hi + fl(lo + d) exactly (Knuth's
// TwoSum on each component; no reassociation, no FMA involved).
template <typename T>
__device__ __forceinline__ void comp_add(cx<T> hi, cx<T> lo, cx<T> d, cx<T>& s_hi, cx<T>& s_lo)
{
    auto two_sum = [](T h, T t, T& s, T& e) {
        s = h + t;
        const T bb = s - h;
        e = (h - (s - bb)) + (t - bb);
    };
    T sx, ex, sy, ey;
    two_sum(hi.x, lo.x + d.x, sx, ex);
    two_sum(hi.y, lo.y + d.y, sy, ey);
    s_hi = mk<T>(sx, sy);
    s_lo = mk<T>(ex, ey);
}

// Storage of the lo part of a compensated state: for FP32 one bf16 pair per
// complex value (8 significant bits below the 24 of the hi part: the pair
// carries about 33 bits, 2^-33 relative per update), else the value type.
template <typename T> struct lo_of { using type = cx<T>; };
template <> struct lo_of<float> { using type = __nv_bfloat162; };
template <typename T> using lo_t = typename lo_of<T>::type;

template <typename T>
__device__ __forceinline__ cx<T> lo_load(const lo_t<T>* p)
{
    if constexpr (sizeof(lo_t<T>) == 4) {
        const unsigned w = __ldcg(reinterpret_cast<const unsigned*>(p));
        __nv_bfloat162 b;
        memcpy(&b, &w, 4);
        return __bfloat1622float2(b);
    } else {
        return __ldcg(p);
    }
}
template <typename T>
__device__ __forceinline__ void lo_store(lo_t<T>* p, cx<T> v)
{
    if constexpr (sizeof(lo_t<T>) == 4) *p = __float22bfloat162_rn(v);
    else *p = v;
}

__host__ __device__ __forceinline__ int ilog2(unsigned v)
{
    int r = 0;
    while ((1u << r) < v) ++r;
    return r;
}

// Device clock in nanoseconds (bounds every wait in the kernels).
__device__ __forceinline__ long long global_ns()
{
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Launch-time error flags (bit set in plan->flags by device code).
enum : int { FLAG_TIMEOUT = 1, FLAG_BAD_LAUNCH = 2 };

}  // namespace kzk
