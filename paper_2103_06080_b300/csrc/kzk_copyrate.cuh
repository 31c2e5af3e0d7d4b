// kzk_copyrate.cuh -- measurement kernel behind kzk_tile_copy_rate: the rate
// at which the tensor memory accelerator copies the FP32 column-pair tiles
// (kzk_colpair.cuh) from HBM into shared memory, with nothing else running.
#pragma once
#include "kzk_colpipe.cuh"

namespace kzk {

// Copy-rate ceiling of the column-pair tiles (measurement, no arithmetic):
// CTA q takes the column pair q of two [ny][n] complex-FP32 arrays -- the
// tile rows of 16 bytes, ny rows at a pitch of 8 n bytes -- through the tensor
// memory accelerator in the same boxes as the column-pair kernels (strip), or
// the same number of bytes as contiguous runs by plain bulk copies
// (contiguous), waits for both, and leaves.  Shared memory is sized by the
// launch so that as many CTAs share an SM as in the column passes.
struct TileCopyArgs {
    CUtensorMap ma, mb;
    const unsigned char* a;
    const unsigned char* b;
    int by, nby, total, contiguous;
    unsigned tile_bytes;
    int* flag;
    long long timeout_ns;
};

__global__ void __launch_bounds__(256) tile_copy_kernel(const __grid_constant__ TileCopyArgs P)
{
    extern __shared__ __align__(128) unsigned char tcopy_smem[];
    unsigned char* smem = tcopy_smem;
    const int q = blockIdx.x;
    if (q >= P.total) return;
    if (smem_addr(smem) & 127u) {
        if (threadIdx.x == 0) atomicOr(P.flag, FLAG_BAD_LAUNCH);
        return;
    }
    unsigned long long* bar = reinterpret_cast<unsigned long long*>(smem);
    unsigned char* ta = smem + 128;
    unsigned char* tb = ta + P.tile_bytes;
    const unsigned box = P.tile_bytes / P.nby;
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        mbar_fence_init();
        mbar_expect(bar, 2 * P.tile_bytes);
        for (int k = 0; k < P.nby; k++) {
            if (P.contiguous) {
                const size_t off = (size_t)q * P.tile_bytes + (size_t)k * box;
                bulk_load(ta + k * box, P.a + off, box, bar);
                bulk_load(tb + k * box, P.b + off, box, bar);
            } else {
                tma_load_3d(ta + k * box, &P.ma, 4 * q, k * P.by, 0, bar);
                tma_load_3d(tb + k * box, &P.mb, 4 * q, k * P.by, 0, bar);
            }
        }
    }
    __syncthreads();   // barrier initialisation visible to every waiting thread
    colp_wait(smem, 0, 0u, P.timeout_ns, P.flag);
}

}  // namespace kzk
