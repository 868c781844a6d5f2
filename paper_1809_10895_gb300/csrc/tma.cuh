// tma.cuh -- tensor-memory-accelerator (TMA) plane staging for the stencil
// kernels: 3-D tensor maps of the FP32 solver arrays, bulk tensor copies into
// shared memory completed on mbarriers, and bounded waits.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace rf {

// Box of one staged plane: 136 x 10 cells around a 128 x 8 tile.  The box
// starts 4 cells before the tile in x so that its x coordinate is a multiple
// of 4 floats (16 bytes), as every tensor copy requires; the -x halo cell is
// box column 3, the tile's first cell column 4.  Rows: y from j0 - 1.
constexpr int TMA_TX = 128;
constexpr int TMA_BX = TMA_TX + 8, TMA_BY = 10, TMA_X0 = 4;
constexpr int TMA_BOX_BYTES = TMA_BX * TMA_BY * 4;       // 5440
constexpr int TMA_SLOT_BYTES = (TMA_BOX_BYTES + 127) / 128 * 128;
// Box of an array read at the tile's own cells only (cb): 128 x 8, no halo.
constexpr int TMA_OWN_BY = 8;
constexpr int TMA_OWN_BYTES = TMA_TX * TMA_OWN_BY * 4;   // 4096

// Tensor maps of the FP32 inner-solve arrays (one 3-D map per array, dims
// nx, ny, nz), with the device pointers they describe.
struct TmaMaps32 {
    CUtensorMap z, p0, p1, K, cb;
    const float *z_ptr, *p_ptr[2], *K_ptr, *cb_ptr;
};

#ifdef __CUDACC__
__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_init_fence()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Non-blocking test of phase `parity` of an mbarrier.
__device__ __forceinline__ bool mbar_test_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Order this thread's generic-proxy shared-memory writes before later
// async-proxy (tensor copy) accesses of the same memory.
__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// try_wait that may suspend the thread for up to about hint_ns nanoseconds
// (it resumes as soon as the phase completes).
__device__ __forceinline__ bool mbar_try_wait_sleep(uint64_t *bar, uint32_t parity, uint32_t hint_ns)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity), "r"(hint_ns)
        : "memory");
    return ok != 0;
}

// Wait for phase `parity` of an mbarrier, at most max_tries suspending polls
// of about a microsecond each; false on timeout.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, int max_tries)
{
    for (int t = 0; t < max_tries; t++)
        if (mbar_try_wait_sleep(bar, parity, 1000u)) return true;
    return false;
}

// Bulk tensor copy of the box at (x, y, z) of a 3-D map into shared memory,
// completing transaction bytes on bar.  x * 4 bytes must be a multiple of 16.
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, uint64_t *bar, int x, int y, int z)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], [%2];"
        ::"r"(smem_addr(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_addr(bar)), "r"(x), "r"(y), "r"(z)
        : "memory");
}
#endif

// Host: encode the maps for arrays of nx * ny * nz floats (nx a multiple of
// 4, pointers 16-byte aligned).  Returns false when the driver entry point is
// unavailable or an encoding fails (the caller then uses the untiled path).
bool make_tma_maps32(int nx, int ny, int nz, const float *z, const float *p0, const float *p1, const float *K,
                     const float *cb, TmaMaps32 *out);

}  // namespace rf
