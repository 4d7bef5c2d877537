// tma.cuh -- tensor-memory-accelerator loads and bounded shared-memory
// mbarrier waits (inline PTX for sm_100 and later), shared by the push kernel
// (a supercell's E/B tile per work item) and the fused field update (E planes
// of a z-marching tile).
//
// A tensor load names a CUtensorMap in global memory (encoded on the host
// over this GPU's own field arrays) and completes on an mbarrier with a byte
// count.  Every wait is bounded: after kWaitCycles SM clocks it gives up and
// the caller reports ST_TIMEOUT instead of spinning on.
#pragma once

#include "pic_internal.cuh"

namespace pic {

constexpr long long kWaitCycles = 4000000000LL;  // about 2 s at 2 GHz

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* mb, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(mb)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory"); }

// shared memory read by generic loads is about to be written by the async proxy
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

__device__ __forceinline__ void mbar_expect_tx(unsigned long long* mb, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(mb)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long* mb, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n"
        " .reg .pred p;\n"
        " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n"
        "}\n"
        : "=r"(ok)
        : "r"(smem_u32(mb)), "r"(parity)
        : "memory");
    return ok != 0;
}

// the phase of parity `parity` completed (false: gave up after kWaitCycles)
__device__ __forceinline__ bool mbar_wait(unsigned long long* mb, unsigned parity)
{
    const long long t0 = clock64();
    while (!mbar_try_wait(mb, parity))
        if (clock64() - t0 > kWaitCycles)
            return false;
    return true;
}

// the tile box at padded coordinates (x, y, z) of the map's field, all three
// components, into dst ([3][tz][ty][px] floats)
__device__ __forceinline__ void tma_load_tile(float* dst, const CUtensorMap* map, int x, int y, int z,
                                              unsigned long long* mb)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
        "%5}], [%6];\n" ::"r"(smem_u32(dst)),
        "l"(map), "r"(x), "r"(y), "r"(z), "r"(0), "r"(smem_u32(mb))
        : "memory");
}

__device__ __forceinline__ void tma_prefetch_tile(const CUtensorMap* map, int x, int y, int z)
{
    asm volatile("cp.async.bulk.prefetch.tensor.4d.L2.global.tile [%0, {%1, %2, %3, %4}];\n" ::"l"(map), "r"(x),
                 "r"(y), "r"(z), "r"(0)
                 : "memory");
}

}  // namespace pic
