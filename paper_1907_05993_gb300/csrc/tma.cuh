// Tensor-memory-accelerator (TMA) tile loads and mbarrier waits for sm_103a.
//
// Host side: tensor maps are encoded through the driver entry point
// cuTensorMapEncodeTiled (looked up once through the runtime).  Device side:
// one thread arms an mbarrier with the expected byte count and issues the
// bulk tensor copy; every consumer waits on the barrier phase.  Waits are
// bounded: after kSpinLimit polls the wait gives up and reports failure, so
// a lost copy can never hang the GPU.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace hr_tma {

constexpr uint32_t kSpinLimit = 1u << 26;   // polls before a wait reports failure (~seconds)

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
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
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Plain arrival (no transaction bytes).
__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Bounded wait for phase `parity`; false if the limit ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity)
{
    for (uint32_t i = 0; i < kSpinLimit; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// 3-D tiled bulk tensor load of the box at (x, y, z) into shared memory.
__device__ __forceinline__ void load_3d(void *dst, const CUtensorMap *tm, uint64_t *bar, int x, int y, int z)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(tm)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

// 4-D tiled bulk tensor load of the box at (x, y, z, w) into shared memory.
__device__ __forceinline__ void load_4d(void *dst, const CUtensorMap *tm, uint64_t *bar, int x, int y, int z, int w)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(tm)), "r"(x), "r"(y), "r"(z), "r"(w), "r"(smem_u32(bar))
        : "memory");
}

// Plain (untiled) bulk copy of `bytes` (multiple of 16, both addresses 16-byte aligned).
__device__ __forceinline__ void load_bulk(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

}  // namespace hr_tma

// Host: encode a 3-D FP32 tiled tensor map (dims innermost first, strides in
// bytes of dims 1 and 2).  Returns 0 on success, nonzero if the driver
// refuses the shape (the caller then uses a path without TMA).
int hr_encode_tmap_3d(CUtensorMap *tm, const void *base, uint64_t d0, uint64_t d1, uint64_t d2, uint64_t s1,
                      uint64_t s2, uint32_t b0, uint32_t b1, uint32_t b2);

// Host: encode a 4-D BF16 tiled tensor map (dims innermost first, byte strides
// of dims 1..3, box b0..b3; out-of-range elements read as zero).  swizzle_bytes
// 0 (none), 32, 64 or 128: the box's inner extent must then equal it.  Same
// return convention as hr_encode_tmap_3d.
int hr_encode_tmap_bf16_4d(CUtensorMap *tm, const void *base, const uint64_t dims[4], const uint64_t strides[3],
                           const uint32_t box[4], int swizzle_bytes = 0);
