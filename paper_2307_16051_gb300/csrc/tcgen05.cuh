// tcgen05.cuh — the pieces of the 5th-generation tensor-core path shared by
// the trailing-update kernels (gemm_tc.cu) and the persistent grouped LU
// (lu.cu): shared-memory operand descriptors for 128-byte-swizzled K-major
// slabs (written by TMA, or with plain stores at sw128_off), the kind::f16
// instruction descriptor, bounded mbarrier waits and the 2-D TMA load.
#pragma once
#include <cuda.h>
#include <cstdint>

namespace nl {

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor for a K-major operand slab written by TMA
// with 128-byte swizzle: 8-row x 128-byte swizzle atoms stacked every 1024 B.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t addr)
{
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFFu) >> 4);      // start address
    d |= (uint64_t)(16u >> 4) << 16;              // leading-dimension byte offset (unused for this layout)
    d |= (uint64_t)(1024u >> 4) << 32;            // stride-dimension byte offset: 8 rows x 128 B
    d |= (uint64_t)1 << 46;                       // descriptor version for tcgen05
    d |= (uint64_t)2 << 61;                       // 128-byte swizzle
    return d;
}

// Byte offset of 16-byte chunk `chunk` (0..7) of row `row` in a 128-byte-swizzled
// K-major slab (the layout TMA writes with 128-byte swizzle), for operands staged
// with plain shared-memory stores.
__device__ __forceinline__ uint32_t sw128_off(int row, int chunk)
{
    return (uint32_t)((row >> 3) * 1024 + (row & 7) * 128 + ((chunk ^ (row & 7)) << 4));
}

// Instruction descriptor: kind::f16, A = B = binary16, D = binary32, both
// operands K-major, M x N.
__host__ __device__ constexpr uint32_t tc_idesc_mn(int M, int N)
{
    return (1u << 4)                        // D format: f32
           | (0u << 7) | (0u << 10)         // A, B format: f16
           | (0u << 15) | (0u << 16)        // A, B K-major
           | ((uint32_t)(N >> 3) << 17)     // N / 8
           | ((uint32_t)(M >> 4) << 24);    // M / 16
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t phase, long long limit)
{
    long long t0 = clock64();
    uint32_t done = 0;
    while (true) {
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(bar), "r"(phase)
            : "memory");
        if (done) return true;
        if (clock64() - t0 > limit) return false;
    }
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            dst),
        "l"(map), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

}  // namespace nl
