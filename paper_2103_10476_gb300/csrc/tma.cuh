// tma.cuh -- bulk asynchronous copies (cp.async.bulk, the Tensor Memory Accelerator's
// non-tensor form) from global into shared memory, completed through an mbarrier.
//
// Rules kept by every caller: source and destination 16-byte aligned, size a multiple of 16;
// the source arrays carry at least 16 bytes of padding after their last element, so a range
// widened to 16-byte boundaries stays inside the allocation.  Waits are bounded: a wait that
// runs out sets the caller's error flag, waits (bounded) once more for the copies in flight,
// and reports failure so the block can return without using the tile.
#pragma once

#include <stdint.h>

namespace amgk {

constexpr int kWaitSpins = 1 << 22;

// Shared-memory tile of a CSR row range staged by two bulk copies: `cap` values of type T
// (plus one 16-byte widening on each side) and cap + 8 column indices.
template <typename T>
__host__ __device__ constexpr int tile_values_bytes(int cap)
{
    return ((cap + 2 * (16 / (int)sizeof(T))) * (int)sizeof(T) + 127) / 128 * 128;
}
template <typename T>
__host__ __device__ constexpr int tile_bytes(int cap)
{
    return cap > 0 ? tile_values_bytes<T>(cap) + (cap + 8) * 4 : 0;
}

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_g2s(void *dst_smem, const void *src_gmem, unsigned bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_u32(dst_smem)), "l"(src_gmem), "r"(bytes), "r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity)
{
    unsigned done;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(done) : "r"(smem_u32(bar)), "r"(parity) : "memory");
    return done != 0;
}

// bounded wait on phase `parity`; false (and *err incremented once per block) on timeout
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, unsigned parity, int *err)
{
    for (int it = 0; it < kWaitSpins; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    if (threadIdx.x == 0 && err) atomicAdd(err, 1);
    for (int it = 0; it < kWaitSpins; ++it)
        if (mbar_try_wait(bar, parity)) break;
    return false;
}

}  // namespace amgk
