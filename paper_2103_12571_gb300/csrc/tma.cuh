// Tensor-memory-accelerator (TMA) tile loads from this GPU's memory into
// shared memory, completed on an mbarrier (sm_90+ PTX: cp.async.bulk.tensor).
//
// Rules kept by the callers: the tensor map lives in kernel parameter space
// (__grid_constant__) and describes 16-byte aligned global memory with row
// strides that are multiples of 16 bytes; the innermost box coordinate times
// the element size is a multiple of 16 bytes; the shared destination is
// 128-byte aligned; the expected byte count (whole boxes, out-of-range rows
// included, which the copy engine fills with zeros) is registered on the
// barrier before its copies complete; every wait is bounded.
#pragma once
#include <cuda.h>
#include <stdint.h>

namespace ac {

__device__ __forceinline__ unsigned smem_addr(const void* p) {
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

// Orders this thread's earlier shared-memory accesses (and, after a block
// barrier, those of the whole CTA) before later copy-engine accesses.
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// One arrival that also announces `bytes` of copies completing this phase.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

// 2D tile (box of the tensor map) at element coordinates (x inner, y outer)
// into shared memory at dst, completion counted on bar.
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Waits for phase `parity` of bar, at most about a second (2^24 polls with
// a short sleep after the first few).  Returns false on timeout.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity) {
    for (int it = 0; it < (1 << 24); ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if (it > 32) __nanosleep(64);
    }
    return false;
}

}  // namespace ac
