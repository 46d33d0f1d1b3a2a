// Tensor Memory Accelerator (TMA) and mbarrier helpers for sm_103a (private).
//
// Tiles move between global and shared memory with cp.async.bulk.tensor
// (loads complete on an mbarrier, stores drain through a bulk group), issued by
// one thread per block; the rest of the block only waits. Every wait on an
// mbarrier is bounded by the global timer: on time-out the block sets a bit in
// the plan's device status word and leaves without touching the tile.
#pragma once

#include <cuda.h>

#include "pd_common.cuh"

namespace pd {

constexpr unsigned long long kWaitLimitNs = 2000000000ull;  // 2 s
constexpr int kErrTmaTimeout = 1;

__device__ __forceinline__ unsigned smem_u32(const void *p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(unsigned long long *mbar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long *mbar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(mbar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long *mbar, unsigned phase)
{
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(mbar)), "r"(phase)
        : "memory");
    return ok != 0;
}

// Bounded wait for phase `phase` of the barrier. Returns false on time-out
// (after recording it in *err).
__device__ __forceinline__ bool mbar_wait(unsigned long long *mbar, unsigned phase, int *err)
{
    if (mbar_try_wait(mbar, phase)) return true;
    const unsigned long long t0 = global_ns();
    while (!mbar_try_wait(mbar, phase)) {
        if (global_ns() - t0 > kWaitLimitNs) {
            if (err) atomicOr(err, kErrTmaTimeout);
            return false;
        }
    }
    return true;
}

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *m, int x, int y, int z,
                                            unsigned long long *mbar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(smem_u32(dst)), "l"(m), "r"(x), "r"(y), "r"(z), "r"(smem_u32(mbar))
        : "memory");
}

__device__ __forceinline__ void tma_store_3d(const CUtensorMap *m, int x, int y, int z, const void *src)
{
    asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%1, %2, %3}], [%4];" ::"l"(m),
                 "r"(x), "r"(y), "r"(z), "r"(smem_u32(src))
                 : "memory");
}

// 1D bulk copy global -> shared (16-byte aligned addresses, size multiple of 16)
__device__ __forceinline__ void bulk_load(void *dst, const void *src, unsigned bytes, unsigned long long *mbar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(mbar))
                 : "memory");
}

// Bulk prefetch of [src, src + bytes) into L2 (16-byte aligned address, size a
// multiple of 16; no shared memory, no completion to wait for)
__device__ __forceinline__ void bulk_prefetch_l2(const void *src, unsigned bytes)
{
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

// 1D bulk copy shared -> global
__device__ __forceinline__ void bulk_store(void *dst, const void *src, unsigned bytes)
{
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_u32(src)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
// Programmatic dependent launch: wait for the preceding grid of the stream to
// complete (its memory visible); a no-op when the grid was launched without
// the programmatic-serialization attribute. The trigger lets the next grid's
// blocks start their prologue once every block of this grid has issued it.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
// make this thread's generic-proxy shared-memory writes visible to the async proxy
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Host: encode a 3D tiled tensor map (dims/box in elements, dim 0 innermost;
// strides in bytes for dims 1 and 2).
pd_status encode_tmap_3d(CUtensorMap *m, void *base, bool fp64, const unsigned long long dims[3],
                         const unsigned long long strides[2], const unsigned box[3]);

}  // namespace pd
