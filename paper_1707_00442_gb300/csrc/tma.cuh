// tma.cuh -- Tensor Memory Accelerator loads (cp.async.bulk.tensor) with mbarrier
// completion, written as inline PTX, plus the host-side tensor-map encoder.
//
// Every wait is bounded: if a barrier phase does not complete within the limit the
// waiting thread records it in the library's device error word (reported by
// shw_sync_status as SHW_ETIMEOUT) and the caller abandons its work.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace shw {

constexpr unsigned kErrWaitTimeout = 1u;
constexpr unsigned kErrTmaAlign = 2u;
constexpr int kWaitPolls = 1 << 20;       // bounded waits: polls of at most ...
constexpr uint32_t kWaitSleepNs = 1000;  // ... this many nanoseconds each, about a second in all
constexpr int kFaultWaitPolls = 1000;    // the bound under SHW_DEBUG_FAULT_TIMEOUT: about a millisecond

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// make barrier initialisation visible to the async (TMA) proxy
__device__ __forceinline__ void fence_barrier_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// order this thread's generic-proxy shared-memory writes before later async-proxy
// (tensor copy) accesses of the same bytes
__device__ __forceinline__ void fence_proxy_async()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// plain arrival (release semantics at CTA scope): a consumer hands a stage back
__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// One 3-D box of a tensor map into shared memory; completion is signalled on `bar`.
// The innermost coordinate x times the element size must be a multiple of 16 bytes.
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int x, int y, int z, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

// A tensor copy's shared-memory destination must start on 128 bytes: refuse (and
// report) a copy that would not, instead of issuing it.
__device__ __forceinline__ bool tma_dst_ok(const void *dst, unsigned *err)
{
    if ((smem_u32(dst) & 127u) == 0u) return true;
    if (err) atomicOr(err, kErrTmaAlign);
    return false;
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// As mbar_try_wait, but the thread may sleep up to `ns` nanoseconds waiting for the
// phase (it wakes as soon as the phase completes): polling without spinning.
__device__ __forceinline__ bool mbar_try_wait_sleep(uint64_t *bar, uint32_t parity, uint32_t ns)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(ns)
        : "memory");
    return ok != 0;
}

// Wait for phase `parity` of `bar`, the thread suspended between polls (so waiting warps
// leave the issue slots to others); false (and the error word set) after `polls` polls.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, unsigned *err, int polls = kWaitPolls)
{
    for (int i = 0; i < polls; ++i)
        if (mbar_try_wait_sleep(bar, parity, kWaitSleepNs)) return true;
    if (err) atomicOr(err, kErrWaitTimeout);
    return false;
}

// host: the library's device error word on the current device (nullptr if unavailable)
unsigned *device_error_word();

// host: encode a 3-D float32 tile map over a [nz][ny][nx] array with box {bx, by, 1};
// out-of-bounds elements of a box read as zero.  Returns false if the driver refuses.
bool encode_tmap_3d_f32(CUtensorMap *map, const float *base, int nx, int ny, int nz, int bx, int by);

// host: a 3-D tile map over [nz][ny][nx] elements of elem_bytes (2, 4 or 8; copied as raw
// bits) with box {bx, by, bz}; out-of-bounds elements of a box read as zero.  nx * elem_bytes
// must be a multiple of 16 and base 16-byte aligned.  False if the driver refuses.
bool encode_tmap_3d(CUtensorMap *map, const void *base, int elem_bytes, int nx, int ny, int nz, int bx, int by,
                    int bz);

}  // namespace shw
