// pf_tma.cuh -- Tensor Memory Accelerator copies (cp.async.bulk.tensor) and
// mbarrier waits used by the y and z passes.  Every wait is bounded: after a
// limited number of polls the kernel records an error code in *err and gives
// up, so a lost transfer ends the launch instead of hanging the GPU.
//
// Error block: err[0] is the error word; the 64-bit value at err + 2 (byte
// offset 8) is the poll limit of the first wait on a copy (kSpinLimit unless
// the handle was created with another one).  The drain wait after giving up
// always uses kSpinLimit, so no bulk copy is still writing a CTA's shared
// memory when the CTA exits.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "pf_internal.h"

namespace pfk {

constexpr int kErrTmaLoad = 1;
constexpr int kErrTmaDrain = 2;
constexpr int kErrCheck = kErrCheckBit;  // a check of the PF_CHECK build failed

// Checks of the PF_CHECK build (compiled out otherwise): a kernel verifies,
// before it touches shared memory, that the layout it derives from its
// arguments fits the launch's dynamic shared memory and that its tile
// coordinates lie inside the field; on failure it records kErrCheck in the
// error word and every thread of the CTA leaves before any barrier or copy.
#ifdef PF_CHECK
__device__ __forceinline__ uint32_t dyn_smem_bytes() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%dynamic_smem_size;" : "=r"(r));
    return r;
}
// true when the CTA may go on (cond holds); the same value in every thread
__device__ __forceinline__ bool pf_check(bool cond, int* err) {
    if (!cond && threadIdx.x == 0 && err) atomicOr(err, kErrCheck);
    return cond;
}
// bytes from the dynamic shared-memory base up to `end` (a pointer into it)
__device__ __forceinline__ bool pf_check_smem(const void* base, const void* end, int* err) {
    const size_t used = (size_t)((const char*)end - (const char*)base);
    return pf_check(used <= dyn_smem_bytes(), err);
}
#else
__device__ __forceinline__ bool pf_check(bool, int*) { return true; }
__device__ __forceinline__ bool pf_check_smem(const void*, const void*, int*) { return true; }
#endif

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// one arrival that also announces `bytes` of incoming transactions
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
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

// Wait for phase `parity` of the barrier; false (and *err set) after `limit`
// polls.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int* err, int code,
                                          long long limit = kSpinLimit) {
    for (long long it = 0; it < limit; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    if (err) atomicExch(err, code);
    return false;
}

// Poll limit of a first wait: the value the error block carries.
__device__ __forceinline__ long long first_wait_limit(const int* err) {
    if (!err) return kSpinLimit;
    const long long v = *reinterpret_cast<const volatile long long*>(err + 2);
    return v >= 0 ? v : kSpinLimit;
}

// Non-blocking test of phase `parity` (acquire when it returns true).
__device__ __forceinline__ bool mbar_test_wait(uint64_t* bar, uint32_t parity) {
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

// Thread 0 polls phase `parity` while the other threads sleep in the CTA
// barrier (a barrier wait takes no issue slots, a poll loop does); the
// outcome is agreed across the CTA so that all threads continue or all give
// up together, and each thread then observes the completed phase itself.  On
// giving up, thread 0 waits once more (bounded) for the copies still in
// flight on `bar` and, if given, on `bar2` (phase parity2) before the caller
// leaves.
__device__ __forceinline__ bool cta_wait(uint64_t* bar, uint32_t parity, int* err, uint64_t* bar2 = nullptr,
                                         uint32_t parity2 = 0) {
    bool ok = true;
    if (threadIdx.x == 0) ok = mbar_wait(bar, parity, err, kErrTmaLoad, first_wait_limit(err));
    if (!__syncthreads_or(!ok)) {
        mbar_test_wait(bar, parity);
        return true;
    }
    if (threadIdx.x == 0) {
        mbar_wait(bar, parity, err, kErrTmaDrain);
        if (bar2) mbar_wait(bar2, parity2, err, kErrTmaDrain);
    }
    __syncthreads();
    return false;
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0, int c1,
                                            int c2) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], "
        "[%2];" ::"r"(smem_addr(dst)),
        "l"(map), "r"(smem_addr(bar)), "r"(c0), "r"(c1), "r"(c2)
        : "memory");
}

__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0, int c1,
                                            int c2, int c3) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5, "
        "%6}], [%2];" ::"r"(smem_addr(dst)),
        "l"(map), "r"(smem_addr(bar)), "r"(c0), "r"(c1), "r"(c2), "r"(c3)
        : "memory");
}

// Prefetch of a TMA box into L2 (a hint: no completion, no shared memory).
__device__ __forceinline__ void tma_prefetch_4d(const CUtensorMap* map, int c0, int c1, int c2, int c3) {
    asm volatile("cp.async.bulk.prefetch.tensor.4d.L2.global.tile [%0, {%1, %2, %3, %4}];" ::"l"(map), "r"(c0),
                 "r"(c1), "r"(c2), "r"(c3)
                 : "memory");
}

__device__ __forceinline__ void tma_store_3d(const CUtensorMap* map, const void* src, int c0, int c1, int c2) {
    asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%2, %3, %4}], [%1];" ::"l"(map),
                 "r"(smem_addr(src)), "r"(c0), "r"(c1), "r"(c2)
                 : "memory");
}

__device__ __forceinline__ void tma_store_4d(const CUtensorMap* map, const void* src, int c0, int c1, int c2,
                                             int c3) {
    asm volatile("cp.async.bulk.tensor.4d.global.shared::cta.bulk_group [%0, {%2, %3, %4, %5}], [%1];" ::"l"(map),
                 "r"(smem_addr(src)), "r"(c0), "r"(c1), "r"(c2), "r"(c3)
                 : "memory");
}

// Contiguous bulk copies (both addresses 16-byte aligned, size a multiple of 16).
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// Prefetch of a contiguous global range into L2 (a hint: no completion, no
// shared memory; 16-byte aligned address and size).
__device__ __forceinline__ void bulk_prefetch_l2(const void* src, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

__device__ __forceinline__ void bulk_store(void* dst, const void* src, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_addr(src)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }

// Block until every committed bulk store has finished reading shared memory.
__device__ __forceinline__ void bulk_wait_read_all() {
    asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}

// Make this thread's generic-proxy shared-memory writes visible to the async
// (TMA) proxy; follow with a barrier before a TMA store reads them.
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

}  // namespace pfk
