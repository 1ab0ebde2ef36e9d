// Intra-CTA hand-off primitives of the persistent kernels: shared-memory mbarriers,
// bounded waits that report a time-out instead of hanging, and bulk asynchronous
// copies of sample blocks into shared memory.  Shared by the pipelined
// (rx_pipe.cu) and balanced (rx_balance.cu) schedules.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "rx_device.cuh"

namespace rxd {

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// Arrive (release semantics at CTA scope).
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile(
        "{\n\t.reg .b64 st;\n\t"
        "mbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_u32(bar))
        : "memory");
}

// One poll of the phase with the given parity (acquire semantics at CTA scope).
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
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

// Arrive and add tx bytes that the phase must also see completed.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile(
        "{\n\t.reg .b64 st;\n\t"
        "mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(smem_u32(bar)), "r"(bytes)
        : "memory");
}

// Bulk copy global -> this CTA's shared memory, completion reported to bar.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Barrier 1 over the NT correlation threads; returns true when every one passes ok.
template <int NT>
__device__ __forceinline__ bool corr_barrier_and(bool ok) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.and.pred q, 1, %2, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)ok), "n"(NT)
        : "memory");
    return r != 0;
}

// As mbar_try_wait, but the thread may stay suspended in the instruction for up to
// hint_ns (it resumes as soon as the phase completes), so that a waiting warp polls
// rarely and leaves the issue slots to the warps that work.
__device__ __forceinline__ bool mbar_try_wait_hint(uint64_t *bar, uint32_t parity, uint32_t hint_ns) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(hint_ns)
        : "memory");
    return ok != 0;
}

// Bounded wait for the phase with the given parity.  Warp-uniform result: false when
// this or any other thread of the CTA gave up.
__device__ __forceinline__ bool pipe_wait(uint64_t *bar, uint32_t parity, volatile uint32_t *abort,
                                          uint32_t *err, uint64_t timeout_ns, uint32_t block) {
    bool ok = mbar_try_wait(bar, parity);
    if (!ok) {
        const uint64_t t0 = globaltimer_ns();
        for (uint32_t it = 0;; ++it) {
            if (mbar_try_wait_hint(bar, parity, 100000u)) {
                ok = true;
                break;
            }
            if (*abort) break;
            if (it > (1u << 24) || globaltimer_ns() - t0 > timeout_ns) {
                *abort = 1u;
                if (atomicCAS(err, 0u, 1u) == 0u) {
                    err[1] = 0xffffffffu;
                    err[2] = blockIdx.x;
                    err[3] = block;
                }
                break;
            }
        }
    }
    return __all_sync(0xffffffffu, ok);
}

// Wait, bounded, for the phase with the given parity whatever the abort flag says
// (used to let this CTA's own bulk copies land before it exits).
__device__ __forceinline__ void drain_wait(uint64_t *bar, uint32_t parity, uint64_t timeout_ns) {
    const uint64_t t0 = globaltimer_ns();
    for (uint32_t it = 0; it < (1u << 24); ++it) {
        if (mbar_try_wait(bar, parity)) return;
        if (globaltimer_ns() - t0 > timeout_ns) return;
    }
}

// Thread 0: start the copy of one block (bytes at src, 2-byte aligned, even length)
// into buf (128-byte aligned).  The block begins at buf + (src mod 16).
__device__ __forceinline__ void stage_block(const int8_t *src, uint32_t bytes, unsigned char *buf,
                                            uint64_t *bar) {
    const uintptr_t s = (uintptr_t)src, e = s + bytes;
    const uintptr_t a0 = s & ~(uintptr_t)15, a1 = e & ~(uintptr_t)15;
    for (uintptr_t q = (a1 > s ? a1 : s); q < e; q += 2)
        *reinterpret_cast<uint16_t *>(buf + (q - a0)) = __ldg(reinterpret_cast<const uint16_t *>(q));
    const uint32_t n = a1 > a0 ? (uint32_t)(a1 - a0) : 0u;
    mbar_arrive_expect_tx(bar, n);
    if (n) bulk_g2s(buf, reinterpret_cast<const void *>(a0), n, bar);
}

// Bounded spin (thread-wise) until *flag >= want with acquire semantics at GPU
// scope.  Returns false when the CTA's abort flag is up or after recording a
// time-out in err (code, 0xfffffffe, cta, block).
__device__ __forceinline__ bool flag_wait(const uint32_t *flag, uint32_t want, volatile uint32_t *abort,
                                          uint32_t *err, uint64_t timeout_ns, uint32_t block) {
    if (ld_acquire(flag) >= want) return true;
    const uint64_t t0 = globaltimer_ns();
    uint32_t ns = 64;
    for (uint32_t it = 0;; ++it) {
        if (ld_acquire(flag) >= want) return true;
        if (*abort) return false;
        if (it > (1u << 24) || globaltimer_ns() - t0 > timeout_ns) {
            *abort = 1u;
            if (atomicCAS(err, 0u, 1u) == 0u) {
                err[1] = 0xfffffffeu;
                err[2] = blockIdx.x;
                err[3] = block;
            }
            return false;
        }
        __nanosleep(ns);
        if (ns < 2048) ns <<= 1;
    }
}

}  // namespace rxd
