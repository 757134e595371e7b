// tma.cuh -- bulk global->shared copies with mbarrier completion (sm_90+ PTX,
// used here on sm_103a), and the two-buffer stager of instruction streams.
//
// Every wait is bounded: after kMaxPolls polls the waiting thread gives up,
// the kernel records STAB_KSTATUS_TIMEOUT in its status word and returns.
#pragma once

#include <cstdint>

#include "stab_internal.h"

namespace stab {

constexpr uint32_t kMaxPolls = 1u << 24;
constexpr int32_t STAB_KSTATUS_TIMEOUT = 1;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void mbar_fence_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

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

__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity) {
    for (uint32_t it = 0; it < kMaxPolls; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// Orders earlier generic-proxy accesses to shared memory before later
// async-proxy (bulk copy) writes to it.
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// 1-D bulk copy: 16-byte aligned addresses, size a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes,
                                         uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Named barrier over `count` threads (ids 1 .. 15; 0 is __syncthreads).
__device__ __forceinline__ void named_sync(uint32_t id, uint32_t count) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// Two-buffer stager of a sequence of instruction chunks taken from up to two
// streams (chunk c < n0 from s0, else from s1).  The lead thread issues the
// copies and waits; the others learn the outcome through `flag` after a
// barrier.  By default the stager serves the whole CTA (thread 0, CTA
// barrier); a part of a CTA that runs on its own sets lead / bar_id / bar_n
// (its first thread, a named barrier over its threads).
struct Stager {
    const Rec *s0, *s1;
    int n0, n_total;
    Rec *buf;          // 2 x kChunkRecs records in shared memory
    uint64_t *bar;     // 2 mbarriers in shared memory
    int *flag;         // shared flag: 1 = chunk ready, 0 = gave up
    uint32_t ph0 = 0, ph1 = 0;   // phases each barrier completed before this sequence
    uint32_t lead = 0, bar_id = 0, bar_n = 0;

    __device__ bool is_lead() const { return threadIdx.x == lead; }
    __device__ void sync() const {
        if (bar_n) named_sync(bar_id, bar_n);
        else __syncthreads();
    }

    __device__ uint32_t parity(int c) const {
        return ((c & 1 ? ph1 : ph0) + (uint32_t)(c >> 1)) & 1u;
    }
    // Phases completed once all n_total chunks of this sequence are consumed.
    __device__ void advance_phases() {
        ph0 += (uint32_t)((n_total + 1) / 2);
        ph1 += (uint32_t)(n_total / 2);
    }
    // Later sequences on the same barriers (persistent kernels): issue the
    // first chunks without re-initialising the barriers.
    __device__ void restart() {
        if (is_lead()) {
            if (n_total > 0) issue(0);
            if (n_total > 1) issue(1);
        }
        sync();
    }

    __device__ const Rec *src(int c) const {
        return c < n0 ? s0 + (size_t)c * kChunkRecs : s1 + (size_t)(c - n0) * kChunkRecs;
    }
    __device__ void issue(int c) {
        uint64_t *b = bar + (c & 1);
        mbar_expect_tx(b, kChunkRecs * sizeof(Rec));
        bulk_g2s(buf + (c & 1) * kChunkRecs, src(c), kChunkRecs * sizeof(Rec), b);
    }
    // Called by all threads once, before any wait.
    __device__ void start() {
        if (is_lead()) {
            mbar_init(bar, 1);
            mbar_init(bar + 1, 1);
            mbar_fence_init();
            if (n_total > 0) issue(0);
            if (n_total > 1) issue(1);
        }
        sync();
    }
    // All threads: wait until chunk c is in buf[c & 1].  Returns false (for
    // every thread) when the bounded wait gave up; *status is then set.
    __device__ bool wait(int c, int32_t *status) {
        if (is_lead()) {
            bool ok = mbar_wait_bounded(bar + (c & 1), parity(c));
            *flag = ok ? 1 : 0;
            if (!ok) {
                if (status) atomicExch(status, STAB_KSTATUS_TIMEOUT);
                // let the copies in flight land before the block exits (bounded)
                mbar_wait_bounded(bar + (c & 1), parity(c));
                if (c + 1 < n_total) mbar_wait_bounded(bar + ((c + 1) & 1), parity(c + 1));
            }
        }
        sync();
        return *flag != 0;
    }
    // All threads, after their last read of buf[c & 1]: refill it with c + 2.
    __device__ void release(int c) {
        sync();
        if (is_lead() && c + 2 < n_total) {
            fence_proxy_async_smem();
            issue(c + 2);
        }
    }
    __device__ const Rec *chunk(int c) const { return buf + (c & 1) * kChunkRecs; }
};

}  // namespace stab
