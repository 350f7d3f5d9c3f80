// Device helpers shared by the library's kernels: status latching, bounded
// waits, gpu-scope relaxed/acquire memory operations, the grid barrier of the
// persistent level-set solve and the "not yet computed" sentinels of the
// synchronisation-free solve.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "sptrsv.h"

namespace sptrsv {

constexpr unsigned FULL_MASK = 0xffffffffu;
// Entry encoding of the solve structure: col >= 0 reads x[col], col < 0
// (but not PAD) reads b[~col] (a right-hand-side term of a rewritten row),
// PAD is a padding slot.
constexpr int32_t PAD_COL = INT32_MIN;
// Single-CTA tail records: a row whose coefficients are stored as they are
// (not divided by its diagonal); the record's count field holds it above
// the count (bits 0-7) and the mask of terms read from x (bits 8-23).
constexpr int32_t kTailUnscaled = 1 << 30;
// Features of one candidate segment (kept level t, depth d) for the
// per-segment cost network of SELECT_SEGMODEL.
constexpr int kSegFeatures = 8;

// Device status block of a plan (zeroed at creation):
//  [0] error code (first one wins), [1] row or index involved,
//  [2] abort flag (set on any error: every wait returns), [3] spare,
//  [4..5] barrier arrival counter (u64), [6..7] exit counter (u64).
struct DevStatus {
    int32_t code;
    int32_t where;
    int32_t abort;
    int32_t ir_iters;
    unsigned long long bar_count;
    unsigned long long exit_count;
    unsigned long long ir_flag;   // refinement converged flag
    double norms[4];              // scratch for infinity norms (as u64 bits)
};

__device__ __forceinline__ void latch_error(DevStatus *st, int code, int where) {
    if (atomicCAS(&st->code, 0, code) == 0) st->where = where;
    atomicExch(&st->abort, 1);
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ int ld_relaxed_i32(const int32_t *p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long ld_relaxed_u64(const void *p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned ld_relaxed_u32(const void *p) {
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed_u64(void *p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" :: "l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void st_relaxed_u32(void *p, unsigned v) {
    asm volatile("st.relaxed.gpu.global.b32 [%0], %1;" :: "l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void red_release_add_u64(unsigned long long *p, unsigned long long v) {
    asm volatile("red.release.gpu.global.add.u64 [%0], %1;" :: "l"(p), "l"(v) : "memory");
}

// "Not computed yet" markers of the synchronisation-free solve: signalling
// NaNs with a payload.  Arithmetic never produces a signalling NaN, so a
// computed unknown can never look like the marker.
template <typename T> struct Sentinel;
template <> struct Sentinel<double> {
    using Bits = unsigned long long;
    static constexpr Bits bits = 0x7FF4DEADBEEF0001ull;
};
template <> struct Sentinel<float> {
    using Bits = unsigned;
    static constexpr Bits bits = 0x7FA0BEEFu;
};

// Bounded wait bookkeeping: every spin in the library checks the plan's
// abort flag and a deadline on the global timer every `kPollMask + 1`
// iterations and gives up (latching SPTRSV_ERR_TIMEOUT) past the deadline.
constexpr int kPollMask = 63;

struct WaitBudget {
    uint64_t deadline;
    __device__ __forceinline__ explicit WaitBudget(uint64_t timeout_ns)
        : deadline(0) { deadline = globaltimer_ns() + timeout_ns; }
    // true if the wait must stop (timeout latched or someone else aborted)
    __device__ __forceinline__ bool expired(DevStatus *st, int where) {
        if (ld_relaxed_i32(&st->abort)) return true;
        if (globaltimer_ns() > deadline) {
            latch_error(st, SPTRSV_ERR_TIMEOUT, where);
            return true;
        }
        return false;
    }
};

// Grid-wide barrier for a co-resident (cooperatively launched) grid.  The
// arrival counter only grows inside one launch; `target` is
// (barrier index + 1) * gridDim.x.  Returns false if the wait gave up.
__device__ __forceinline__ bool grid_barrier(DevStatus *st, unsigned long long target,
                                             uint64_t timeout_ns, int where) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        __threadfence();  // publish this CTA's stores before arriving
        red_release_add_u64(&st->bar_count, 1ull);
        if (ld_acquire_u64(&st->bar_count) < target) {
            WaitBudget wb(timeout_ns);
            unsigned it = 0;
            while (ld_acquire_u64(&st->bar_count) < target) {
                if ((++it & kPollMask) == 0 && wb.expired(st, where)) { ok = 0; break; }
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Split form of grid_barrier: grid_arrive publishes this CTA's stores and
// counts it in; the CTA may then issue loads of data that does not depend on
// other CTAs (they stay in flight across the wait); grid_wait spins until
// every CTA arrived.  Thread 0 does both, so the fence in grid_arrive never
// has to wait for the loads issued in between.
__device__ __forceinline__ void grid_arrive(DevStatus *st) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        red_release_add_u64(&st->bar_count, 1ull);
    }
}
__device__ __forceinline__ bool grid_wait(DevStatus *st, unsigned long long target,
                                          uint64_t timeout_ns, int where) {
    __shared__ int s_ok2;
    if (threadIdx.x == 0) {
        int ok = 1;
        if (ld_acquire_u64(&st->bar_count) < target) {
            WaitBudget wb(timeout_ns);
            unsigned it = 0;
            while (ld_acquire_u64(&st->bar_count) < target) {
                if ((++it & kPollMask) == 0 && wb.expired(st, where)) { ok = 0; break; }
            }
        }
        s_ok2 = ok;
    }
    __syncthreads();
    return s_ok2 != 0;
}

// Bulk prefetch of [p, p + bytes) into L2 (TMA engine), shared out over the
// grid: CTA b takes the b-th slice.  Only whole 16-byte units inside the
// range are requested (the engine needs 16-byte aligned address and size).
__device__ __forceinline__ void l2_prefetch_slice(const void *p, size_t bytes) {
    if (threadIdx.x != 0 || p == nullptr || bytes == 0) return;
    uintptr_t a = ((uintptr_t)p + 15) & ~(uintptr_t)15;
    const uintptr_t e = ((uintptr_t)p + bytes) & ~(uintptr_t)15;
    if (e <= a) return;
    const uintptr_t total = e - a;
    uintptr_t slice = (total / gridDim.x + 15) & ~(uintptr_t)15;
    if (slice < 4096) slice = 4096;
    uintptr_t lo = a + slice * blockIdx.x;
    if (lo >= e) return;
    uintptr_t hi = lo + slice < e ? lo + slice : e;
    constexpr uintptr_t kPiece = 1u << 16;
    for (; lo < hi; lo += kPiece) {
        const uint32_t sz = (uint32_t)(hi - lo < kPiece ? hi - lo : kPiece);
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" :: "l"(lo), "r"(sz) : "memory");
    }
}

// ---------------------------------------------------------------------------
// Shared-memory mbarriers and bulk (TMA) copies global -> shared memory.
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint32_t bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(bar), "r"(count) : "memory");
}
// makes mbarrier initialisations visible to the bulk-copy (async) proxy
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// orders this thread's earlier generic-proxy accesses of shared memory before
// later bulk copies into it
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                 :: "r"(bar), "r"(bytes) : "memory");
}
// Bulk copy of `bytes` (a positive multiple of 16; both addresses 16-byte
// aligned) from global memory into this CTA's shared memory, completing on
// the mbarrier's transaction count.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes,
                                         uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes "
                 "[%0], [%1], %2, [%3];"
                 :: "r"(dst), "l"(src), "r"(bytes), "r"(bar) : "memory");
}
// 16-byte asynchronous copy global -> shared memory (through L2 only) and
// the arrival on an mbarrier once all of this thread's earlier such copies
// have landed (the barrier's expected count includes this arrival).
__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" :: "r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_mbar_arrive(uint32_t bar) {
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" :: "r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                 " selp.u32 %0, 1, 0, p;\n}"
                 : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
    return ok != 0;
}
// Bounded wait for the completion of phase `parity`; false if it gave up
// (timeout latched, or another wait of the launch aborted).
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, DevStatus *st,
                                          uint64_t timeout_ns, int where) {
    if (mbar_try_wait(bar, parity)) return true;
    WaitBudget wb(timeout_ns);
    unsigned it = 0;
    while (!mbar_try_wait(bar, parity)) {
        if ((++it & 15) == 0 && wb.expired(st, where)) return false;
    }
    return true;
}
// Bounded wait that latches nothing (draining copies after an abort).
__device__ __forceinline__ void mbar_drain(uint32_t bar, uint32_t parity, uint64_t timeout_ns) {
    const uint64_t deadline = globaltimer_ns() + timeout_ns;
    while (!mbar_try_wait(bar, parity))
        if (globaltimer_ns() > deadline) return;
}

// Called once by every CTA at the very end of a kernel that used
// grid_barrier: the last CTA to leave resets the counters for the next
// launch on the same stream.
__device__ __forceinline__ void grid_exit(DevStatus *st) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        unsigned long long prev = atomicAdd(&st->exit_count, 1ull);
        if (prev == gridDim.x - 1) {
            atomicExch(&st->bar_count, 0ull);
            atomicExch(&st->exit_count, 0ull);
        }
    }
}

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

}  // namespace sptrsv
