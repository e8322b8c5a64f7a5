// Bulk asynchronous copies (cp.async.bulk), mbarriers and named barriers, as inline PTX,
// shared by the staged LOWD sweeps.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace lowd {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
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

// try_wait that lets the hardware suspend the thread for up to hint_ns before returning
__device__ __forceinline__ bool mbar_try_wait_sleep(uint64_t* bar, uint32_t parity, uint32_t hint_ns) {
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

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void bulk_s2g(void* dst, const void* src, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_u32(src)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }

template <int N>
__device__ __forceinline__ void bulk_wait_read() {
    asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory");
}

template <int N>
__device__ __forceinline__ void bulk_wait() {
    asm volatile("cp.async.bulk.wait_group %0;" ::"n"(N) : "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// orders this thread's generic-proxy accesses (shared and global) before later
// async-proxy ones, e.g. plain stores of a buffer before a bulk copy reads it
__device__ __forceinline__ void fence_proxy_async_all() {
    asm volatile("fence.proxy.async;" ::: "memory");
}

__device__ __forceinline__ void mbar_inval(uint64_t* bar) {
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Bounded wait for the bulk loads of fills [first, issued) of a ring of S stages: fill i
// completes phase i / S of stage i mod S's barrier.  Used on the abort path so that no
// copy is still landing in shared memory when the block moves on or exits.
__device__ __forceinline__ void drain_fills(uint64_t* full, int32_t S, int32_t first, int32_t issued,
                                            uint32_t limit) {
    for (int32_t i = first; i < issued; ++i) {
        uint32_t spins = 0;
        const uint32_t par = (uint32_t)((i / S) & 1);
        while (!mbar_try_wait(&full[i % S], par) && ++spins < limit) {
        }
    }
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void consumer_sync(int nc) {  // bar.sync over the consumer warps
    asm volatile("bar.sync 1, %0;" ::"r"(nc) : "memory");
}

// bar.sync over the consumer warps that also ORs a predicate across them
__device__ __forceinline__ bool consumer_sync_or(int nc, bool pred) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.or.pred q, 1, %2, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)pred), "r"(nc)
        : "memory");
    return r != 0;
}


constexpr uint32_t kGridSpins = 1u << 24;    // bounded waits: grid barrier (with 64 ns sleeps)

// Grid barrier of a cooperative launch: arrive on a counter, the last block to arrive opens
// the next generation (count and gen start at zero; the counter is back at zero after every
// barrier, so later launches reuse the words).  Bounded: on expiry bit 1 of the error word
// is set and false is returned.
__device__ __forceinline__ unsigned ld_acquire_gpu(const volatile unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Arrival: an acquire-release add (publishes this block's writes, which the block barrier
// ordered before it, and lets the last arriver see every other block's); the last arriver
// re-arms the counter and opens the generation with a release; the others poll it with
// acquire loads.
__device__ __forceinline__ bool grid_barrier(unsigned* count, volatile unsigned* gen, unsigned nblocks, int32_t* err,
                                             uint32_t max_spins = kGridSpins) {
    __syncthreads();
    bool ok = true;
    if (threadIdx.x == 0) {
        const unsigned g = ld_acquire_gpu(gen);
        unsigned old;
        asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;" : "=r"(old) : "l"(count) : "memory");
        if (old == nblocks - 1) {
            asm volatile("st.relaxed.gpu.global.u32 [%0], 0;" ::"l"(count) : "memory");
            asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(gen) : "memory");
        } else {
            uint32_t spins = 0;
            while (ld_acquire_gpu(gen) == g) {
                if (++spins > max_spins) { ok = false; atomicOr(err, 2); break; }
                if (spins > 4096) __nanosleep(64);   // poll fast at first, then back off
            }
        }
    }
    __shared__ int okb;
    if (threadIdx.x == 0) okb = ok ? 1 : 0;
    __syncthreads();
    return okb != 0;
}

}  // namespace lowd
