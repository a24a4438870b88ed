// Thin inline-PTX wrappers for sm_103a: mbarriers, cluster/DSMEM access,
// asynchronous copies and timers.  Every wait loop built on these
// is bounded by a time limit (see wait_parity_bounded).
#pragma once
#include <cstdint>

namespace jac {

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint32_t cluster_ctarank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ uint64_t globaltimer_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void cluster_sync_all()
{
    asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
}

// ---------------------------------------------------------------- mbarrier
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init_cluster()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ bool mbar_try_wait_parity(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Arrivals that only signal "this slot was read": the reads they follow
// have completed (their values were consumed), so no memory ordering is
// requested.  A release arrive would instead wait for every earlier global
// store of the thread to drain, which costs thousands of cycles per plane.
__device__ __forceinline__ void mbar_arrive_local(uint32_t bar)
{
    asm volatile(
        "{\n\t.reg .b64 st;\n\t"
        "mbarrier.arrive.relaxed.cta.shared::cta.b64 st, [%0];\n\t}" ::"r"(bar)
        : "memory");
}

// Same, on a barrier given by a shared::cluster address (any CTA of the
// cluster).
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t cluster_bar)
{
    asm volatile("mbarrier.arrive.relaxed.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_bar)
                 : "memory");
}

// ----------------------------------------------------------- cluster / DSMEM
// Address of the same shared-memory location in CTA `rank` of this cluster.
__device__ __forceinline__ uint32_t mapa(uint32_t local, uint32_t rank)
{
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(local), "r"(rank));
    return r;
}

// Asynchronous 16-byte store into another CTA's shared memory whose byte
// count completes on that CTA's mbarrier (addresses are shared::cluster).
__device__ __forceinline__ void st_async_v(uint32_t addr, const float (&v)[4], uint32_t mbar)
{
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.f32 [%0], {%1, %2, %3, %4}, [%5];" ::"r"(addr),
                 "f"(v[0]), "f"(v[1]), "f"(v[2]), "f"(v[3]), "r"(mbar)
                 : "memory");
}
__device__ __forceinline__ void st_async_v(uint32_t addr, const double (&v)[2], uint32_t mbar)
{
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.f64 [%0], {%1, %2}, [%3];" ::"r"(addr),
                 "d"(v[0]), "d"(v[1]), "r"(mbar)
                 : "memory");
}

// Arrival on a barrier of this CTA that also raises its expected byte count.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile(
        "{\n\t.reg .b64 st;\n\t"
        "mbarrier.arrive.expect_tx.relaxed.cta.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(bar),
        "r"(bytes)
        : "memory");
}

// Element-wise asynchronous copy global -> shared (4 or 8 bytes, naturally
// aligned), and an arrival on `bar` once all of this thread's earlier
// cp.async operations have completed (the arrival does not raise the
// pending count: the barrier's expected count includes these arrivals).
__device__ __forceinline__ void cp_async_4(uint32_t dst, const void *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_8(uint32_t dst, const void *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_16(uint32_t dst, const void *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_arrive_noinc(uint32_t bar)
{
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.wait_all;" ::: "memory");
}

// Closes this thread's current group of cp.async operations; waits until at
// most N of its groups are still pending.
__device__ __forceinline__ void cp_async_commit()
{
    asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait_group()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Wait for completion of the barrier phase with the given parity (acquire at
// CTA scope: data that completed the phase through cp.async or st.async
// transaction counts is visible to the waiting thread afterwards).  Gives up
// (returns false) once `limit_ns` has passed, or early when `abort_flag`
// (if not null) becomes nonzero.  Never traps.
__device__ __forceinline__ bool wait_parity_bounded(uint32_t bar, uint32_t parity, uint64_t limit_ns,
                                                    const volatile int *abort_flag)
{
    if (mbar_try_wait_parity(bar, parity)) return true;
    const uint64_t t0 = globaltimer_ns();
    for (uint32_t it = 1;; ++it) {
        if (mbar_try_wait_parity(bar, parity)) return true;
        if ((it & 63u) == 0u) {
            if (abort_flag && *abort_flag != 0) return false;
            if (globaltimer_ns() - t0 > limit_ns) return false;
        }
    }
}

}  // namespace jac
