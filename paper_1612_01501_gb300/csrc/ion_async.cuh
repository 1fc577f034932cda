// ion_async.cuh -- mbarrier, bulk async copy, timer and compensated-sum helpers (sm_90+ PTX).
#pragma once
#include <cstdint>

namespace ion {

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t phase) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(phase)
        : "memory");
    return ok != 0;
}
// Programmatic dependent launch (griddepcontrol, sm_90+).  A kernel launched with
// programmatic stream serialization may be scheduled while the kernel before it in the
// stream is still draining.  pdl_enter() first waits until that kernel has completed and
// its writes are visible (at once for an ordinary launch), then allows the next kernel
// launched that way to be scheduled.  Every kernel so launched calls it before its first
// global-memory access.
__device__ __forceinline__ void pdl_enter() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}
// Bounded wait on an mbarrier phase: gives up after ~0.5 s (then flags ST_TIMEOUT).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t phase) {
    if (mbar_try_wait(bar, phase)) return true;
    const uint64_t t0 = globaltimer_ns();
    for (uint32_t it = 0; it < (1u << 26); ++it) {
        if (mbar_try_wait(bar, phase)) return true;
        if ((it & 255u) == 255u && globaltimer_ns() - t0 > 500000000ull) break;
    }
    return mbar_try_wait(bar, phase);
}
// 1-D bulk copy global -> shared, completion counted in bytes on `bar`
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Ask for [src, src + bytes) to be brought into L2, without completion tracking (a hint).
// src 16-byte aligned, bytes a multiple of 16, the range inside one allocation.
__device__ __forceinline__ void bulk_prefetch_l2(const void *src, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

__device__ __forceinline__ void kahan_add(float &sum, float &comp, float x) {
    const float y = x - comp;
    const float t = sum + y;
    comp = (t - sum) - y;
    sum = t;
}

// ---- grid-wide barrier of a cooperative launch (bounded) --------------------------
__device__ __forceinline__ uint32_t ld_acquire_gpu(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void red_release_gpu_add(uint32_t *p, uint32_t v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// true once the 32-bit arrival counter has reached `target`, comparing modulo 2^32: a long
// persistent launch arrives more than 2^32 times in total, so both the counter and the
// targets wrap; the two never drift apart by 2^31 (the counter exceeds the current target
// by at most the grid size), so the sign of their difference decides
__device__ __forceinline__ bool arrivals_reached(uint32_t count, uint32_t target) {
    return (int32_t)(count - target) >= 0;
}

// Every CTA arrives once per barrier on a monotonically increasing counter (zeroed before
// the launch); barrier k completes when the counter reaches k * gridDim.x (mod 2^32).  A
// wait that exceeds timeout_ns (or 2^30 polls) sets `status` bit 2 (timeout) and the shared
// abort word, so every other CTA leaves its own wait too; the function then returns false
// in every thread of the CTA.
__device__ __forceinline__ bool grid_barrier(uint32_t *count, uint32_t *abort_flag, uint32_t target,
                                             uint64_t timeout_ns, uint32_t *status, int *ok_sh) {
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        // release at GPU scope: the CTA's writes, ordered before this by the bar.sync above,
        // become visible before the arrival does
        red_release_gpu_add(count, 1u);
        if (!arrivals_reached(ld_acquire_gpu(count), target)) {
            const uint64_t t0 = globaltimer_ns();
            for (uint32_t it = 1;; ++it) {
                if (arrivals_reached(ld_acquire_gpu(count), target)) break;
                if ((it & 63u) == 0u) {          // the abort word and the clock every 64 polls
                    if (ld_acquire_gpu(abort_flag) != 0u) {
                        ok = 0;
                        break;
                    }
                    if (globaltimer_ns() - t0 > timeout_ns || it > (1u << 30)) {
                        atomicOr(status, 2u);
                        atomicExch(abort_flag, 1u);
                        ok = 0;
                        break;
                    }
                }
            }
        }
        // order the async-proxy (bulk copy) reads that follow after the acquire above
        asm volatile("fence.proxy.async;" ::: "memory");
        *ok_sh = ok;
    }
    __syncthreads();
    return *ok_sh != 0;
}

// ---- grid-wide barrier with a release flag (bounded) ------------------------------------
__device__ __forceinline__ uint32_t atom_add_acqrel_gpu(uint32_t *p, uint32_t v) {
    uint32_t old;
    asm volatile("atom.add.acq_rel.gpu.global.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}
__device__ __forceinline__ void st_release_gpu(uint32_t *p, uint32_t v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Every CTA arrives once on `count` (acquire-release); the CTA that brings it to `target`
// (mod 2^32) is the last and stores `target` to `flag` (release); the others poll `flag`,
// which lives on its own cache line, until it reaches `target`.  So the arrivals are not
// slowed by pollers on their line, and a poll sees the release of one store.  Bounded
// like grid_barrier (timeout_ns or 2^30 polls: status bit 2 and the abort word).
__device__ __forceinline__ bool grid_barrier_flag(uint32_t *count, uint32_t *flag, uint32_t *abort_flag,
                                                  uint32_t target, uint64_t timeout_ns, uint32_t *status, int *ok_sh) {
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        const uint32_t old = atom_add_acqrel_gpu(count, 1u);
        if (old + 1u == target) {
            st_release_gpu(flag, target);
        } else if (!arrivals_reached(ld_acquire_gpu(flag), target)) {
            const uint64_t t0 = globaltimer_ns();
            for (uint32_t it = 1;; ++it) {
                if (arrivals_reached(ld_acquire_gpu(flag), target)) break;
                if ((it & 63u) == 0u) {
                    if (ld_acquire_gpu(abort_flag) != 0u) {
                        ok = 0;
                        break;
                    }
                    if (globaltimer_ns() - t0 > timeout_ns || it > (1u << 30)) {
                        atomicOr(status, 2u);
                        atomicExch(abort_flag, 1u);
                        ok = 0;
                        break;
                    }
                }
            }
        }
        asm volatile("fence.proxy.async;" ::: "memory");
        *ok_sh = ok;
    }
    __syncthreads();
    return *ok_sh != 0;
}

}  // namespace ion
