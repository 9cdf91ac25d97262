// hcg_async.cuh -- shared-memory barriers (mbarrier) and bulk asynchronous
// copies (the TMA unit's 1-D form) used by the staged kernels, written as
// inline PTX for sm_100-class GPUs.  Every wait is bounded in global time: it
// raises HCG_DERR_TIMEOUT and returns false instead of spinning forever.
#pragma once

#include "hcg_dev.cuh"

HCG_DEV uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

HCG_DEV uint64_t gtimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

HCG_DEV void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(bar), "r"(count) : "memory");
}

// Make the initialised barriers visible to the async proxy (bulk copies).
HCG_DEV void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

HCG_DEV void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" :: "r"(bar) : "memory");
}

// Arrive and announce `bytes` of asynchronous copies completing on bar.
HCG_DEV void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" :: "r"(bar), "r"(bytes)
                 : "memory");
}

// Wait for the phase of `bar` with the given parity; gives up after limit_ns
// of global time (then the TIMEOUT bit is raised and false returned).
HCG_DEV bool mbar_wait(uint32_t bar, uint32_t parity, int *err, uint64_t limit_ns) {
    uint64_t t0 = 0;
    for (uint32_t it = 0;; it++) {
        uint32_t done;
        asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
                     : "=r"(done) : "r"(bar), "r"(parity) : "memory");
        if (done) return true;
        if ((it & 255) == 0) {
            uint64_t t = gtimer();
            if (t0 == 0) t0 = t;
            else if (t - t0 > limit_ns) { set_err(err, HCG_DERR_TIMEOUT); return false; }
        }
    }
}

// Bulk copy of `bytes` (a multiple of 16; both addresses 16-byte aligned)
// from global to shared memory, completing as transaction bytes on bar.
HCG_DEV void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 :: "r"(dst), "l"(src), "r"(bytes), "r"(bar) : "memory");
}

// Named barrier over `count` threads (a multiple of 32) that also ORs a
// predicate across them: every participant gets the OR.
HCG_DEV bool bar_red_or(int id, int count, bool pred) {
    uint32_t r;
    asm volatile("{\n.reg .pred p, q;\nsetp.ne.u32 p, %1, 0;\nbar.red.or.pred q, %2, %3, p;\nselp.u32 %0, 1, 0, q;\n}"
                 : "=r"(r) : "r"((uint32_t)pred), "r"(id), "r"(count) : "memory");
    return r != 0;
}

HCG_DEV void bar_sync(int id, int count) { asm volatile("bar.sync %0, %1;" :: "r"(id), "r"(count) : "memory"); }
