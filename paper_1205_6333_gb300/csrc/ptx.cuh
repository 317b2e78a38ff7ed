// ptx.cuh -- hand-written inline PTX used by the kernels (sm_103a):
// mbarrier set-up and bounded waits, 1-D bulk copies global -> shared
// (cp.async.bulk with mbarrier completion), and the SFU reciprocal square root.
#pragma once
#include <cstdint>

namespace sd {

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

// Make the initialised barriers visible to the async (bulk-copy) proxy.
__device__ __forceinline__ void fence_barrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
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

// Wait for phase `parity` of `bar` to complete, giving up after `limit` polls.
// Returns false on time-out (the caller records an error and carries on).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, long long limit) {
    for (long long it = 0; it < limit; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// Poll budget for draining this CTA's own bulk copies before it exits after a
// time-out: at least 2^20 polls whatever the watchdog, since a copy that is still
// in flight must land before the shared memory it targets is released.
__device__ __forceinline__ long long drain_limit(long long wd) { return wd > (1LL << 20) ? 4 * wd : (1LL << 22); }

// 1-D bulk copy of `bytes` (multiple of 16, both addresses 16-byte aligned) from
// global to this CTA's shared memory; completion is signalled on `bar` as
// transaction bytes.
__device__ __forceinline__ void bulk_g2s(void *dst_smem, const void *src_gmem, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst_smem)),
        "l"(src_gmem), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// SFU reciprocal square root, approximate (PTX rsqrt.approx.ftz.f32).
__device__ __forceinline__ float rsqrt_sfu(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rcp_sfu(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// FP64 reciprocal square root from the FP32 SFU seed y0 (relative error below
// 2^-22) and one third-order correction: with e = 1 - x y0^2,
//   x^(-1/2) = y0 (1 - e)^(-1/2) = y0 (1 + e/2 + 3e^2/8 + 5e^3/16 + ...),
// and the truncated e^3 term is below 2^-64 relative.  Five FP64 operations instead
// of the seven of two Newton steps (FP64 issues at a small fraction of the FP32 rate
// on this GPU, so the operation count is the cost).
__device__ __forceinline__ double rsqrt_nr64(double x) {
    const double y0 = static_cast<double>(rsqrt_sfu(static_cast<float>(x)));
    const double e = fma(-x * y0, y0, 1.0);
    return fma(y0 * e, fma(0.375, e, 0.5), y0);
}

}  // namespace sd
