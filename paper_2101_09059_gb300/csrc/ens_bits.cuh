// binary32 <-> binary64 conversions on the integer pipe, and the PTX wrappers for the
// bulk-copy engine (TMA, non-tensor form) and mbarriers used by the staged step kernel.
//
// On GB300 the binary64 pipe issues about 2 operations per SM per clock, and the
// hardware F2F conversions between binary32 and binary64 run on that same pipe. The
// FP32-force update converts twice per dof and step, so the conversions below rebuild
// the IEEE-754 bit patterns with integer operations instead (sign, exponent rebias
// 127 <-> 1023, mantissa shift by 29 bits), falling back to the hardware conversion only
// for the rare operands outside the normal range.
#pragma once

#include <cstdint>

namespace ens {

// Exact binary32 -> binary64 for every input (normal values via bit rebuild).
__device__ __forceinline__ double f32_to_f64(float x) {
    const uint32_t b = __float_as_uint(x);
    const uint32_t e = (b >> 23) & 0xffu;
    if (e == 0u || e == 0xffu) return (double)x;  // zero, subnormal, Inf, NaN
    const uint32_t hi = (b & 0x80000000u) | ((e + 896u) << 20) | ((b & 0x7fffffu) >> 3);
    const uint32_t lo = b << 29;
    return __hiloint2double((int)hi, (int)lo);
}

// binary64 -> binary32 rounding toward zero. Magnitudes below the smallest normal
// binary32 (2^-126) become signed zero; Inf, NaN and overflow use the hardware path.
__device__ __forceinline__ float f64_to_f32_rz(double d) {
    const uint32_t hi = (uint32_t)__double2hiint(d);
    const uint32_t lo = (uint32_t)__double2loint(d);
    const uint32_t e = (hi >> 20) & 0x7ffu;
    const uint32_t s = hi & 0x80000000u;
    if (e < 897u) return __uint_as_float(s);
    if (e > 1150u) return __double2float_rz(d);
    const uint32_t m = ((hi & 0xfffffu) << 3) | (lo >> 29);
    return __uint_as_float(s | ((e - 896u) << 23) | m);
}

// ---- mbarrier and bulk copies (PTX ISA: mbarrier, cp.async.bulk) --------------------
__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}

// Make the initialised barrier visible to the bulk-copy (async) proxy.
__device__ __forceinline__ void fence_barrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile(
        "{ .reg .b64 st; mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1; }" ::"r"(
            smem_addr(bar)),
        "r"(bytes)
        : "memory");
}

// Global -> shared bulk copy completing on `bar`. dst, src 16-byte aligned, bytes % 16 == 0.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes,
                                         uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, "
        "[%3];" ::"r"(smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// Bring a 16-byte-aligned global range (bytes % 16 == 0) into L2 ahead of use.
__device__ __forceinline__ void bulk_prefetch_l2(const void *src, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

// Wait for phase `parity` of `bar` with at most `limit` polls; returns false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, uint32_t limit) {
    const uint32_t a = smem_addr(bar);
    for (uint32_t it = 0; it < limit; ++it) {
        uint32_t done;
        asm volatile(
            "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; "
            "selp.u32 %0, 1, 0, p; }"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

}  // namespace ens
