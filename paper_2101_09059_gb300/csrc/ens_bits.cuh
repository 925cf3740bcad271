// binary32 <-> binary64 conversions on the integer pipe, and the PTX wrappers for the
// bulk-copy engine (TMA, non-tensor form) and mbarriers used by the staged step kernel.
//
// On GB300 the binary64 pipe issues about 2 operations per SM per clock, and the
// hardware F2F conversions between binary32 and binary64 run on that same pipe. The
// FP32-force update converts twice per dof and step, so the conversions below rebuild
// the IEEE-754 bit patterns with integer operations only (sign, exponent rebias
// 127 <-> 1023, mantissa shift by 29 bits, and the special classes), never issuing a
// binary64 instruction.
#pragma once

#include <cstdint>

namespace ens {

// Exact binary32 -> binary64 for every input, integer operations only: normal values by
// rebiasing the exponent (127 -> 1023) and shifting the mantissa 29 bits; subnormals are
// normalised with a count of leading zeros; zero, Inf and NaN keep their class and sign.
__device__ __forceinline__ double f32_to_f64(float x) {
    const uint32_t b = __float_as_uint(x);
    const uint64_t sign = (uint64_t)(b >> 31) << 63;
    const uint32_t e = (b >> 23) & 0xffu;
    const uint32_t m = b & 0x7fffffu;
    uint64_t bits;
    if (e == 0u) {
        if (m == 0u) {
            bits = sign;
        } else {  // subnormal: value m * 2^-149, leading one at bit p
            const int p = 31 - __clz(m);
            const uint64_t mm = ((uint64_t)m << (52 - p)) & 0xfffffffffffffull;
            bits = sign | ((uint64_t)(p - 149 + 1023) << 52) | mm;
        }
    } else if (e == 0xffu) {
        bits = sign | (0x7ffull << 52) | ((uint64_t)m << 29);
    } else {
        bits = sign | ((uint64_t)(e + 896u) << 52) | ((uint64_t)m << 29);
    }
    return __longlong_as_double((long long)bits);
}

// binary64 -> binary32 rounding toward zero, integer operations only. Magnitudes below
// the smallest normal binary32 (2^-126) become signed zero; finite values beyond the
// largest binary32 become the largest finite value (toward zero); Inf stays Inf and NaN
// stays NaN.
__device__ __forceinline__ float f64_to_f32_rz(double d) {
    const uint64_t bits = (uint64_t)__double_as_longlong(d);
    const uint32_t sign = (uint32_t)(bits >> 32) & 0x80000000u;
    const uint32_t e = (uint32_t)(bits >> 52) & 0x7ffu;
    const uint64_t m = bits & 0xfffffffffffffull;
    uint32_t out;
    if (e < 897u) {
        out = sign;
    } else if (e == 0x7ffu) {
        out = sign | 0x7f800000u | (m ? 0x400000u : 0u);
    } else if (e > 1150u) {
        out = sign | 0x7f7fffffu;
    } else {
        out = sign | ((e - 896u) << 23) | (uint32_t)(m >> 29);
    }
    return __uint_as_float(out);
}

// binary32 -> binary64 for normal values and zeros (exact), integer operations only, in
// fewer steps than f32_to_f64: subnormal inputs become signed zero, and Inf / NaN map to
// finite magnitudes >= 2^128, which split_state below reports as out of range.
__device__ __forceinline__ double f32_to_f64_ftz(float x) {
    const uint32_t b = __float_as_uint(x);
    const uint32_t mag = b & 0x7fffffffu;
    const bool normal = mag >= 0x00800000u;
    const uint32_t hw = (b & 0x80000000u) | (normal ? (mag >> 3) + (896u << 20) : 0u);
    const uint32_t lw = normal ? (b << 29) : 0u;
    return __longlong_as_double((long long)(((uint64_t)hw << 32) | lw));
}

// ---- bit-split binary64 state ---------------------------------------------------------
// The FP32-force form keeps each binary64 displacement u as two 32-bit words:
//   head = u truncated to binary32 (the value neighbours gather for the forces), and
//   tail = the 29 low mantissa bits of u that the truncation drops.
// For |u| in [2^-126, 2^128) the pair holds u exactly (binary32 and binary64 mantissas
// differ by 29 bits); smaller magnitudes are stored as signed zero, and larger ones or
// non-finite u are reported as out of range. The state then needs 8 bytes per dof with
// no separate binary32 copy for the gather.

// Split u into (head, tail); returns false when |u| >= 2^128 or u is not finite.
__device__ __forceinline__ bool split_state(double u, float &head, uint32_t &tail) {
    const uint32_t hw = (uint32_t)((uint64_t)__double_as_longlong(u) >> 32);
    const uint32_t lw = (uint32_t)__double_as_longlong(u);
    const uint32_t mag = hw & 0x7fffffffu;
    const uint32_t sign = hw & 0x80000000u;
    // binary64 exponent field e in [897, 1150] <=> mag in [897 << 20, 1151 << 20)
    const bool normal = mag - (897u << 20) < ((1151u - 897u) << 20);
    // (e mod 2^9, top 23 mantissa bits), then the exponent rebiased by 896: subtracting
    // 896 * 2^23 mod 2^32 = 0xC0000000 leaves e - 896 in bits 23..31, exact for e in
    // range since 1 <= e - 896 < 2^8
    const uint32_t hb = (__funnelshift_l(lw, hw, 3) - 0xC0000000u) & 0x7fffffffu;
    head = __uint_as_float(normal ? (sign | hb) : sign);
    tail = normal ? (lw & 0x1fffffffu) : 0u;
    return mag < (1151u << 20);
}

// Rebuild u from (head, tail) written by split_state (head is a normal binary32 or zero).
__device__ __forceinline__ double join_state(float head, uint32_t tail) {
    const uint32_t b = __float_as_uint(head);
    const uint32_t mag = b & 0x7fffffffu;
    const uint32_t hw = mag ? ((b & 0x80000000u) | ((mag >> 3) + (896u << 20))) : b;
    const uint32_t lw = (b << 29) | tail;
    return __longlong_as_double((long long)(((uint64_t)hw << 32) | lw));
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

// Programmatic dependent launch (PTX griddepcontrol). launch_dependents lets the next
// kernel on the stream, launched with programmatic stream serialisation, start its
// blocks before this grid finishes; wait blocks the calling thread until the grids this
// one depends on have completed and their memory is visible (a no-op when the kernel
// was launched without the attribute).
__device__ __forceinline__ void grid_launch_dependents() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void grid_dependency_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

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
