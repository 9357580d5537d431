// tcgen05 building blocks of the split-FP16 radix-32 tensor-core stages:
// operand sizes, the shared-memory descriptor of the K-major B table, the
// kind::f16 instruction descriptors, MMA / TMEM load / TMEM store wrappers,
// bounded mbarrier waits and the float16 pair packing.  Shared by the
// tensor-core row and column kernels (fft_tc32.cu, fft_tc_stream.cu).
#pragma once
#include <cuda_fp16.h>

#include "fft_common.cuh"

namespace gb300fft {

constexpr int kT32E = 32;                 // elements per thread = the tensor-core radix
constexpr int kT32Group = 128;            // threads (butterflies) per MMA group
constexpr int kT32ABytes = 128 * 64 * 2;  // one float16 A operand of a group: 128 rows x 64 halves (16 KiB)
constexpr int kT32GroupStage = 2 * kT32ABytes;  // A_hi + A_lo of a group: 32 KiB
constexpr int kT32BBytes = 64 * 64 * 2;   // one float16 B operand (8 KiB)
static_assert(kT32GroupStage == 32768, "A_hi + A_lo of a group");

// Shared-memory descriptor of a K-major operand without swizzle: core
// matrices of 8 rows x 16 bytes, K-adjacent ones 128 bytes apart, 8-row
// groups 1024 bytes apart (K = 64 halves).
__device__ __forceinline__ uint64_t t32_desc(uint32_t saddr) {
    return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46);
}
// kind::f16: D = F32 (bit 4), A = B = F16, both K-major, N = 64, M = 128
constexpr uint32_t kT32Idesc = (1u << 4) | ((64u >> 3) << 17) | ((128u >> 4) << 24);
// the same with N = 32 (one diagonal block of the even/odd table)
constexpr uint32_t kT32IdescN32 = (1u << 4) | ((32u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ void t32_mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(kT32Idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void t32_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
}

__device__ __forceinline__ void t32_st8(uint32_t taddr, const uint32_t (&r)[8]) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(taddr), "r"(r[0]),
                 "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7])
                 : "memory");
}

// MMA with A read from tensor memory (rows = lanes, two float16 per column).
__device__ __forceinline__ void t32_mma_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t b, uint32_t accumulate,
                                           uint32_t idesc = kT32Idesc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
        "r"(a_tmem), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}

// try_wait that may suspend the thread up to `ns` nanoseconds in hardware
// instead of returning at once, so waiting threads do not spin.
__device__ __forceinline__ bool t32_try_wait_sleep(uint64_t *bar, uint32_t parity, uint32_t ns) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(ns)
        : "memory");
    return ok != 0;
}
// Bounded wait (~limit_ns of global time, at most 2^20 suspended polls).
__device__ __forceinline__ bool t32_wait(uint64_t *bar, uint32_t parity, uint64_t limit_ns = 2000000000ull) {
    const uint64_t t0 = globaltimer_ns();
    for (uint32_t it = 0; it < (1u << 20); ++it) {
        if (t32_try_wait_sleep(bar, parity, 20000)) return true;
        if (globaltimer_ns() - t0 > limit_ns) break;
    }
    return false;
}

__device__ __forceinline__ void named_sync(int id, int nthreads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

__device__ __forceinline__ uint32_t f2h2_bits(float lo_elem, float hi_elem) {
    const __half2 h = __floats2half2_rn(lo_elem, hi_elem);  // .x (low half) = lo_elem
    uint32_t u;
    memcpy(&u, &h, 4);
    return u;
}

}  // namespace gb300fft
