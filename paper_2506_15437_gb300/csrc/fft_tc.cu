// Split-FP16 tensor-core form: every radix-16 butterfly of the Stockham
// engine runs as a small dense DFT-matrix product on the tensor cores.
//
// A radix-16 butterfly is y = W16 x with W16[k][r] = exp(-2*pi*i*k*r/16).  In
// real arithmetic, with x = (xr, xi) stacked as a 32-vector,
//     [yr; yi] = [[Wr, -Wi], [Wi, Wr]] [xr; xi],   Wr = Re W16, Wi = Im W16.
// Float16 operands keep 11 significant bits, so both sides are split into a
// high and a low half (after Ootomo & Yokota's error-corrected tensor-core
// GEMM): W = W_hi + 2^-11 W_lo, with hi/lo computed from the FP64 matrix, and
// per butterfly x = s (x_hi + 2^-11 x_lo) with s a power of two at least the
// largest |component| (so x_hi, x_lo never overflow and the scaling is exact).
// Three products are kept and accumulated in float32:
//     y = s (W_hi x_hi + 2^-11 (W_hi x_lo + W_lo x_hi));
// the dropped W_lo x_lo term is below 2^-22 relative.  The twiddles between
// stages stay float32 on the CUDA cores; so do stages of radix below 16.
//
// The products use mma.sync.m16n8k16 (f16 inputs, f32 accumulate): one
// instruction multiplies a 16x16 tile of the 32x32 matrix by eight butterflies.
// Each warp handles its 32 butterflies in four groups of eight: the owners of
// a group write their split halves to a small per-warp staging area, all 32
// lanes load the operand fragments with ldmatrix, issue 12 MMAs, recombine,
// and hand the 16 outputs back to each owner through the staging area.  To the
// engine this is just another butterfly<16>, so the row and column passes, the
// fused reorders and the column pre-split are the same as on the FP32 path.
#include <cuda_fp16.h>

#include <mutex>

#include "fft_common.cuh"
#include "fft_internal.h"

namespace gb300fft {

constexpr int kTcStageIn = 144;                            // bytes per butterfly record (hi/lo, re/im, + pad)
constexpr int kTcStageOutRec = 17;                         // float2 per output record (16 + pad)
constexpr int kTcStageBytes = 8 * kTcStageIn + 8 * kTcStageOutRec * 8;  // per warp: 1152 + 1088
constexpr int kTcStageStride = 2304;                       // per-warp staging stride (bytes)

// W16 split table, half precision: [Wr_hi][Wr_lo][Wi_hi][Wi_lo], each 16x16
// row-major (row = output k, column = input r).  Generated in FP64.
__global__ void k_w16_table(__half *t) {
    const int idx = threadIdx.x;  // 256 threads
    const int k = idx / 16, r = idx % 16;
    double sv, cv;
    sincospi(2.0 * (double)((k * r) % 16) / 16.0, &sv, &cv);
    const double wr = cv, wi = -sv;
    const __half wr_hi = __double2half(wr);
    const __half wi_hi = __double2half(wi);
    t[0 * 256 + idx] = wr_hi;
    t[1 * 256 + idx] = __double2half((wr - (double)__half2float(wr_hi)) * 2048.0);
    t[2 * 256 + idx] = wi_hi;
    t[3 * 256 + idx] = __double2half((wi - (double)__half2float(wi_hi)) * 2048.0);
}

cudaError_t build_w16_table(void *t, cudaStream_t s) {
    k_w16_table<<<1, 256, 0, s>>>(static_cast<__half *>(t));
    return cudaGetLastError();
}

// the two halves of h as one 32-bit word (low half first)
__device__ __forceinline__ uint32_t h2bits(__half2 h) {
    uint32_t u;
    memcpy(&u, &h, 4);
    return u;
}
__device__ __forceinline__ uint32_t pack_half2(__half a, __half b) {
    return (uint32_t)__half_as_ushort(a) | ((uint32_t)__half_as_ushort(b) << 16);
}

__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void ldmatrix_x4(uint32_t (&r)[4], const void *p) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(smem_u32(p)));
}

struct TcPolicy {
    using T = float2;
    static constexpr bool kUsesTwiddles = true;
    uint32_t wr_hi[4], wi_hi[4], wr_lo[4], wi_lo[4];
    unsigned char *stage;  // this warp's staging area (shared memory)

    // per-CTA extra shared memory: one staging area per warp
    static constexpr size_t stage_bytes(int threads) { return (size_t)((threads + 31) / 32) * kTcStageStride; }
    __device__ __forceinline__ void init(const __half *__restrict__ table, unsigned char *stage_base, int *) {
        load(table, stage_base + (threadIdx.x >> 5) * kTcStageStride);
    }
    __device__ __forceinline__ void finish() {}

    // A-operand fragments of the four 16x16 parts, from the FP64-built table.
    __device__ __forceinline__ void load(const __half *__restrict__ table, unsigned char *warp_stage) {
        stage = warp_stage;
        const int lane = threadIdx.x & 31;
        const int g = lane >> 2, q = lane & 3;
        // register j of an m16k16 A fragment: rows g (+8 for j odd), columns 2q (+8 for j >= 2)
        for (int j = 0; j < 4; ++j) {
            const int row = g + ((j & 1) ? 8 : 0);
            const int col = 2 * q + ((j & 2) ? 8 : 0);
            const int o = row * 16 + col;
            wr_hi[j] = pack_half2(table[0 * 256 + o], table[0 * 256 + o + 1]);
            wr_lo[j] = pack_half2(table[1 * 256 + o], table[1 * 256 + o + 1]);
            wi_hi[j] = pack_half2(table[2 * 256 + o], table[2 * 256 + o + 1]);
            wi_lo[j] = pack_half2(table[3 * 256 + o], table[3 * 256 + o + 1]);
        }
    }

    template <int R>
    __device__ __forceinline__ void butterfly(float2 *a) const {
        if constexpr (R == 16)
            tc_dft16(a);
        else
            dft<R>(a);
    }
    __device__ __forceinline__ float2 twiddle(float2 a, float2 w) const { return cmul(a, w); }

    // The calling thread's length-16 DFT, computed by the warp on the tensor
    // cores.  Every lane of the warp must call it (warp-synchronous).
    __device__ __forceinline__ void tc_dft16(float2 *v) const {
        const int lane = threadIdx.x & 31;
        const int g = lane >> 2, q = lane & 3;
        // power-of-two scale s > max |component| of this butterfly
        float m = 0.f;
#pragma unroll
        for (int r = 0; r < 16; ++r) m = fmaxf(m, fmaxf(fabsf(v[r].x), fabsf(v[r].y)));
        const int eb = (__float_as_int(m) >> 23) & 0xff;          // m < 2^(eb - 126)
        const float s = __int_as_float((eb + 1) << 23);            // 2^(eb - 126)
        const float inv_s = __int_as_float((253 - eb) << 23);      // 2^(126 - eb)
        unsigned char *in_rec = stage;
        float2 *out_rec = reinterpret_cast<float2 *>(stage + 8 * kTcStageIn);
#pragma unroll 1
        for (int G = 0; G < 4; ++G) {
            if ((lane >> 3) == G) {
                // record: hi_re[16] hi_im[16] lo_re[16] lo_im[16] (halves)
                uint32_t *dst = reinterpret_cast<uint32_t *>(in_rec + (lane & 7) * kTcStageIn);
#pragma unroll
                for (int r = 0; r < 16; r += 2) {
                    const float xr0 = v[r].x * inv_s, xr1 = v[r + 1].x * inv_s;
                    const float xi0 = v[r].y * inv_s, xi1 = v[r + 1].y * inv_s;
                    const __half2 hr = __floats2half2_rn(xr0, xr1), hi = __floats2half2_rn(xi0, xi1);
                    const float2 hrf = __half22float2(hr), hif = __half22float2(hi);
                    dst[r / 2] = h2bits(hr);
                    dst[8 + r / 2] = h2bits(hi);
                    dst[16 + r / 2] = h2bits(__floats2half2_rn((xr0 - hrf.x) * 2048.f, (xr1 - hrf.y) * 2048.f));
                    dst[24 + r / 2] = h2bits(__floats2half2_rn((xi0 - hif.x) * 2048.f, (xi1 - hif.y) * 2048.f));
                }
            }
            __syncwarp();
            // lane l addresses row (l & 7) of matrix (l >> 3): matrices
            // (re, k 0-7), (re, k 8-15), (im, k 0-7), (im, k 8-15)
            const int mat = lane >> 3;
            const unsigned char *row = in_rec + (lane & 7) * kTcStageIn + (mat >> 1) * 32 + (mat & 1) * 16;
            uint32_t bh[4], bl[4];
            ldmatrix_x4(bh, row);       // hi: b(re) = bh[0], bh[1]; b(im) = bh[2], bh[3]
            ldmatrix_x4(bl, row + 64);  // lo
            float d1[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
            float d2[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
            // yr = Wr xr - Wi xi ; yi = Wi xr + Wr xi   (-Wi: flip the sign bits
            // of the imaginary-part operand halves instead of storing -Wi)
            const uint32_t nbh2 = bh[2] ^ 0x80008000u, nbh3 = bh[3] ^ 0x80008000u;
            const uint32_t nbl2 = bl[2] ^ 0x80008000u, nbl3 = bl[3] ^ 0x80008000u;
            mma16816(d1[0], wr_hi, bh[0], bh[1]);
            mma16816(d1[0], wi_hi, nbh2, nbh3);
            mma16816(d1[1], wi_hi, bh[0], bh[1]);
            mma16816(d1[1], wr_hi, bh[2], bh[3]);
            mma16816(d2[0], wr_hi, bl[0], bl[1]);
            mma16816(d2[0], wi_hi, nbl2, nbl3);
            mma16816(d2[1], wi_hi, bl[0], bl[1]);
            mma16816(d2[1], wr_hi, bl[2], bl[3]);
            mma16816(d2[0], wr_lo, bh[0], bh[1]);
            mma16816(d2[0], wi_lo, nbh2, nbh3);
            mma16816(d2[1], wi_lo, bh[0], bh[1]);
            mma16816(d2[1], wr_lo, bh[2], bh[3]);
            // this lane holds outputs k = g, g+8 of butterflies 2q, 2q+1 of the group
            const float s0 = __shfl_sync(0xffffffffu, s, 8 * G + 2 * q);
            const float s1 = __shfl_sync(0xffffffffu, s, 8 * G + 2 * q + 1);
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const float se = e ? s1 : s0;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int c = 2 * h + e;
                    const float yr = se * fmaf(d2[0][c], 1.f / 2048.f, d1[0][c]);
                    const float yi = se * fmaf(d2[1][c], 1.f / 2048.f, d1[1][c]);
                    out_rec[(2 * q + e) * kTcStageOutRec + g + 8 * h] = make_float2(yr, yi);
                }
            }
            __syncwarp();
            if ((lane >> 3) == G) {
                const float2 *src = out_rec + (lane & 7) * kTcStageOutRec;
#pragma unroll
                for (int k = 0; k < 16; ++k) v[k] = src[k];
            }
            __syncwarp();
        }
    }
};


// ---------------------------------------------------------------------------
// The same split-FP16 radix-16 butterfly on the 5th-generation tensor cores:
// tcgen05.mma with operands in shared memory and accumulators in TMEM.
//
// Per group of 128 threads (one butterfly each) and per stage:
//   A = the group's 128 butterflies as rows, K = 32 (16 re, 16 im) halves,
//       once as x_hi and once as x_lo, in the K-major canonical layout
//       (core matrices of 8 rows x 16 bytes; K-adjacent cores 128 bytes
//       apart, 8-row groups 512 bytes apart);
//   B = the 32 x 32 real DFT-16 matrix [[Wr,-Wi],[Wi,Wr]] split hi/lo,
//       rows = outputs, K-major, built once per CTA from the FP64 table;
//   D1 = A_hi B_hi^T, D2 = A_lo B_hi^T + A_hi B_lo^T in TMEM (32 columns
//       each; M = 128, N = 32, K = 16 per instruction, 6 instructions),
// issued by one thread, committed to the group's mbarrier; then every
// thread reads its own row (lane) of D1 and D2 with tcgen05.ld and forms
// y = s (D1 + 2^-11 D2).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr) {
    // start >> 4 | LBO (K-adjacent cores: 128 B) | SBO (8-row groups: 512 B) | version 1
    return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(512 >> 4) << 32) |
           ((uint64_t)1 << 46);
}
// kind::f16, D = F32, A = B = F16, both K-major, N = 32, M = 128
constexpr uint32_t kUmmaIdesc = (1u << 4) | ((32u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ void umma_f16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(kUmmaIdesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
}

constexpr int kTcgGroupStage = 2 * 128 * 64;  // A_hi + A_lo of one 128-thread group (bytes)

struct TcgPolicy {
    using T = float2;
    static constexpr bool kUsesTwiddles = true;
    unsigned char *bmat;   // B_hi at bmat, B_lo at bmat + 2048
    unsigned char *astage; // this group's A_hi (8 KiB) then A_lo (8 KiB)
    uint64_t *bar;         // this group's mbarrier
    uint32_t tmem;         // this group's first accumulator column (lane field 0)
    int *status;
    mutable uint32_t phase;

    // layout: [B: 4 KiB][mbarriers: 16 x 8 B][TMEM base: 16 B][A staging: groups x 16 KiB]
    static constexpr size_t stage_bytes(int threads) {
        return 4096 + 128 + 16 + (size_t)(threads / 128) * kTcgGroupStage;
    }
    static constexpr int tmem_cols(int threads) {
        return (threads / 128) * 64 <= 32 ? 32 : (threads / 128) * 64 <= 64 ? 64 : (threads / 128) * 64 <= 128 ? 128 : 256;
    }

    // Per-CTA set-up; every thread of the CTA must call it (it synchronises).
    __device__ void init(const __half *__restrict__ table, unsigned char *base, int *status_word) {
        const int t = threadIdx.x;
        const int nthreads = blockDim.x;
        status = status_word;
        bmat = base;
        bar = reinterpret_cast<uint64_t *>(base + 4096) + (t >> 7);
        uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(base + 4096 + 128);
        astage = base + 4096 + 128 + 16 + (t >> 7) * kTcgGroupStage;
        phase = 0;
        // B = [[Wr, -Wi], [Wi, Wr]] (rows n = outputs re 0-15 / im 16-31,
        // columns k = inputs re 0-15 / im 16-31), hi then lo
        for (int idx = t; idx < 2 * 32 * 32; idx += nthreads) {
            const int part = idx >> 10;  // 0 hi, 1 lo
            const int n = (idx >> 5) & 31, k = idx & 31;
            const int kr = k & 15, nr = n & 15;
            const bool wr = (n < 16) == (k < 16);
            __half h = table[(wr ? 0 : 2) * 256 + part * 256 + nr * 16 + kr];
            if (n < 16 && k >= 16) h = __hneg(h);
            *reinterpret_cast<__half *>(base + part * 2048 + (n >> 3) * 512 + (k >> 3) * 128 + (n & 7) * 16 +
                                        (k & 7) * 2) = h;
        }
        if (t < 32) {
            const int cols = tmem_cols(nthreads);
            asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                         "r"(cols)
                         : "memory");
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
        }
        if (t == 0) {
            for (int g = 0; g < nthreads / 128; ++g)
                mbar_init(reinterpret_cast<uint64_t *>(base + 4096) + g, 1);
            fence_mbar_init();
        }
        fence_proxy_async_smem();
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        tmem = *tmem_slot + (uint32_t)((t >> 7) * 64);
    }

    // Per-CTA tear-down: every thread calls it; frees the TMEM columns.
    __device__ void finish() {
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (threadIdx.x < 32) {
            const uint32_t base_col = tmem - (uint32_t)((threadIdx.x >> 7) * 64);
            asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(base_col),
                         "r"(tmem_cols(blockDim.x))
                         : "memory");
        }
    }

    template <int R>
    __device__ __forceinline__ void butterfly(float2 *a) const {
        if constexpr (R == 16)
            tc_dft16(a);
        else
            dft<R>(a);
    }
    __device__ __forceinline__ float2 twiddle(float2 a, float2 w) const { return cmul(a, w); }

    // The calling thread's length-16 DFT; every thread of the CTA must call it.
    __device__ __forceinline__ void tc_dft16(float2 *v) const {
        const int r = threadIdx.x & 127;
        float m = 0.f;
#pragma unroll
        for (int k = 0; k < 16; ++k) m = fmaxf(m, fmaxf(fabsf(v[k].x), fabsf(v[k].y)));
        const int eb = (__float_as_int(m) >> 23) & 0xff;
        const float s = __int_as_float((eb + 1) << 23);
        const float inv_s = __int_as_float((253 - eb) << 23);
        // row r of A_hi / A_lo: 4 core-matrix chunks of 8 halves (re 0-7, re 8-15, im 0-7, im 8-15)
        unsigned char *row_hi = astage + (r >> 3) * 512 + (r & 7) * 16;
        unsigned char *row_lo = row_hi + 8192;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            uint32_t wh[4], wl[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int k0 = (c & 1) * 8 + 2 * q;
                const float x0 = ((c & 2) ? v[k0].y : v[k0].x) * inv_s;
                const float x1 = ((c & 2) ? v[k0 + 1].y : v[k0 + 1].x) * inv_s;
                const __half2 h = __floats2half2_rn(x0, x1);
                const float2 hf = __half22float2(h);
                wh[q] = h2bits(h);
                wl[q] = h2bits(__floats2half2_rn((x0 - hf.x) * 2048.f, (x1 - hf.y) * 2048.f));
            }
            *reinterpret_cast<uint4 *>(row_hi + c * 128) = make_uint4(wh[0], wh[1], wh[2], wh[3]);
            *reinterpret_cast<uint4 *>(row_lo + c * 128) = make_uint4(wl[0], wl[1], wl[2], wl[3]);
        }
        fence_proxy_async_smem();  // generic-proxy writes -> visible to the tensor core
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (r == 0) {
            const uint32_t a_hi = smem_u32(astage), a_lo = a_hi + 8192;
            const uint32_t b_hi = smem_u32(bmat), b_lo = b_hi + 2048;
#pragma unroll
            for (int ks = 0; ks < 2; ++ks) {  // K = 32 as two K = 16 steps (two core chunks each)
                umma_f16(tmem, umma_desc(a_hi + ks * 256), umma_desc(b_hi + ks * 256), ks);
                umma_f16(tmem + 32, umma_desc(a_lo + ks * 256), umma_desc(b_hi + ks * 256), ks);
                umma_f16(tmem + 32, umma_desc(a_hi + ks * 256), umma_desc(b_lo + ks * 256), 1);
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(bar))
                         : "memory");
        }
        if (!mbar_wait_bounded(bar, phase)) record_status(status, kStatusTimeout);
        phase ^= 1;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t lane = (uint32_t)((threadIdx.x & 96)) << 16;  // this warp's 32 TMEM lanes
        uint32_t d1[32], d2[32];
        tmem_ld32(tmem + lane, d1);
        tmem_ld32(tmem + 32 + lane, d2);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const float yr = s * fmaf(__int_as_float(d2[k]), 1.f / 2048.f, __int_as_float(d1[k]));
            const float yi = s * fmaf(__int_as_float(d2[16 + k]), 1.f / 2048.f, __int_as_float(d1[16 + k]));
            v[k] = make_float2(yr, yi);
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    }
};

// ---------------------------------------------------------------------------
// Row pass (E = 16), optional column pre-split P = 2: the FP32 row kernel's
// structure with the tensor-core butterfly.
// ---------------------------------------------------------------------------
template <int N, class Pol>
struct TcRowShape {
    static constexpr int E = N >= 16 ? 16 : N;
    static constexpr int T = N / E;
    static constexpr int ROWS = (T >= 256) ? 1 : 256 / T;
    static constexpr int THREADS = ROWS * T;
    using Eng = Engine<N, E, 1, PadShift<E>::value>;
    static constexpr size_t EX_BYTES = sizeof(float2) * (size_t)ROWS * Eng::SMEM_ELEMS;
    static constexpr size_t STAGE_OFF = (EX_BYTES + 1023) / 1024 * 1024;
    static constexpr size_t SMEM = STAGE_OFF + Pol::stage_bytes(THREADS);
};

// 256-thread CTAs are held to 128 registers so two fit an SM (the kernel
// waits on its MMA groups and needs the second CTA's warps to cover them);
// 512-thread CTAs would spill at 64 and stay one per SM
template <int N, int P, class Pol>
__global__ void __launch_bounds__(TcRowShape<N, Pol>::THREADS, TcRowShape<N, Pol>::THREADS <= 256 ? 2 : 1)
    k_rows_tc(const float2 *__restrict__ in, float2 *out, const float2 *__restrict__ tw,
              const float2 *__restrict__ twp, const __half *__restrict__ w16, long long nrows, int ny, int conj_in,
              int conj_out, int *status) {
    using Sh = TcRowShape<N, Pol>;
    using Eng = typename Sh::Eng;
    constexpr int E = Sh::E;
    constexpr int T = Sh::T;
    constexpr int R0 = Eng::R0;
    extern __shared__ __align__(1024) unsigned char raw[];
    float2 *smem = reinterpret_cast<float2 *>(raw);
    Pol pol;
    pol.init(w16, raw + Sh::STAGE_OFF, status);
    const int g = threadIdx.x / T;
    const int tt = threadIdx.x - g * T;
    const long long row = (long long)blockIdx.x * Sh::ROWS + g;
    const bool active = row < nrows;
    const float si = conj_in ? -1.f : 1.f;
    const float so = conj_out ? -1.f : 1.f;
    const int Q = ny / P;
    int kp = 0, q = 0;
    long long in0 = row;
    if constexpr (P > 1) {
        const long long b = active ? row / ny : 0;
        const int y = active ? (int)(row - b * ny) : 0;
        kp = y % P;
        q = y / P;
        in0 = b * ny + q;
    }
    float2 v[E];
#pragma unroll
    for (int b = 0; b < E / R0; ++b) {
        const int j = tt + b * T;
#pragma unroll
        for (int r = 0; r < R0; ++r) {
            const int i = j + r * (N / R0);
            float2 x = active ? __ldg(in + in0 * N + i) : make_float2(0.f, 0.f);
            x.y *= si;
            if constexpr (P == 2) {
                float2 y = active ? __ldg(in + (in0 + Q) * N + i) : make_float2(0.f, 0.f);
                y.y *= si;
                x = kp ? csub(x, y) : cadd(x, y);
            }
            v[b * R0 + r] = x;
        }
    }
    if constexpr (P == 2) {
        if (kp) {
            const float2 w = __ldg(twp + q);
#pragma unroll
            for (int k = 0; k < E; ++k) v[k] = cmul(v[k], w);
        }
    }
    float2 *dst = out + row * N;
    auto store = [&](int i, int, float2 x) {
        if (active) {
            x.y *= so;
            dst[i] = x;
        }
    };
    auto none = [] {};
    if constexpr (Eng::NT >= 32)
        Eng::template run_with<Pol, false>(pol, v, smem + g * Eng::SMEM_ELEMS, tw, tt, 0, SyncBlock{}, none, store);
    else
        Eng::template run_with<Pol, false>(pol, v, smem + g * Eng::SMEM_ELEMS, tw, tt, 0, SyncWarp{}, none, store);
    pol.finish();
}

// ---------------------------------------------------------------------------
// Column pass (E = 16): the TMA-staged persistent column kernel with the
// tensor-core butterfly.
// ---------------------------------------------------------------------------
template <int N, int W, class Pol>
struct TcColShape {
    static constexpr int E = N >= 16 ? 16 : N;
    static constexpr int T = N / E;
    static constexpr int THREADS = T * W;
    using Eng = Engine<N, E, W, PadShift<E>::value>;
    static constexpr int ELEMS = Eng::SMEM_ELEMS > N * W ? Eng::SMEM_ELEMS : N * W;
    static constexpr int BOXR = N < 256 ? N : 256;
    static constexpr uint32_t TILE_BYTES = (uint32_t)N * W * sizeof(float2);
    static constexpr size_t BAR_OFF = ((size_t)ELEMS * sizeof(float2) + 127) / 128 * 128;
    static constexpr size_t STAGE_OFF = (BAR_OFF + 128 + 1023) / 1024 * 1024;
    static constexpr size_t SMEM = STAGE_OFF + Pol::stage_bytes(THREADS);
};

template <int N, int W, class Pol>
__global__ void __launch_bounds__(TcColShape<N, W, Pol>::THREADS, 1)
    k_cols_tc(const __grid_constant__ CUtensorMap map, float2 *out, const float2 *__restrict__ tw,
              const __half *__restrict__ w16, int nx, int batch, int P, int conj_out, int *status) {
    using Sh = TcColShape<N, W, Pol>;
    using Eng = typename Sh::Eng;
    constexpr int E = Sh::E;
    constexpr int R0 = Eng::R0;
    constexpr int T = Sh::T;
    extern __shared__ __align__(1024) unsigned char raw[];
    float2 *tile = reinterpret_cast<float2 *>(raw);
    uint64_t *bar = reinterpret_cast<uint64_t *>(raw + Sh::BAR_OFF);
    __shared__ int s_ok;
    Pol pol;
    pol.init(w16, raw + Sh::STAGE_OFF, status);

    const int t = threadIdx.x;
    const int c = t % W;
    const int tt = t / W;
    const int groups_x = nx / W;
    const long long ntiles = (long long)groups_x * P * batch;
    const float so = conj_out ? -1.f : 1.f;
    auto tile_x = [&](long long id) { return (int)(id % groups_x) * 2 * W; };
    auto tile_kp = [&](long long id) { return (int)((id / groups_x) % P); };
    auto tile_z = [&](long long id) { return (int)((id / groups_x) / P) * N; };
    auto issue = [&](long long id) {
        const int x = tile_x(id), kp = tile_kp(id), z0 = tile_z(id);
        mbar_expect_tx(bar, Sh::TILE_BYTES);
#pragma unroll 1
        for (int k = 0; k < N / Sh::BOXR; ++k)
            tma_load_3d(tile + k * Sh::BOXR * W, &map, x, kp, z0 + k * Sh::BOXR, bar);
    };
    if (t == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
        fence_proxy_async_smem();
    }
    __syncthreads();
    long long id = blockIdx.x;
    uint32_t phase = 0;
    if (t == 0 && id < ntiles) issue(id);
    for (; id < ntiles; id += gridDim.x) {
        if (t == 0) s_ok = mbar_wait_bounded(bar, phase) ? 1 : 0;
        __syncthreads();
        if (!s_ok) {
            if (t == 0) {
                record_status(status, kStatusTimeout);
                mbar_wait_bounded(bar, phase);
            }
            break;  // leave through finish(): the TMEM columns must be freed
        }
        phase ^= 1;
        const long long next = id + gridDim.x;
        const long long blk = id / groups_x;
        const long long b = blk / P;
        const int kp = (int)(blk - b * P);
        float2 *dst = out + (b * N * P + kp) * (long long)nx + (long long)(id % groups_x) * W;
        const long long rstride = (long long)P * nx;
        float2 v[E];
#pragma unroll
        for (int bb = 0; bb < E / R0; ++bb) {
            const int j = tt + bb * T;
#pragma unroll
            for (int r = 0; r < R0; ++r) v[bb * R0 + r] = tile[(j + r * (N / R0)) * W + c];
        }
        auto after_reads = [&] {
            __syncthreads();
            if (t == 0 && next < ntiles) {
                fence_proxy_async_smem();
                issue(next);
            }
        };
        auto store = [&](int i, int cc, float2 x) {
            x.y *= so;
            dst[(long long)i * rstride + cc] = x;
        };
        Eng::template run_with<Pol, true>(pol, v, tile, tw, tt, c, SyncBlock{}, after_reads, store);
    }
    pol.finish();
}

// ---------------------------------------------------------------------------
// Variant tables and launchers.
// ---------------------------------------------------------------------------
namespace {
// [policy: 0 mma.sync, 1 tcgen05]
struct TcRowEntry {
    const void *fn[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};  // [policy][P == 2]
    int threads = 0, rows_per_cta = 0;
    size_t smem[2] = {0, 0};
};
struct TcColEntry {
    const void *fn[2] = {nullptr, nullptr};
    int threads = 0, w = 0, box_rows = 0;
    size_t smem[2] = {0, 0};
};
TcRowEntry g_tc_rows[kMaxLog2 + 1];
TcColEntry g_tc_cols[kMaxLog2 + 1][5];  // W slot: 2, 4, 8, 16, 32
std::once_flag g_tc_once;  // registry filled once, safe across host threads

int tc_w_slot(int w) { return w == 2 ? 0 : w == 4 ? 1 : w == 8 ? 2 : w == 16 ? 3 : w == 32 ? 4 : -1; }

template <int N>
void reg_tc_row() {
    using Sh0 = TcRowShape<N, TcPolicy>;
    using Sh1 = TcRowShape<N, TcgPolicy>;
    TcRowEntry &en = g_tc_rows[ilog2(N)];
    en.fn[0][0] = (const void *)k_rows_tc<N, 1, TcPolicy>;
    en.fn[0][1] = (const void *)k_rows_tc<N, 2, TcPolicy>;
    if constexpr (Sh1::THREADS % 128 == 0) {
        en.fn[1][0] = (const void *)k_rows_tc<N, 1, TcgPolicy>;
        en.fn[1][1] = (const void *)k_rows_tc<N, 2, TcgPolicy>;
    }
    en.threads = Sh0::THREADS;
    en.rows_per_cta = Sh0::ROWS;
    en.smem[0] = Sh0::SMEM;
    en.smem[1] = Sh1::SMEM;
}
template <int N, int W>
void reg_tc_col() {
    using Sh0 = TcColShape<N, W, TcPolicy>;
    using Sh1 = TcColShape<N, W, TcgPolicy>;
    TcColEntry &en = g_tc_cols[ilog2(N)][tc_w_slot(W)];
    en.fn[0] = (const void *)k_cols_tc<N, W, TcPolicy>;
    if constexpr (Sh1::THREADS % 128 == 0 && Sh1::SMEM <= 227 * 1024) en.fn[1] = (const void *)k_cols_tc<N, W, TcgPolicy>;
    en.threads = Sh0::THREADS;
    en.w = W;
    en.box_rows = Sh0::BOXR;
    en.smem[0] = Sh0::SMEM;
    en.smem[1] = Sh1::SMEM;
}
template <int N>
void reg_tc_cols() {
    // widths with 32..1024 threads per CTA and at most a 128 KiB tile
    if constexpr (N * 2 <= 16384 && (N / 16) * 2 >= 32) reg_tc_col<N, 2>();
    if constexpr (N * 4 <= 16384 && (N / 16) * 4 >= 32 && (N / 16) * 4 <= 1024) reg_tc_col<N, 4>();
    if constexpr (N * 8 <= 16384 && (N / 16) * 8 >= 32 && (N / 16) * 8 <= 1024) reg_tc_col<N, 8>();
    if constexpr (N * 16 <= 16384 && (N / 16) * 16 >= 32 && (N / 16) * 16 <= 1024) reg_tc_col<N, 16>();
    if constexpr (N * 32 <= 16384 && (N / 16) * 32 >= 32 && (N / 16) * 32 <= 1024) reg_tc_col<N, 32>();
}
void init_tc() {
    std::call_once(g_tc_once, [] {
        reg_tc_row<16>();
        reg_tc_row<32>();
        reg_tc_row<64>();
        reg_tc_row<128>();
        reg_tc_row<256>();
        reg_tc_row<512>();
        reg_tc_row<1024>();
        reg_tc_row<2048>();
        reg_tc_row<4096>();
        reg_tc_row<8192>();
        reg_tc_cols<16>();
        reg_tc_cols<32>();
        reg_tc_cols<64>();
        reg_tc_cols<128>();
        reg_tc_cols<256>();
        reg_tc_cols<512>();
        reg_tc_cols<1024>();
        reg_tc_cols<2048>();
        reg_tc_cols<4096>();
        reg_tc_cols<8192>();
    });
}
}  // namespace

bool tc_rows_available(int n) {
    init_tc();
    return n >= 16 && n <= 8192 && (n & (n - 1)) == 0 && g_tc_rows[ilog2(n)].fn[0][0] != nullptr;
}

// Column tile for length n with at most nx columns: the widest one with at
// most 512 threads (the tensor-core butterfly needs many registers), else the
// narrowest available.
int tc_col_width(int n, int nx) {
    init_tc();
    if (n < 16 || n > 8192 || (n & (n - 1))) return 0;
    int best = 0;
    for (int w = 2; w <= 32 && w <= nx; w <<= 1) {
        const TcColEntry &en = g_tc_cols[ilog2(n)][tc_w_slot(w)];
        if (!en.fn[0]) continue;
        if (en.threads <= 512 || best == 0) best = w;
    }
    return best;
}

int tc_col_box_rows(int n) { return n < 256 ? n : 256; }

// Whether the tcgen05 kernels exist for this row length / column shape.
bool tcg_available(int rown, int coln, int colw) {
    init_tc();
    if (!g_tc_rows[ilog2(rown)].fn[1][0]) return false;
    if (coln > 1 && (tc_w_slot(colw) < 0 || !g_tc_cols[ilog2(coln)][tc_w_slot(colw)].fn[1])) return false;
    return true;
}

cudaError_t launch_rows_tc(int n, int tcg, const float2 *in, float2 *out, const float2 *tw, const float2 *twp,
                           const void *w16, long long nrows, int ny, int split, int conj_in, int conj_out, int *status,
                           cudaStream_t s) {
    init_tc();
    if (!tc_rows_available(n) || (split != 1 && split != 2)) return cudaErrorInvalidValue;
    if (nrows <= 0) return cudaSuccess;
    const TcRowEntry &en = g_tc_rows[ilog2(n)];
    const int pk = tcg ? 1 : 0;
    const void *fn = en.fn[pk][split == 2 ? 1 : 0];
    if (!fn) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)en.smem[pk]);
    if (e != cudaSuccess) return e;
    const long long grid = (nrows + en.rows_per_cta - 1) / en.rows_per_cta;
    const __half *w = static_cast<const __half *>(w16);
    void *args[] = {(void *)&in,    (void *)&out, (void *)&tw,      (void *)&twp,      (void *)&w,
                    (void *)&nrows, (void *)&ny,  (void *)&conj_in, (void *)&conj_out, (void *)&status};
    return cudaLaunchKernel(fn, dim3((unsigned)grid), dim3(en.threads), args, en.smem[pk], s);
}

int tc_cols_grid(int n, int w, int tcg, long long ntiles, int num_sms) {
    init_tc();
    const int slot = tc_w_slot(w);
    if (slot < 0 || !g_tc_cols[ilog2(n)][slot].fn[tcg ? 1 : 0]) return 0;
    const TcColEntry &en = g_tc_cols[ilog2(n)][slot];
    const void *fn = en.fn[tcg ? 1 : 0];
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)en.smem[tcg ? 1 : 0]);
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, en.threads, en.smem[tcg ? 1 : 0]) != cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    long long grid = (long long)num_sms * per_sm;
    if (grid > ntiles) grid = ntiles;
    return grid < 1 ? 1 : (int)grid;
}

cudaError_t launch_cols_tc(int n, int w, int tcg, const CUtensorMap &map, float2 *out, const float2 *tw,
                           const void *w16, int nx, int batch, int split, int conj_out, int *status, int grid,
                           cudaStream_t s) {
    init_tc();
    const int slot = tc_w_slot(w);
    const int pk = tcg ? 1 : 0;
    if (slot < 0 || !g_tc_cols[ilog2(n)][slot].fn[pk]) return cudaErrorInvalidValue;
    const TcColEntry &en = g_tc_cols[ilog2(n)][slot];
    cudaError_t e = cudaFuncSetAttribute(en.fn[pk], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)en.smem[pk]);
    if (e != cudaSuccess) return e;
    CUtensorMap m = map;
    const __half *wt = static_cast<const __half *>(w16);
    void *args[] = {(void *)&m,     (void *)&out,   (void *)&tw,       (void *)&wt,     (void *)&nx,
                    (void *)&batch, (void *)&split, (void *)&conj_out, (void *)&status};
    return cudaLaunchKernel(en.fn[pk], dim3(grid), dim3(en.threads), args, en.smem[pk], s);
}

}  // namespace gb300fft
