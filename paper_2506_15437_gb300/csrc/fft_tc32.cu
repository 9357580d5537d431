// Split-FP16 tensor-core form with radix-32 stages on tcgen05.
//
// Every radix-32 butterfly of the Stockham engine (Section 2.2's butterflies,
// 32 points at a time) is the product y = W32 x with W32[k][r] =
// exp(-2*pi*i*k*r/32).  In real arithmetic, x = (xr, xi) stacked as a
// 64-vector, y = B x with the 64 x 64 matrix B = [[Wr, -Wi], [Wi, Wr]].  B is
// split once, in FP64, as B = B_hi + B_lo (both float16; B_lo holds the
// rounding error of B_hi unscaled).  Each butterfly is scaled by 2048 / s, s
// the power of two just above its largest |component|, so every scaled value
// has |xs| < 2048, and split as xs = hi + lo: hi keeps the top 11 significant
// bits of xs (mask of the float32 mantissa, exact in float16), lo = xs - hi
// (exact in float32, rounded once to float16).  Three products are kept,
// B_hi hi, B_hi lo and B_lo hi, accumulated in float32 (after Ootomo &
// Yokota's error-corrected tensor-core GEMM; B_lo lo is below 2^-21
// relative), the small corrections first.
//
// One 128-thread group holds 128 butterflies, one per thread and one per row
// of A.  Default (A in TMEM): each thread writes its row's hi / lo halves into
// its TMEM lane, and B is the even/odd table -- two 32 x 32 diagonal blocks,
// E_k = sum_m W16^(km) x_{2m} and O_k = sum_m W32^(k(2m+1)) x_{2m+1} -- so the
// product is 12 tcgen05.mma of M = 128, N = 32, K = 16 (kind::f16, f32
// accumulate) into one accumulator, issued by one thread and committed to
// the group's mbarrier, and y_k = E_k + O_k, y_{k+16} = E_k - O_k are formed
// in float32 on the way out of TMEM.  With A staged in shared memory (the
// stage's exchange, whose reads are complete by then) the full table and two
// accumulators are used instead.  A 8192-point transform is radix 8 (float32)
// + two radix-32 tensor-core stages; 4096 is 4 + 32 + 32, 2048 is 2 + 32 +
// 32, 1024 is 32 + 32.
#include <mutex>

#include "fft_internal.h"
#include "fft_tc32.cuh"

namespace gb300fft {

// Two B tables, each B_hi then B_lo (64 x 64 float16) in the canonical
// K-major layout of the tensor-core descriptors: element (n, k) at byte
// (n/8)*1024 + (k/8)*128 + (n%8)*16 + (k%8)*2.  Built in FP64 once per plan.
//   Table 0, the full real form of W32: [[Wr, -Wi], [Wi, Wr]], rows 0-31 the
//   real outputs, 32-63 the imaginary; columns 0-31 Re x, 32-63 Im x.
//   Table 1, the even/odd form: y_k = E_k + O_k, y_{k+16} = E_k - O_k (k < 16)
//   with E_k = sum_m W16^(k m) x_{2m} and O_k = sum_m W32^(k (2m+1)) x_{2m+1}:
//   block-diagonal, rows 0-15 Re E, 16-31 Im E, 32-47 Re O, 48-63 Im O;
//   columns 0-15 Re x_even, 16-31 Im x_even, 32-47 Re x_odd, 48-63 Im x_odd.
__global__ void k_w32_table(__half *t) {
    const int gidx = blockIdx.x * blockDim.x + threadIdx.x;  // 2 x 4096 entries
    if (gidx >= 2 * 64 * 64) return;
    const int table = gidx >> 12, idx = gidx & 4095;
    const int n = idx >> 6, k = idx & 63;
    double b = 0.0;
    if (table == 0) {
        const int kr = k & 31, nr = n & 31;
        double sv, cv;
        sincospi(2.0 * (double)((nr * kr) & 31) / 32.0, &sv, &cv);
        const double wr = cv, wi = -sv;
        b = (n < 32) ? (k < 32 ? wr : -wi) : (k < 32 ? wi : wr);
    } else if ((n < 32) == (k < 32)) {  // the two diagonal blocks
        const int odd = n >= 32;
        const int nq = n & 15, mq = k & 15;           // output k', input m
        const int nim = (n >> 4) & 1, kim = (k >> 4) & 1;  // imaginary row / column
        const int a = odd ? (nq * (2 * mq + 1)) & 31 : (2 * nq * mq) & 31;  // angle in units of 2 pi / 32
        double sv, cv;
        sincospi(2.0 * (double)a / 32.0, &sv, &cv);
        const double wr = cv, wi = -sv;
        b = nim == 0 ? (kim == 0 ? wr : -wi) : (kim == 0 ? wi : wr);
    }
    const __half hi = __double2half(b);
    const __half lo = __double2half(b - (double)__half2float(hi));
    const int off = ((n >> 3) * 1024 + (k >> 3) * 128 + (n & 7) * 16 + (k & 7) * 2) / 2;
    __half *tb = t + table * kT32BBytes;  // kT32BBytes halves = two 8 KiB operands
    tb[off] = hi;
    tb[kT32BBytes / 2 + off] = lo;
}

cudaError_t build_w32_table(void *t, cudaStream_t s) {
    k_w32_table<<<32, 256, 0, s>>>(static_cast<__half *>(t));
    return cudaGetLastError();
}

// Per-CTA tensor-core state of the radix-32 butterflies.  TA: the A operand
// lives in tensor memory (each thread writes its own row with tcgen05.st;
// one accumulator D = B_hi hi + B_hi lo + B_lo hi), so the stage needs no
// shared-memory staging at all; otherwise A is staged in shared memory (the
// caller's exchange) and the two products accumulate separately.
// TMEM columns of a group: [0, 64) D (D1), [64, 96) A_hi or D2, [96, 128) A_lo.
template <bool TA>
struct Tc32 {
    unsigned char *bsm;    // B_hi, B_lo (16 KiB) in shared memory
    unsigned char *stage;  // this group's A_hi (16 KiB) then A_lo (16 KiB)
    uint64_t *bar;         // this group's mbarrier
    uint32_t tmem;         // this group's D1 column (D2 = +64), lane field 0
    int *status;
    uint32_t phase;
    int group, row;        // group index, row of A (thread within the group)

    // Every thread of the CTA calls init (it synchronises).  `bsrc` is the
    // global B table, `bsm_p` 16 KiB of shared memory, `bars` one mbarrier
    // per group, `slot` a shared word for the TMEM base, `stage_base` the
    // (exchange) memory the groups stage A in, 32 KiB per group.
    __device__ void init(const __half *__restrict__ bsrc, unsigned char *bsm_p, uint64_t *bars, uint32_t *slot,
                         unsigned char *stage_base, int *status_word) {
        const int t = threadIdx.x;
        const int ngroups = blockDim.x / kT32Group;
        status = status_word;
        bsm = bsm_p;
        group = t / kT32Group;
        row = t % kT32Group;
        bar = bars + group;
        stage = stage_base + (size_t)group * kT32GroupStage;
        phase = 0;
        // the A-in-TMEM form multiplies by the even/odd table (the second one)
        const uint4 *src = reinterpret_cast<const uint4 *>(bsrc + (TA ? kT32BBytes : 0));
        uint4 *dst = reinterpret_cast<uint4 *>(bsm);
        for (int i = t; i < 2 * kT32BBytes / 16; i += blockDim.x) dst[i] = __ldg(src + i);
        const uint32_t cols = (uint32_t)ngroups * 128;  // 128, 256 or 512: powers of two
        if (t < 32) {
            asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
                         "r"(cols)
                         : "memory");
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
        }
        if (t == 0) {
            for (int g = 0; g < ngroups; ++g) mbar_init(bars + g, 1);
            fence_mbar_init();
        }
        fence_proxy_async_smem();
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        tmem = *slot + (uint32_t)(group * 128);
    }

    // Every thread calls finish once all its tensor-core work is done.
    __device__ void finish() {
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (threadIdx.x < 32) {
            const uint32_t base_col = tmem - (uint32_t)(group * 128);
            asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(base_col),
                         "r"((uint32_t)(blockDim.x / kT32Group) * 128)
                         : "memory");
        }
    }

    // TA form of dft32: split into TMEM, then the even/odd product: 12 MMAs
    // of N = 32 (one accumulator, each diagonal block of the table into its
    // own half of D), and the radix-2 recombination y_k = E_k + O_k,
    // y_{k+16} = E_k - O_k in float32.  Every thread of the group calls it;
    // no CTA barrier, no shared memory.
    __device__ __forceinline__ void dft32_ta(float2 (&v)[kT32E]) {
        float m = 0.f;
#pragma unroll
        for (int k = 0; k < kT32E; ++k) m = fmaxf(m, fmaxf(fabsf(v[k].x), fabsf(v[k].y)));
        int eb = (__float_as_int(m) >> 23) & 0xff;
        eb = eb < 11 ? 11 : eb;
        const float up = __int_as_float((264 - eb) << 23);   // 2048 / s
        const float down = __int_as_float((eb - 10) << 23);  // s / 2048
        const uint32_t lane = (uint32_t)(threadIdx.x & 96) << 16;
        // A row, 16 halves per chunk q: Re x_even, Im x_even, Re x_odd, Im x_odd
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            uint32_t wh[8], wl[8];
#pragma unroll
            for (int p = 0; p < 8; ++p) {
                const int k0 = 4 * p + (q >> 1);  // x_{2j} (q < 2) or x_{2j+1}, j = 2p and 2p + 1
                const float x0 = ((q & 1) ? v[k0].y : v[k0].x) * up;
                const float x1 = ((q & 1) ? v[k0 + 2].y : v[k0 + 2].x) * up;
                const float h0 = __int_as_float(__float_as_int(x0) & 0xFFFFE000);
                const float h1 = __int_as_float(__float_as_int(x1) & 0xFFFFE000);
                wh[p] = f2h2_bits(h0, h1);
                wl[p] = f2h2_bits(x0 - h0, x1 - h1);
            }
            t32_st8(tmem + lane + 64 + 8 * q, wh);
            t32_st8(tmem + lane + 96 + 8 * q, wl);
        }
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        named_sync(1 + group, kT32Group);
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (row == 0) {
            const uint32_t b_hi = smem_u32(bsm), b_lo = b_hi + kT32BBytes;
            // block e (0: even, 1: odd): K steps 2e, 2e + 1 (A columns 16e ..),
            // table rows 32e .. (4 core-matrix groups of 1024 bytes), D
            // columns 32e ..  The small correction products accumulate
            // first, at their own scale; the large B_hi hi terms come last.
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const uint32_t d = tmem + 32 * e, bo = 4096 * e;
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    const int ks = 2 * e + j;
                    t32_mma_ts(d, tmem + 96 + 8 * ks, t32_desc(b_hi + bo + ks * 256), j, kT32IdescN32);
                }
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    const int ks = 2 * e + j;
                    t32_mma_ts(d, tmem + 64 + 8 * ks, t32_desc(b_lo + bo + ks * 256), 1, kT32IdescN32);
                }
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    const int ks = 2 * e + j;
                    t32_mma_ts(d, tmem + 64 + 8 * ks, t32_desc(b_hi + bo + ks * 256), 1, kT32IdescN32);
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(bar))
                         : "memory");
        }
        if (!t32_wait(bar, phase)) record_status(status, kStatusTimeout);
        phase ^= 1;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // D columns: 0-15 Re E, 16-31 Im E, 32-47 Re O, 48-63 Im O (all four
        // loads in flight before the one wait)
        uint32_t d[4][16];
#pragma unroll
        for (int q = 0; q < 4; ++q) t32_ld16(tmem + lane + 16 * q, d[q]);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const float er = __int_as_float(d[0][k]), ei = __int_as_float(d[1][k]);
            const float orr = __int_as_float(d[2][k]), oi = __int_as_float(d[3][k]);
            v[k] = make_float2((er + orr) * down, (ei + oi) * down);
            v[k + 16] = make_float2((er - orr) * down, (ei - oi) * down);
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    }

    // The calling thread's length-32 DFT (forward sign) of v, in place.
    // Every thread of the CTA must call it: it starts with a CTA barrier
    // (the staging area is the exchange the stage has just read).  If `hook`
    // is true, `after_mma()` runs once every group's products are complete
    // (all threads, after a CTA barrier): the staging memory is free again.
    template <class AfterMma>
    __device__ __forceinline__ void dft32(float2 (&v)[kT32E], bool hook, AfterMma after_mma) {
        if constexpr (TA) {
            dft32_ta(v);
            return;
        }
        // scale: s = 2^(eb - 126) > max |component|; xs = x * 2048 / s
        float m = 0.f;
#pragma unroll
        for (int k = 0; k < kT32E; ++k) m = fmaxf(m, fmaxf(fabsf(v[k].x), fabsf(v[k].y)));
        int eb = (__float_as_int(m) >> 23) & 0xff;
        eb = eb < 11 ? 11 : eb;  // keeps both scale factors normal (tiny or zero rows)
        const float up = __int_as_float((264 - eb) << 23);  // 2^(137 - eb) = 2048 / s
        const float down = __int_as_float((eb - 10) << 23);  // 2^(eb - 137) = s / 2048
        __syncthreads();  // every thread has read the exchange: it becomes the staging area
        // row `row` of A_hi / A_lo: 8 chunks of 8 halves (re 0-31, then im 0-31)
        unsigned char *row_hi = stage + (row >> 3) * 1024 + (row & 7) * 16;
        unsigned char *row_lo = row_hi + kT32ABytes;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            uint32_t wh[4], wl[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int k0 = (c & 3) * 8 + 2 * q;
                const float x0 = ((c & 4) ? v[k0].y : v[k0].x) * up;
                const float x1 = ((c & 4) ? v[k0 + 1].y : v[k0 + 1].x) * up;
                const float h0 = __int_as_float(__float_as_int(x0) & 0xFFFFE000);
                const float h1 = __int_as_float(__float_as_int(x1) & 0xFFFFE000);
                wh[q] = f2h2_bits(h0, h1);
                wl[q] = f2h2_bits(x0 - h0, x1 - h1);
            }
            *reinterpret_cast<uint4 *>(row_hi + c * 128) = make_uint4(wh[0], wh[1], wh[2], wh[3]);
            *reinterpret_cast<uint4 *>(row_lo + c * 128) = make_uint4(wl[0], wl[1], wl[2], wl[3]);
        }
        fence_proxy_async_smem();  // generic-proxy writes -> visible to the tensor core
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        named_sync(1 + group, kT32Group);
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (row == 0) {
            const uint32_t a_hi = smem_u32(stage), a_lo = a_hi + kT32ABytes;
            const uint32_t b_hi = smem_u32(bsm), b_lo = b_hi + kT32BBytes;
#pragma unroll
            for (int ks = 0; ks < 4; ++ks) {  // K = 64 as four K = 16 steps (two core chunks each)
                t32_mma(tmem, t32_desc(a_hi + ks * 256), t32_desc(b_hi + ks * 256), ks);
                t32_mma(tmem + 64, t32_desc(a_lo + ks * 256), t32_desc(b_hi + ks * 256), ks);
                t32_mma(tmem + 64, t32_desc(a_hi + ks * 256), t32_desc(b_lo + ks * 256), 1);
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(bar))
                         : "memory");
        }
        if (!t32_wait(bar, phase)) record_status(status, kStatusTimeout);
        phase ^= 1;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (hook) {
            __syncthreads();
            after_mma();
        }
        // this warp's 32 TMEM lanes; columns 0-31 real outputs, 32-63 imaginary
        const uint32_t lane = (uint32_t)(threadIdx.x & 96) << 16;
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            uint32_t d1[16], d2[16];
            t32_ld16(tmem + lane + h * 16, d1);
            t32_ld16(tmem + 64 + lane + h * 16, d2);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                const float y = (__int_as_float(d1[k]) + __int_as_float(d2[k])) * down;
                if (h < 2)
                    v[(h & 1) * 16 + k].x = y;
                else
                    v[(h & 1) * 16 + k].y = y;
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    }
};

// ---------------------------------------------------------------------------
// Row pass: T = N/32 threads per row, 256 threads per CTA (two groups), two
// CTAs per SM (128 registers, 86 KiB of shared memory, 256 TMEM columns
// each), one CTA per row group.  Optional column pre-split P = 2 as in the
// FP32 row pass (the 2-point DFT across rows q and q + ny/2 and the twiddle
// w_ny^q), so the column pass runs on blocks of ny/2 rows.
// ---------------------------------------------------------------------------
template <int N>
struct T32RowShape {
    static constexpr int E = kT32E;
    static constexpr int T = N / E;
    static constexpr int ROWS = 256 / T;
    static constexpr int THREADS = 256;
    using Eng = Engine<N, E, 1, PadShift<E>::value, RowPadShift1<E>::value>;
    static constexpr int R0 = Eng::R0;
    static constexpr int S = Eng::S;
    static constexpr size_t EX_BYTES = sizeof(float2) * (size_t)ROWS * Eng::SMEM_ELEMS;
    static constexpr size_t B_OFF = (EX_BYTES + 1023) / 1024 * 1024;
    static constexpr size_t BAR_OFF = B_OFF + 2 * kT32BBytes;
    static constexpr size_t SMEM = BAR_OFF + 64;
    static_assert(T >= 32 && 256 % T == 0, "rows of 1024..8192 points");
    static_assert(EX_BYTES >= 2 * (size_t)kT32GroupStage, "the exchange holds both groups' A staging");
    static_assert(S >= 2 && (R0 == E || R0 < E), "stage 0 radix");
};

// Barrier over the T threads of one row (row h of the CTA): a named barrier
// (ids 5 and up; 1-4 are the MMA groups'), or the warp for 32-thread rows.
template <int T>
struct RowSync {
    int h;
    __device__ __forceinline__ void operator()() const {
        if constexpr (T == 32)
            __syncwarp();
        else
            named_sync(5 + h, T);
    }
};

// Stages 0 .. S-1 of one N-point row held as v (stage-0 operands, already
// loaded) by thread tt of its row's T threads, exchanging through sm (the
// row's padded span).  first() runs before the first exchange write (a
// barrier when the span may still be read as input).  `sync` orders the
// accesses to the row's own span (a CTA barrier, or one over the row's
// threads when the span is the row's alone).  after_reads() runs, on every
// thread, once the last stage has read its operands from the exchange.
template <int N, bool TA, class First, class Sync, class AfterReads>
__device__ __forceinline__ void t32_row_stages(Tc32<TA> &tc, float2 (&v)[kT32E], float2 *sm, const float2 *tw, int tt,
                                               First first, Sync sync, AfterReads after_reads) {
    using Sh = T32RowShape<N>;
    using Eng = typename Sh::Eng;
    using Sc = Sched<N, kT32E>;
    constexpr int E = kT32E;
    constexpr int T = Sh::T;
    constexpr int R0 = Sh::R0;
    constexpr int S = Sh::S;
    auto none = [] {};
    // stage 0
    if constexpr (R0 == E) {
        tc.dft32(v, false, none);
    } else {
#pragma unroll
        for (int b = 0; b < E / R0; ++b) dft<R0>(&v[b * R0]);
    }
    // stages 1 .. S-1: exchange, twiddles, tensor-core radix-32
#pragma unroll
    for (int s = 1; s < S; ++s) {
        const int Rp = (s == 1) ? R0 : E;
        const int Nsp = Sc::ns(s - 1);
        // the previous staging / exchange reads are done; before the first
        // exchange write, first() orders it after the reads of whatever input
        // the span aliases (a no-op if none)
        if (s == 1) first();
        if (s > 1 || R0 == E) sync();
#pragma unroll
        for (int b = 0; b < E / Rp; ++b) {
            const int j = tt + b * T;
            const int m = j & (Nsp - 1);
#pragma unroll
            for (int k = 0; k < Rp; ++k) sm[Eng::pad_s((j - m) * Rp + m + k * Nsp, s)] = v[b * Rp + k];
        }
        sync();
        const int Ns = Sc::ns(s);
        const int m = tt & (Ns - 1);
#pragma unroll
        for (int r = 0; r < E; ++r) v[r] = sm[Eng::pad_s(tt + r * T, s)];
        if (s == S - 1) after_reads();
        const float4 *tws = reinterpret_cast<const float4 *>(tw + Sc::tw_off(s)) + m;
#pragma unroll
        for (int k = 0; k < E / 2; ++k) {
            const float4 w2 = __ldg(tws + k * Ns);
            v[2 * k + 1] = cmul(v[2 * k + 1], make_float2(w2.x, w2.y));
            if (2 * k + 2 < E) v[2 * k + 2] = cmul(v[2 * k + 2], make_float2(w2.z, w2.w));
        }
        tc.dft32(v, false, none);
    }
}

template <int N, int P, bool TA>
__global__ void __launch_bounds__(256, 2)
    k_rows_tc32(const float2 *__restrict__ in, float2 *out, const float2 *__restrict__ tw,
                const float2 *__restrict__ twp, const __half *__restrict__ w32, long long nrows, int ny, int conj_in,
                int conj_out, int *status) {
    using Sh = T32RowShape<N>;
    using Eng = typename Sh::Eng;
    constexpr int E = kT32E;
    constexpr int T = Sh::T;
    constexpr int R0 = Sh::R0;
    static_assert(P == 1 || P == 2, "pre-split of 1 or 2");
    extern __shared__ __align__(1024) unsigned char raw[];
    float2 *ex = reinterpret_cast<float2 *>(raw);
    uint64_t *bars = reinterpret_cast<uint64_t *>(raw + Sh::BAR_OFF);
    uint32_t *slot = reinterpret_cast<uint32_t *>(raw + Sh::BAR_OFF + 32);
    Tc32<TA> tc;
    tc.init(w32, raw + Sh::B_OFF, bars, slot, raw, status);
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
    t32_row_stages<N, TA>(tc, v, ex + g * Eng::SMEM_ELEMS, tw, tt, [] {}, SyncBlock{}, [] {});
    if (active) {
        float2 *dst = out + row * N;
#pragma unroll
        for (int k = 0; k < E; ++k) {
            float2 x = v[k];
            x.y *= so;
            dst[tt + k * T] = x;
        }
    }
    tc.finish();
}

// ---------------------------------------------------------------------------
// Row pass from landed rows: one persistent 512-thread CTA per SM (four MMA
// groups, all 512 TMEM columns), L = 512 / T output rows per unit.  Compiled
// for the pre-split rows (P = 2); unsplit rows take k_rows_tc32_land1 below.  The unit's
// input rows land in shared memory through bulk copies on one mbarrier (P = 1:
// L consecutive rows, one copy; P = 2: L/2 consecutive pairs q, q + ny/2, two
// copies, each input row crossing HBM once for both of its output rows).
// Output h of the unit is formed by threads [h*T, (h+1)*T) and transformed in
// its own padded span of the same buffer, which the landed rows no longer
// need by then; the next unit's copies start as soon as every thread has read
// its last-stage operands, so they run under the last stage's products and
// the stores.  Arithmetic per output row: the plain tensor-core row pass's.
// ---------------------------------------------------------------------------
template <int N>
struct T32LandShape {
    static constexpr int T = N / kT32E;
    static constexpr int THREADS = 512;
    static constexpr int L = THREADS / T;  // output rows per unit
    using Eng = typename T32RowShape<N>::Eng;
    static constexpr size_t LAND_BYTES = (size_t)L * N * sizeof(float2);
    static constexpr size_t XBYTES = (size_t)L * Eng::SMEM_ELEMS * sizeof(float2);
    static constexpr size_t BUF = XBYTES > LAND_BYTES ? XBYTES : LAND_BYTES;
    static constexpr size_t B_OFF = (BUF + 1023) / 1024 * 1024;
    static constexpr size_t BAR_OFF = B_OFF + 2 * kT32BBytes;  // 4 group barriers, the landing barrier, TMEM slot
    static constexpr size_t SMEM = BAR_OFF + 64;
    static_assert(L >= 2 && L % 2 == 0, "pairs of outputs per unit");
    static_assert(LAND_BYTES < (1u << 20), "one mbarrier transaction count");
};

template <int N, int P>
__global__ void __launch_bounds__(512, 1)
    k_rows_tc32_land(const float2 *__restrict__ in, float2 *out, const float2 *__restrict__ tw,
                     const float2 *__restrict__ twp, const __half *__restrict__ w32, long long nunits, int ny,
                     int conj_in, int conj_out, int perm_t, int perm_g, int *status) {
    using Sh = T32LandShape<N>;
    using Eng = typename Sh::Eng;
    constexpr int E = kT32E;
    constexpr int T = Sh::T;
    constexpr int L = Sh::L;
    constexpr int R0 = T32RowShape<N>::R0;
    static_assert(P == 1 || P == 2, "pre-split of 1 or 2");
    extern __shared__ __align__(1024) unsigned char raw[];
    float2 *land = reinterpret_cast<float2 *>(raw);  // [L][N]
    uint64_t *bars = reinterpret_cast<uint64_t *>(raw + Sh::BAR_OFF);
    uint64_t *lbar = bars + 4;
    uint32_t *slot = reinterpret_cast<uint32_t *>(raw + Sh::BAR_OFF + 48);
    __shared__ int s_ok;
    Tc32<true> tc;
    tc.init(w32, raw + Sh::B_OFF, bars, slot, raw, status);
    const int t = threadIdx.x;
    const int h = t / T;  // output row of the unit
    const int tt = t - h * T;
    const float si = conj_in ? -1.f : 1.f;
    const float so = conj_out ? -1.f : 1.f;
    const int Q = ny / P;
    constexpr int UQ = L / P;        // input rows per copy (P = 2: pairs per unit)
    const int upb = Q / UQ;          // units per slice
    // first input row of unit u's (first) copy
    auto first_row = [&](long long u) -> long long {
        if constexpr (P == 1) return u * L;
        const long long b = u / upb;
        return b * ny + (long long)(u - b * upb) * UQ;
    };
    auto issue = [&](long long u) {  // thread 0: the unit's copies
        const long long r0 = first_row(u);
        mbar_expect_tx(lbar, (uint32_t)Sh::LAND_BYTES);
        constexpr uint32_t CB = (uint32_t)UQ * N * sizeof(float2);
        bulk_load(land, in + r0 * N, CB, lbar);
        if constexpr (P == 2) bulk_load(land + UQ * N, in + (r0 + Q) * N, CB, lbar);
    };
    auto prefetch = [&](long long u) {
        const long long r0 = first_row(u);
        constexpr uint32_t CB = (uint32_t)UQ * N * sizeof(float2);
        bulk_prefetch_l2(in + r0 * N, CB);
        if constexpr (P == 2) bulk_prefetch_l2(in + (r0 + Q) * N, CB);
    };
    if (t == 0) {
        mbar_init(lbar, 1);
        fence_mbar_init();
        fence_proxy_async_smem();
    }
    __syncthreads();
    long long u = blockIdx.x;
    uint32_t phase = 0;
    if (t == 0 && u < nunits) issue(u);
    for (; u < nunits; u += gridDim.x) {
        if (t == 0 && u + gridDim.x < nunits) prefetch(u + gridDim.x);
        if (t == 0) s_ok = mbar_wait_bounded(lbar, phase) ? 1 : 0;
        __syncthreads();
        if (!s_ok) {
            if (t == 0) {
                record_status(status, kStatusTimeout);
                mbar_wait_bounded(lbar, phase);  // give the copies in flight a last chance to land
            }
            break;  // leave through finish(): the TMEM columns must be freed
        }
        phase ^= 1;
        const long long next = u + gridDim.x;
        const long long r0 = first_row(u);
        // output h: P = 1, row r0 + h; P = 2, pair i = h / 2 (rows r0 + i and
        // r0 + i + Q landed at i and UQ + i), kp = h % 2, stored at row
        // (slice) + 2 q + kp with q = (r0 - slice) + i
        const int i = P == 2 ? h >> 1 : h;
        const int kp = P == 2 ? h & 1 : 0;
        float2 v[E];
#pragma unroll
        for (int b = 0; b < E / R0; ++b) {
            const int j = tt + b * T;
#pragma unroll
            for (int r = 0; r < R0; ++r) {
                const int e = j + r * (N / R0);
                float2 x = land[i * N + e];
                x.y *= si;
                if constexpr (P == 2) {
                    float2 y = land[(UQ + i) * N + e];
                    y.y *= si;
                    x = kp ? csub(x, y) : cadd(x, y);
                }
                v[b * R0 + r] = x;
            }
        }
        // output row: element q of column block kp of slice b, stored at
        // block row pos (permuted for the streaming column pass if perm_t:
        // q = j + perm_t r goes to (j / perm_g) perm_g (Q / perm_t) + r perm_g
        // + j % perm_g)
        const long long b = r0 / ny;
        const int q = (int)(r0 - b * ny) + (P == 2 ? i : h);
        if constexpr (P == 2) {
            if (kp) {
                const float2 w = __ldg(twp + q);
#pragma unroll
                for (int k = 0; k < E; ++k) v[k] = cmul(v[k], w);
            }
        }
        int pos = q;
        if (perm_t) {
            const int j = q & (perm_t - 1), r = q / perm_t;
            pos = (j / perm_g) * perm_g * (Q / perm_t) + r * perm_g + (j & (perm_g - 1));
        }
        const long long orow = b * ny + (long long)P * pos + kp;
        auto after_reads = [&] {
            __syncthreads();
            if (t == 0 && next < nunits) {
                fence_proxy_async_smem();
                issue(next);
            }
        };
        t32_row_stages<N, true>(tc, v, land + h * Eng::SMEM_ELEMS, tw, tt, [] { __syncthreads(); }, RowSync<T>{h},
                                after_reads);
        float2 *dst = out + orow * N;
#pragma unroll
        for (int k = 0; k < E; ++k) {
            float2 x = v[k];
            x.y *= so;
            dst[tt + k * T] = x;
        }
    }
    tc.finish();
}

// Unsplit rows from landed rows in independent sub-units: without the
// pre-split no output row needs another row's input, so the CTA's 512 threads
// form K sub-units of U = RS * T threads (RS rows each, U = 128 or 256), each
// with its own landing barrier and its own persistent loop over units of RS
// rows: it lands its rows (one bulk copy per row, into the row's own exchange
// span), transforms them, and starts its next unit's copies once its rows'
// last-stage operands are read.  No barrier spans two sub-units, so their
// tensor-core products and waits interleave instead of running in step.
template <int N>
struct T32Land1Shape {
    static constexpr int T = N / kT32E;
    static constexpr int THREADS = 512;
    static constexpr int L = THREADS / T;                // rows in the CTA
    static constexpr int RS = T >= kT32Group ? 1 : kT32Group / T;  // rows per sub-unit
    static constexpr int U = RS * T;                     // threads per sub-unit
    static constexpr int K = THREADS / U;                // sub-units
    using Eng = typename T32RowShape<N>::Eng;
    static constexpr int SPAN = (Eng::SMEM_ELEMS + 1) / 2 * 2;  // float2 per row span, 16-byte multiple
    static constexpr size_t BUF = (size_t)L * SPAN * sizeof(float2);
    static constexpr size_t B_OFF = (BUF + 1023) / 1024 * 1024;
    static constexpr size_t BAR_OFF = B_OFF + 2 * kT32BBytes;  // [0, 4) MMA groups, [4, 4 + K) landing
    static constexpr size_t SLOT_OFF = BAR_OFF + 8 * (4 + K);
    static constexpr size_t SMEM = SLOT_OFF + 16;
    static_assert(U == 128 || U == 256, "one or two MMA groups per sub-unit");
    static_assert(SPAN >= N, "a span holds a landed row");
};

template <int N>
__global__ void __launch_bounds__(512, 1)
    k_rows_tc32_land1(const float2 *__restrict__ in, float2 *out, const float2 *__restrict__ tw,
                      const __half *__restrict__ w32, long long nrows, int ny, int conj_in, int conj_out, int perm_t,
                      int perm_g, int *status) {
    using Sh = T32Land1Shape<N>;
    constexpr int E = kT32E;
    constexpr int T = Sh::T;
    constexpr int RS = Sh::RS;
    constexpr int U = Sh::U;
    constexpr int K = Sh::K;
    constexpr int R0 = T32RowShape<N>::R0;
    extern __shared__ __align__(1024) unsigned char raw[];
    float2 *spans = reinterpret_cast<float2 *>(raw);  // [L][SPAN]
    uint64_t *bars = reinterpret_cast<uint64_t *>(raw + Sh::BAR_OFF);
    uint32_t *slot = reinterpret_cast<uint32_t *>(raw + Sh::SLOT_OFF);
    __shared__ int s_ok[K];
    Tc32<true> tc;
    tc.init(w32, raw + Sh::B_OFF, bars, slot, raw, status);
    const int t = threadIdx.x;
    const int h = t / T;  // row of the CTA (its span)
    const int tt = t - h * T;
    const int k = t / U;  // sub-unit
    const bool lead = (t % U) == 0;
    uint64_t *lbar = bars + 4 + k;
    const float si = conj_in ? -1.f : 1.f;
    const float so = conj_out ? -1.f : 1.f;
    // the sub-unit's barrier: its MMA group (U = 128) or its row (U = 256)
    auto sub_sync = [&] {
        if constexpr (U == kT32Group)
            named_sync(1 + t / kT32Group, kT32Group);
        else
            named_sync(5 + k, U);
    };
    const long long nsub = nrows / RS;
    const long long stride = (long long)gridDim.x * K;
    auto issue = [&](long long su) {  // lead thread: the RS rows of unit su
        mbar_expect_tx(lbar, (uint32_t)(RS * N * sizeof(float2)));
#pragma unroll
        for (int i = 0; i < RS; ++i)
            bulk_load(spans + (size_t)(k * RS + i) * Sh::SPAN, in + (su * RS + i) * N, N * sizeof(float2), lbar);
    };
    if (t == 0) {
        for (int j = 0; j < K; ++j) mbar_init(bars + 4 + j, 1);
        fence_mbar_init();
        fence_proxy_async_smem();
    }
    __syncthreads();
    long long su = (long long)blockIdx.x * K + k;
    uint32_t phase = 0;
    if (lead && su < nsub) issue(su);
    for (; su < nsub; su += stride) {
        const long long next = su + stride;
        if (lead && next < nsub) bulk_prefetch_l2(in + next * RS * N, RS * N * sizeof(float2));
        if (lead) s_ok[k] = mbar_wait_bounded(lbar, phase) ? 1 : 0;
        sub_sync();
        if (!s_ok[k]) {
            if (lead) {
                record_status(status, kStatusTimeout);
                mbar_wait_bounded(lbar, phase);  // give the copies in flight a last chance to land
            }
            break;  // leave through finish(): the TMEM columns must be freed
        }
        phase ^= 1;
        float2 *sm = spans + (size_t)h * Sh::SPAN;
        float2 v[E];
#pragma unroll
        for (int b = 0; b < E / R0; ++b) {
            const int j = tt + b * T;
#pragma unroll
            for (int r = 0; r < R0; ++r) {
                float2 x = sm[j + r * (N / R0)];
                x.y *= si;
                v[b * R0 + r] = x;
            }
        }
        // output row; with perm_t, row y of slice b goes to block row pos
        // (the streaming column pass's order, as in the pre-split form)
        long long orow = su * RS + (h - k * RS);
        if (perm_t) {
            const long long b = orow / ny;
            const int y = (int)(orow - b * ny);
            const int j = y & (perm_t - 1), r = y / perm_t;
            orow = b * ny + (j / perm_g) * perm_g * (ny / perm_t) + r * perm_g + (j & (perm_g - 1));
        }
        auto after_reads = [&] {
            sub_sync();
            if (lead && next < nsub) {
                fence_proxy_async_smem();
                issue(next);
            }
        };
        // the row's span is its own landed row: a row barrier orders the
        // stage-0 reads before the first exchange write
        t32_row_stages<N, true>(tc, v, sm, tw, tt, RowSync<T>{h}, RowSync<T>{h}, after_reads);
        float2 *dst = out + orow * N;
#pragma unroll
        for (int e = 0; e < E; ++e) {
            float2 x = v[e];
            x.y *= so;
            dst[tt + e * T] = x;
        }
    }
    tc.finish();
}

// ---------------------------------------------------------------------------
// Column pass: tiles of W adjacent columns x N rows staged by TMA (3D map,
// rows P apart), T*W threads = 128, 256 or 512 (one to four groups), one CTA
// per SM, persistent.  The tile buffer is also the exchange and the A staging;
// the next tile's copy starts once the last stage's products are complete.
// ---------------------------------------------------------------------------
template <int N, int W>
struct T32ColShape {
    static constexpr int E = kT32E;
    static constexpr int T = N / E;
    static constexpr int THREADS = T * W;
    static constexpr int GROUPS = THREADS / kT32Group;
    using Sc = Sched<N, E>;
    static constexpr int R0 = Sc::R0;
    static constexpr int S = Sc::S;
    // exchange index swizzle: element i of the [N][W] tile lives at
    // i ^ (((i >> 4) & (16/W - 1)) * W), a permutation within each 16-element
    // group that puts the 16 lanes of every half-warp access on distinct
    // bank pairs for all stage writes and reads (half-warp bank model), so
    // the exchange needs no padding
    static_assert(W >= 2 && W <= 16, "tile widths 2..16");
    __host__ __device__ static constexpr int sw(int i) { return i ^ (((i >> 4) & (16 / W - 1)) * W); }
    static constexpr int ELEMS = N * W;
    static constexpr int BOXR = N < 256 ? N : 256;
    static constexpr uint32_t TILE_BYTES = (uint32_t)N * W * sizeof(float2);
    static constexpr size_t B_OFF = ((size_t)ELEMS * sizeof(float2) + 1023) / 1024 * 1024;
    static constexpr size_t BAR_OFF = B_OFF + 2 * kT32BBytes;
    static constexpr size_t SMEM = BAR_OFF + 64;
    static_assert(THREADS % kT32Group == 0 && THREADS <= 512, "one to four MMA groups");
    static_assert((size_t)ELEMS * sizeof(float2) >= (size_t)GROUPS * kT32GroupStage, "tile holds the staging");
    static_assert(S >= 2, "at least one exchange");
    static_assert(2 * W * sizeof(float) >= 16, "TMA rows of at least 16 bytes");
};

template <int N, int W, bool TA>
__global__ void __launch_bounds__(T32ColShape<N, W>::THREADS, 1)
    k_cols_tc32(const __grid_constant__ CUtensorMap map, float2 *out, const float2 *__restrict__ tw,
                const __half *__restrict__ w32, int nx, int batch, int P, int conj_out, int *status) {
    using Sh = T32ColShape<N, W>;
    using Sc = Sched<N, kT32E>;
    constexpr int E = kT32E;
    constexpr int T = Sh::T;
    constexpr int R0 = Sh::R0;
    constexpr int S = Sh::S;
    extern __shared__ __align__(1024) unsigned char raw[];
    float2 *tile = reinterpret_cast<float2 *>(raw);
    uint64_t *bars = reinterpret_cast<uint64_t *>(raw + Sh::BAR_OFF);  // [0, 4): groups, [4]: tile
    uint32_t *slot = reinterpret_cast<uint32_t *>(raw + Sh::BAR_OFF + 48);
    uint64_t *tbar = bars + 4;
    __shared__ int s_ok;
    Tc32<TA> tc;
    tc.init(w32, raw + Sh::B_OFF, bars, slot, raw, status);

    const int t = threadIdx.x;
    const int c = t % W;
    const int tt = t / W;
    const int groups_x = nx / W;
    const long long ntiles = (long long)groups_x * P * batch;
    const float so = conj_out ? -1.f : 1.f;
    auto issue = [&](long long id) {  // thread 0: TMA loads of tile `id`
        const int x = (int)(id % groups_x) * 2 * W;
        const int kp = (int)((id / groups_x) % P);
        const int z0 = (int)((id / groups_x) / P) * N;
        mbar_expect_tx(tbar, Sh::TILE_BYTES);
#pragma unroll 1
        for (int k = 0; k < N / Sh::BOXR; ++k) tma_load_3d(tile + k * Sh::BOXR * W, &map, x, kp, z0 + k * Sh::BOXR, tbar);
    };
    if (t == 0) {
        mbar_init(tbar, 1);
        fence_mbar_init();
        fence_proxy_async_smem();
    }
    __syncthreads();
    long long id = blockIdx.x;
    uint32_t tphase = 0;
    if (t == 0 && id < ntiles) issue(id);
    for (; id < ntiles; id += gridDim.x) {
        if (t == 0) s_ok = mbar_wait_bounded(tbar, tphase) ? 1 : 0;
        __syncthreads();
        if (!s_ok) {
            if (t == 0) {
                record_status(status, kStatusTimeout);
                mbar_wait_bounded(tbar, tphase);  // give the copy in flight a last chance to land
            }
            break;  // leave through finish(): the TMEM columns must be freed
        }
        tphase ^= 1;
        const long long next = id + gridDim.x;
        const long long blk = id / groups_x;
        const long long b = blk / P;
        const int kp = (int)(blk - b * P);
        float2 v[E];
#pragma unroll
        for (int bb = 0; bb < E / R0; ++bb) {
            const int j = tt + bb * T;
#pragma unroll
            for (int r = 0; r < R0; ++r) v[bb * R0 + r] = tile[(j + r * (N / R0)) * W + c];
        }
        auto next_copy = [&] {  // every group's products are complete: the tile is free
            if (t == 0 && next < ntiles) {
                fence_proxy_async_smem();
                issue(next);
            }
        };
        if constexpr (R0 == E) {
            tc.dft32(v, false, next_copy);
        } else {
#pragma unroll
            for (int bb = 0; bb < E / R0; ++bb) dft<R0>(&v[bb * R0]);
        }
#pragma unroll
        for (int s = 1; s < S; ++s) {
            const int Rp = (s == 1) ? R0 : E;
            const int Nsp = Sc::ns(s - 1);
            __syncthreads();  // tile reads (s = 1) or the previous staging are done
#pragma unroll
            for (int bb = 0; bb < E / Rp; ++bb) {
                const int j = tt + bb * T;
                const int m = j & (Nsp - 1);
#pragma unroll
                for (int k = 0; k < Rp; ++k) tile[Sh::sw(((j - m) * Rp + m + k * Nsp) * W + c)] = v[bb * Rp + k];
            }
            __syncthreads();
            const int Ns = Sc::ns(s);
            const int m = tt & (Ns - 1);
#pragma unroll
            for (int r = 0; r < E; ++r) v[r] = tile[Sh::sw((tt + r * T) * W + c)];
            if constexpr (TA) {
                if (s == S - 1) {  // A goes to tensor memory: the tile is free once every thread has read it
                    __syncthreads();
                    next_copy();
                }
            }
            const float4 *tws = reinterpret_cast<const float4 *>(tw + Sc::tw_off(s)) + m;
#pragma unroll
            for (int k = 0; k < E / 2; ++k) {
                const float4 w2 = __ldg(tws + k * Ns);
                v[2 * k + 1] = cmul(v[2 * k + 1], make_float2(w2.x, w2.y));
                if (2 * k + 2 < E) v[2 * k + 2] = cmul(v[2 * k + 2], make_float2(w2.z, w2.w));
            }
            tc.dft32(v, !TA && s == S - 1, next_copy);
        }
        float2 *dst = out + (b * N * P + kp) * (long long)nx + (long long)(id % groups_x) * W + c;
        const long long rstride = (long long)P * nx;
#pragma unroll
        for (int k = 0; k < E; ++k) {
            float2 x = v[k];
            x.y *= so;
            dst[(long long)(tt + k * T) * rstride] = x;
        }
    }
    tc.finish();
}

// ---------------------------------------------------------------------------
// Variant tables and launchers.
// ---------------------------------------------------------------------------
namespace {
struct T32RowEntry {
    const void *fn[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};  // [A in TMEM][P = 1, 2]
    int rows_per_cta = 0;
    size_t smem = 0;
};
struct T32LandEntry {
    const void *fn2 = nullptr;  // pre-split rows (P = 2), landed in row pairs
    int rows_per_unit = 0;
    size_t smem = 0;
    const void *fn1 = nullptr;  // unsplit rows (P = 1) in independent sub-units
    int rows_per_sub = 0, subs = 0;
    size_t smem1 = 0;
};
struct T32ColEntry {
    const void *fn[2] = {nullptr, nullptr};  // [A in TMEM]
    int threads = 0, w = 0;
    size_t smem = 0;
};
T32RowEntry g_t32_rows[kMaxLog2 + 1];
T32LandEntry g_t32_land[kMaxLog2 + 1];
T32ColEntry g_t32_cols[kMaxLog2 + 1][4];  // W slot: 2, 4, 8, 16
std::once_flag g_t32_once;

int t32_w_slot(int w) { return w == 2 ? 0 : w == 4 ? 1 : w == 8 ? 2 : w == 16 ? 3 : -1; }

template <int N>
void reg_t32_row() {
    using Sh = T32RowShape<N>;
    T32RowEntry &en = g_t32_rows[ilog2(N)];
    en.fn[0][0] = (const void *)k_rows_tc32<N, 1, false>;
    en.fn[0][1] = (const void *)k_rows_tc32<N, 2, false>;
    en.fn[1][0] = (const void *)k_rows_tc32<N, 1, true>;
    en.fn[1][1] = (const void *)k_rows_tc32<N, 2, true>;
    en.rows_per_cta = Sh::ROWS;
    en.smem = Sh::SMEM;
}
template <int N>
void reg_t32_land() {
    using Sh = T32LandShape<N>;
    T32LandEntry &en = g_t32_land[ilog2(N)];
    en.fn2 = (const void *)k_rows_tc32_land<N, 2>;
    en.rows_per_unit = Sh::L;
    en.smem = Sh::SMEM;
    using S1 = T32Land1Shape<N>;
    en.fn1 = (const void *)k_rows_tc32_land1<N>;
    en.rows_per_sub = S1::RS;
    en.subs = S1::K;
    en.smem1 = S1::SMEM;
}
template <int N, int W>
void reg_t32_col() {
    using Sh = T32ColShape<N, W>;
    T32ColEntry &en = g_t32_cols[ilog2(N)][t32_w_slot(W)];
    en.fn[0] = (const void *)k_cols_tc32<N, W, false>;
    en.fn[1] = (const void *)k_cols_tc32<N, W, true>;
    en.threads = Sh::THREADS;
    en.w = W;
    en.smem = Sh::SMEM;
}
void init_t32() {
    std::call_once(g_t32_once, [] {
        reg_t32_row<1024>();
        reg_t32_row<2048>();
        reg_t32_row<4096>();
        reg_t32_row<8192>();
        reg_t32_land<1024>();
        reg_t32_land<2048>();
        reg_t32_land<4096>();
        reg_t32_land<8192>();
        // 512-thread tiles (the split form's rows are at least 16 long, so
        // every 2D shape has nx >= 16 columns to fill them)
        reg_t32_col<1024, 16>();
        reg_t32_col<2048, 8>();
        reg_t32_col<4096, 4>();
        reg_t32_col<8192, 2>();
    });
}
}  // namespace

bool tc32_rows_available(int n) {
    init_t32();
    return n >= 1024 && n <= 8192 && (n & (n - 1)) == 0 && g_t32_rows[ilog2(n)].fn[0][0] != nullptr;
}

// Compile-time layout of the landed tensor-core row kernels (host only):
// kind 0, the pre-split pair form; kind 1, the unsplit sub-unit form.
template <int N>
static void land_layout(int kind, long long *v) {
    if (kind == 0) {
        using Sh = T32LandShape<N>;
        const long long a[] = {Sh::THREADS, Sh::T, Sh::L, Sh::Eng::SMEM_ELEMS, (long long)Sh::BUF,
                               (long long)Sh::B_OFF, (long long)Sh::BAR_OFF, (long long)Sh::SMEM, (long long)Sh::LAND_BYTES};
        for (int i = 0; i < 9; ++i) v[i] = a[i];
    } else {
        using Sh = T32Land1Shape<N>;
        const long long a[] = {Sh::THREADS, Sh::T,          Sh::L,           Sh::Eng::SMEM_ELEMS, Sh::RS,
                               Sh::U,       Sh::K,          Sh::SPAN,        (long long)Sh::BUF,  (long long)Sh::B_OFF,
                               (long long)Sh::BAR_OFF, (long long)Sh::SLOT_OFF, (long long)Sh::SMEM};
        for (int i = 0; i < 13; ++i) v[i] = a[i];
    }
}

int tc32_land_layout(int n, int kind, long long *v) {
    if (kind != 0 && kind != 1) return -1;
    switch (n) {
        case 1024: land_layout<1024>(kind, v); return 0;
        case 2048: land_layout<2048>(kind, v); return 0;
        case 4096: land_layout<4096>(kind, v); return 0;
        case 8192: land_layout<8192>(kind, v); return 0;
        default: return -1;
    }
}

// Widest compiled tile (at most 512 threads) that fits nx columns; 0 if none.
int tc32_col_width(int n, int nx) {
    init_t32();
    if (n < 1024 || n > 8192 || (n & (n - 1))) return 0;
    int best = 0;
    for (int w = 2; w <= 16 && w <= nx; w <<= 1)
        if (g_t32_cols[ilog2(n)][t32_w_slot(w)].fn[0]) best = w;
    return best;
}

int tc32_cols_grid(int n, int w, long long ntiles, int num_sms) {
    init_t32();
    const int slot = t32_w_slot(w);
    if (slot < 0 || !g_t32_cols[ilog2(n)][slot].fn[0]) return 0;
    const T32ColEntry &en = g_t32_cols[ilog2(n)][slot];
    cudaFuncSetAttribute(en.fn[0], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)en.smem);
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, en.fn[0], en.threads, en.smem) != cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    // TMEM: 128 columns per group, 512 per SM
    const int tmem_per_sm = 512 / ((en.threads / kT32Group) * 128);
    if (per_sm > tmem_per_sm) per_sm = tmem_per_sm;
    long long grid = (long long)num_sms * per_sm;
    if (grid > ntiles) grid = ntiles;
    return grid < 1 ? 1 : (int)grid;
}

cudaError_t launch_rows_tc32(int n, int tmem_a, const float2 *in, float2 *out, const float2 *tw, const float2 *twp,
                             const void *w32, long long nrows, int ny, int split, int conj_in, int conj_out,
                             int *status, cudaStream_t s) {
    init_t32();
    if (!tc32_rows_available(n) || (split != 1 && split != 2) || ny % split) return cudaErrorInvalidValue;
    if (nrows <= 0) return cudaSuccess;
    const T32RowEntry &en = g_t32_rows[ilog2(n)];
    const void *fn = en.fn[tmem_a ? 1 : 0][split == 2 ? 1 : 0];
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)en.smem);
    if (e != cudaSuccess) return e;
    const long long grid = (nrows + en.rows_per_cta - 1) / en.rows_per_cta;  // one CTA per row group
    const __half *w = static_cast<const __half *>(w32);
    void *args[] = {(void *)&in,    (void *)&out, (void *)&tw,      (void *)&twp,      (void *)&w,
                    (void *)&nrows, (void *)&ny,  (void *)&conj_in, (void *)&conj_out, (void *)&status};
    return cudaLaunchKernel(fn, dim3((unsigned)grid), dim3(256), args, en.smem, s);
}

// Landed-row form: whether it covers nrows rows of n points (P = 1) or the
// pre-split rows of ny-row slices (P = 2); 0 if not.
int tc32_land_rows(int n) {
    init_t32();
    if (n < 1024 || n > 8192 || (n & (n - 1))) return 0;
    return g_t32_land[ilog2(n)].fn2 ? g_t32_land[ilog2(n)].rows_per_unit : 0;
}

bool tc32_land_available(int n, long long nrows, int ny, int split) {
    const int L = tc32_land_rows(n);
    if (L == 0 || (split != 1 && split != 2)) return false;
    if (split == 1) return nrows % g_t32_land[ilog2(n)].rows_per_sub == 0;
    return ny % 2 == 0 && (ny / 2) % (L / 2) == 0;
}

cudaError_t launch_rows_tc32_land(int n, const float2 *in, float2 *out, const float2 *tw, const float2 *twp,
                                  const void *w32, long long nrows, int ny, int split, int conj_in, int conj_out,
                                  int perm_t, int perm_g, int *status, int num_sms, cudaStream_t s) {
    init_t32();
    if (!tc32_land_available(n, nrows, ny, split)) return cudaErrorInvalidValue;
    if (perm_t && (perm_g < 1 || (perm_g & (perm_g - 1)) || (perm_t & (perm_t - 1)) || (ny / split) % perm_t ||
                   perm_t % perm_g))
        return cudaErrorInvalidValue;
    if (nrows <= 0) return cudaSuccess;
    const T32LandEntry &en = g_t32_land[ilog2(n)];
    const __half *w = static_cast<const __half *>(w32);
    if (split == 1) {
        // independent sub-units of rows_per_sub rows, subs per CTA, one CTA per SM
        cudaError_t e = cudaFuncSetAttribute(en.fn1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)en.smem1);
        if (e != cudaSuccess) return e;
        const long long nsub = nrows / en.rows_per_sub;
        const long long ctas = (nsub + en.subs - 1) / en.subs;
        const long long grid = num_sms < ctas ? num_sms : ctas;
        void *args[] = {(void *)&in,      (void *)&out,      (void *)&tw,     (void *)&w,
                        (void *)&nrows,   (void *)&ny,       (void *)&conj_in, (void *)&conj_out,
                        (void *)&perm_t,  (void *)&perm_g,   (void *)&status};
        return cudaLaunchKernel(en.fn1, dim3((unsigned)grid), dim3(512), args, en.smem1, s);
    }
    const void *fn = en.fn2;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)en.smem);
    if (e != cudaSuccess) return e;
    long long nunits = nrows / en.rows_per_unit;
    long long grid = num_sms < nunits ? num_sms : nunits;  // one CTA per SM: it holds all 512 TMEM columns
    void *args[] = {(void *)&in,       (void *)&out,     (void *)&tw,     (void *)&twp,
                    (void *)&w,        (void *)&nunits,  (void *)&ny,     (void *)&conj_in,
                    (void *)&conj_out, (void *)&perm_t,  (void *)&perm_g, (void *)&status};
    return cudaLaunchKernel(fn, dim3((unsigned)grid), dim3(512), args, en.smem, s);
}

cudaError_t launch_cols_tc32(int n, int w, int tmem_a, const CUtensorMap &map, float2 *out, const float2 *tw,
                             const void *w32, int nx, int batch, int split, int conj_out, int *status, int grid,
                             cudaStream_t s) {
    init_t32();
    const int slot = t32_w_slot(w);
    if (slot < 0 || !g_t32_cols[ilog2(n)][slot].fn[0] || grid < 1) return cudaErrorInvalidValue;
    const T32ColEntry &en = g_t32_cols[ilog2(n)][slot];
    const void *fn = en.fn[tmem_a ? 1 : 0];
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)en.smem);
    if (e != cudaSuccess) return e;
    CUtensorMap m = map;
    const __half *wt = static_cast<const __half *>(w32);
    void *args[] = {(void *)&m,     (void *)&out,   (void *)&tw,       (void *)&wt,     (void *)&nx,
                    (void *)&batch, (void *)&split, (void *)&conj_out, (void *)&status};
    return cudaLaunchKernel(fn, dim3(grid), dim3(en.threads), args, en.smem, s);
}

}  // namespace gb300fft
