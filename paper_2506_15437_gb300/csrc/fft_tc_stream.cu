// Streaming split-FP16 tensor-core column pass (4096-point column blocks).
//
// The radix-32 tensor-core column pass (fft_tc32.cu) stages a whole [N x W]
// tile, runs three stages (radix 4 in float32, two radix-32 products) with two
// exchanges, and starts the next tile's copy only after the last exchange.
// Here the schedule and the data movement are those of the streaming float32
// pass (fft_cols_stream.cu): two radix-64 stages and one exchange, each
// warp's stage-0 operands one contiguous 16 KiB segment of a row-permuted
// intermediate (the row pass stores column element j + 64 r at block row
// (j / 8) * 512 + 8 r + j % 8), on the warp's own mbarrier, with a ring of
// segment slots so most of the next tile lands under this tile's work.
//
// Each radix-64 butterfly (a thread's 64 elements) is one radix-2
// decimation-in-frequency level in float32,
//     a_n = x_n + x_{n+32},   b_n = (x_n - x_{n+32}) w64^n     (n < 32),
// and two radix-32 DFTs on the tensor cores, X_{2k} = DFT32(a)_k and
// X_{2k+1} = DFT32(b)_k, each split and multiplied exactly as the radix-32
// stages of fft_tc32.cu do (per-butterfly power-of-two scale, hi/lo float16
// split, three products by the even/odd B table, E_k +/- O_k).  A 128-thread
// group holds 2 x 128 radix-32 rows: tensor memory per group is D of both
// halves (2 x 64 columns) and A_hi / A_lo of both (4 x 32 columns), 256
// columns, so the CTA's two groups use all 512.
#include <mutex>

#include "fft_internal.h"
#include "fft_tc32.cuh"

namespace gb300fft {

template <int N, int W, int S>
struct TcStreamShape {
    static constexpr int E = 64;
    using Eng = Engine<N, E, W, PadShift<E>::value>;
    static constexpr int T = N / E;  // stage-0 butterflies per column
    static constexpr int R0 = Eng::R0;
    static_assert(Eng::S == 2 && R0 == E, "two radix-64 stages");
    static constexpr int THREADS = T * W;
    static constexpr int WARPS = THREADS / 32;
    static constexpr int GROUPS = THREADS / kT32Group;
    static constexpr int G = 32 / W;  // butterflies per warp
    static constexpr int SEG_ROWS = G * R0;
    static constexpr int SEG_ELEMS = SEG_ROWS * W;
    static constexpr int BOXR = SEG_ROWS < 256 ? SEG_ROWS : 256;
    static constexpr uint32_t SEG_BYTES = (uint32_t)SEG_ELEMS * sizeof(float2);
    static constexpr int xch_seg(int w) { return Eng::pad(w * SEG_ELEMS); }
    static constexpr size_t RING_OFF = ((size_t)Eng::SMEM_ELEMS * sizeof(float2) + 127) / 128 * 128;
    static constexpr size_t B_OFF = (RING_OFF + (size_t)S * SEG_BYTES + 1023) / 1024 * 1024;
    static constexpr size_t BAR_OFF = B_OFF + 2 * kT32BBytes;  // WARPS segment barriers, 2 MMA barriers per group
    static constexpr size_t SLOT_OFF = BAR_OFF + 8 * (WARPS + 2 * GROUPS);
    static constexpr size_t SMEM = SLOT_OFF + 16;
    static_assert(GROUPS * 256 <= 512, "256 TMEM columns per group");
    static_assert(WARPS * G == T, "one warp per G butterflies");
    static_assert(S >= 1 && S <= WARPS, "ring slots");
    static_assert(Eng::pad((WARPS - 1) * SEG_ELEMS) + SEG_ELEMS <= Eng::SMEM_ELEMS, "landing span");
    // the kernel's static shared memory (status words, the 1024-byte
    // alignment of the dynamic buffer) takes 1 KiB of the CTA's 227 KiB
    static_assert(SMEM + 1024 <= 232448, "shared memory of one CTA");
};

// Tensor-core state of one 128-thread group: its TMEM columns, its MMA
// barrier and phase, the even/odd B table in shared memory.
struct Tc64Group {
    uint32_t tmem;   // group base column, lane field 0
    uint32_t b_hi;   // shared address of B_hi (B_lo follows)
    uint64_t *bar;   // two: the products of half a, of half b
    uint32_t phase;
    int group, row;
    int *status;

    // split one radix-32 half (v[off .. off+31]) into A_hi / A_lo of half h
    template <int OFF>
    __device__ __forceinline__ float split_half(const float2 (&v)[64], uint32_t a_hi, uint32_t lane) {
        float m = 0.f;
#pragma unroll
        for (int k = 0; k < 32; ++k) m = fmaxf(m, fmaxf(fabsf(v[OFF + k].x), fabsf(v[OFF + k].y)));
        int eb = (__float_as_int(m) >> 23) & 0xff;
        eb = eb < 11 ? 11 : eb;
        const float up = __int_as_float((264 - eb) << 23);  // 2048 / s
        // chunks of 16 halves: Re x_even, Im x_even, Re x_odd, Im x_odd
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            uint32_t wh[8], wl[8];
#pragma unroll
            for (int p = 0; p < 8; ++p) {
                const int k0 = OFF + 4 * p + (q >> 1);
                const float x0 = ((q & 1) ? v[k0].y : v[k0].x) * up;
                const float x1 = ((q & 1) ? v[k0 + 2].y : v[k0 + 2].x) * up;
                const float h0 = __int_as_float(__float_as_int(x0) & 0xFFFFE000);
                const float h1 = __int_as_float(__float_as_int(x1) & 0xFFFFE000);
                wh[p] = f2h2_bits(h0, h1);
                wl[p] = f2h2_bits(x0 - h0, x1 - h1);
            }
            t32_st8(a_hi + lane + 8 * q, wh);
            t32_st8(a_hi + 32 + lane + 8 * q, wl);
        }
        return __int_as_float((eb - 10) << 23);  // s / 2048
    }

    // Half h's twelve products (even/odd table, small corrections first), on
    // the elected thread, committed to barrier h.
    __device__ __forceinline__ void issue_half(int h) {
        const uint32_t b_lo = b_hi + kT32BBytes;
        const uint32_t a = tmem + 128 + 64 * h;
#pragma unroll
        for (int e = 0; e < 2; ++e) {  // diagonal block e of the even/odd table
            const uint32_t d = tmem + 64 * h + 32 * e, bo = 4096 * e;
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int ks = 2 * e + j;
                t32_mma_ts(d, a + 32 + 8 * ks, t32_desc(b_hi + bo + ks * 256), j, kT32IdescN32);
            }
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int ks = 2 * e + j;
                t32_mma_ts(d, a + 8 * ks, t32_desc(b_lo + bo + ks * 256), 1, kT32IdescN32);
            }
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int ks = 2 * e + j;
                t32_mma_ts(d, a + 8 * ks, t32_desc(b_hi + bo + ks * 256), 1, kT32IdescN32);
            }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(bar + h))
                     : "memory");
    }

    // All of the group's A rows of half h are in TMEM: one thread issues.
    __device__ __forceinline__ void rows_written_issue(int h) {
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        named_sync(1 + group, kT32Group);
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (row == 0) issue_half(h);
    }

    // Half h's products are complete: X_{2k + h} = E_k + O_k, X_{2k + 32 + h}
    // = E_k - O_k (D columns 0-15 Re E, 16-31 Im E, 32-47 Re O, 48-63 Im O).
    template <int H>
    __device__ __forceinline__ void read_half(float2 (&v)[64], float down, uint32_t lane) {
        if (!t32_wait(bar + H, phase)) record_status(status, kStatusTimeout);
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        uint32_t d[4][16];
#pragma unroll
        for (int q = 0; q < 4; ++q) t32_ld16(tmem + lane + 64 * H + 16 * q, d[q]);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const float er = __int_as_float(d[0][k]), ei = __int_as_float(d[1][k]);
            const float orr = __int_as_float(d[2][k]), oi = __int_as_float(d[3][k]);
            v[2 * k + H] = make_float2((er + orr) * down, (ei + oi) * down);
            v[2 * (k + 16) + H] = make_float2((er - orr) * down, (ei - oi) * down);
        }
    }

    // The calling thread's length-64 DFT (forward sign) of v, natural order
    // in and out.  Every thread of the group calls it.  Half a's products
    // run while half b is split, half b's while half a is read back.
    __device__ __forceinline__ void dft64(float2 (&v)[64]) {
#pragma unroll
        for (int n = 0; n < 32; ++n) {
            const float2 u = v[n], w = v[n + 32];
            v[n] = cadd(u, w);
            v[n + 32] = mul_root64(csub(u, w), n);
        }
        const uint32_t lane = (uint32_t)(threadIdx.x & 96) << 16;
        // TMEM of the group: D_a [0, 64), D_b [64, 128), A_a [128, 192), A_b [192, 256)
        const float down_a = split_half<0>(v, tmem + 128, lane);
        rows_written_issue(0);
        const float down_b = split_half<32>(v, tmem + 192, lane);
        rows_written_issue(1);
        // X_{2k} from half a lands in even registers, which half b's inputs
        // (v[32..63], already in TMEM) no longer need
        read_half<0>(v, down_a, lane);
        read_half<1>(v, down_b, lane);
        phase ^= 1;
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    }
};

template <int N, int W, int S>
__global__ void __launch_bounds__(TcStreamShape<N, W, S>::THREADS, 1)
    k_cols_tc_stream(const __grid_constant__ CUtensorMap map, float2 *out, const float2 *__restrict__ tw,
                     const __half *__restrict__ w32, int nx, int batch, int P, int conj_out, int *status) {
    using Sh = TcStreamShape<N, W, S>;
    using Eng = typename Sh::Eng;
    constexpr int E = Sh::E;
    constexpr int T = Sh::T;
    constexpr int R0 = Sh::R0;
    constexpr int G = Sh::G;
    constexpr int WARPS = Sh::WARPS;
    extern __shared__ __align__(1024) unsigned char raw[];
    float2 *xch = reinterpret_cast<float2 *>(raw);
    float2 *ring = reinterpret_cast<float2 *>(raw + Sh::RING_OFF);
    uint64_t *full = reinterpret_cast<uint64_t *>(raw + Sh::BAR_OFF);  // one per warp
    uint64_t *mbar = full + WARPS;                                       // two per group (halves a, b)
    uint32_t *slot = reinterpret_cast<uint32_t *>(raw + Sh::SLOT_OFF);
    __shared__ int s_fail;
    __shared__ int s_armed[WARPS];

    const int t = threadIdx.x;
    const int c = t % W;
    const int tt = t / W;  // stage-0 butterfly j
    const int warp = t >> 5;
    const int lane = t & 31;
    const int ttl = tt - warp * G;
    const int groups_x = nx / W;
    const long long ntiles = (long long)groups_x * P * batch;
    const long long mt = blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const float so = conj_out ? -1.f : 1.f;
    auto seg_buf = [&](int w) -> float2 * {
        return w < S ? ring + (size_t)w * Sh::SEG_ELEMS : xch + Sh::xch_seg(w);
    };
    auto issue = [&](long long m, int w) {  // segment w of local tile m
        const long long id = blockIdx.x + m * (long long)gridDim.x;
        const int x = (int)(id % groups_x) * 2 * W;
        const int kp = (int)((id / groups_x) % P);
        const int z0 = (int)((id / groups_x) / P) * N + w * Sh::SEG_ROWS;
        float2 *dst = seg_buf(w);
        mbar_expect_tx(full + w, Sh::SEG_BYTES);
#pragma unroll
        for (int k = 0; k < Sh::SEG_ROWS / Sh::BOXR; ++k)
            tma_load_3d(dst + k * Sh::BOXR * W, &map, x, kp, z0 + k * Sh::BOXR, full + w);
        s_armed[w] += 1;
    };

    // the even/odd B table (second table of w32) into shared memory, TMEM
    Tc64Group tc;
    {
        const uint4 *src = reinterpret_cast<const uint4 *>(w32 + kT32BBytes);
        uint4 *dst = reinterpret_cast<uint4 *>(raw + Sh::B_OFF);
        for (int i = t; i < 2 * kT32BBytes / 16; i += Sh::THREADS) dst[i] = __ldg(src + i);
    }
    if (t < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
                     "r"(512u)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (t == 0) {
        s_fail = 0;
        for (int w = 0; w < WARPS; ++w) {
            mbar_init(full + w, 1);
            s_armed[w] = 0;
        }
        for (int gi = 0; gi < 2 * Sh::GROUPS; ++gi) mbar_init(mbar + gi, 1);
        fence_mbar_init();
        fence_proxy_async_smem();
        if (mt > 0)
            for (int w = 0; w < WARPS; ++w) issue(0, w);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    tc.group = t / kT32Group;
    tc.row = t % kT32Group;
    tc.tmem = *slot + (uint32_t)(tc.group * 256);
    tc.b_hi = smem_u32(raw + Sh::B_OFF);
    tc.bar = mbar + 2 * tc.group;
    tc.phase = 0;
    tc.status = status;

    long long m = 0;
    for (; m < mt; ++m) {
        const long long id = blockIdx.x + m * (long long)gridDim.x;
        // stage 0: this warp's segment, read, then the ring slot refilled
        float2 v[E];
        const bool ok = mbar_wait_bounded(full + warp, (uint32_t)(m & 1));
        if (ok) {
            const float2 *seg = seg_buf(warp);
#pragma unroll
            for (int r = 0; r < R0; ++r) v[r] = seg[(r * G + ttl) * W + c];
        } else {
            atomicOr(&s_fail, 1);
#pragma unroll
            for (int r = 0; r < R0; ++r) v[r] = make_float2(0.f, 0.f);
        }
        __syncwarp();
        if (warp < S && lane == 0 && ok && m + 1 < mt) {
            fence_proxy_async_smem();
            issue(m + 1, warp);
        }
        // every thread of the group takes part in the products (a failed
        // segment transforms zeros; the status word records the failure)
        tc.dft64(v);
#pragma unroll
        for (int k = 0; k < R0; ++k) xch[Eng::pad((tt * R0 + k) * W + c)] = v[k];
        __syncthreads();
        if (s_fail) break;
        // stage 1: exchange reads, twiddles, DFT-64, natural-order stores
        constexpr int Ns = R0;
        const int mm = tt & (Ns - 1);
#pragma unroll
        for (int r = 0; r < E; ++r) v[r] = xch[Eng::pad((tt + r * T) * W + c)];
        __syncthreads();  // the exchange is free: the next tile's remaining segments land in it
        if (t == 0 && m + 1 < mt) {
            fence_proxy_async_smem();
            for (int w = S; w < WARPS; ++w) issue(m + 1, w);
        }
        const float4 *tws = reinterpret_cast<const float4 *>(tw + Sched<N, E>::tw_off(1)) + mm;
#pragma unroll
        for (int k = 0; k < E / 2; ++k) {
            const float4 w2 = __ldg(tws + k * Ns);
            v[2 * k + 1] = cmul(v[2 * k + 1], make_float2(w2.x, w2.y));
            if (2 * k + 2 < E) v[2 * k + 2] = cmul(v[2 * k + 2], make_float2(w2.z, w2.w));
        }
        tc.dft64(v);
        const long long blk = id / groups_x;  // b*P + kp
        const long long b = blk / P;
        const int kp = (int)(blk - b * P);
        float2 *dst = out + (b * N * P + kp) * (long long)nx + (long long)(id % groups_x) * W + c;
        const long long rstride = (long long)P * nx;
#pragma unroll
        for (int k = 0; k < E; ++k) {
            float2 x = v[k];
            x.y *= so;
            dst[(long long)(tt + k * T) * rstride] = x;
        }
    }
    if (s_fail && t == 0) {
        record_status(status, kStatusTimeout);
        for (int w = 0; w < WARPS; ++w)
            for (long long ph = m; ph < s_armed[w]; ++ph)
                mbar_wait_bounded(full + w, (uint32_t)(ph & 1), 10000000ull);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (t < 32)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(*slot), "r"(512u) : "memory");
}

namespace {
const void *g_tcs_fn = nullptr;
size_t g_tcs_smem = 0;
int g_tcs_threads = 0;
std::once_flag g_tcs_once;
constexpr int kTcsN = 4096, kTcsW = 4, kTcsS = 4;
void init_tcs() {
    std::call_once(g_tcs_once, [] {
        using Sh = TcStreamShape<kTcsN, kTcsW, kTcsS>;
        g_tcs_fn = (const void *)k_cols_tc_stream<kTcsN, kTcsW, kTcsS>;
        g_tcs_smem = Sh::SMEM;
        g_tcs_threads = Sh::THREADS;
    });
}
}  // namespace

bool tc_stream_available(int n, int nx) { return n == kTcsN && nx >= kTcsW && nx % kTcsW == 0; }

void tc_stream_perm(int *perm_t, int *perm_g) {
    using Sh = TcStreamShape<kTcsN, kTcsW, kTcsS>;
    *perm_t = kTcsN / Sh::R0;
    *perm_g = Sh::G;
}

int tc_stream_width() { return kTcsW; }

int tc_stream_twiddle_e() { return TcStreamShape<kTcsN, kTcsW, kTcsS>::E; }

// Compile-time layout of the streaming tensor-core column kernel (host only).
int tc_stream_layout(long long *v) {
    using Sh = TcStreamShape<kTcsN, kTcsW, kTcsS>;
    const long long a[] = {kTcsN,       kTcsW,          kTcsS,        Sh::THREADS,           Sh::WARPS,
                           Sh::GROUPS,  Sh::G,          Sh::SEG_ROWS, Sh::SEG_ELEMS,         Sh::BOXR,
                           Sh::SEG_BYTES, Sh::Eng::SMEM_ELEMS, (long long)Sh::RING_OFF, (long long)Sh::B_OFF,
                           (long long)Sh::BAR_OFF, (long long)Sh::SLOT_OFF, (long long)Sh::SMEM};
    for (int i = 0; i < 17; ++i) v[i] = a[i];
    for (int w = 0; w < Sh::WARPS && w < 16; ++w) v[17 + w] = Sh::xch_seg(w);
    return 0;
}

cudaError_t launch_cols_tc_stream(const CUtensorMap &map, float2 *out, const float2 *tw, const void *w32, int nx,
                                  int batch, int split, int conj_out, int *status, int num_sms, cudaStream_t s) {
    init_tcs();
    if (nx % kTcsW) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(g_tcs_fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)g_tcs_smem);
    if (e != cudaSuccess) return e;
    const long long ntiles = (long long)(nx / kTcsW) * split * batch;
    const int grid = (int)(ntiles < num_sms ? ntiles : num_sms);  // one CTA per SM: all 512 TMEM columns
    if (grid < 1) return cudaSuccess;
    CUtensorMap m = map;
    const __half *wt = static_cast<const __half *>(w32);
    void *args[] = {(void *)&m,     (void *)&out,   (void *)&tw,       (void *)&wt,    (void *)&nx,
                    (void *)&batch, (void *)&split, (void *)&conj_out, (void *)&status};
    return cudaLaunchKernel(g_tcs_fn, dim3(grid), dim3(g_tcs_threads), args, g_tcs_smem, s);
}

}  // namespace gb300fft
