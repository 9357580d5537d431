// Row pass with the column pre-split from a landed pair of rows.
//
// With the pre-split (P = 2, see fft_rows.cu) output rows kp = 0 and kp = 1
// of pair q both need input rows q and q + ny/2: x0 + x1 and
// (x0 - x1) * w_ny^q.  The plain row pass gives each output row its own CTA,
// which loads both input rows from global memory, so every input row is
// fetched twice (the second time mostly from L2).  Here one 512-thread CTA
// takes the whole pair: two bulk copies (one per input row, completion on an
// mbarrier) land the rows in shared memory once, the first half of the
// threads forms and transforms output kp = 0, the second half kp = 1, each
// with the plain Stockham engine in its own half of the buffer, which the
// landed rows no longer need by then.  The next pair's copies start as soon
// as every thread has read its last-stage operands.  The arithmetic (sum or
// difference, then the twiddle, then the same engine) is the plain row
// pass's, operation for operation.
#include <mutex>

#include "fft_common.cuh"
#include "fft_internal.h"

namespace gb300fft {

template <int N, int E>
struct LandShape {
    static constexpr int T = N / E;        // threads per output row
    static constexpr int THREADS = 2 * T;  // one half per output row kp
    using Eng = Engine<N, E, 1, PadShift<E>::value, RowPadShift1<E>::value>;
    static constexpr size_t LAND_BYTES = 2 * (size_t)N * sizeof(float2);
    static constexpr size_t XBYTES = 2 * (size_t)Eng::SMEM_ELEMS * sizeof(float2);
    static constexpr size_t BUF = XBYTES > LAND_BYTES ? XBYTES : LAND_BYTES;
    static constexpr size_t BAR_OFF = (BUF + 15) / 16 * 16;
    static constexpr size_t SMEM = BAR_OFF + 16;
};

template <int N, int E>
__global__ void __launch_bounds__(LandShape<N, E>::THREADS, 1)
    k_rows_land(const float2 *__restrict__ in, float2 *out, const float2 *__restrict__ tw,
                const float2 *__restrict__ twp, int ny, long long npairs, int conj_in, int perm_t, int perm_g,
                int planar, int *status, int pf) {
    using Sh = LandShape<N, E>;
    using Eng = typename Sh::Eng;
    constexpr int T = Sh::T;
    constexpr int R0 = Eng::R0;
    extern __shared__ __align__(128) unsigned char raw[];
    float2 *land = reinterpret_cast<float2 *>(raw);  // [2][N]: input rows q, q + ny/2
    uint64_t *bar = reinterpret_cast<uint64_t *>(raw + Sh::BAR_OFF);
    __shared__ int s_ok;
    const int t = threadIdx.x;
    const int h = t / T;  // output row kp of the pair
    const int tt = t - h * T;
    float2 *sm = reinterpret_cast<float2 *>(raw) + h * Eng::SMEM_ELEMS;
    const int Q = ny / 2;
    const float si = conj_in ? -1.f : 1.f;

    auto issue = [&](long long id) {  // thread 0: the pair's two row copies
        const long long b = id / Q;
        const int q = (int)(id - b * Q);
        mbar_expect_tx(bar, (uint32_t)Sh::LAND_BYTES);
        bulk_load(land, in + (b * ny + q) * (long long)N, N * sizeof(float2), bar);
        bulk_load(land + N, in + (b * ny + q + Q) * (long long)N, N * sizeof(float2), bar);
    };
    if (t == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
        fence_proxy_async_smem();
    }
    __syncthreads();
    // L2 bulk prefetch of pair `pid`'s two input rows (thread 0)
    auto prefetch = [&](long long pid) {
        const long long b = pid / Q;
        const int q = (int)(pid - b * Q);
        bulk_prefetch_l2(in + (b * ny + q) * (long long)N, N * sizeof(float2));
        bulk_prefetch_l2(in + (b * ny + q + Q) * (long long)N, N * sizeof(float2));
    };
    long long id = blockIdx.x;
    uint32_t phase = 0;
    if (t == 0 && id < npairs) {
        issue(id);
        for (int d = 1; d < pf; ++d)
            if (id + (long long)d * gridDim.x < npairs) prefetch(id + (long long)d * gridDim.x);
    }
    for (; id < npairs; id += gridDim.x) {
        // the pair pf steps ahead starts moving into L2 while this one computes
        if (t == 0 && pf > 0 && id + (long long)pf * gridDim.x < npairs) prefetch(id + (long long)pf * gridDim.x);
        if (t == 0) s_ok = mbar_wait_bounded(bar, phase) ? 1 : 0;
        __syncthreads();
        if (!s_ok) {
            if (t == 0) {
                record_status(status, kStatusTimeout);
                mbar_wait_bounded(bar, phase);  // give the copies in flight a last chance to land
            }
            return;
        }
        phase ^= 1;
        const long long next = id + gridDim.x;
        const long long b = id / Q;
        const int q = (int)(id - b * Q);
        float2 v[E];
#pragma unroll
        for (int bb = 0; bb < E / R0; ++bb) {
            const int j = tt + bb * T;
#pragma unroll
            for (int r = 0; r < R0; ++r) {
                const int i = j + r * (N / R0);
                float2 x0 = land[i], x1 = land[N + i];
                x0.y *= si;
                x1.y *= si;
                const float2 acc = cadd(make_float2(0.f, 0.f), x0);
                v[bb * R0 + r] = h ? csub(acc, x1) : cadd(acc, x1);
            }
        }
        if (h) {
            const float2 w = __ldg(twp + q);
#pragma unroll
            for (int k = 0; k < E; ++k) v[k] = cmul(v[k], w);
        }
        // output row of (kp = h, block element q), as the plain row pass stores it
        int pos = q;
        if (perm_t) {
            const int j = q & (perm_t - 1), r = q / perm_t;
            pos = (j / perm_g) * perm_g * (Q / perm_t) + r * perm_g + (j & (perm_g - 1));
        }
        float2 *dst = out + (b * ny + (planar ? (long long)h * Q + pos : h + 2LL * pos)) * N;
        auto after_reads = [&] {
            __syncthreads();
            if (t == 0 && next < npairs) {
                fence_proxy_async_smem();
                issue(next);
            }
        };
        auto store = [&](int i, int, float2 x) { dst[i] = x; };
        Eng::template run<FftPolicy, true>(v, sm, tw, tt, 0, SyncBlock{}, after_reads, store);
    }
}

namespace {
struct LandEntry {
    const void *fn = nullptr;
    size_t smem = 0;
    int threads = 0;
    int per_sm = 0;
    std::once_flag occ_once;
};
// E = 32 only: the E = 16 form (1024 threads, 64 registers, radices 2, 16,
// 16, 16) measured 0.354 against 0.267 ms on the same box
LandEntry g_land;
std::once_flag g_land_once;
void init_land() {
    std::call_once(g_land_once, [] {
        constexpr int N = 8192, E = 32;
        g_land.fn = (const void *)k_rows_land<N, E>;
        g_land.smem = LandShape<N, E>::SMEM;
        g_land.threads = LandShape<N, E>::THREADS;
    });
}
}  // namespace

bool land_rows_available(int n, int e) { return n == 8192 && e == 32; }

cudaError_t launch_rows_land(int e, const float2 *in, float2 *out, const float2 *tw, const float2 *twp, int ny,
                             int batch, int conj_in, int perm_t, int perm_g, int planar, int *status, int num_sms,
                             int pf, cudaStream_t s) {
    init_land();
    if (ny < 2 || ny % 2 || !land_rows_available(8192, e)) return cudaErrorInvalidValue;
    LandEntry &en = g_land;
    cudaError_t err = cudaFuncSetAttribute(en.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)en.smem);
    if (err != cudaSuccess) return err;
    std::call_once(en.occ_once, [&en] {
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, en.fn, en.threads, en.smem) != cudaSuccess)
            per_sm = 1;
        en.per_sm = per_sm > 0 ? per_sm : 1;
    });
    long long npairs = (long long)batch * (ny / 2);
    long long grid = (long long)num_sms * en.per_sm;
    if (grid > npairs) grid = npairs;
    void *args[] = {(void *)&in,     (void *)&out,    (void *)&tw,     (void *)&twp,   (void *)&ny,    (void *)&npairs,
                    (void *)&conj_in, (void *)&perm_t, (void *)&perm_g, (void *)&planar, (void *)&status,
                    (void *)&pf};
    return cudaLaunchKernel(en.fn, dim3((unsigned)grid), dim3(en.threads), args, en.smem, s);
}

}  // namespace gb300fft
