// Small square 2D transforms (n x n, n = 256 .. 1024, up to 2^20 points in
// all) in one cooperative launch.
//
// Section 5's row FFTs, then column FFTs, both from and to the output array.
// At these sizes the array fits the L2 and each pass is a handful of
// microseconds, so the launch of the second pass and its ramp-up cost as much
// as its work.  Here one persistent grid runs both phases:
// - phase 1: the rows, ROWS rows per 256-thread item, read from the input and
//   written in natural order to the output;
// - a grid-wide barrier;
// - phase 2: the columns, tiles of W = ROWS adjacent columns, read from and
//   written back to the output.
// Each phase runs the same Stockham engine, twiddle table and stage order as
// the separate row and column kernels (E = 16), so the results are the same
// arithmetic.  The launch is cooperative, so every CTA is resident and the
// barrier can complete.  The barrier is a generation counter: the last CTA
// to arrive resets the count and advances the generation, so it works across
// launches and CUDA-graph replays with no host-side state.  Its spin is
// bounded; a timeout records FFT_ERR_TIMEOUT in the status word and the
// kernel finishes.
#include <mutex>

#include "fft_common.cuh"
#include "fft_internal.h"

namespace gb300fft {

template <int N>
struct Small2DShape {
    static constexpr int E = 16;
    static constexpr int T = N / E;        // threads per row / per column
    static constexpr int THREADS = 256;
    static constexpr int ROWS = THREADS / T;  // rows per item, columns per tile
    using RowEng = Engine<N, E, 1, PadShift<E>::value, RowPadShift1<E>::value>;
    using ColEng = Engine<N, E, ROWS, PadShift<E>::value>;
    static constexpr size_t ROW_SMEM = sizeof(float2) * (size_t)ROWS * RowEng::SMEM_ELEMS;
    static constexpr size_t COL_SMEM = sizeof(float2) * (size_t)ColEng::SMEM_ELEMS;
    static constexpr size_t SMEM = ROW_SMEM > COL_SMEM ? ROW_SMEM : COL_SMEM;
    static_assert(T <= THREADS && THREADS % T == 0, "whole rows per item");
    static_assert(ROWS * 8 >= 16, "column tiles of at least 16 bytes per row");
};

// Grid-wide barrier over gridDim.x CTAs (all resident: cooperative launch).
// bar[0]: arrivals of the current generation, bar[1]: generation.
__device__ __forceinline__ void grid_barrier(unsigned *bar, int *status) {
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *gen = bar + 1;
        const unsigned g0 = *gen;
        __threadfence();  // this CTA's phase-1 stores before its arrival
        if (atomicAdd(bar, 1u) == gridDim.x - 1) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            const uint64_t t0 = globaltimer_ns();
            uint32_t it = 0;
            while (*gen == g0) {
                __nanosleep(64);
                if ((++it & 1023u) == 0 && globaltimer_ns() - t0 > 2000000000ull) {
                    record_status(status, kStatusTimeout);
                    break;
                }
            }
        }
        __threadfence();  // the other CTAs' stores before this CTA's phase 2
    }
    __syncthreads();
}

template <int N>
__global__ void __launch_bounds__(256) k_fft2_small(const float2 *__restrict__ in, float2 *out,
                                                    const float2 *__restrict__ tw, int batch, int conj,
                                                    unsigned *bar, int *status) {
    using Sh = Small2DShape<N>;
    using RowEng = typename Sh::RowEng;
    using ColEng = typename Sh::ColEng;
    constexpr int E = Sh::E;
    constexpr int T = Sh::T;
    constexpr int ROWS = Sh::ROWS;
    constexpr int W = ROWS;
    extern __shared__ __align__(16) float2 sm[];
    const int t = threadIdx.x;
    const float s = conj ? -1.f : 1.f;
    // phase 1: rows (conjugated on load for the inverse)
    {
        constexpr int R0 = RowEng::R0;
        const int g = t / T, tt = t - g * T;
        float2 *rs = sm + g * RowEng::SMEM_ELEMS;
        const long long items = (long long)N * batch / ROWS;
        for (long long it = blockIdx.x; it < items; it += gridDim.x) {
            const long long row = it * ROWS + g;
            const float2 *src = in + row * N;
            float2 v[E];
#pragma unroll
            for (int b = 0; b < E / R0; ++b) {
                const int j = tt + b * T;
#pragma unroll
                for (int r = 0; r < R0; ++r) {
                    float2 x = src[j + r * (N / R0)];
                    x.y *= s;
                    v[b * R0 + r] = x;
                }
            }
            float2 *dst = out + row * N;
            auto store = [&](int i, int, float2 x) { dst[i] = x; };
            // the previous item's last exchange reads are behind the engine's
            // first barrier, so the spans can be reused at once
            RowEng::template run<FftPolicy, true>(v, rs, tw, tt, 0, SyncBlock{}, [] {}, store);
        }
    }
    grid_barrier(bar, status);
    // phase 2: columns, in place in the output (conjugated on store)
    {
        constexpr int R0 = ColEng::R0;
        const int c = t % W, tt = t / W;
        const long long tiles = (long long)(N / W) * batch;
        for (long long it = blockIdx.x; it < tiles; it += gridDim.x) {
            const long long b = it / (N / W);
            const int x0 = (int)(it - b * (N / W)) * W;
            float2 *base = out + b * (long long)N * N + x0 + c;
            float2 v[E];
#pragma unroll
            for (int bb = 0; bb < E / R0; ++bb) {
                const int j = tt + bb * T;
#pragma unroll
                for (int r = 0; r < R0; ++r)  // L2, not this SM's L1: other CTAs wrote these rows
                    v[bb * R0 + r] = __ldcg(base + (long long)(j + r * (N / R0)) * N);
            }
            auto store = [&](int i, int, float2 x) {
                x.y *= s;
                base[(long long)i * N] = x;
            };
            ColEng::template run<FftPolicy, true>(v, sm, tw, tt, c, SyncBlock{}, [] {}, store);
        }
    }
}

namespace {
struct SmallEntry {
    const void *fn = nullptr;
    size_t smem = 0;
    int per_sm = 0;
};
SmallEntry g_small[kMaxLog2 + 1];
std::once_flag g_small_once;
template <int N>
void reg_small() {
    SmallEntry &en = g_small[ilog2(N)];
    en.fn = (const void *)k_fft2_small<N>;
    en.smem = Small2DShape<N>::SMEM;
}
void init_small() {
    std::call_once(g_small_once, [] {
        // 2048 x 2048 measured slower in one launch (0.053 against 0.037 ms:
        // 16-byte column tiles against the column pass's 64-byte ones)
        reg_small<256>();
        reg_small<512>();
        reg_small<1024>();
    });
}
}  // namespace

// Up to 2^20 points in all (one 1024 x 1024 array): measured 512^2 0.0123 ->
// 0.0103 ms, 1024^2 0.0164 -> 0.0144 ms; a batch of eight 1024^2 arrays
// gains nothing (0.0685 against 0.0693 ms).
bool small2d_available(int nx, int ny, int batch, int row_e) {
    init_small();
    return nx == ny && nx >= 256 && nx <= 1024 && (nx & (nx - 1)) == 0 && row_e == 16 &&
           (long long)nx * ny * batch <= (1LL << 20) && g_small[ilog2(nx)].fn;
}

// Grid: every CTA resident (cooperative launch), no more than the larger
// phase has items.
int small2d_grid(int n, int batch, int num_sms) {
    init_small();
    SmallEntry &en = g_small[ilog2(n)];
    if (!en.fn) return 0;
    if (en.per_sm == 0) {
        if (en.smem > 48 * 1024)
            cudaFuncSetAttribute(en.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)en.smem);
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, en.fn, 256, en.smem) != cudaSuccess || per_sm < 1)
            return 0;
        en.per_sm = per_sm;
    }
    const int rows_per_item = 256 / (n / 16);
    const long long items = (long long)n * batch / rows_per_item;  // = column tiles too (W = rows per item)
    long long grid = (long long)num_sms * en.per_sm;
    if (grid > items) grid = items;
    return grid < 1 ? 1 : (int)grid;
}

cudaError_t launch_small2d(int n, const float2 *in, float2 *out, const float2 *tw, int batch, int conj,
                           unsigned *bar, int *status, int grid, cudaStream_t s) {
    init_small();
    SmallEntry &en = g_small[ilog2(n)];
    if (!en.fn || grid < 1) return cudaErrorInvalidValue;
    if (en.smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(en.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)en.smem);
        if (e != cudaSuccess) return e;
    }
    void *args[] = {(void *)&in, (void *)&out, (void *)&tw, (void *)&batch, (void *)&conj, (void *)&bar,
                    (void *)&status};
    return cudaLaunchCooperativeKernel(en.fn, dim3(grid), dim3(256), args, en.smem, s);
}

}  // namespace gb300fft
