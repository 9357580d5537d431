// Row pass for long rows (N >= 2048): persistent CTAs fed by a TMA landing
// ring.  The paper overlaps its reader, compute and writer kernels by
// splitting the domain into chunks (Section 4, "chunked"); here the same
// overlap comes from asynchronous bulk copies.
//
// Shared memory holds two landing slots (dense rows, filled by 1D bulk
// copies that complete on an mbarrier) and one padded exchange buffer.  A
// slot is consumed only by the stage-0 loads; as soon as every thread has
// read it, the CTA refills it with a later row, so the copy runs under the
// remaining butterfly stages and the stores.  Results leave through ordinary
// coalesced stores straight from registers.
//
// P = 1: a unit is one row, units alternate between the two slots.
// P = 2: a unit is one row pair (q, q + ny/2) of the column pre-split (see
// fft_rows.cu); both slots hold the pair, and the CTA produces both output
// rows 2q (a + b) and 2q + 1 ((a - b) * w_ny^q) from one copy of the inputs.
#include <mutex>

#include "fft_common.cuh"
#include "fft_internal.h"

namespace gb300fft {

template <int N, int E>
struct RingShape {
    static constexpr int THREADS = N / E;
    using Eng = Engine<N, E, 1, PadShift<E>::value>;
    static constexpr size_t SLOT_BYTES = (size_t)N * sizeof(float2);
    static constexpr size_t X_OFF = 2 * SLOT_BYTES;
    static constexpr size_t BAR_OFF = (X_OFF + (size_t)Eng::SMEM_ELEMS * sizeof(float2) + 15) / 16 * 16;
    static constexpr size_t SMEM = BAR_OFF + 2 * sizeof(uint64_t);
    // the landing ring takes most of shared memory: N = 8192 runs one CTA per
    // SM (registers up to 128), shorter rows two or more
    static constexpr int MINB = N >= 8192 ? 1 : 2;
};

template <int N, int E, int P, bool WEIGHTED>
__global__ void __launch_bounds__(RingShape<N, E>::THREADS, RingShape<N, E>::MINB)
    k_rows_ring(const float2 *__restrict__ in, float2 *out, const float2 *__restrict__ tw,
                const float2 *__restrict__ twp, long long nrows, int ny, int conj_in, int conj_out,
                const float *__restrict__ weight, float wscale, const float *__restrict__ wscale_dev, int *status) {
    using Sh = RingShape<N, E>;
    using Eng = typename Sh::Eng;
    constexpr int T = Sh::THREADS;
    constexpr int R0 = Eng::R0;
    extern __shared__ __align__(128) unsigned char raw[];
    float2 *slot0 = reinterpret_cast<float2 *>(raw);  // slot s starts at slot0 + s * N
    float2 *xbuf = reinterpret_cast<float2 *>(raw + Sh::X_OFF);
    uint64_t *bar = reinterpret_cast<uint64_t *>(raw + Sh::BAR_OFF);
    __shared__ int s_ok;

    const int tt = threadIdx.x;
    if constexpr (WEIGHTED) {
        if (wscale_dev) wscale *= __ldg(wscale_dev);  // a scale that lives on the device (no host read)
    }
    const float si = conj_in ? -1.f : 1.f;
    const float so = conj_out ? -1.f : 1.f;
    const int Q = ny / P;
    const long long nunits = nrows / P;
    const long long grid = gridDim.x;

    // first input row of unit u (P == 2: the pair's upper row is + Q)
    auto unit_row = [&](long long u) -> long long {
        if constexpr (P == 1) {
            return u;
        } else {
            const long long b = u / Q;
            return b * ny + (u - b * Q);
        }
    };
    auto issue = [&](long long u, int s) {  // thread 0
        const long long r = unit_row(u);
        if constexpr (P == 1) {
            mbar_expect_tx(&bar[s], (uint32_t)Sh::SLOT_BYTES);
            bulk_load(slot0 + s * N, in + r * N, (uint32_t)Sh::SLOT_BYTES, &bar[s]);
        } else {
            mbar_expect_tx(&bar[0], (uint32_t)(2 * Sh::SLOT_BYTES));
            bulk_load(slot0, in + r * N, (uint32_t)Sh::SLOT_BYTES, &bar[0]);
            bulk_load(slot0 + N, in + (r + Q) * N, (uint32_t)Sh::SLOT_BYTES, &bar[0]);
        }
    };
    auto prefetch = [&](long long u) {  // thread 0
        const long long r = unit_row(u);
        bulk_prefetch_l2(in + r * N, (uint32_t)Sh::SLOT_BYTES);
        if constexpr (P == 2) bulk_prefetch_l2(in + (r + Q) * N, (uint32_t)Sh::SLOT_BYTES);
    };

    if (tt == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
        fence_proxy_async_smem();
    }
    __syncthreads();
    const long long u0 = blockIdx.x;
    if (tt == 0) {
        if (u0 < nunits) issue(u0, 0);
        if constexpr (P == 1) {
            if (u0 + grid < nunits) issue(u0 + grid, 1);
            if (u0 + 2 * grid < nunits) prefetch(u0 + 2 * grid);
        } else {
            if (u0 + grid < nunits) prefetch(u0 + grid);
        }
    }

    long long k = 0;
    for (long long u = u0; u < nunits; u += grid, ++k) {
        const int s = (P == 1) ? (int)(k & 1) : 0;
        const uint32_t parity = (P == 1) ? (uint32_t)((k >> 1) & 1) : (uint32_t)(k & 1);
        if (tt == 0) s_ok = mbar_wait_bounded(&bar[s], parity) ? 1 : 0;
        __syncthreads();
        if (!s_ok) {
            if (tt == 0) {
                record_status(status, kStatusTimeout);
                mbar_wait_bounded(&bar[s], parity);
            }
            return;
        }
        const long long r_in = unit_row(u);
#pragma unroll 1
        for (int kp = 0; kp < P; ++kp) {
            float2 v[E];
            float2 w = make_float2(1.f, 0.f);
            if constexpr (P == 2) {
                if (kp == 1) w = __ldg(twp + (r_in % ny));
            }
#pragma unroll
            for (int b = 0; b < E / R0; ++b) {
                const int j = tt + b * T;
#pragma unroll
                for (int r = 0; r < R0; ++r) {
                    const int i = j + r * (N / R0);
                    float2 x = slot0[s * N + i];
                    if constexpr (WEIGHTED) {
                        const float wv = __ldg(weight + r_in * N + i) * wscale;
                        x.x *= wv;
                        x.y *= wv;
                    }
                    x.y *= si;
                    if constexpr (P == 2) {
                        float2 y = slot0[N + i];
                        if constexpr (WEIGHTED) {
                            const float wv = __ldg(weight + (r_in + Q) * N + i) * wscale;
                            y.x *= wv;
                            y.y *= wv;
                        }
                        y.y *= si;
                        x = (kp == 0) ? cadd(x, y) : cmul(csub(x, y), w);
                    }
                    v[b * R0 + r] = x;
                }
            }
            // every thread has read the slot(s) and finished the previous
            // transform's exchanges: release the slot(s), reuse the buffer
            __syncthreads();
            if (tt == 0 && kp == P - 1) {
                const long long nu = u + ((P == 1) ? 2 : 1) * grid;
                if (nu < nunits) {
                    fence_proxy_async_smem();
                    issue(nu, s);
                }
                if (nu + grid < nunits) prefetch(nu + grid);
            }
            const long long r_out = (P == 1) ? u : (r_in - (r_in % ny)) + 2 * (r_in % ny) + kp;
            float2 *dst = out + r_out * N;
            auto store = [&](int i, int, float2 x) {
                x.y *= so;
                dst[i] = x;
            };
            auto none = [] {};
            Eng::template run<FftPolicy, false>(v, xbuf, tw, tt, 0, SyncBlock{}, none, store);
        }
    }
}

namespace {
struct RingEntry {
    const void *fn[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};  // [weighted][P == 2]
    int threads = 0;
    size_t smem = 0;
};
RingEntry g_ring[kMaxLog2 + 1];
std::once_flag g_ring_once;  // registry filled once, safe across host threads

template <int N>
void reg_ring() {
    constexpr int E = 16;
    using Sh = RingShape<N, E>;
    RingEntry &en = g_ring[ilog2(N)];
    en.fn[0][0] = (const void *)k_rows_ring<N, E, 1, false>;
    en.fn[1][0] = (const void *)k_rows_ring<N, E, 1, true>;
    en.fn[0][1] = (const void *)k_rows_ring<N, E, 2, false>;
    en.fn[1][1] = (const void *)k_rows_ring<N, E, 2, true>;
    en.threads = Sh::THREADS;
    en.smem = Sh::SMEM;
}

const RingEntry *ring_entry(int n) {
    std::call_once(g_ring_once, [] {
        reg_ring<2048>();
        reg_ring<4096>();
        reg_ring<8192>();
    });
    if (n < 2048 || n > 8192 || (n & (n - 1))) return nullptr;
    return &g_ring[ilog2(n)];
}
}  // namespace

bool ring_rows_available(int n) { return ring_entry(n) != nullptr; }

int ring_rows_grid(int n, long long nrows, int split, int num_sms, bool weighted) {
    const RingEntry *en = ring_entry(n);
    if (!en) return 0;
    const void *fn = en->fn[weighted ? 1 : 0][split == 2 ? 1 : 0];
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)en->smem);
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, en->threads, en->smem) != cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    const long long units = nrows / split;
    long long grid = (long long)num_sms * per_sm;
    if (grid > units) grid = units;
    return grid < 1 ? 1 : (int)grid;
}

cudaError_t launch_rows_ring(int n, const float2 *in, float2 *out, const float2 *tw, const float2 *twp,
                             long long nrows, int ny, int split, int conj_in, int conj_out, const float *weight,
                             float wscale, const float *wscale_dev, int *status, int grid, cudaStream_t s) {
    const RingEntry *en = ring_entry(n);
    if (!en || (split != 1 && split != 2) || grid < 1) return cudaErrorInvalidValue;
    if (nrows <= 0) return cudaSuccess;
    const void *fn = en->fn[weight ? 1 : 0][split == 2 ? 1 : 0];
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)en->smem);
    if (e != cudaSuccess) return e;
    void *args[] = {(void *)&in,       (void *)&out,    (void *)&tw,     (void *)&twp,
                    (void *)&nrows,    (void *)&ny,     (void *)&conj_in, (void *)&conj_out,
                    (void *)&weight,   (void *)&wscale, (void *)&wscale_dev, (void *)&status};
    return cudaLaunchKernel(fn, dim3(grid), dim3(en->threads), args, en->smem, s);
}

}  // namespace gb300fft
