// Large 1D FFTs, n = 2^14 .. 2^26, beyond what one CTA holds: the four-step
// decomposition the paper names as its next step (Section 6: stage through
// on-chip memory, reorder from DRAM).  With n = n1 * n2 and the input viewed
// as [n1][n2] (element i1*n2 + i2),
//
//   X[k1 + n1*k2] = sum_{i2} w_n2^{i2*k2} * ( w_n^{i2*k1} * sum_{i1} x[i1*n2 + i2] * w_n1^{i1*k1} ).
//
// Pass A is the plain TMA column pass (fft_cols.cu, k_cols) run out of place:
// length-n1 FFTs down the columns into a plan-owned workspace [n1][n2].
// Pass B (this file) multiplies by the inter-pass twiddle w_n^{i2*k1} as it
// loads, runs the length-n2 FFTs along the workspace rows and writes element
// k2 of row k1 to out[k1 + n1*k2]: the transpose that natural output order
// needs is folded into its store.  The inverse needs no conjugation: it is the
// forward transform read at index (n - k) mod n, so pass B stores to the
// reflected position instead.  A CTA takes W adjacent rows (thread t owns row c = t % W,
// butterfly index tt = t / W), so every output position k2 receives W
// consecutive values, W*8 bytes, at once -- whole 32-byte sectors for W >= 4.
// Two HBM passes, 32 bytes per point, as for the 2D transform.
//
// The twiddle of a thread's stage-0 operand e (butterfly b = e / R0, leg
// r = e % R0) is w_n^{k1*(tt + m_e)} with m_e = b*T + r*n2/R0, the same m_e
// for every thread.  So it factors into a per-thread base w_n^{k1*tt} and a
// per-row table G[c][e] = w_n^{k1*m_e} of W*E entries that the CTA builds in
// shared memory; each value comes from two FP64-built tables,
// w_n^a = hi[a >> 13] * lo[a & 8191] with lo[k] = w_n^k, hi[k] = w_n^{8192 k}.
//
// Three passes for n = 2^25, 2^26: a length-8192 axis allows only 16-byte
// tiles (two columns or rows of 64 KiB in one CTA), which halves the DRAM
// efficiency of both passes.  So the row length n / 4096 is split once more,
// n = n1 * M * n3 with n1 = n3 = 4096 and M = 2 or 4 (i2 < M the middle
// digit, i' = i2*n3 + i3):
//   pass A   the length-4096 column FFTs, as above (32-byte tiles);
//   pass M   per (k1, i3): u[i2] = Y[k1][i2][i3] w_n^{i' k1}, an M-point DFT
//            over i2, then the twiddle w_n^{i3 k2 n1} (= w_{M n3}^{i3 k2}) --
//            elementwise and in place, coalesced over i3 (k_fs_mid);
//   pass B   length-4096 row FFTs of row (k1, k2) without twiddle, stored at
//            k1 + n1 k2 + n1 M k3, W = 4 rows of adjacent k1 per CTA.
// 48 bytes per point instead of 32, every pass with 32-byte tiles.
#include <mutex>

#include "fft_common.cuh"
#include "fft_internal.h"

namespace gb300fft {

template <int N, int E, int W>
struct FsRowShape {
    static constexpr int T = N / E;
    static constexpr int THREADS = T * W;
    using Eng = Engine<N, E, W, PadShift<E>::value>;
    // landing layout of a tile: row c at c*ROWP.  A half-warp's 8-byte reads
    // cover 16/W consecutive elements of each of its W rows; a padding of
    // 16/W elements (at least 2, to keep each row's bulk copy 16-byte
    // aligned) puts those W runs on disjoint banks.
    static constexpr int ROWP = N + (16 / W > 2 ? 16 / W : 2);
    static constexpr int ELEMS = Eng::SMEM_ELEMS > W * ROWP ? Eng::SMEM_ELEMS : W * ROWP;
    static constexpr int GROW = E + 1;  // padded row of the twiddle-factor table
    static constexpr size_t G_OFF = (size_t)ELEMS * sizeof(float2);
    static constexpr size_t BAR_OFF = (G_OFF + (size_t)W * GROW * sizeof(float2) + 15) / 16 * 16;
    static constexpr size_t SMEM = BAR_OFF + 16;
    static constexpr uint32_t TILE_BYTES = (uint32_t)W * N * sizeof(float2);
    // E = 16: cap at 64 registers (several CTAs per SM); larger E: one CTA
    static constexpr int MINB_RAW = E <= 16 ? 1024 / THREADS : 1;
    static constexpr int MINB = MINB_RAW < 1 ? 1 : (MINB_RAW > 32 ? 32 : MINB_RAW);
};

__device__ __forceinline__ float2 root_n(const float2 *__restrict__ lohi, int a) {
    return cmul(__ldg(lohi + 8192 + (a >> 13)), __ldg(lohi + (a & 8191)));
}

// Persistent: CTA k takes tiles k, k + gridDim.x, ...  A tile's W rows are
// contiguous in the workspace; W bulk copies (one per row, completion on an
// mbarrier) land them in shared memory, the stage-0 operands are read from
// there, and the buffer then serves as the Stockham exchange.  The next
// tile's copies start as soon as every thread has read its last-stage
// operands, so they overlap the last butterflies and the stores.
// MID: the last pass of the three-pass form (middle digit m, no twiddle);
// otherwise pass B of the four-step form (m = 1, twiddle on load).
template <int N, int E, int W, bool MID>
__global__ void __launch_bounds__(FsRowShape<N, E, W>::THREADS, FsRowShape<N, E, W>::MINB)
    k_rows_fourstep(const float2 *__restrict__ work, float2 *__restrict__ out, const float2 *__restrict__ tw,
                    const float2 *__restrict__ lohi, int n1, long long ntiles, int reverse, int *status,
                    int m_arg) {
    using Sh = FsRowShape<N, E, W>;
    using Eng = typename Sh::Eng;
    constexpr int R0 = Eng::R0;
    constexpr int T = Sh::T;
    extern __shared__ __align__(128) unsigned char raw[];
    float2 *tile = reinterpret_cast<float2 *>(raw);
    float2 *G = reinterpret_cast<float2 *>(raw + Sh::G_OFF);  // [W][E + 1]
    uint64_t *bar = reinterpret_cast<uint64_t *>(raw + Sh::BAR_OFF);
    __shared__ int s_ok;
    const int m = MID ? m_arg : 1;
    const int groups = n1 / W;
    const int t = threadIdx.x;
    const int c = t % W;
    const int tt = t / W;
    const int mask = reverse ? n1 * m * N - 1 : -1;  // n = n1 * m * N is a power of two
    const int sgn = reverse ? -1 : 1;
    // tile id: transform tr, middle digit k2 (m > 1: three passes), rows
    // k1 = k10 .. k10 + W - 1; workspace row (k1, k2) of transform tr at
    // ((tr * n1 + k1) * m + k2) * N
    auto issue = [&](long long id) {  // thread 0: the W row copies of tile `id`
        mbar_expect_tx(bar, Sh::TILE_BYTES);
        const long long tb = id / groups, tr = tb / m;
        const int k2 = (int)(tb - tr * m), k10 = (int)(id - tb * groups) * W;
        const float2 *src = work + ((tr * n1 + k10) * m + k2) * (long long)N;
#pragma unroll 1
        for (int r = 0; r < W; ++r)
            bulk_load(tile + r * Sh::ROWP, src + (long long)r * m * N, N * sizeof(float2), bar);
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
        const long long tb = id / groups;  // transform and middle digit
        const long long b = tb / m;        // transform within the batch
        const int k2m = (int)(tb - b * m);
        const int k10 = (int)(id - tb * groups) * W;
        float2 base = make_float2(1.f, 0.f);
        if constexpr (!MID) {
            for (int q = t; q < W * E; q += Sh::THREADS) {
                const int cq = q / E, e = q % E;
                const int me = (e / R0) * T + (e % R0) * (N / R0);
                G[cq * Sh::GROW + e] = root_n(lohi, (k10 + cq) * me);  // k1 * m_e < n1 * n2
            }
            base = root_n(lohi, (k10 + c) * tt);
        }
        if (t == 0) s_ok = mbar_wait_bounded(bar, phase) ? 1 : 0;
        __syncthreads();
        if (!s_ok) {
            if (t == 0) {
                record_status(status, kStatusTimeout);
                mbar_wait_bounded(bar, phase);  // give the copy in flight a last chance to land
            }
            return;
        }
        phase ^= 1;
        const long long next = id + gridDim.x;
        float2 v[E];
#pragma unroll
        for (int bb = 0; bb < E / R0; ++bb) {
            const int j = tt + bb * T;
#pragma unroll
            for (int r = 0; r < R0; ++r) {
                const int e = bb * R0 + r;
                const float2 x = tile[c * Sh::ROWP + j + r * (N / R0)];
                if constexpr (MID) v[e] = x;
                else v[e] = cmul(x, cmul(base, G[c * Sh::GROW + e]));
            }
        }
        float2 *dst = out + b * (long long)n1 * m * N;
        const int off = k10 + n1 * k2m, ostride = n1 * m;
        auto after_reads = [&] {
            __syncthreads();
            if (t == 0 && next < ntiles) {
                fence_proxy_async_smem();
                issue(next);
            }
        };
        auto store = [&](int i, int cc, float2 x) { dst[(sgn * (off + cc + i * ostride)) & mask] = x; };
        Eng::template run<FftPolicy, true>(v, tile, tw, tt, c, SyncBlock{}, after_reads, store);
    }
}

namespace {
ColVariant g_fs_rows[kMaxLog2 + 1][3][4];  // [log2 n2][E slot: 16, 32, 64][W slot: 2, 4, 8, 16]
const void *g_fs_mid_fn = nullptr;         // the three-pass form's last pass (4096, E = 64, W = 4)
std::once_flag g_fs_rows_once;  // registry filled once, safe across host threads

int e_slot(int e) { return e == 16 ? 0 : e == 32 ? 1 : e == 64 ? 2 : -1; }
int w_slot(int w) { return w == 2 ? 0 : w == 4 ? 1 : w == 8 ? 2 : w == 16 ? 3 : -1; }

// Row length n2 = 128 .. 8192 with W rows per CTA, N*W <= 16384 (an
// exchange buffer of at most 128 KiB plus padding).
template <int N, int E, int W>
void reg_fs_row() {
    static_assert(N * W <= 16384, "exchange buffer");
    using Sh = FsRowShape<N, E, W>;
    ColVariant &v = g_fs_rows[ilog2(N)][e_slot(E)][w_slot(W)];
    v.fn = (const void *)k_rows_fourstep<N, E, W, false>;
    v.n = N;
    v.e = E;
    v.w = W;
    v.threads = Sh::THREADS;
    v.smem = Sh::SMEM;
    v.box_rows = 0;
    v.tw_size = Sched<N, E>::tw_size;
}
template <int N>
void reg_fs_row_ws() {
    reg_fs_row<N, 16, 4>();
    reg_fs_row<N, 16, 8>();
    if constexpr (N <= 1024) reg_fs_row<N, 16, 16>();
}
void init_fs_rows() {
    std::call_once(g_fs_rows_once, [] {
        reg_fs_row_ws<128>();
        reg_fs_row_ws<256>();
        reg_fs_row_ws<512>();
        reg_fs_row_ws<1024>();
        reg_fs_row_ws<2048>();
        reg_fs_row<4096, 16, 4>();
        reg_fs_row<4096, 64, 4>();
        g_fs_mid_fn = (const void *)k_rows_fourstep<4096, 64, 4, true>;
        reg_fs_row<8192, 16, 2>();
        reg_fs_row<8192, 32, 2>();
    });
}
}  // namespace

// Elements per thread pass B prefers for row length n: 64 at 4096 (one
// shared-memory exchange), 32 at 8192 (two), otherwise 16.
int fourstep_row_e(int n) { return n == 4096 ? 64 : n == 8192 ? 32 : 16; }

// Rows per CTA pass B prefers for row length n: 4 (32-byte store chunks;
// measured fastest from 256 to 4096), 8 at 128, 2 at 8192 (the exchange
// buffer's limit).
int fourstep_row_w(int n) { return n >= 8192 ? 2 : n <= 128 ? 8 : 4; }

const ColVariant *fourstep_row_variant(int log2n, int e, int w) {
    init_fs_rows();
    const int es = e_slot(e), ws = w_slot(w);
    if (log2n < 1 || log2n > kMaxLog2 || es < 0 || ws < 0) return nullptr;
    const ColVariant *v = &g_fs_rows[log2n][es][ws];
    return v->fn ? v : nullptr;
}

cudaError_t launch_rows_fourstep(const ColVariant &v, const float2 *work, float2 *out, const float2 *tw,
                                 const float2 *lohi, int n1, int batch, int reverse, int *status, cudaStream_t s,
                                 int m) {
    if (v.w < 1 || n1 % v.w || m < 1) return cudaErrorInvalidValue;
    init_fs_rows();
    // m > 1: the three-pass form's last pass, compiled for 4096-point rows only
    const void *fn = v.fn;
    if (m > 1) {
        if (v.n != 4096 || v.e != 64 || v.w != 4) return cudaErrorInvalidValue;
        fn = g_fs_mid_fn;
    }
    const long long ntiles = (long long)batch * m * (n1 / v.w);
    if (ntiles < 1 || ntiles > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    if (v.smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)v.smem);
        if (e != cudaSuccess) return e;
    }
    // persistent grid: every resident CTA slot once
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, v.threads, v.smem) != cudaSuccess)
        return cudaErrorInvalidConfiguration;
    long long grid = (long long)sms * (per_sm > 0 ? per_sm : 1);
    if (grid > ntiles) grid = ntiles;
    void *args[] = {(void *)&work,   (void *)&out,     (void *)&tw,     (void *)&lohi, (void *)&n1,
                    (void *)&ntiles, (void *)&reverse, (void *)&status, (void *)&m};
    return cudaLaunchKernel(fn, dim3((unsigned)grid), dim3(v.threads), args, v.smem, s);
}

// Middle pass of the three-pass form: one thread per (transform, k1, i3).
template <int M>
__global__ void __launch_bounds__(256) k_fs_mid(float2 *work, const float2 *__restrict__ lohi, int n1, int n3,
                                                long long groups) {
    const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= groups) return;
    const long long tk = gid / n3;  // tr * n1 + k1
    const int i3 = (int)(gid - tk * n3);
    const int k1 = (int)(tk % n1);
    float2 *p = work + tk * M * n3 + i3;  // element (tr, k1, i2, i3)
    float2 v[M];
#pragma unroll
    for (int i2 = 0; i2 < M; ++i2) v[i2] = cmul(p[(long long)i2 * n3], root_n(lohi, (i2 * n3 + i3) * k1));
    dft<M>(v);
#pragma unroll
    for (int k2 = 0; k2 < M; ++k2) p[(long long)k2 * n3] = k2 ? cmul(v[k2], root_n(lohi, i3 * k2 * n1)) : v[k2];
}

cudaError_t launch_fs_mid(float2 *work, const float2 *lohi, int n1, int m, int n3, int batch, cudaStream_t s) {
    const long long groups = (long long)batch * n1 * n3;
    const long long grid = (groups + 255) / 256;
    if (grid > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    if (m == 2) k_fs_mid<2><<<(unsigned)grid, 256, 0, s>>>(work, lohi, n1, n3, groups);
    else if (m == 4) k_fs_mid<4><<<(unsigned)grid, 256, 0, s>>>(work, lohi, n1, n3, groups);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

}  // namespace gb300fft
