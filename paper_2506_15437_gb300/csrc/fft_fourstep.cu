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
#include "fft_common.cuh"
#include "fft_internal.h"

namespace gb300fft {

template <int N, int E, int W>
struct FsRowShape {
    static constexpr int T = N / E;
    static constexpr int THREADS = T * W;
    using Eng = Engine<N, E, W, PadShift<E>::value>;
    static constexpr int GROW = E + 1;  // padded row of the twiddle-factor table
    static constexpr size_t SMEM = sizeof(float2) * ((size_t)Eng::SMEM_ELEMS + (size_t)W * GROW);
};

__device__ __forceinline__ float2 root_n(const float2 *__restrict__ lohi, int a) {
    return cmul(__ldg(lohi + 8192 + (a >> 13)), __ldg(lohi + (a & 8191)));
}

template <int N, int E, int W>
__global__ void __launch_bounds__(FsRowShape<N, E, W>::THREADS)
    k_rows_fourstep(const float2 *__restrict__ work, float2 *__restrict__ out, const float2 *__restrict__ tw,
                    const float2 *__restrict__ lohi, int n1, long long ntiles, int reverse) {
    using Sh = FsRowShape<N, E, W>;
    using Eng = typename Sh::Eng;
    constexpr int R0 = Eng::R0;
    constexpr int T = Sh::T;
    extern __shared__ __align__(16) float2 smem[];
    float2 *G = smem + Eng::SMEM_ELEMS;  // [W][E + 1]
    const long long id = blockIdx.x;
    if (id >= ntiles) return;
    const int groups = n1 / W;
    const long long b = id / groups;  // transform within the batch
    const int k10 = (int)(id - b * groups) * W;
    const int t = threadIdx.x;
    const int c = t % W;
    const int tt = t / W;
    const float2 *src = work + (b * n1 + k10 + c) * (long long)N;
    float2 v[E];
#pragma unroll
    for (int bb = 0; bb < E / R0; ++bb) {
        const int j = tt + bb * T;
#pragma unroll
        for (int r = 0; r < R0; ++r) v[bb * R0 + r] = __ldcs(src + j + r * (N / R0));  // read once
    }
    for (int q = t; q < W * E; q += Sh::THREADS) {
        const int cq = q / E, e = q % E;
        const int me = (e / R0) * T + (e % R0) * (N / R0);
        G[cq * Sh::GROW + e] = root_n(lohi, (k10 + cq) * me);  // k1 * m_e < n1 * n2
    }
    const float2 base = root_n(lohi, (k10 + c) * tt);
    __syncthreads();
#pragma unroll
    for (int e = 0; e < E; ++e) v[e] = cmul(v[e], cmul(base, G[c * Sh::GROW + e]));
    float2 *dst = out + b * (long long)n1 * N;
    const int mask = reverse ? n1 * N - 1 : -1;  // n = n1 * N is a power of two
    const int sgn = reverse ? -1 : 1;
    auto none = [] {};
    auto store = [&](int i, int cc, float2 x) { dst[(sgn * (k10 + cc + i * n1)) & mask] = x; };
    Eng::template run<FftPolicy, false>(v, smem, tw, tt, c, SyncBlock{}, none, store);
}

namespace {
ColVariant g_fs_rows[kMaxLog2 + 1][3][4];  // [log2 n2][E slot: 16, 32, 64][W slot: 2, 4, 8, 16]
bool g_fs_rows_init = false;

int e_slot(int e) { return e == 16 ? 0 : e == 32 ? 1 : e == 64 ? 2 : -1; }
int w_slot(int w) { return w == 2 ? 0 : w == 4 ? 1 : w == 8 ? 2 : w == 16 ? 3 : -1; }

// Row length n2 = 128 .. 8192 with W rows per CTA, N*W <= 16384 (an
// exchange buffer of at most 128 KiB plus padding).
template <int N, int E, int W>
void reg_fs_row() {
    static_assert(N * W <= 16384, "exchange buffer");
    using Sh = FsRowShape<N, E, W>;
    ColVariant &v = g_fs_rows[ilog2(N)][e_slot(E)][w_slot(W)];
    v.fn = (const void *)k_rows_fourstep<N, E, W>;
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
    if (g_fs_rows_init) return;
    reg_fs_row_ws<128>();
    reg_fs_row_ws<256>();
    reg_fs_row_ws<512>();
    reg_fs_row_ws<1024>();
    reg_fs_row_ws<2048>();
    reg_fs_row<4096, 16, 4>();
    reg_fs_row<4096, 64, 4>();
    reg_fs_row<8192, 16, 2>();
    reg_fs_row<8192, 32, 2>();
    g_fs_rows_init = true;
}
}  // namespace

// Elements per thread pass B prefers for row length n: 64 at 4096 (one
// shared-memory exchange), 32 at 8192 (two), otherwise 16.
int fourstep_row_e(int n) { return n == 4096 ? 64 : n == 8192 ? 32 : 16; }

// Rows per CTA pass B prefers for row length n: 4 (32-byte store chunks,
// 64-byte row segments per load; measured fastest from 128 to 4096), 2 at
// 8192 (the exchange buffer's limit).
int fourstep_row_w(int n) { return n >= 8192 ? 2 : 4; }

const ColVariant *fourstep_row_variant(int log2n, int e, int w) {
    init_fs_rows();
    const int es = e_slot(e), ws = w_slot(w);
    if (log2n < 1 || log2n > kMaxLog2 || es < 0 || ws < 0) return nullptr;
    const ColVariant *v = &g_fs_rows[log2n][es][ws];
    return v->fn ? v : nullptr;
}

cudaError_t launch_rows_fourstep(const ColVariant &v, const float2 *work, float2 *out, const float2 *tw,
                                 const float2 *lohi, int n1, int batch, int reverse, cudaStream_t s) {
    if (v.w < 1 || n1 % v.w) return cudaErrorInvalidValue;
    const long long ntiles = (long long)batch * (n1 / v.w);
    if (ntiles < 1 || ntiles > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    if (v.smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(v.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)v.smem);
        if (e != cudaSuccess) return e;
    }
    void *args[] = {(void *)&work, (void *)&out,    (void *)&tw,     (void *)&lohi,
                    (void *)&n1,   (void *)&ntiles, (void *)&reverse};
    return cudaLaunchKernel(v.fn, dim3((unsigned)ntiles), dim3(v.threads), args, v.smem, s);
}

}  // namespace gb300fft
