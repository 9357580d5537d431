// Column pass by CTA pairs (thread-block clusters of 2).
//
// A column block of length N = 2*N2 is split once more, by decimation in
// frequency:  X[2k + r] = sum_{i<N2} w_N2^{i*k} * w_N^{r*i} * (a[i] + (-1)^r a[i + N2]),
// r in {0, 1}.  The two CTAs of a cluster take the same W columns of a block;
// CTA r loads both halves a[i], a[i + N2] straight from global memory (rows of
// W*8 = 32 bytes, whole DRAM sectors), forms the bracket while loading, and
// runs a length-N2 column FFT whose outputs go to rows 2k + r.  The pair runs
// concurrently by construction, so the second read of each half is an L2 hit
// rather than an HBM read, and each CTA needs only an N2 x W exchange buffer:
// 64 KiB for N2 = 2048, W = 4, instead of the single 128 KiB tile (one CTA per
// SM) a length-4096 block would need.
//
// In place: both CTAs read every row of the block before either writes one,
// which a cluster-wide barrier between the loads and the first store
// guarantees (the loaded values feed the bracket before the barrier, so the
// loads have completed).
//
// Rows of a block are P apart (column pre-split of the row pass): element i
// of block (slice b, kp) is row b*P*N + kp + P*i.
#include <cooperative_groups.h>

#include <mutex>

#include "fft_common.cuh"
#include "fft_internal.h"

namespace gb300fft {

template <int N2, int E, int W>
struct PairShape {
    static constexpr int T = N2 / E;
    static constexpr int THREADS = T * W;
    using Eng = Engine<N2, E, W, PadShift<E>::value>;
    static constexpr size_t SMEM = sizeof(float2) * (size_t)Eng::SMEM_ELEMS;
    static constexpr int MINB = E >= 32 ? 2 : (THREADS >= 512 ? 2 : 3);
};

__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

template <int N2, int E, int W>
__global__ void __launch_bounds__(PairShape<N2, E, W>::THREADS, PairShape<N2, E, W>::MINB)
    k_cols_pair(float2 *data, const float2 *__restrict__ tw, const float2 *__restrict__ roots, int nx,
                long long nblocks, int P, int conj_out) {
    using Sh = PairShape<N2, E, W>;
    using Eng = typename Sh::Eng;
    constexpr int T = Sh::T;
    constexpr int R0 = Eng::R0;
    constexpr int N = 2 * N2;
    extern __shared__ __align__(16) float2 smem[];
    const int r = blockIdx.x & 1;  // rank in the cluster: output parity
    const long long tile = blockIdx.x >> 1;
    const int groups_x = nx / W;
    const long long blk = tile / groups_x;  // b * P + kp
    const int gx = (int)(tile - blk * groups_x);
    const long long b = blk / P;
    const int kp = (int)(blk - b * P);
    float2 *base = data + (b * (long long)P * N + kp) * nx + (long long)gx * W;
    const long long rstride = (long long)P * nx;  // between consecutive block elements
    const int t = threadIdx.x;
    const int c = t % W;
    const int tt = t / W;
    const float sgn = r ? -1.f : 1.f;
    const float so = conj_out ? -1.f : 1.f;
    const bool valid = blk < nblocks;

    float2 v[E];
#pragma unroll
    for (int bb = 0; bb < E / R0; ++bb) {
        const int j = tt + bb * T;
#pragma unroll
        for (int q = 0; q < R0; ++q) {
            const int i = j + q * (N2 / R0);  // 0 <= i < N2
            float2 x = make_float2(0.f, 0.f);
            if (valid) {
                const float2 lo = __ldcg(base + (long long)i * rstride + c);
                const float2 hi = __ldcg(base + (long long)(i + N2) * rstride + c);
                x = make_float2(fmaf(sgn, hi.x, lo.x), fmaf(sgn, hi.y, lo.y));
                if (r) x = cmul(x, __ldg(roots + i));  // w_N^i
            }
            v[bb * R0 + q] = x;
        }
    }
    // both CTAs of the pair hold every input they need: writes may start
    cluster_sync_all();
    auto store = [&](int i, int cc, float2 x) {
        if (valid) {
            x.y *= so;
            base[(long long)(2 * i + r) * rstride + cc] = x;
        }
    };
    auto none = [] {};
    Eng::template run<FftPolicy, false>(v, smem, tw, tt, c, SyncBlock{}, none, store);
}

namespace {
struct PairEntry {
    const void *fn = nullptr;
    int threads = 0, w = 0, e = 0;
    size_t smem = 0;
    int tw_size = 0;
};
PairEntry g_pair[kMaxLog2 + 1][2];  // [log2 N2][E slot: 16, 32]
std::once_flag g_pair_once;  // registry filled once, safe across host threads

template <int N2, int E, int W>
void reg_pair() {
    using Sh = PairShape<N2, E, W>;
    PairEntry &en = g_pair[ilog2(N2)][E == 32 ? 1 : 0];
    en.fn = (const void *)k_cols_pair<N2, E, W>;
    en.threads = Sh::THREADS;
    en.w = W;
    en.e = E;
    en.smem = Sh::SMEM;
    en.tw_size = Sched<N2, E>::tw_size;
}
void init_pair() {
    std::call_once(g_pair_once, [] {
        reg_pair<1024, 16, 8>();
        reg_pair<1024, 32, 8>();
        reg_pair<2048, 16, 4>();
        reg_pair<2048, 32, 4>();
        reg_pair<4096, 16, 2>();
        reg_pair<4096, 32, 2>();
    });
}
const PairEntry *pair_entry(int n2, int e) {
    init_pair();
    if (n2 < 1024 || n2 > 4096 || (n2 & (n2 - 1))) return nullptr;
    const PairEntry *en = &g_pair[ilog2(n2)][e == 32 ? 1 : 0];
    return en->fn ? en : nullptr;
}
}  // namespace

// Column block length n = 2 * N2 handled by the pair kernel with E elements
// per thread: its tile width, or 0 if no variant exists for nx columns.
int pair_cols_width(int n, int e, int nx) {
    const PairEntry *en = pair_entry(n / 2, e);
    return (en && en->w <= nx) ? en->w : 0;
}
int pair_cols_tw_size(int n, int e) {
    const PairEntry *en = pair_entry(n / 2, e);
    return en ? en->tw_size : -1;
}

cudaError_t launch_cols_pair(int n, int e, float2 *data, const float2 *tw, const float2 *roots, int nx, int batch,
                             int split, int conj_out, cudaStream_t s) {
    const PairEntry *en = pair_entry(n / 2, e);
    if (!en || en->w > nx) return cudaErrorInvalidValue;
    if (en->smem > 48 * 1024) {
        cudaError_t err = cudaFuncSetAttribute(en->fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)en->smem);
        if (err != cudaSuccess) return err;
    }
    const long long nblocks = (long long)batch * split;
    const long long ntiles = nblocks * (nx / en->w);
    if (2 * ntiles > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(2 * ntiles));
    cfg.blockDim = dim3(en->threads);
    cfg.dynamicSmemBytes = en->smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    void *args[] = {(void *)&data, (void *)&tw, (void *)&roots, (void *)&nx,
                    (void *)&nblocks, (void *)&split, (void *)&conj_out};
    return cudaLaunchKernelExC(&cfg, en->fn, args);
}

}  // namespace gb300fft
