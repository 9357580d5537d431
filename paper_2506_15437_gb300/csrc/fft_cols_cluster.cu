// Column pass by thread-block clusters sharing one column block through
// distributed shared memory (DSMEM).
//
// A column block of length N = C * NQ (C = 2 or 4 CTAs per cluster) is split
// by decimation in frequency:
//   X[C*k + q] = sum_{i<NQ} w_NQ^{i*k} * w_N^{q*i} * (sum_{r<C} x[i + NQ*r] w_C^{r*q}).
// CTA r of the cluster stages rows [r*NQ, (r+1)*NQ) of the block (W adjacent
// columns) in its own shared memory with 2D/3D TMA copies -- rows of W*8 = 32
// bytes, whole DRAM sectors, each byte read from HBM once.  After a cluster
// barrier, CTA q forms the bracket for its outputs by reading slice r of
// every partner through DSMEM, multiplies by w_N^{q*i}, and after a second
// cluster barrier (nobody reads a partner's slice any more) transforms its
// length-NQ column FFT in its own buffer and writes rows C*k + q of the block.
// So the block is spread over C SMs: each CTA needs one NQ x W slice (64 KiB
// for NQ = 2048, W = 4) instead of a whole N x W tile, which lets two or three
// CTAs share an SM where a single 128 KiB tile allowed only one.
//
// In place: every CTA finished reading every slice before the second barrier,
// and no CTA stores before it.  Rows of a block are P apart (the row pass's
// column pre-split): element i of block (slice b, kp) is row b*P*N + kp + P*i.
#include <cooperative_groups.h>

#include <mutex>

#include "fft_common.cuh"
#include "fft_internal.h"

namespace cg = cooperative_groups;

namespace gb300fft {

template <int NQ, int E, int W, int C>
struct ClusterShape {
    static constexpr int T = NQ / E;
    static constexpr int THREADS = T * W;
    using Eng = Engine<NQ, E, W, PadShift<E>::value>;
    static constexpr int ELEMS = Eng::SMEM_ELEMS > NQ * W ? Eng::SMEM_ELEMS : NQ * W;
    static constexpr int BOXR = NQ < 256 ? NQ : 256;
    static constexpr uint32_t SLICE_BYTES = (uint32_t)NQ * W * sizeof(float2);
    static constexpr size_t BAR_OFF = ((size_t)ELEMS * sizeof(float2) + 127) / 128 * 128;
    static constexpr size_t SMEM = BAR_OFF + 16;
    static constexpr int MINB = E >= 32 ? 2 : (THREADS >= 512 ? 2 : 3);
};

__device__ __forceinline__ float2 mul_pow_minus_i(float2 x, int k) {  // x * (-i)^k
    switch (k & 3) {
        case 0: return x;
        case 1: return make_float2(x.y, -x.x);
        case 2: return make_float2(-x.x, -x.y);
        default: return make_float2(-x.y, x.x);
    }
}

template <int NQ, int E, int W, int C>
__global__ void __launch_bounds__(ClusterShape<NQ, E, W, C>::THREADS, ClusterShape<NQ, E, W, C>::MINB)
    k_cols_cluster(const __grid_constant__ CUtensorMap map, float2 *out, const float2 *__restrict__ tw,
                   const float2 *__restrict__ roots, int nx, int P, int conj_out, int *status) {
    using Sh = ClusterShape<NQ, E, W, C>;
    using Eng = typename Sh::Eng;
    constexpr int T = Sh::T;
    constexpr int R0 = Eng::R0;
    constexpr int N = C * NQ;
    extern __shared__ __align__(128) unsigned char raw[];
    float2 *tile = reinterpret_cast<float2 *>(raw);
    uint64_t *bar = reinterpret_cast<uint64_t *>(raw + Sh::BAR_OFF);
    __shared__ int s_ok;
    cg::cluster_group cluster = cg::this_cluster();
    const int q = (int)cluster.block_rank();
    const long long tid = blockIdx.x / C;  // (block, column group)
    const int groups_x = nx / W;
    const long long blk = tid / groups_x;  // b * P + kp
    const int gx = (int)(tid - blk * groups_x);
    const long long b = blk / P;
    const int kp = (int)(blk - b * P);
    const int t = threadIdx.x;
    const int c = t % W;
    const int tt = t / W;

    if (t == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
        fence_proxy_async_smem();
        mbar_expect_tx(bar, Sh::SLICE_BYTES);
        // this CTA's slice: block elements [q*NQ, (q+1)*NQ) -> coordinates
        // (float within row, kp, b*N + i) of the 3D map
        const int x = gx * 2 * W;
        const int z0 = (int)(b * N) + q * NQ;
#pragma unroll 1
        for (int k = 0; k < NQ / Sh::BOXR; ++k) tma_load_3d(tile + k * Sh::BOXR * W, &map, x, kp, z0 + k * Sh::BOXR, bar);
        s_ok = mbar_wait_bounded(bar, 0) ? 1 : 0;
        if (!s_ok) record_status(status, kStatusTimeout);
    }
    // every slice of the cluster has landed (a CTA whose copy timed out still
    // takes part in both barriers, so its partners never wait forever)
    cluster.sync();
    const float2 *slice[C];
#pragma unroll
    for (int r = 0; r < C; ++r) slice[r] = cluster.map_shared_rank(tile, r);

    float2 v[E];
#pragma unroll
    for (int bb = 0; bb < E / R0; ++bb) {
        const int j = tt + bb * T;
#pragma unroll
        for (int rr = 0; rr < R0; ++rr) {
            const int i = j + rr * (NQ / R0);  // 0 <= i < NQ
            const int off = i * W + c;
            float2 acc = slice[0][off];
#pragma unroll
            for (int r = 1; r < C; ++r)  // w_C^{r*q} = (-i)^{r*q*4/C}
                acc = cadd(acc, mul_pow_minus_i(slice[r][off], (4 / C) * r * q));
            if (q) acc = cmul(acc, __ldg(roots + q * i));  // w_N^{q*i}
            v[bb * R0 + rr] = acc;
        }
    }
    // nobody reads a partner's slice after this point
    cluster.sync();
    const bool ok = s_ok != 0;
    float2 *base = out + (b * (long long)P * N + kp) * nx + (long long)gx * W;
    const long long rstride = (long long)P * nx;
    const float so = conj_out ? -1.f : 1.f;
    auto store = [&](int i, int cc, float2 x) {
        if (ok) {
            x.y *= so;
            base[(long long)(C * i + q) * rstride + cc] = x;
        }
    };
    auto none = [] {};
    Eng::template run<FftPolicy, false>(v, tile, tw, tt, c, SyncBlock{}, none, store);
}

namespace {
struct ClusterEntry {
    const void *fn = nullptr;
    int threads = 0, w = 0, box_rows = 0;
    size_t smem = 0;
    int tw_size = 0;
};
ClusterEntry g_cl[3][2][2];  // [C slot: 2, 4][NQ slot: 1024, 2048][E slot: 16, 32]
std::once_flag g_cl_once;  // registry filled once, safe across host threads

template <int NQ, int E, int C>
void reg_cl() {
    constexpr int W = 4;
    using Sh = ClusterShape<NQ, E, W, C>;
    ClusterEntry &en = g_cl[C == 2 ? 0 : 1][NQ == 1024 ? 0 : 1][E == 32 ? 1 : 0];
    en.fn = (const void *)k_cols_cluster<NQ, E, W, C>;
    en.threads = Sh::THREADS;
    en.w = W;
    en.box_rows = Sh::BOXR;
    en.smem = Sh::SMEM;
    en.tw_size = Sched<NQ, E>::tw_size;
}
void init_cl() {
    std::call_once(g_cl_once, [] {
        reg_cl<1024, 16, 2>();
        reg_cl<1024, 32, 2>();
        reg_cl<2048, 16, 2>();
        reg_cl<2048, 32, 2>();
        reg_cl<1024, 16, 4>();
        reg_cl<1024, 32, 4>();
        reg_cl<2048, 16, 4>();
        reg_cl<2048, 32, 4>();
    });
}
const ClusterEntry *cl_entry(int n, int e, int C) {
    init_cl();
    if (C != 2 && C != 4) return nullptr;
    const int nq = n / C;
    if (nq != 1024 && nq != 2048) return nullptr;
    const ClusterEntry *en = &g_cl[C == 2 ? 0 : 1][nq == 1024 ? 0 : 1][e == 32 ? 1 : 0];
    return en->fn ? en : nullptr;
}
}  // namespace

int cluster_cols_width(int n, int e, int C, int nx) {
    const ClusterEntry *en = cl_entry(n, e, C);
    return (en && en->w <= nx) ? en->w : 0;
}
int cluster_cols_tw_size(int n, int e, int C) {
    const ClusterEntry *en = cl_entry(n, e, C);
    return en ? en->tw_size : -1;
}
int cluster_cols_box_rows(int n, int e, int C) {
    const ClusterEntry *en = cl_entry(n, e, C);
    return en ? en->box_rows : 0;
}

cudaError_t launch_cols_cluster(int n, int e, int C, const CUtensorMap &map, float2 *out, const float2 *tw,
                                const float2 *roots, int nx, int batch, int split, int conj_out, int *status,
                                cudaStream_t s) {
    const ClusterEntry *en = cl_entry(n, e, C);
    if (!en || en->w > nx) return cudaErrorInvalidValue;
    cudaError_t err = cudaFuncSetAttribute(en->fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)en->smem);
    if (err != cudaSuccess) return err;
    const long long ntiles = (long long)batch * split * (nx / en->w);
    if ((long long)C * ntiles > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(C * ntiles));
    cfg.blockDim = dim3(en->threads);
    cfg.dynamicSmemBytes = en->smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    CUtensorMap m = map;
    void *args[] = {(void *)&m, (void *)&out, (void *)&tw, (void *)&roots, (void *)&nx,
                    (void *)&split, (void *)&conj_out, (void *)&status};
    return cudaLaunchKernelExC(&cfg, en->fn, args);
}

}  // namespace gb300fft
