// Streaming column pass over a row-permuted intermediate.
//
// The plain column pass (fft_cols.cu) must hold a whole [N x W] tile before
// its first stage can start: a stage-0 butterfly combines the column elements
// j + r*T (r < R0), spread over the whole column.  So a tile's loads and its
// compute alternate, and with one 128 KiB tile per SM the HBM sits idle
// while the first stage runs.
//
// Here the row pass (which writes the intermediate anyway) stores column
// element i = j + r*T (j < T butterflies of stage 0, r < R0 legs) at block
// row
//     sigma(i) = (j / G) * G*R0 + r*G + (j % G),      G = 32 / W,
// so the G butterflies one warp owns read one contiguous run of G*R0 rows --
// a 16 KiB segment for N = 4096, W = 4.  Each warp waits only for its own
// segment, on its own mbarrier.  Warps 0 .. S-1 own a ring slot each, which
// they refill with their segment of the next tile right after reading it;
// the segments of warps S and up land in those warps' own spans of the
// exchange buffer, issued as soon as stage 1 has read the exchange.  So the
// next tile's copies run during this tile's butterflies and stores, every
// barrier has one consumer warp that takes its phases in tile order, and the
// first butterflies of a tile start when their own segment has landed.  The
// schedule is the two-stage one of the plain pass with E = R0 = 64: stage 0
// from the landed segments, one exchange, stage 1 with twiddles,
// natural-order stores.
//
// Rows of a block are P apart (the row pass's column pre-split) and the
// output goes to the same rows it came from in natural order, so the pass is
// in place on the intermediate; or (planar) the row pass wrote each block as
// a plane of its own in a workspace, read here through a P = 1 map, and the
// output goes to the interleaved rows of the destination.
#include <mutex>

#include "fft_common.cuh"
#include "fft_internal.h"

namespace gb300fft {

template <int N, int E, int W, int S, bool TS>
struct StreamShape {
    using Eng = Engine<N, E, W, PadShift<E>::value>;
    static constexpr int T = N / E;   // stage-0 butterflies per column
    static constexpr int R0 = Eng::R0;
    static_assert(Eng::S == 2 && R0 == E, "two-stage schedule with E = R0");
    static constexpr int THREADS = T * W;
    static constexpr int WARPS = THREADS / 32;       // = segments per tile
    static constexpr int G = 32 / W;                 // butterflies per warp
    static constexpr int SEG_ROWS = G * R0;          // rows per segment
    static constexpr int SEG_ELEMS = SEG_ROWS * W;
    static constexpr int BOXR = SEG_ROWS < 256 ? SEG_ROWS : 256;
    static constexpr uint32_t SEG_BYTES = (uint32_t)SEG_ELEMS * sizeof(float2);
    // warp w's stage-0 exchange writes fill the padded span starting at
    // pad(w * SEG_ELEMS); a warp without a ring slot lands its segment there
    static constexpr int xch_seg(int w) { return Eng::pad(w * SEG_ELEMS); }
    static constexpr size_t RING_OFF = ((size_t)Eng::SMEM_ELEMS * sizeof(float2) + 127) / 128 * 128;
    // TS: outputs leave through TMA stores.  Stage-1 output k of thread
    // (tt, c) is output row tt + T*k; a warp's G butterflies are G adjacent
    // rows tt, so KB consecutive k form a box of KB x G rows x W columns,
    // staged per warp in two alternating chunks.
    static constexpr int KB = 8;
    static constexpr int CHUNK_ELEMS = KB * G * W;
    static constexpr size_t STG_OFF = RING_OFF + (size_t)S * SEG_BYTES;
    static constexpr size_t STG_BYTES = TS ? (size_t)WARPS * 2 * CHUNK_ELEMS * sizeof(float2) : 0;
    static constexpr size_t BAR_OFF = STG_OFF + STG_BYTES;
    static constexpr size_t SMEM = BAR_OFF + 8 * WARPS + 16;
    static_assert(E % KB == 0 && (CHUNK_ELEMS * sizeof(float2)) % 128 == 0, "store chunks");
    static_assert(WARPS * G == T, "one warp per G butterflies");
    static_assert(S >= 1 && S <= WARPS, "ring slots");
    static_assert(Eng::pad((WARPS - 1) * SEG_ELEMS) + SEG_ELEMS <= Eng::SMEM_ELEMS, "landing span");
};

template <int N, int E, int W, int S, bool TS>
__global__ void __launch_bounds__(StreamShape<N, E, W, S, TS>::THREADS, 1)
    k_cols_stream(const __grid_constant__ CUtensorMap map, const __grid_constant__ CUtensorMap omap, float2 *out,
                  const float2 *__restrict__ tw, int nx, int batch, int P, int conj_out, int *status, int planar) {
    using Sh = StreamShape<N, E, W, S, TS>;
    using Eng = typename Sh::Eng;
    constexpr int T = Sh::T;
    constexpr int R0 = Sh::R0;
    constexpr int G = Sh::G;
    constexpr int WARPS = Sh::WARPS;
    extern __shared__ __align__(128) unsigned char raw[];
    float2 *xch = reinterpret_cast<float2 *>(raw);
    float2 *ring = reinterpret_cast<float2 *>(raw + Sh::RING_OFF);
    float2 *stg = reinterpret_cast<float2 *>(raw + Sh::STG_OFF);  // TS: [warp][2][CHUNK_ELEMS]
    uint64_t *full = reinterpret_cast<uint64_t *>(raw + Sh::BAR_OFF);  // one per warp
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
    // this CTA's tiles: blockIdx.x + m * gridDim.x, m < mt
    const long long mt = blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const float so = conj_out ? -1.f : 1.f;
    // segment w of a tile lands in ring slot w (w < S) or in warp w's own
    // span of the exchange buffer (w >= S)
    auto seg_buf = [&](int w) -> float2 * {
        return w < S ? ring + (size_t)w * Sh::SEG_ELEMS : xch + Sh::xch_seg(w);
    };
    // TMA copies of segment w of local tile m, completing on full[w]
    auto issue = [&](long long m, int w) {
        const long long id = blockIdx.x + m * (long long)gridDim.x;
        const int x = (int)(id % groups_x) * 2 * W;
        // block b*P + kp: rows kp + P*i of slice b (map over the output), or
        // planar, rows (b*P + kp)*N + i of a workspace whose map has P = 1
        const int kp = planar ? 0 : (int)((id / groups_x) % P);
        const int z0 = (int)(planar ? (id / groups_x) : (id / groups_x) / P) * N + w * Sh::SEG_ROWS;
        float2 *dst = seg_buf(w);
        mbar_expect_tx(full + w, Sh::SEG_BYTES);
#pragma unroll
        for (int k = 0; k < Sh::SEG_ROWS / Sh::BOXR; ++k)
            tma_load_3d(dst + k * Sh::BOXR * W, &map, x, kp, z0 + k * Sh::BOXR, full + w);
        s_armed[w] += 1;
    };
    if (t == 0) {
        s_fail = 0;
        for (int w = 0; w < WARPS; ++w) {
            mbar_init(full + w, 1);
            s_armed[w] = 0;
        }
        fence_mbar_init();
        fence_proxy_async_smem();
        if (mt > 0)
            for (int w = 0; w < WARPS; ++w) issue(0, w);
    }
    __syncthreads();

    long long m = 0;
    for (; m < mt; ++m) {
        const long long id = blockIdx.x + m * (long long)gridDim.x;
        // stage 0: this warp's segment (one barrier, one consumer, phases in
        // tile order), read, then the ring slot refilled for the next tile
        float2 v[E];
        const bool ok = mbar_wait_bounded(full + warp, (uint32_t)(m & 1));
        if (ok) {
            const float2 *seg = seg_buf(warp);
#pragma unroll
            for (int r = 0; r < R0; ++r) v[r] = seg[(r * G + ttl) * W + c];
        } else {
            atomicOr(&s_fail, 1);
        }
        __syncwarp();
        if (warp < S && lane == 0 && ok && m + 1 < mt) {
            fence_proxy_async_smem();
            issue(m + 1, warp);
        }
        if (ok) {
            dft<R0>(v);
            // into this warp's own exchange span (its landed segment, if any,
            // is already in registers)
#pragma unroll
            for (int k = 0; k < R0; ++k) xch[Eng::pad((tt * R0 + k) * W + c)] = v[k];
        }
        __syncthreads();
        if (s_fail) break;
        // stage 1: exchange reads, twiddles, DFT-E, natural-order stores
        constexpr int Ns = R0;  // span of stage 1
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
        dft<E>(v);
        const long long blk = id / groups_x;  // b*P + kp
        const long long b = blk / P;
        const int kp = (int)(blk - b * P);
        if constexpr (TS) {
            // output box (x, kp, rows tt of this warp, k-blocks) of the map
            // {floats of a row, kp, ky mod T, slice*E + ky / T}
            float2 *wst = stg + (size_t)warp * 2 * Sh::CHUNK_ELEMS;
            const int xo = (int)(id % groups_x) * 2 * W;
            const int kb0 = (int)b * E;
#pragma unroll
            for (int rr = 0; rr < E / Sh::KB; ++rr) {
                float2 *cb = wst + (rr & 1) * Sh::CHUNK_ELEMS;
                if (lane == 0) bulk_wait_read_1();  // the chunk's store of two rounds ago has read it
                __syncwarp();
#pragma unroll
                for (int kk = 0; kk < Sh::KB; ++kk) {
                    float2 x = v[rr * Sh::KB + kk];
                    x.y *= so;
                    cb[(kk * G + ttl) * W + c] = x;
                }
                fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0) {
                    tma_store_4d(&omap, cb, xo, kp, warp * G, kb0 + rr * Sh::KB);
                    bulk_commit();
                }
            }
        } else {
            float2 *dst = out + (b * N * P + kp) * (long long)nx + (long long)(id % groups_x) * W + c;
            const long long rstride = (long long)P * nx;
#pragma unroll
            for (int k = 0; k < E; ++k) {
                float2 x = v[k];
                x.y *= so;
                dst[(long long)(tt + k * (N / E)) * rstride] = x;
            }
        }
    }
    if constexpr (TS) {
        if (lane == 0) bulk_wait_all();  // this warp's stores are complete before the CTA leaves
    }
    if (s_fail && t == 0) {
        record_status(status, kStatusTimeout);
        // let the copies still in flight land before the CTA leaves: barrier
        // w has completed min(m, armed) phases of the s_armed[w] it was given
        for (int w = 0; w < WARPS; ++w)
            for (long long ph = m; ph < s_armed[w]; ++ph)
                mbar_wait_bounded(full + w, (uint32_t)(ph & 1), 10000000ull);
    }
}

namespace {
struct StreamEntry {
    ColVariant v;
    int g = 0, r0 = 0, t = 0, kb = 0;
};
StreamEntry g_stream[2];  // [TMA stores]
std::once_flag g_stream_once;  // registry filled once, safe across host threads

template <int N, int E, int W, int S, bool TS>
void reg_stream(StreamEntry &en) {
    using Sh = StreamShape<N, E, W, S, TS>;
    en.v.fn = (const void *)k_cols_stream<N, E, W, S, TS>;
    en.v.n = N;
    en.v.e = E;
    en.v.w = W;
    en.v.threads = Sh::THREADS;
    en.v.smem = Sh::SMEM;
    en.v.box_rows = Sh::BOXR;
    en.v.tw_size = Sched<N, E>::tw_size;
    en.g = Sh::G;
    en.r0 = Sh::R0;
    en.t = Sh::T;
    en.kb = Sh::KB;
}

void init_stream() {
    std::call_once(g_stream_once, [] {
        // 130 KiB exchange + 80 KiB ring; with TMA stores 130 KiB + 64 KiB
        // ring + 32 KiB store staging
        reg_stream<4096, 64, 4, 5, false>(g_stream[0]);
        reg_stream<4096, 64, 4, 4, true>(g_stream[1]);
    });
}
}  // namespace

const ColVariant *stream_col_variant(int n, int nx, int *perm_t, int *perm_g, int tstore) {
    init_stream();
    const StreamEntry &en = g_stream[tstore ? 1 : 0];
    if (n != en.v.n || nx < en.v.w) return nullptr;
    if (perm_t) *perm_t = n / en.r0;
    if (perm_g) *perm_g = en.g;
    return &en.v;
}

bool stream_tstore(const ColVariant &v) {
    init_stream();
    return v.fn == g_stream[1].v.fn;
}

int encode_stream_store_map(CUtensorMap *map, const ColVariant &v, const void *base, int nx, long long rows,
                            int split) {
    init_stream();
    const StreamEntry &en = g_stream[1];
    if (v.fn != en.v.fn) return -1;
    const int T = en.t;  // output row ky = tt + T*k
    if (split < 1 || rows % ((long long)split * T) != 0) return -1;
    return encode_map4(map, base, nx, rows, split, T, en.v.w, en.g, en.kb);
}

cudaError_t launch_cols_stream(const ColVariant &v, const CUtensorMap &map, const CUtensorMap *omap, float2 *out,
                               const float2 *tw, int nx, int batch, int split, int conj_out, int *status, int grid,
                               int planar, cudaStream_t s) {
    const bool ts = stream_tstore(v);
    if (ts && !omap) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(v.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)v.smem);
    if (e != cudaSuccess) return e;
    CUtensorMap m = map;
    CUtensorMap om = ts ? *omap : map;  // unused by the plain-store kernel
    void *args[] = {(void *)&m,     (void *)&om,    (void *)&out,      (void *)&tw,     (void *)&nx, (void *)&batch,
                    (void *)&split, (void *)&conj_out, (void *)&status, (void *)&planar};
    return cudaLaunchKernel(v.fn, dim3(grid), dim3(v.threads), args, v.smem, s);
}

}  // namespace gb300fft
