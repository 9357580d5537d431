// Column pass: batched length-N FFTs down the columns of each [N][nx] slice
// (the second half of the paper's Section 5 decomposition).  The paper moves
// data between the two halves with a global transpose (Fig. 6); here there is
// none.  Each CTA stages a tile of W adjacent columns x N rows into shared
// memory with 2D TMA copies (cp.async.bulk.tensor, completion on an mbarrier),
// transforms the W columns with the same Stockham engine as the row pass, and
// stores natural-order results back into the same columns.
//
// CTAs are persistent: each walks tiles blockIdx.x, blockIdx.x + gridDim.x,
// ...  While tile k is being transformed, tile k+1 sits in L2 (bulk L2
// prefetch issued one tile ahead) and its TMA load into shared memory starts
// as soon as every thread has read its last-stage operands of tile k, so the
// load overlaps the last butterflies and the stores of tile k.
#include <mutex>

#include "fft_common.cuh"
#include "fft_internal.h"

namespace gb300fft {

template <int N, int E, int W>
struct ColShape {
    static constexpr int T = N / E;
    static constexpr int THREADS = T * W;
    static constexpr int MINB = THREADS >= 512 ? (E >= 32 ? 512 : 1024) / THREADS : (THREADS >= 256 && E < 32 ? 3 : 1);
    using Eng = Engine<N, E, W, PadShift<E>::value>;
    static constexpr int ELEMS = Eng::SMEM_ELEMS > N * W ? Eng::SMEM_ELEMS : N * W;
    static constexpr int BOXR = N < 256 ? N : 256;
    static constexpr uint32_t TILE_BYTES = (uint32_t)N * W * sizeof(float2);
    static constexpr size_t BAR_OFF = ((size_t)ELEMS * sizeof(float2) + 127) / 128 * 128;
    static constexpr size_t SMEM = BAR_OFF + 16;
};

// With a column pre-split of P (see the row pass), each [ny][nx] slice holds
// P independent column blocks of N = ny/P rows: block kp is the row set
// {kp + P*i : i < N}, and its output element i belongs in row kp + P*i too, so
// every tile reads and writes the same rows and the pass stays in place.  The
// tensor map is 3D -- (float within row, kp, slice*N + i) -- so one TMA box
// gathers BOXR rows P apart.
template <int N, int E, int W>
__global__ void __launch_bounds__(ColShape<N, E, W>::THREADS, ColShape<N, E, W>::MINB)
    k_cols(const __grid_constant__ CUtensorMap map, float2 *out, const float2 *__restrict__ tw, int nx,
           int batch, int P, int conj_out, int *status, int pf_dist) {
    using Sh = ColShape<N, E, W>;
    using Eng = typename Sh::Eng;
    constexpr int R0 = Eng::R0;
    constexpr int T = Sh::T;
    extern __shared__ __align__(128) unsigned char raw[];
    float2 *tile = reinterpret_cast<float2 *>(raw);
    uint64_t *bar = reinterpret_cast<uint64_t *>(raw + Sh::BAR_OFF);
    __shared__ int s_ok;

    const int t = threadIdx.x;
    const int c = t % W;
    const int tt = t / W;
    const int groups_x = nx / W;
    const long long ntiles = (long long)groups_x * P * batch;
    // conj_out bit 0: conjugate the outputs; bit 1: conjugate the inputs (a
    // column-only inverse, conj(F(conj x)), has no row pass to do it)
    const float so = (conj_out & 1) ? -1.f : 1.f;
    const bool conj_in = (conj_out & 2) != 0;
    // tile id -> (column group, kp, first row coordinate of its block)
    auto tile_x = [&](long long id) { return (int)(id % groups_x) * 2 * W; };
    auto tile_kp = [&](long long id) { return (int)((id / groups_x) % P); };
    auto tile_z = [&](long long id) { return (int)((id / groups_x) / P) * N; };

    auto issue = [&](long long id) {  // thread 0: TMA loads of tile `id`
        const int x = tile_x(id), kp = tile_kp(id), z0 = tile_z(id);
        mbar_expect_tx(bar, Sh::TILE_BYTES);
#pragma unroll 1
        for (int k = 0; k < N / Sh::BOXR; ++k)
            tma_load_3d(tile + k * Sh::BOXR * W, &map, x, kp, z0 + k * Sh::BOXR, bar);
    };
    auto prefetch = [&](long long id) {  // thread 0: bulk L2 prefetch of tile `id`
        const int x = tile_x(id), kp = tile_kp(id), z0 = tile_z(id);
#pragma unroll 1
        for (int k = 0; k < N / Sh::BOXR; ++k) tma_prefetch_3d(&map, x, kp, z0 + k * Sh::BOXR);
    };

    if (t == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
        fence_proxy_async_smem();
    }
    __syncthreads();
    long long id = blockIdx.x;
    uint32_t phase = 0;
    if (t == 0 && id < ntiles) {
        issue(id);
        for (int d = 1; d <= pf_dist; ++d)
            if (id + (long long)d * gridDim.x < ntiles) prefetch(id + (long long)d * gridDim.x);
    }
    for (; id < ntiles; id += gridDim.x) {
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
        const long long blk = id / groups_x;  // b*P + kp
        const long long b = blk / P;
        const int kp = (int)(blk - b * P);
        float2 *dst = out + (b * N * P + kp) * (long long)nx + (long long)(id % groups_x) * W;
        const long long rstride = (long long)P * nx;

        float2 v[E];
#pragma unroll
        for (int bb = 0; bb < E / R0; ++bb) {
            const int j = tt + bb * T;
#pragma unroll
            for (int r = 0; r < R0; ++r) v[bb * R0 + r] = tile[(j + r * (N / R0)) * W + c];
        }
        if (conj_in) {
#pragma unroll
            for (int k = 0; k < E; ++k) v[k].y = -v[k].y;
        }
        auto after_reads = [&] {
            __syncthreads();
            if (t == 0 && next < ntiles) {
                fence_proxy_async_smem();
                issue(next);
                const long long pf = next + (long long)pf_dist * gridDim.x;
                if (pf_dist > 0 && pf < ntiles) prefetch(pf);
            }
        };
        auto store = [&](int i, int cc, float2 x) {
            x.y *= so;
            dst[(long long)i * rstride + cc] = x;
        };
        Eng::template run<FftPolicy, true>(v, tile, tw, tt, c, SyncBlock{}, after_reads, store);
    }
}

// Differentiation form, column half (P = 1).  For L = sum w |F x|^2 the
// gradient is 2 F^H (w (.) X) with X = F x, and F^H = F_rows^H F_cols^H.
// Each tile: the forward column transform, its outputs X written back into
// the tile in natural order; one sweep over the tile that adds the tile's
// loss partial sum of w |X|^2 (float, one per tile) and replaces X by
// conj(w (.) X); the same forward engine over that, whose conjugated outputs
// are F_cols^H (w (.) X), stored in place of the tile's input.  X itself
// never reaches HBM: the pass reads the row pass's output and w and writes
// the adjoint's column half.
template <int N, int E, int W>
__global__ void __launch_bounds__(ColShape<N, E, W>::THREADS, ColShape<N, E, W>::MINB)
    k_cols_wadj(const __grid_constant__ CUtensorMap map, float2 *out, const float2 *__restrict__ tw,
                const float *__restrict__ w, float *partials, int nx, int batch, int *status, int pf_dist) {
    using Sh = ColShape<N, E, W>;
    using Eng = typename Sh::Eng;
    constexpr int R0 = Eng::R0;
    constexpr int T = Sh::T;
    constexpr int WARPS = Sh::THREADS / 32;
    extern __shared__ __align__(128) unsigned char raw[];
    float2 *tile = reinterpret_cast<float2 *>(raw);
    uint64_t *bar = reinterpret_cast<uint64_t *>(raw + Sh::BAR_OFF);
    __shared__ int s_ok;
    __shared__ float s_red[WARPS];

    const int t = threadIdx.x;
    const int c = t % W;
    const int tt = t / W;
    const int groups_x = nx / W;
    const long long ntiles = (long long)groups_x * batch;
    auto issue = [&](long long id) {  // thread 0: TMA loads of tile `id` (map over `out`, P = 1)
        const int x = (int)(id % groups_x) * 2 * W, z0 = (int)(id / groups_x) * N;
        mbar_expect_tx(bar, Sh::TILE_BYTES);
#pragma unroll 1
        for (int k = 0; k < N / Sh::BOXR; ++k) tma_load_3d(tile + k * Sh::BOXR * W, &map, x, 0, z0 + k * Sh::BOXR, bar);
    };
    auto prefetch = [&](long long id) {
        const int x = (int)(id % groups_x) * 2 * W, z0 = (int)(id / groups_x) * N;
#pragma unroll 1
        for (int k = 0; k < N / Sh::BOXR; ++k) tma_prefetch_3d(&map, x, 0, z0 + k * Sh::BOXR);
    };
    auto load_v = [&](float2 (&v)[E]) {
#pragma unroll
        for (int bb = 0; bb < E / R0; ++bb) {
            const int j = tt + bb * T;
#pragma unroll
            for (int r = 0; r < R0; ++r) v[bb * R0 + r] = tile[(j + r * (N / R0)) * W + c];
        }
    };

    if (t == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
        fence_proxy_async_smem();
    }
    __syncthreads();
    long long id = blockIdx.x;
    uint32_t phase = 0;
    if (t == 0 && id < ntiles) {
        issue(id);
        for (int d = 1; d <= pf_dist; ++d)
            if (id + (long long)d * gridDim.x < ntiles) prefetch(id + (long long)d * gridDim.x);
    }
    for (; id < ntiles; id += gridDim.x) {
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
        const long long b = id / groups_x;
        const long long off = b * (long long)N * nx + (long long)(id % groups_x) * W;
        float2 *dst = out + off;
        const float *wt = w + off;

        float part = 0.f;
        float2 v[E];
        load_v(v);
        auto all_read = [] { __syncthreads(); };
        auto fwd_store = [&](int i, int cc, float2 x) { tile[i * W + cc] = x; };
        Eng::template run<FftPolicy, true>(v, tile, tw, tt, c, SyncBlock{}, all_read, fwd_store);
        __syncthreads();  // X complete in the tile, natural order
        // w (.) X, its power and the conjugate, element by element: each row
        // of W adjacent w values is one coalesced run (offsets < N * nx)
#pragma unroll 4
        for (int k = t; k < N * W; k += Sh::THREADS) {
            const int i = k / W, cc = k % W;
            const float wv = __ldg(wt + (i * nx + cc));
            const float2 x = tile[k];
            part = fmaf(wv, fmaf(x.x, x.x, x.y * x.y), part);
            tile[k] = make_float2(wv * x.x, -(wv * x.y));
        }
        __syncthreads();  // conj(w (.) X) complete in the tile
        load_v(v);
        auto after_reads = [&] {
            __syncthreads();
            if (t == 0 && next < ntiles) {
                fence_proxy_async_smem();
                issue(next);
                const long long pf = next + (long long)pf_dist * gridDim.x;
                if (pf_dist > 0 && pf < ntiles) prefetch(pf);
            }
        };
        auto adj_store = [&](int i, int cc, float2 x) { dst[i * nx + cc] = make_float2(x.x, -x.y); };
        // the same table, through a pointer the compiler cannot equate with
        // `tw`: otherwise it keeps the first run's twiddle loads live for the
        // second and spills
        const float2 *tw2 = tw;
        asm volatile("" : "+l"(tw2));
        Eng::template run<FftPolicy, true>(v, tile, tw2, tt, c, SyncBlock{}, after_reads, adj_store);
        // the tile's partial: warps, then thread 0 (s_red is next written a
        // whole tile later, after several block barriers)
#pragma unroll
        for (int m = 16; m > 0; m >>= 1) part += __shfl_xor_sync(0xffffffffu, part, m);
        if ((t & 31) == 0) s_red[t >> 5] = part;
        __syncthreads();
        if (t == 0) {
            float sum = 0.f;
#pragma unroll
            for (int k = 0; k < WARPS; ++k) sum += s_red[k];
            partials[id] = sum;
        }
    }
}

// Movement-only twin: one tile of W columns whose dense staging buffer holds
// integer tags exactly where the TMA copy would put the data.  map[i] = final
// row of the element that started in row i of column 0.
template <int N, int E, int W>
__global__ void __launch_bounds__(ColShape<N, E, W>::THREADS) k_cols_movemap(int *map) {
    using Sh = ColShape<N, E, W>;
    using Eng = typename Sh::Eng;
    constexpr int R0 = Eng::R0;
    constexpr int T = Sh::T;
    extern __shared__ __align__(128) unsigned char raw[];
    float2 *tile = reinterpret_cast<float2 *>(raw);
    const int t = threadIdx.x;
    const int c = t % W;
    const int tt = t / W;
    for (int k = t; k < N * W; k += blockDim.x) tile[k] = make_float2(__int_as_float(k / W), __int_as_float(k % W));
    __syncthreads();
    float2 v[E];
#pragma unroll
    for (int bb = 0; bb < E / R0; ++bb) {
        const int j = tt + bb * T;
#pragma unroll
        for (int r = 0; r < R0; ++r) v[bb * R0 + r] = tile[(j + r * (N / R0)) * W + c];
    }
    auto after = [] { __syncthreads(); };
    auto store = [&](int i, int cc, float2 x) {
        if (cc == 0 && __float_as_int(x.y) == 0) map[__float_as_int(x.x)] = i;
    };
    Eng::template run<MovePolicy, true>(v, tile, nullptr, tt, c, SyncBlock{}, after, store);
}

// ---------------------------------------------------------------------------
// Variant table: (log2 n, E, W) with W in {2, 4, 8, 16} and N*W <= 16384
// (a tile of at most 128 KiB plus padding).
// ---------------------------------------------------------------------------
namespace {
struct ColEntry {
    ColVariant v;
    const void *movemap = nullptr;
    const void *wadj = nullptr;  // the differentiation form's fused column half (N <= 2048)
};
constexpr int kWSlots = 4;  // W = 2, 4, 8, 16
ColEntry g_cols[kMaxLog2 + 1][3][kWSlots];  // [log2n][E slot: default, 32, 64][W slot]
std::once_flag g_cols_once;  // registry filled once, safe across host threads

int w_slot(int w) { return w == 2 ? 0 : w == 4 ? 1 : w == 8 ? 2 : w == 16 ? 3 : -1; }

// the fused column half reduces per warp: whole warps only
template <int N, int E, int W>
struct THREADS_OK {
    static constexpr bool value = ColShape<N, E, W>::THREADS % 32 == 0;
};

template <int N, int E, int W>
void reg_col(int eslot) {
    using Sh = ColShape<N, E, W>;
    ColEntry &en = g_cols[ilog2(N)][eslot][w_slot(W)];
    en.v.fn = (const void *)k_cols<N, E, W>;
    en.v.n = N;
    en.v.e = E;
    en.v.w = W;
    en.v.threads = Sh::THREADS;
    en.v.smem = Sh::SMEM;
    en.v.box_rows = Sh::BOXR;
    en.v.tw_size = Sched<N, E>::tw_size;
    en.movemap = (const void *)k_cols_movemap<N, E, W>;
    if constexpr (N >= 32 && N <= 2048 && THREADS_OK<N, E, W>::value) en.wadj = (const void *)k_cols_wadj<N, E, W>;
}

template <int N, int E>
void reg_col_ws(int eslot) {
    reg_col<N, E, 2>(eslot);
    if constexpr (N * 4 <= 16384) reg_col<N, E, 4>(eslot);
    if constexpr (N * 8 <= 16384) reg_col<N, E, 8>(eslot);
    if constexpr (N * 16 <= 16384) reg_col<N, E, 16>(eslot);
}

template <int N>
void reg_cols_n() {
    constexpr int E = N >= 16 ? 16 : N;
    reg_col_ws<N, E>(0);
    if constexpr (N >= 4096) reg_col_ws<N, 32>(1);
    if constexpr (N >= 4096) reg_col_ws<N, 64>(2);
}

void init_cols() {
    std::call_once(g_cols_once, [] {
        reg_cols_n<2>();
        reg_cols_n<4>();
        reg_cols_n<8>();
        reg_cols_n<16>();
        reg_cols_n<32>();
        reg_cols_n<64>();
        reg_cols_n<128>();
        reg_cols_n<256>();
        reg_cols_n<512>();
        reg_cols_n<1024>();
        reg_cols_n<2048>();
        reg_cols_n<4096>();
        reg_cols_n<8192>();
    });
}

const ColEntry *col_entry(int log2n, int e, int w) {
    init_cols();
    if (log2n < 1 || log2n > kMaxLog2) return nullptr;
    const int ws = w_slot(w);
    if (ws < 0) return nullptr;
    const int n = 1 << log2n;
    const int es = (e == default_col_e(n)) ? 0 : (e == 32 ? 1 : e == 64 ? 2 : -1);
    if (es < 0) return nullptr;
    const ColEntry *en = &g_cols[log2n][es][ws];
    return en->v.fn ? en : nullptr;
}
}  // namespace

int default_col_e(int n) { return n >= 16 ? 16 : n; }

// Elements per thread the column pass prefers for length n and tile width w:
// E = 64 makes a 4096-point column two stages with one shared-memory
// exchange, so the tile is free for the next TMA copy after half the work
// (measured 0.35 -> 0.26 ms for the 8192^2 column pass).
int preferred_col_e(int n, int w) {
    if (n == 4096 && col_variant(ilog2(n), 64, w)) return 64;
    return default_col_e(n);
}

// Widest tile that keeps the staged tile within 128 KiB (columns of 4096
// points and more) or 64 KiB (shorter columns: two CTAs per SM, one
// transforming while the other loads; measured against 128 KiB tiles,
// 4 x 2048^2 0.136 -> 0.127 ms, 16 x 1024^2 0.124 -> 0.119) and the row
// length: rows of at least 32 bytes (W >= 4) make whole DRAM sectors, which
// the TMA moves far faster than 16-byte rows.
int default_col_w(int n, int nx) {
    int w = (n >= 4096 ? 16384 : 8192) / n;
    if (w > 16) w = 16;
    if (w < 2) w = 2;
    while (w > nx) w >>= 1;
    return w;
}

const ColVariant *col_variant(int log2n, int e, int w) {
    const ColEntry *en = col_entry(log2n, e, w);
    return en ? &en->v : nullptr;
}

int col_ctas_per_sm(const ColVariant &v) {
    int blocks = 0;
    if (v.smem > 48 * 1024)
        cudaFuncSetAttribute(v.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)v.smem);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, v.fn, v.threads, v.smem) != cudaSuccess)
        return 1;
    return blocks > 0 ? blocks : 1;
}

cudaError_t launch_cols(const ColVariant &v, const CUtensorMap &map, float2 *out, const float2 *tw,
                        int nx, int batch, int split, int conj_out, int *status, int grid, int pf_dist,
                        cudaStream_t s) {
    if (v.smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(v.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)v.smem);
        if (e != cudaSuccess) return e;
    }
    CUtensorMap m = map;
    void *args[] = {(void *)&m,     (void *)&out,   (void *)&tw,       (void *)&nx,     (void *)&batch,
                    (void *)&split, (void *)&conj_out, (void *)&status, (void *)&pf_dist};
    return cudaLaunchKernel(v.fn, dim3(grid), dim3(v.threads), args, v.smem, s);
}

bool cols_wadj_available(const ColVariant &v) {
    const ColEntry *en = col_entry(ilog2(v.n), v.e, v.w);
    return en && en->wadj;
}

int cols_wadj_ctas_per_sm(const ColVariant &v) {
    const ColEntry *en = col_entry(ilog2(v.n), v.e, v.w);
    if (!en || !en->wadj) return 1;
    int blocks = 0;
    if (v.smem > 48 * 1024) cudaFuncSetAttribute(en->wadj, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)v.smem);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, en->wadj, v.threads, v.smem) != cudaSuccess) return 1;
    return blocks > 0 ? blocks : 1;
}

cudaError_t launch_cols_wadj(const ColVariant &v, const CUtensorMap &map, float2 *out, const float2 *tw,
                             const float *w, float *partials, int nx, int batch, int *status, int grid, int pf_dist,
                             cudaStream_t s) {
    const ColEntry *en = col_entry(ilog2(v.n), v.e, v.w);
    if (!en || !en->wadj) return cudaErrorInvalidValue;
    if (v.smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(en->wadj, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)v.smem);
        if (e != cudaSuccess) return e;
    }
    CUtensorMap m = map;
    void *args[] = {(void *)&m,  (void *)&out,   (void *)&tw,     (void *)&w,      (void *)&partials,
                    (void *)&nx, (void *)&batch, (void *)&status, (void *)&pf_dist};
    return cudaLaunchKernel(en->wadj, dim3(grid), dim3(v.threads), args, v.smem, s);
}

cudaError_t launch_cols_movemap(int log2n, int *map, cudaStream_t s) {
    const int n = 1 << log2n;
    const ColEntry *en = col_entry(log2n, default_col_e(n), 2);
    if (!en) return cudaErrorInvalidValue;
    if (en->v.smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(en->movemap, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)en->v.smem);
        if (e != cudaSuccess) return e;
    }
    void *args[] = {(void *)&map};
    return cudaLaunchKernel(en->movemap, dim3(1), dim3(en->v.threads), args, en->v.smem, s);
}

int schedule_radices(int n, int e, int *radices) {
    if (n < 1 || (n & (n - 1)) || e < 1 || (e & (e - 1))) return -1;
    if (e > n) e = n;
    const int L = ilog2(n), LE = ilog2(e);
    if (n == 1) {
        radices[0] = 1;
        return 1;
    }
    const int S = (L + LE - 1) / LE;
    radices[0] = n >> (LE * (S - 1));
    for (int s = 1; s < S; ++s) radices[s] = e;
    return S;
}

}  // namespace gb300fft
