// Row pass: batched length-N FFTs along contiguous rows (the first half of the
// paper's Section 5 row-then-column 2D decomposition).
//
// One group of N/E threads owns one row; a CTA holds ROWS rows.  Stage-0
// operands come straight from HBM with coalesced loads (thread tt reads
// elements tt + r*N/R0, so each warp load is 256 contiguous bytes), later
// stages exchange through padded shared memory, and the last stage stores
// natural-order results straight to HBM, again 256 contiguous bytes per warp.
// So each element crosses HBM exactly once in each direction; the reorders
// between butterfly steps never leave the SM.
#include <cstdio>

#include "fft_common.cuh"
#include "fft_internal.h"

namespace gb300fft {

template <int N, int E>
struct RowShape {
    static constexpr int T = N / E;
    static constexpr int ROWS = (T >= 256) ? 1 : 256 / T;
    static constexpr int THREADS = ROWS * T;
    using Eng = Engine<N, E, 1, PadShift<E>::value>;
    static constexpr size_t SMEM = sizeof(float2) * (size_t)ROWS * Eng::SMEM_ELEMS;
};

template <int N, int E, bool WEIGHTED>
__global__ void __launch_bounds__(RowShape<N, E>::THREADS)
    k_rows(const float2 *__restrict__ in, float2 *out, const float2 *__restrict__ tw, long long nrows,
           int conj_in, int conj_out, const float *__restrict__ weight, float wscale) {
    using Sh = RowShape<N, E>;
    using Eng = typename Sh::Eng;
    constexpr int T = Sh::T;
    constexpr int R0 = Eng::R0;
    extern __shared__ __align__(16) float2 smem[];
    const int g = threadIdx.x / T;
    const int tt = threadIdx.x - g * T;
    const long long row = (long long)blockIdx.x * Sh::ROWS + g;
    const bool active = row < nrows;
    const float2 *src = in + row * N;
    float2 *dst = out + row * N;
    const float si = conj_in ? -1.f : 1.f;
    const float so = conj_out ? -1.f : 1.f;

    float2 v[E];
#pragma unroll
    for (int b = 0; b < E / R0; ++b) {
        const int j = tt + b * T;
#pragma unroll
        for (int r = 0; r < R0; ++r) {
            const int i = j + r * (N / R0);
            float2 x = active ? __ldg(src + i) : make_float2(0.f, 0.f);
            if constexpr (WEIGHTED) {
                const float wv = active ? __ldg(weight + row * N + i) * wscale : 0.f;
                x.x *= wv;
                x.y *= wv;
            }
            x.y *= si;
            v[b * R0 + r] = x;
        }
    }
    float2 *sm = smem + g * Eng::SMEM_ELEMS;
    auto store = [&](int i, int, float2 x) {
        if (active) {
            x.y *= so;
            dst[i] = x;
        }
    };
    auto none = [] {};
    if constexpr (Eng::NT >= 32)
        Eng::template run<FftPolicy, false>(v, sm, tw, tt, 0, SyncBlock{}, none, store);
    else
        Eng::template run<FftPolicy, false>(v, sm, tw, tt, 0, SyncWarp{}, none, store);
}

// Movement-only twin of k_rows for one row: integer tags instead of values,
// identity butterflies, identical addresses.  map[tag] = final position.
template <int N, int E>
__global__ void __launch_bounds__(N / E) k_rows_movemap(int *map) {
    using Eng = Engine<N, E, 1, PadShift<E>::value>;
    constexpr int T = N / E;
    constexpr int R0 = Eng::R0;
    extern __shared__ __align__(16) float2 smem[];
    const int tt = threadIdx.x;
    float2 v[E];
#pragma unroll
    for (int b = 0; b < E / R0; ++b)
#pragma unroll
        for (int r = 0; r < R0; ++r) v[b * R0 + r] = make_float2(__int_as_float(tt + b * T + r * (N / R0)), 0.f);
    auto store = [&](int i, int, float2 x) { map[__float_as_int(x.x)] = i; };
    auto none = [] {};
    if constexpr (Eng::NT >= 32)
        Eng::template run<MovePolicy, false>(v, smem, nullptr, tt, 0, SyncBlock{}, none, store);
    else
        Eng::template run<MovePolicy, false>(v, smem, nullptr, tt, 0, SyncWarp{}, none, store);
}

// ---------------------------------------------------------------------------
// Variant table: one entry per (log2 n, E).  Lengths below 8 have a single
// stage and use E = n in every slot.
// ---------------------------------------------------------------------------
namespace {
struct RowEntry {
    RowVariant plain, weighted;
    const void *movemap = nullptr;
    size_t movemap_smem = 0;
    int movemap_threads = 0;
};
RowEntry g_rows[kMaxLog2 + 1][3];  // [log2n][E slot: 8, 16, 32]
bool g_rows_init = false;

int e_slot(int e) { return e == 8 ? 0 : e == 16 ? 1 : e == 32 ? 2 : -1; }

template <int N, int E>
RowEntry make_row_entry() {
    using Sh = RowShape<N, E>;
    RowEntry en;
    RowVariant v;
    v.n = N;
    v.e = E;
    v.threads = Sh::THREADS;
    v.rows_per_cta = Sh::ROWS;
    v.smem = Sh::SMEM;
    v.tw_size = Sched<N, E>::tw_size;
    v.fn = (const void *)k_rows<N, E, false>;
    en.plain = v;
    v.fn = (const void *)k_rows<N, E, true>;
    en.weighted = v;
    en.movemap = (const void *)k_rows_movemap<N, E>;
    en.movemap_smem = sizeof(float2) * (size_t)Sh::Eng::SMEM_ELEMS;
    en.movemap_threads = N / E;
    return en;
}

template <int N>
void reg_rows_n() {
    if constexpr (N < 8) {
        const RowEntry en = make_row_entry<N, N>();
        for (int k = 0; k < 3; ++k) g_rows[ilog2(N)][k] = en;
    } else {
        g_rows[ilog2(N)][0] = make_row_entry<N, 8>();
        if constexpr (N >= 16) g_rows[ilog2(N)][1] = make_row_entry<N, 16>();
        if constexpr (N >= 32) g_rows[ilog2(N)][2] = make_row_entry<N, 32>();
    }
}

void init_rows() {
    if (g_rows_init) return;
    reg_rows_n<2>();
    reg_rows_n<4>();
    reg_rows_n<8>();
    reg_rows_n<16>();
    reg_rows_n<32>();
    reg_rows_n<64>();
    reg_rows_n<128>();
    reg_rows_n<256>();
    reg_rows_n<512>();
    reg_rows_n<1024>();
    reg_rows_n<2048>();
    reg_rows_n<4096>();
    reg_rows_n<8192>();
    g_rows_init = true;
}

const RowEntry *row_entry(int log2n, int e) {
    init_rows();
    if (log2n < 1 || log2n > kMaxLog2) return nullptr;
    const int n = 1 << log2n;
    const int k = n < 8 ? 0 : e_slot(e);
    if (k < 0 || (n >= 8 && e > n)) return nullptr;
    const RowEntry *en = &g_rows[log2n][k];
    return en->plain.fn ? en : nullptr;
}
}  // namespace

int default_row_e(int n) { return n >= 16 ? 16 : (n >= 8 ? 8 : n); }

const RowVariant *row_variant(int log2n, int e) {
    const RowEntry *en = row_entry(log2n, e);
    return en ? &en->plain : nullptr;
}

static const RowVariant *row_variant_weighted(int log2n, int e) {
    const RowEntry *en = row_entry(log2n, e);
    return en ? &en->weighted : nullptr;
}

cudaError_t launch_rows(const RowVariant &v, const float2 *in, float2 *out, const float2 *tw,
                        long long nrows, int conj_in, int conj_out, const float *weight,
                        float wscale, cudaStream_t s) {
    if (nrows <= 0) return cudaSuccess;
    const void *fn = v.fn;
    if (weight) {
        const RowVariant *w = row_variant_weighted(ilog2(v.n), v.e);
        if (!w) return cudaErrorInvalidValue;
        fn = w->fn;
    }
    if (v.smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)v.smem);
        if (e != cudaSuccess) return e;
    }
    const long long grid = (nrows + v.rows_per_cta - 1) / v.rows_per_cta;
    if (grid > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    void *args[] = {(void *)&in, (void *)&out, (void *)&tw, (void *)&nrows, (void *)&conj_in,
                    (void *)&conj_out, (void *)&weight, (void *)&wscale};
    return cudaLaunchKernel(fn, dim3((unsigned)grid), dim3(v.threads), args, v.smem, s);
}

cudaError_t launch_rows_movemap(int log2n, int *map, cudaStream_t s) {
    const RowEntry *en = row_entry(log2n, default_row_e(1 << log2n));
    if (!en) return cudaErrorInvalidValue;
    if (en->movemap_smem > 48 * 1024) {
        cudaError_t err = cudaFuncSetAttribute(en->movemap, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)en->movemap_smem);
        if (err != cudaSuccess) return err;
    }
    void *args[] = {(void *)&map};
    return cudaLaunchKernel(en->movemap, dim3(1), dim3(en->movemap_threads), args, en->movemap_smem, s);
}

}  // namespace gb300fft
