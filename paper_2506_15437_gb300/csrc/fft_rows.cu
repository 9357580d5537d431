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

#include <mutex>

#include "fft_common.cuh"
#include "fft_internal.h"

namespace gb300fft {

#ifndef ROWMINB32
#define ROWMINB32 2  // 256-thread CTAs with E = 32: two per SM (128 registers)
#endif

template <int N, int E>
struct RowShape {
    static constexpr int T = N / E;
    static constexpr int ROWS = (T >= 256) ? 1 : 256 / T;
    static constexpr int THREADS = ROWS * T;
    // resident CTAs the register budget must allow: 64 registers per thread
    // for 512-thread CTAs with E <= 16, at most 85 for 256-thread ones
    static constexpr int MINB = THREADS >= 512 ? (E >= 32 ? 512 : 1024) / THREADS
                                               : (THREADS >= 256 ? (E < 32 ? 3 : ROWMINB32) : 1);
    using Eng = Engine<N, E, 1, PadShift<E>::value, RowPadShift1<E>::value>;
    static constexpr size_t SMEM = sizeof(float2) * (size_t)ROWS * Eng::SMEM_ELEMS;
};

// Column pre-split (P > 1).  A column transform of length ny = P*Q can be
// split as X[kp + P*kq] = sum_q w_Q^{q*kq} * w_ny^{q*kp} * (sum_p x[q + Q*p] w_P^{p*kp}).
// With P > 1 the row pass computes the bracket -- the P-point DFT across the
// rows q + Q*p and the scalar twiddle w_ny^{q*kp} -- while it loads, and
// writes the transformed row to row kp + P*q; the column pass then runs
// length-Q transforms over the row sets {kp + P*q : q < Q} and writes output
// kq of set kp to row kp + P*kq, i.e. back into the rows it read.  Because the
// row FFT acts along x and the split along y, the two commute and the result
// is the same 2D DFT.  Output rows r and r+1 (kp = 0, 1) read the same input
// rows, so neighbouring groups share them through L2.
//
// The grid is either one CTA per row group, or persistent: a CTA walks row
// groups blockIdx.x, blockIdx.x + gridDim.x, ... and asks L2 for its next
// group's rows (bulk prefetch) before transforming the current one.
template <int N, int E, bool WEIGHTED, int P>
__global__ void __launch_bounds__(RowShape<N, E>::THREADS, RowShape<N, E>::MINB)
    k_rows(const float2 *__restrict__ in, float2 *out, const float2 *__restrict__ tw,
           const float2 *__restrict__ twp, long long nrows, int ny, int conj_in, int conj_out,
           const float *__restrict__ weight, float wscale, const float *__restrict__ wscale_dev, int pf_dist,
           int perm_t, int perm_g, int planar) {
    using Sh = RowShape<N, E>;
    using Eng = typename Sh::Eng;
    constexpr int T = Sh::T;
    constexpr int R0 = Eng::R0;
    constexpr int ROWS = Sh::ROWS;
    extern __shared__ __align__(16) float2 smem[];
    const int g = threadIdx.x / T;
    const int tt = threadIdx.x - g * T;
    const float si = conj_in ? -1.f : 1.f;
    const float so = conj_out ? -1.f : 1.f;
    const int Q = ny / P;
    float2 *sm = smem + g * Eng::SMEM_ELEMS;
    const long long step = (long long)gridDim.x * ROWS;
    if constexpr (WEIGHTED) {
        if (wscale_dev) wscale *= __ldg(wscale_dev);  // a scale that lives on the device (no host read)
    }

    // first input row of output row r, for input part p (P == 1: r itself)
    auto in_row = [&](long long r, int p) -> long long {
        if constexpr (P == 1) {
            return r;
        } else {
            const long long b = r / ny;
            const int y = (int)(r - b * ny);
            return b * ny + (y / P) + (long long)Q * p;
        }
    };

    bool first = true;
    if (threadIdx.x == 0 && pf_dist > 1) {  // warm L2 with the groups after the first
        for (int d = 1; d < pf_dist; ++d) {
            const long long nb = (long long)blockIdx.x * ROWS + d * step;
            if (nb >= nrows) break;
            if constexpr (P == 1) {
                const long long cnt = (nrows - nb) < ROWS ? (nrows - nb) : ROWS;
                bulk_prefetch_l2(in + nb * N, (uint32_t)(cnt * N * sizeof(float2)));
            } else {
                for (int gg = 0; gg < ROWS && nb + gg < nrows; ++gg)
#pragma unroll
                    for (int p = 0; p < P; ++p)
                        bulk_prefetch_l2(in + in_row(nb + gg, p) * N, (uint32_t)(N * sizeof(float2)));
            }
        }
    }
    for (long long base = (long long)blockIdx.x * ROWS; base < nrows; base += step) {
        const long long nb = base + (long long)(pf_dist > 0 ? pf_dist : 1) * step;
        if (threadIdx.x == 0 && pf_dist > 0 && nb < nrows) {
            if constexpr (P == 1) {
                const long long cnt = (nrows - nb) < ROWS ? (nrows - nb) : ROWS;
                bulk_prefetch_l2(in + nb * N, (uint32_t)(cnt * N * sizeof(float2)));
            } else {
                for (int gg = 0; gg < ROWS && nb + gg < nrows; ++gg)
#pragma unroll
                    for (int p = 0; p < P; ++p)
                        bulk_prefetch_l2(in + in_row(nb + gg, p) * N, (uint32_t)(N * sizeof(float2)));
            }
        }
        if (!first) __syncthreads();  // the previous group's last shared-memory reads are done
        first = false;

        const long long row = base + g;
        const bool active = row < nrows;
        int kp = 0, q = 0;
        if constexpr (P > 1) {
            const int y = active ? (int)(row % ny) : 0;
            kp = y % P;
            q = y / P;
        }
        float2 v[E];
#pragma unroll
        for (int b = 0; b < E / R0; ++b) {
            const int j = tt + b * T;
#pragma unroll
            for (int r = 0; r < R0; ++r) {
                const int i = j + r * (N / R0);
                float2 acc = make_float2(0.f, 0.f);
#pragma unroll
                for (int p = 0; p < P; ++p) {
                    const long long ir = active ? in_row(row, p) : 0;
                    float2 x = active ? __ldg(in + ir * N + i) : make_float2(0.f, 0.f);
                    if constexpr (WEIGHTED && !(P == 1 && N <= 2048)) {
                        // with the split, the weight belongs to each input row;
                        // no weight array: the scale alone
                        const float wv = active ? (weight ? __ldg(weight + ir * N + i) : 1.f) * wscale : 0.f;
                        x.x *= wv;
                        x.y *= wv;
                    }
                    x.y *= si;
                    if constexpr (P == 1) {
                        acc = x;
                    } else {
                        // P == 2: w_2^{p*kp} = (-1)^{p*kp}
                        acc = (p == 1 && kp == 1) ? csub(acc, x) : cadd(acc, x);
                    }
                }
                v[b * R0 + r] = acc;
            }
        }
        if constexpr (WEIGHTED && P == 1 && N <= 2048) {
            // weights and scale after the data loads, in a sweep of their own:
            // interleaved with the loads, 8 x 2048^2 scaled rows took 0.220 ms
            // instead of 0.102 (the weighted adjoint 0.404 instead of 0.279);
            // 4096-point rows are faster interleaved (0.234 against 0.250)
            if (weight) {
                float wv[E];
#pragma unroll
                for (int b = 0; b < E / R0; ++b)
#pragma unroll
                    for (int r = 0; r < R0; ++r)
                        wv[b * R0 + r] = active ? __ldg(weight + row * N + tt + b * T + r * (N / R0)) : 0.f;
#pragma unroll
                for (int k = 0; k < E; ++k) {
                    v[k].x *= wv[k] * wscale;
                    v[k].y *= wv[k] * wscale;
                }
            } else {
#pragma unroll
                for (int k = 0; k < E; ++k) {
                    v[k].x *= wscale;
                    v[k].y *= wscale;
                }
            }
        }
        if constexpr (P > 1) {
            if (kp != 0) {
                const float2 w = __ldg(twp + (long long)q * kp);
#pragma unroll
                for (int k = 0; k < E; ++k) v[k] = cmul(v[k], w);
            }
        }
        long long orow = row;
        if (perm_t || planar) {
            // column block kq, element i: with perm_t (streaming column pass)
            // at block row (j / G)*G*R0 + r*G + j % G for i = j + r*perm_t
            // (G = perm_g), else at block row i; the block's rows are P apart
            // (kq + P*row) or, planar, a plane of its own (kq*Q + row)
            const long long bb = row / ny;
            const int y = (int)(row - bb * ny);
            const int i = y / P, kq = y - (y / P) * P;
            int pos = i;
            if (perm_t) {
                const int j = i & (perm_t - 1), r = i / perm_t;
                pos = (j / perm_g) * perm_g * (Q / perm_t) + r * perm_g + (j & (perm_g - 1));
            }
            orow = bb * ny + (planar ? (long long)kq * Q + pos : kq + (long long)P * pos);
        }
        float2 *dst = out + orow * N;
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
}

// Movement-only twin of k_rows for one row: integer tags instead of values,
// identity butterflies, identical addresses.  map[tag] = final position.
template <int N, int E>
__global__ void __launch_bounds__(N / E) k_rows_movemap(int *map) {
    using Eng = Engine<N, E, 1, PadShift<E>::value, RowPadShift1<E>::value>;
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
    RowVariant plain, weighted, split2, split2_weighted;
    const void *movemap = nullptr;
    size_t movemap_smem = 0;
    int movemap_threads = 0;
};
RowEntry g_rows[kMaxLog2 + 1][3];  // [log2n][E slot: 8, 16, 32]
std::once_flag g_rows_once;  // registry filled once, safe across host threads

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
    v.fn = (const void *)k_rows<N, E, false, 1>;
    en.plain = v;
    v.fn = (const void *)k_rows<N, E, true, 1>;
    en.weighted = v;
    // Pre-split (P = 2) kernels: the default E of every length, and E = 32
    // for 8192-point rows only.  The E = 32 pre-split kernel of 4096-point
    // rows (two rows per CTA) raised an illegal address on a 4096 x 512 x 2
    // plan; reading its index arithmetic and the CPU index model of the tests
    // found no out-of-range access, so with the cause unknown it is not
    // compiled, and neither plans nor the autotuner can select it.
    if constexpr (E == (N >= 16 ? 16 : N) || (E == 32 && N >= 8192)) {
        v.fn = (const void *)k_rows<N, E, false, 2>;
        en.split2 = v;
        v.fn = (const void *)k_rows<N, E, true, 2>;
        en.split2_weighted = v;
    }
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
    std::call_once(g_rows_once, [] {
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
    });
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

int default_row_e(int n) { return n >= 8192 ? 32 : n >= 16 ? 16 : (n >= 8 ? 8 : n); }

const RowVariant *row_variant(int log2n, int e) {
    const RowEntry *en = row_entry(log2n, e);
    return en ? &en->plain : nullptr;
}

static const void *row_fn(const RowVariant &v, bool weighted, int split) {
    const RowEntry *en = row_entry(ilog2(v.n), v.e);
    if (!en) return nullptr;
    const RowVariant &k = split == 2 ? (weighted ? en->split2_weighted : en->split2)
                                     : (weighted ? en->weighted : en->plain);
    return k.fn;
}

bool row_split_available(int n, int e) {
    const RowEntry *en = row_entry(ilog2(n), e);
    return en && en->split2.fn && en->split2_weighted.fn;
}

bool row_variant_info(int n, int e, int split, int *threads, int *rows_per_cta, int *smem_elems) {
    if (n < 2 || n > 8192 || (n & (n - 1)) || (split != 1 && split != 2)) return false;
    const RowEntry *en = row_entry(ilog2(n), e);
    if (!en || en->plain.e != (e > n ? n : e)) return false;
    if (split == 2 && !(en->split2.fn && en->split2_weighted.fn)) return false;
    *threads = en->plain.threads;
    *rows_per_cta = en->plain.rows_per_cta;
    *smem_elems = (int)(en->plain.smem / sizeof(float2) / en->plain.rows_per_cta);
    return true;
}

int row_grid(const RowVariant &v, long long nrows, int num_sms, bool weighted, int split, bool persistent) {
    const void *fn = row_fn(v, weighted, split);
    if (!fn) return 0;
    if (v.smem > 48 * 1024) cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)v.smem);
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, v.threads, v.smem) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    const long long groups = (nrows + v.rows_per_cta - 1) / v.rows_per_cta;
    long long grid = persistent ? (long long)num_sms * per_sm : groups;
    if (grid > groups) grid = groups;
    if (grid > 0x7fffffffLL) grid = 0x7fffffffLL;
    return grid < 1 ? 1 : (int)grid;
}

cudaError_t launch_rows(const RowVariant &v, const float2 *in, float2 *out, const float2 *tw, const float2 *twp,
                        long long nrows, int ny, int split, int conj_in, int conj_out, const float *weight,
                        float wscale, const float *wscale_dev, int grid, int pf_dist, int perm_t, int perm_g,
                        int planar, cudaStream_t s) {
    if (nrows <= 0) return cudaSuccess;
    if (split != 1 && split != 2) return cudaErrorInvalidValue;
    // the weighted variant also serves a plain scale (no weight array)
    const void *fn = row_fn(v, weight != nullptr || wscale_dev != nullptr || wscale != 1.f, split);
    if (!fn) return cudaErrorInvalidValue;
    if (v.smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)v.smem);
        if (e != cudaSuccess) return e;
    }
    if (grid < 1) return cudaErrorInvalidConfiguration;
    if (perm_t && (perm_t & (perm_t - 1) || perm_g < 1 || (perm_g & (perm_g - 1)) || perm_t % perm_g ||
                   (ny / split) % perm_t))
        return cudaErrorInvalidValue;
    void *args[] = {(void *)&in,      (void *)&out,     (void *)&tw,       (void *)&twp,    (void *)&nrows,
                    (void *)&ny,      (void *)&conj_in, (void *)&conj_out, (void *)&weight, (void *)&wscale,
                    (void *)&wscale_dev, (void *)&pf_dist, (void *)&perm_t, (void *)&perm_g, (void *)&planar};
    return cudaLaunchKernel(fn, dim3(grid), dim3(v.threads), args, v.smem, s);
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
