// Transforms of any length: Bluestein's chirp-z identity on top of the
// power-of-two path.  The paper's future work asks for uneven decompositions
// beyond powers of two (Section 6); this is the general route.
//
// With c[j] = exp(dir*pi*i*j^2/n) (dir = -1 forward) and j*k = (j^2 + k^2 -
// (k-j)^2)/2,
//     X[k] = c[k] * sum_{j<n} (x[j] c[j]) * conj(c[k-j]),
// a linear convolution of a[j] = x[j] c[j] with h[m] = conj(c[m]),
// |m| < n.  Zero-padded to a power of two M >= 2n - 1 it is a circular one,
// computed as conv = F^-1( F(a) . F(h) ) / M with the library's own
// power-of-two transforms (one plan of length M, run forward and inverse).
// H = F(h) / M is built once per plan and direction.  The chirp's phase
// j^2 mod 2n is reduced in integers and evaluated in FP64 (sincospi), then
// rounded once to FP32.
//
// For M <= 8192 the chirp and filter products are fused into the two
// transforms (k_blu below): two HBM passes over the padded rows.
//
// A 2D transform whose sizes are not both powers of two runs axis by axis:
// the x axis over all rows, a tiled transpose, the y axis over the rows of
// the transposed array, and the transpose back.
#include <mutex>
#include <type_traits>

#include "fft_common.cuh"
#include "fft_internal.h"

namespace gb300fft {

// c[j] = exp(sgn*pi*i*(j^2 mod 2n)/n), j < n
__global__ void k_chirp(float2 *c, int n, int sgn) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const long long q = ((long long)j * j) % (2LL * n);
    double sv, cv;
    sincospi((double)q / (double)n, &sv, &cv);
    c[j] = make_float2((float)cv, (float)(sgn * sv));
}

// h[m] = conj(c[|m|]) placed circularly in M slots (m and M - m), zero between
__global__ void k_chirp_filter(float2 *h, const float2 *__restrict__ c, int n, int M) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    int idx = -1;
    if (m < n) idx = m;
    else if (m > M - n) idx = M - m;
    h[m] = idx >= 0 ? make_float2(c[idx].x, -c[idx].y) : make_float2(0.f, 0.f);
}

__global__ void k_scale(float2 *a, long long count, float s) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
         i += (long long)gridDim.x * blockDim.x) {
        float2 v = a[i];
        a[i] = make_float2(v.x * s, v.y * s);
    }
}

// A[r][j] = x[r][j] * c[j] for j < n, 0 for n <= j < M
__global__ void k_blu_pre(const float2 *__restrict__ x, float2 *__restrict__ A, const float2 *__restrict__ c, int n,
                          int M, long long rows) {
    const long long total = rows * M;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long r = i / M;
        const int j = (int)(i - r * M);
        A[i] = j < n ? cmul(__ldg(x + r * n + j), __ldg(c + j)) : make_float2(0.f, 0.f);
    }
}

// A[r][k] *= H[k]
__global__ void k_blu_mul(float2 *A, const float2 *__restrict__ H, int M, long long rows) {
    const long long total = rows * M;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(i % M);
        A[i] = cmul(A[i], __ldg(H + k));
    }
}

// out[r][k] = c[k] * A[r][k], k < n
__global__ void k_blu_post(const float2 *__restrict__ A, float2 *__restrict__ out, const float2 *__restrict__ c,
                           int n, int M, long long rows) {
    const long long total = rows * n;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long r = i / n;
        const int k = (int)(i - r * n);
        out[i] = cmul(__ldg(A + r * M + k), __ldg(c + k));
    }
}

// out[b][cc][rr] = in[b][rr][cc] for [batch][rows][cols] arrays, through
// 32 x 32 tiles in shared memory (one padding column: conflict-free both ways)
__global__ void __launch_bounds__(256) k_transpose(const float2 *__restrict__ in, float2 *__restrict__ out, int rows,
                                                   int cols, long long tiles_c, long long tiles_rc) {
    __shared__ float2 tile[32][33];
    const long long b = blockIdx.x / tiles_rc;
    const long long rem = blockIdx.x - b * tiles_rc;
    const int tr = (int)(rem / tiles_c), tc = (int)(rem - (long long)tr * tiles_c);
    const float2 *src = in + b * (long long)rows * cols;
    float2 *dst = out + b * (long long)rows * cols;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8 threads
#pragma unroll
    for (int k = 0; k < 32; k += 8) {
        const int r = tr * 32 + ty + k, cc = tc * 32 + tx;
        if (r < rows && cc < cols) tile[ty + k][tx] = src[(long long)r * cols + cc];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 32; k += 8) {
        const int cc = tc * 32 + ty + k, r = tr * 32 + tx;
        if (r < rows && cc < cols) dst[(long long)cc * rows + r] = tile[tx][ty + k];
    }
}

// Fused Bluestein for padded lengths M <= 8192 (one row per thread group, as
// in the row pass).  Phase 0: A[r] = F(a) . H with a[j] = x[r][j] c[j] for
// j < n and 0 up to M, the chirp product applied as the rows are loaded and
// the filter product as the transform is stored.  Phase 1: out[r][k] =
// c[k] * F^-1(A[r])[k] for k < n, the inverse as conj(F(conj(.))) and the
// chirp product and truncation applied as it is stored.  Two HBM passes over
// the padded rows instead of five.  Phase 2 does both in one pass: the
// forward transform's outputs stay in registers -- thread tt holds elements
// tt + m*T (m < E) in the last stage's order, exactly the elements its
// stage-0 inputs of the inverse transform are, in another register order --
// so the filter product, the conjugation and that compile-time register
// permutation connect the two transforms without touching HBM.
template <int N, int E>
struct BluShape {
    static constexpr int T = N / E;
    static constexpr int ROWS = (T >= 256) ? 1 : 256 / T;
    static constexpr int THREADS = ROWS * T;
    using Eng = Engine<N, E, 1, PadShift<E>::value, RowPadShift1<E>::value>;
    static constexpr size_t SMEM = sizeof(float2) * (size_t)ROWS * Eng::SMEM_ELEMS;
    static constexpr int MINB = THREADS >= 512 ? (E >= 32 ? 512 : 1024) / THREADS : (THREADS >= 256 ? 2 : 1);
};

template <int N, int E, int PHASE>
__global__ void __launch_bounds__(BluShape<N, E>::THREADS, BluShape<N, E>::MINB)
    k_blu(const float2 *__restrict__ src, float2 *__restrict__ dst, const float2 *__restrict__ tw,
          const float2 *__restrict__ chirp, const float2 *__restrict__ H, int n, long long rows) {
    using Sh = BluShape<N, E>;
    using Eng = typename Sh::Eng;
    constexpr int T = Sh::T;
    constexpr int R0 = Eng::R0;
    extern __shared__ __align__(16) float2 smem[];
    const int g = threadIdx.x / T;
    const int tt = threadIdx.x - g * T;
    float2 *sm = smem + g * Eng::SMEM_ELEMS;
    const long long row = (long long)blockIdx.x * Sh::ROWS + g;
    const bool active = row < rows;
    float2 v[E];
#pragma unroll
    for (int b = 0; b < E / R0; ++b) {
        const int j = tt + b * T;
#pragma unroll
        for (int r = 0; r < R0; ++r) {
            const int i = j + r * (N / R0);
            float2 x = make_float2(0.f, 0.f);
            if constexpr (PHASE == 0) {
                if (active && i < n) x = __ldg(src + row * n + i);  // the chirp below, in a sweep of its own
            } else if constexpr (PHASE == 2) {
                if (active && i < n) x = cmul(__ldg(src + row * n + i), __ldg(chirp + i));
            } else {
                if (active) {
                    x = __ldg(src + row * N + i);
                    x.y = -x.y;
                }
            }
            v[b * R0 + r] = x;
        }
    }
    if constexpr (PHASE == 0) {
        // the chirp product after all the data loads (the zero padding past
        // n stays zero whatever chirp entry multiplies it): 16384 x 4093
        // 0.871 -> 0.811 ms; the one-pass form (phase 2) keeps the product
        // in its loads (1009 x 32768: 0.397 against 0.401 ms)
#pragma unroll
        for (int b = 0; b < E / R0; ++b) {
            const int j = tt + b * T;
#pragma unroll
            for (int r = 0; r < R0; ++r) {
                const int i = j + r * (N / R0);
                v[b * R0 + r] = cmul(v[b * R0 + r], __ldg(chirp + (i < n ? i : n - 1)));
            }
        }
    }
    auto store = [&](int i, int, float2 x) {
        if constexpr (PHASE == 0) {
            if (active) dst[row * N + i] = cmul(x, __ldg(H + i));
        } else {  // phases 1 and 2: the inverse's outputs
            if (active && i < n) {
                x.y = -x.y;
                dst[row * n + i] = cmul(x, __ldg(chirp + i));
            }
        }
    };
    auto none = [] {};
    using Sync = typename std::conditional<(Eng::NT >= 32), SyncBlock, SyncWarp>::type;
    if constexpr (PHASE < 2) {
        Eng::template run<FftPolicy, false>(v, sm, tw, tt, 0, Sync{}, none, store);
    } else if constexpr (Eng::S == 1) {
        // one in-register stage (N = E, one thread per row, no shared
        // memory): v[k] is element k both as the forward's output and as the
        // inverse's input
        Eng::template run<FftPolicy, false>(v, sm, tw, tt, 0, Sync{}, none, [](int, int, float2) {});
#pragma unroll
        for (int k = 0; k < E; ++k) {
            float2 y = cmul(v[k], __ldg(H + k));
            y.y = -y.y;
            v[k] = y;
        }
        Eng::template run<FftPolicy, false>(v, sm, tw, tt, 0, Sync{}, none, store);
    } else {
        // forward transform; its natural-order outputs, times the filter and
        // conjugated, go back into the exchange once every thread has read
        // its last-stage operands, and the inverse loads its stage-0 inputs
        // from there.  The two transforms are one loop body run twice (not
        // unrolled): two inlined copies of the engine would be scheduled into
        // each other and spill.
        static_assert(Eng::SMEM_ELEMS >= N, "the exchange holds the whole padded row");
#pragma unroll 1
        for (int ph = 0; ph < 2; ++ph) {
            if (ph == 1) {
                Sync{}();  // every forward output is in the exchange
#pragma unroll
                for (int b = 0; b < E / R0; ++b) {
                    const int j = tt + b * T;
#pragma unroll
                    for (int r = 0; r < R0; ++r) v[b * R0 + r] = sm[Eng::pad(j + r * (N / R0))];
                }
            }
            auto reads_done = [&] {
                if (ph == 0) Sync{}();  // the forward's outputs overwrite the exchange
            };
            auto out = [&](int i, int c, float2 x) {
                if (ph == 0) {
                    float2 y = cmul(x, __ldg(H + i));
                    y.y = -y.y;
                    sm[Eng::pad(i)] = y;
                } else {
                    store(i, c, x);
                }
            };
            // (ph = 1: the stage-0 reads above precede the first exchange writes)
            Eng::template run<FftPolicy, true>(v, sm, tw, tt, 0, Sync{}, reads_done, out);
        }
    }
}

namespace {
BluVariant g_blu[kMaxLog2 + 1];
std::once_flag g_blu_once;  // registry filled once, safe across host threads

template <int N>
void reg_blu() {
    constexpr int E = N >= 8192 ? 32 : N >= 16 ? 16 : (N >= 8 ? 8 : N);  // the row pass's default E
    using Sh = BluShape<N, E>;
    BluVariant &v = g_blu[ilog2(N)];
    v.fn[0] = (const void *)k_blu<N, E, 0>;
    v.fn[1] = (const void *)k_blu<N, E, 1>;
    v.fn[2] = (const void *)k_blu<N, E, 2>;
    v.n = N;
    v.e = E;
    v.threads = Sh::THREADS;
    v.rows_per_cta = Sh::ROWS;
    v.smem = Sh::SMEM;
}
void init_blu() {
    std::call_once(g_blu_once, [] {
        reg_blu<4>();
        reg_blu<8>();
        reg_blu<16>();
        reg_blu<32>();
        reg_blu<64>();
        reg_blu<128>();
        reg_blu<256>();
        reg_blu<512>();
        reg_blu<1024>();
        reg_blu<2048>();
        reg_blu<4096>();
        reg_blu<8192>();
    });
}

int blocks_for(long long count) {
    long long b = (count + 255) / 256;
    if (b > 152LL * 16) b = 152LL * 16;
    return (int)(b < 1 ? 1 : b);
}
}  // namespace

const BluVariant *blu_variant(int M) {
    init_blu();
    if (M < 4 || M > 8192 || (M & (M - 1))) return nullptr;
    const BluVariant *v = &g_blu[ilog2(M)];
    return v->fn[0] ? v : nullptr;
}

cudaError_t launch_blu(const BluVariant &v, int phase, const float2 *src, float2 *dst, const float2 *tw,
                       const float2 *chirp, const float2 *H, int n, long long rows, cudaStream_t s) {
    if (phase < 0 || phase > 2) return cudaErrorInvalidValue;
    if (v.smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(v.fn[phase], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)v.smem);
        if (e != cudaSuccess) return e;
    }
    const long long grid = (rows + v.rows_per_cta - 1) / v.rows_per_cta;
    if (grid < 1 || grid > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    void *args[] = {(void *)&src, (void *)&dst, (void *)&tw, (void *)&chirp, (void *)&H, (void *)&n, (void *)&rows};
    return cudaLaunchKernel(v.fn[phase], dim3((unsigned)grid), dim3(v.threads), args, v.smem, s);
}

cudaError_t build_chirp(float2 *c, int n, int sgn, cudaStream_t s) {
    k_chirp<<<(n + 255) / 256, 256, 0, s>>>(c, n, sgn);
    return cudaGetLastError();
}

cudaError_t build_chirp_filter(float2 *h, const float2 *c, int n, int M, cudaStream_t s) {
    k_chirp_filter<<<(M + 255) / 256, 256, 0, s>>>(h, c, n, M);
    return cudaGetLastError();
}

cudaError_t launch_scale(float2 *a, long long count, float sc, cudaStream_t s) {
    k_scale<<<blocks_for(count), 256, 0, s>>>(a, count, sc);
    return cudaGetLastError();
}

cudaError_t launch_blu_pre(const float2 *x, float2 *A, const float2 *c, int n, int M, long long rows, cudaStream_t s) {
    k_blu_pre<<<blocks_for(rows * M), 256, 0, s>>>(x, A, c, n, M, rows);
    return cudaGetLastError();
}

cudaError_t launch_blu_mul(float2 *A, const float2 *H, int M, long long rows, cudaStream_t s) {
    k_blu_mul<<<blocks_for(rows * M), 256, 0, s>>>(A, H, M, rows);
    return cudaGetLastError();
}

cudaError_t launch_blu_post(const float2 *A, float2 *out, const float2 *c, int n, int M, long long rows,
                            cudaStream_t s) {
    k_blu_post<<<blocks_for(rows * n), 256, 0, s>>>(A, out, c, n, M, rows);
    return cudaGetLastError();
}

cudaError_t launch_transpose(const float2 *in, float2 *out, int rows, int cols, long long batch, cudaStream_t s) {
    const long long tiles_c = (cols + 31) / 32, tiles_r = (rows + 31) / 32;
    const long long blocks = batch * tiles_r * tiles_c;
    if (blocks < 1 || blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    k_transpose<<<(unsigned)blocks, 256, 0, s>>>(in, out, rows, cols, tiles_c, tiles_r * tiles_c);
    return cudaGetLastError();
}

}  // namespace gb300fft
