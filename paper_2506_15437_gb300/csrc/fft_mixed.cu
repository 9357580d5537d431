// Mixed-radix transforms for lengths of the form 2^a 3^b 5^c 7^d 11^e 13^f.
//
// The paper's kernels take powers of two only and name uneven sizes as
// further work (Sections 6 and 7).  Smooth lengths up to kMixedMaxN run here
// as a Stockham autosort transform whose stages have radix 16, 15, 14, 13,
// 12, 11, 10, 9, 8, 7, 6, 5, 4, 3 or 2, chosen at plan time (15, 14, 12, 10,
// 9 and 6 are two-level DFTs in registers with compile-time inner twiddles;
// the odd primes 3 .. 13 one symmetric-pair DFT each): the
// fewest stages these radices allow, since each stage is one pass through
// shared memory and one barrier.  Stage s of radix R, with Ns
// the product of the radices before it, takes butterfly j (k = j mod Ns)
// from elements j + r n/R, multiplies leg r by w_{Ns R}^{k r}, runs an
// R-point DFT and writes leg r to element (j - k) R + k + r Ns.  After the
// last stage the output is in natural order, so no reorder pass exists.
// One CTA owns whole transforms: the first stage reads global memory, the
// last writes it, and the stages between ping-pong through two padded
// shared-memory buffers.
//
// Two layouts: rows (transforms along contiguous rows, W rows per CTA when
// they are short) and columns (the transforms of W adjacent columns of an
// [ny][nx] slice, element i of column x at i*nx + x), which serves the y axis
// of a 2D plan without a transpose.  Longer smooth lengths run as a
// four-step split n = n1 n2 over both layouts: columns of length n1 into a
// workspace, then rows of length n2 whose first stage multiplies by the
// inter-pass twiddle and whose last stage, with its lanes taken transform
// first, stores the W rows' outputs transposed, W adjacent outputs per row of
// the result (FourStepB).
#include <math.h>

#include "fft_common.cuh"
#include "fft_internal.h"

namespace gb300fft {

namespace {

// cos and sin of 2 pi m / R, evaluated by the compiler: the angle is split
// in integers into a quadrant k (multiples of pi/2) and a remainder phi in
// [0, pi/2), whose sine and cosine are Taylor series summed in double (error
// below 1e-15; exactly 0 and +-1 on the axes), then rounded once to float.
constexpr double kPiD = 3.14159265358979323846264338327950288;
__host__ __device__ constexpr double taylor_sin(double x) {
    double term = x, sum = x;
    for (int k = 1; k < 30; ++k) {
        term *= -x * x / ((2.0 * k) * (2.0 * k + 1.0));
        sum += term;
    }
    return sum;
}
__host__ __device__ constexpr double taylor_cos(double x) {
    double term = 1.0, sum = 1.0;
    for (int k = 1; k < 30; ++k) {
        term *= -x * x / ((2.0 * k - 1.0) * (2.0 * k));
        sum += term;
    }
    return sum;
}
__host__ __device__ constexpr double cos_2pi(int m, int R) {
    const long long q = ((long long)(m % R) + R) % R, t = 4 * q, k = t / R, rem = t - k * R;
    const double phi = (kPiD / 2) * (double)rem / (double)R;
    return k == 0 ? taylor_cos(phi) : k == 1 ? -taylor_sin(phi) : k == 2 ? -taylor_cos(phi) : taylor_sin(phi);
}
__host__ __device__ constexpr double sin_2pi(int m, int R) {
    const long long q = ((long long)(m % R) + R) % R, t = 4 * q, k = t / R, rem = t - k * R;
    const double phi = (kPiD / 2) * (double)rem / (double)R;
    return k == 0 ? taylor_sin(phi) : k == 1 ? taylor_cos(phi) : k == 2 ? -taylor_sin(phi) : -taylor_cos(phi);
}

// cos and sin of 2 pi j / R for j = 1 .. (R-1)/2, rounded to float.  Built
// only in constant initialisers (a constexpr variable), so the double-precision
// series never reach device code.
template <int R>
struct OddRoots {
    float c[(R - 1) / 2], s[(R - 1) / 2];
};
template <int R>
__host__ __device__ constexpr OddRoots<R> odd_roots() {
    OddRoots<R> w{};
    for (int j = 1; j <= (R - 1) / 2; ++j) {
        w.c[j - 1] = (float)cos_2pi(j, R);
        w.s[j - 1] = (float)sin_2pi(j, R);
    }
    return w;
}

// Forward R-point DFT for odd prime R, legs paired as (k, R - k):
//   y_m     = a_0 + sum_k t_k cos(2 pi k m / R) - i sum_k d_k sin(2 pi k m / R)
//   y_{R-m} = a_0 + sum_k t_k cos(2 pi k m / R) + i sum_k d_k sin(2 pi k m / R)
// with t_k = a_k + a_{R-k}, d_k = a_k - a_{R-k}, k, m = 1 .. (R-1)/2.
template <int R>
__device__ __forceinline__ void dft_odd(float2 *a) {
    constexpr int H = (R - 1) / 2;
    constexpr OddRoots<R> W = odd_roots<R>();
    float2 t[H], d[H];
#pragma unroll
    for (int k = 1; k <= H; ++k) {
        t[k - 1] = cadd(a[k], a[R - k]);
        d[k - 1] = csub(a[k], a[R - k]);
    }
    float2 y0 = a[0];
#pragma unroll
    for (int k = 0; k < H; ++k) y0 = cadd(y0, t[k]);
    float2 y[R];
    y[0] = y0;
#pragma unroll
    for (int m = 1; m <= H; ++m) {
        float2 A = a[0], B = make_float2(0.f, 0.f);
#pragma unroll
        for (int k = 1; k <= H; ++k) {
            const int q = (k * m) % R;  // angle index, folded into 1 .. H
            const int j = q <= H ? q : R - q;
            const float c = W.c[j - 1];
            const float sn = q <= H ? W.s[j - 1] : -W.s[j - 1];
            A = make_float2(fmaf(c, t[k - 1].x, A.x), fmaf(c, t[k - 1].y, A.y));
            B = make_float2(fmaf(sn, d[k - 1].x, B.x), fmaf(sn, d[k - 1].y, B.y));
        }
        // -i B = (B.y, -B.x)
        y[m] = make_float2(A.x + B.y, A.y - B.x);
        y[R - m] = make_float2(A.x - B.y, A.y + B.x);
    }
#pragma unroll
    for (int k = 0; k < R; ++k) a[k] = y[k];
}

// x * w_R^M with w_R = exp(-2 pi i / R); powers of -i are exact swaps
template <int M, int R>
__device__ __forceinline__ float2 mul_w(float2 x) {
    if constexpr ((4 * M) % R == 0) {
        constexpr int k = ((4 * M) / R) % 4;
        if constexpr (k == 0) return x;
        else if constexpr (k == 1) return make_float2(x.y, -x.x);
        else if constexpr (k == 2) return make_float2(-x.x, -x.y);
        else return make_float2(-x.y, x.x);
    } else {
        constexpr float wr = (float)cos_2pi(M, R), wi = (float)-sin_2pi(M, R);
        return make_float2(fmaf(x.x, wr, -x.y * wi), fmaf(x.x, wi, x.y * wr));
    }
}

template <int R>
__device__ __forceinline__ void dft_any(float2 *a);

// R = R1 R2 points in registers, natural order in and out: with input index
// i2 + R2 i1 and output index k1 + R1 k2, w_R^{ik} = w_R1^{i1 k1} w_R^{i2 k1}
// w_R2^{i2 k2}, so: R2 transforms of length R1 (over i1), the inner twiddles
// w_R^{i2 k1} (compile-time constants), R1 transforms of length R2 (over i2).
template <int R1, int R2, int I2, int K1>
__device__ __forceinline__ void dft_2lvl_tw(const float2 *t, float2 *b) {
    if constexpr (K1 < R1) {
        b[I2 * R1 + K1] = mul_w<I2 * K1, R1 * R2>(t[K1]);
        dft_2lvl_tw<R1, R2, I2, K1 + 1>(t, b);
    }
}
template <int R1, int R2, int I2 = 0>
__device__ __forceinline__ void dft_2lvl_cols(const float2 *a, float2 *b) {
    if constexpr (I2 < R2) {
        float2 t[R1];
#pragma unroll
        for (int i1 = 0; i1 < R1; ++i1) t[i1] = a[I2 + R2 * i1];
        dft_any<R1>(t);
        dft_2lvl_tw<R1, R2, I2, 0>(t, b);
        dft_2lvl_cols<R1, R2, I2 + 1>(a, b);
    }
}
template <int R1, int R2>
__device__ __forceinline__ void dft_2lvl(float2 *a) {
    float2 b[R1 * R2];
    dft_2lvl_cols<R1, R2>(a, b);
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) {
        float2 t[R2];
#pragma unroll
        for (int i2 = 0; i2 < R2; ++i2) t[i2] = b[i2 * R1 + k1];
        dft_any<R2>(t);
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2) a[k1 + R1 * k2] = t[k2];
    }
}

template <int R>
__device__ __forceinline__ void dft_any(float2 *a) {
    if constexpr ((R & (R - 1)) == 0) dft<R>(a);
    else if constexpr (R == 6) dft_2lvl<2, 3>(a);
    else if constexpr (R == 9) dft_2lvl<3, 3>(a);
    else if constexpr (R == 10) dft_2lvl<2, 5>(a);
    else if constexpr (R == 12) dft_2lvl<4, 3>(a);
    else if constexpr (R == 14) dft_2lvl<2, 7>(a);
    else if constexpr (R == 15) dft_2lvl<3, 5>(a);
    else dft_odd<R>(a);
}

struct MixedGeom {
    int n;        // transform length
    int W;        // transforms per CTA
    int nv;       // valid transforms in this CTA (rows: the last CTA may hold fewer)
    int estride;  // element stride within a transform (1 for rows, nx for columns)
    int tstride;  // offset between the CTA's transforms (n for rows, 1 for columns)
};

// x / d for x * d < 2^32 by a multiply-high with m = ceil(2^32 / d) (d >= 2);
// d = 1 passes x through
__device__ __forceinline__ int fdiv(int x, int d, uint32_t m) {
    return d == 1 ? x : (int)__umulhi((uint32_t)x, m);
}

// Twiddle-table entries per butterfly of a radix-R stage: R - 1 rounded up
// to even, so each butterfly's twiddles are whole 16-byte pairs.
__host__ __device__ constexpr int mixed_tw_stride(int R) { return (R - 1 + 1) & ~1; }

struct StageArgs {
    int nb, Ns;  // butterflies per transform, product of the earlier radices
    uint32_t mag_nb, mag_ns;
    int wlog;
    int pin, pout;  // padding shifts of the buffer read and of the buffer written (31: none)
};

// padded shared-memory index: one spare slot after every 2^ps elements
// (ps = 31: no padding, since every index is below 2^31)
__device__ __forceinline__ int padx(int x, int ps) { return x + (x >> ps); }

// One stage of radix R over the CTA's W transforms, `src` to `dst` (global
// memory in place of `src` in the first stage, of `dst` in the last).  Rows:
// butterfly index fastest within a transform (coalesced rows); columns:
// transform fastest (W adjacent columns of a row together).  Local layout:
// rows [c][i], columns [i][c].  `gin` and `gout` point at the CTA's first
// transform, so every offset within the group fits 32 bits.
template <int R, bool COLS, bool FIRST, bool LAST, bool FS>
__device__ __forceinline__ void mixed_stage(const MixedGeom &g, const StageArgs a, const float2 *src, float2 *dst,
                                            const float2 *gin, float2 *gout, const float2 *__restrict__ tws,
                                            float si, const FourStepB &fs) {
    const int nb = a.nb, Ns = a.Ns;
    const int total = g.nv * nb;
    // lanes by transform first (c fastest) for the column layout, and for
    // the last stage of a four-step row pass, whose outputs go to global
    // memory transposed: W adjacent outputs per row of the result
    constexpr bool CFAST = COLS || (LAST && FS);
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
        int c, j;
        if (CFAST) {
            c = idx & (g.W - 1);
            j = idx >> a.wlog;
        } else {
            c = fdiv(idx, nb, a.mag_nb);
            j = idx - c * nb;
        }
        const int k = j - fdiv(j, Ns, a.mag_ns) * Ns;
        float2 v[R];
        // four-step: element i2 = j + r nb of row m = k1 + c times w_n^{i2 m}
        // = w_n^{j m} w_n^{r nb m}, each from the two factor tables w_n^a =
        // hi[a >> L] lo[a & (2^L - 1)].  The first factor is one gather per
        // thread; the second is the same for every lane of a row, so its
        // loads are broadcasts (one gather per element, lanes m entries
        // apart, cost a cache line each)
        float2 wj = make_float2(1.f, 0.f);
        if (FIRST && FS) {
            const int e = j * (fs.k1 + c);
            wj = cmul(__ldg(fs.hi + (e >> fs.lshift)), __ldg(fs.lo + (e & fs.lmask)));
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int i = j + r * nb;
            if (FIRST) {
                float2 x = gin[c * g.tstride + i * g.estride];
                x.y *= si;
                if (FS) {
                    float2 w = wj;
                    if (r > 0) {
                        const int e = r * nb * (fs.k1 + c);
                        w = cmul(w, cmul(__ldg(fs.hi + (e >> fs.lshift)), __ldg(fs.lo + (e & fs.lmask))));
                    }
                    x = cmul(x, w);
                }
                v[r] = x;
            } else {
                v[r] = src[padx(COLS ? i * g.W + c : c * g.n + i, a.pin)];
            }
        }
        if (!FIRST) {
            // twiddles r, r + 1 of butterfly k as one 16-byte load, pair p =
            // (r - 1) / 2 of every butterfly in one row of the table: lanes
            // with consecutive k read consecutive 16-byte words.  (With the
            // pairs of one butterfly together, lanes read words M/2 apart,
            // which conflict in the L1 banks when M/2 is even.  Measured
            // against that layout: 16384 x 3000 0.251 -> 0.236 ms, 1920 x
            // 1080 x 8 0.183 -> 0.175, 6^9 0.231 -> 0.224, 1000^2 x 32 0.310
            // -> 0.305; 10^6 x 32 0.360 -> 0.369, 15360 x 1024 0.123 -> 0.130)
            const float4 *w = reinterpret_cast<const float4 *>(tws) + k;
#pragma unroll
            for (int r = 1; r < R; r += 2) {
                const float4 w2 = __ldg(w + ((r - 1) / 2) * Ns);
                v[r] = cmul(v[r], make_float2(w2.x, w2.y));
                if (r + 1 < R) v[r + 1] = cmul(v[r + 1], make_float2(w2.z, w2.w));
            }
        }
        dft_any<R>(v);
        const int o0 = (j - k) * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int o = o0 + r * Ns;
            if (LAST && FS) {
                // output o of row k1 + c goes to k1 + c + n1 o (gout points at k1)
                float2 x = v[r];
                x.y *= si;
                gout[c + (long long)fs.n1 * o] = x;
            } else if (LAST) {
                float2 x = v[r];
                x.y *= si;
                gout[c * g.tstride + o * g.estride] = x;
            } else {
                dst[padx(COLS ? o * g.W + c : c * g.n + o, a.pout)] = v[r];
            }
        }
    }
}

template <bool COLS, bool FIRST, bool LAST, bool FS>
__device__ __forceinline__ void mixed_dispatch(int R, const MixedGeom &g, const StageArgs a, const float2 *src,
                                               float2 *dst, const float2 *gin, float2 *gout, const float2 *tws,
                                               float si, const FourStepB &fs) {
    switch (R) {
        case 2: mixed_stage<2, COLS, FIRST, LAST, FS>(g, a, src, dst, gin, gout, tws, si, fs); break;
        case 3: mixed_stage<3, COLS, FIRST, LAST, FS>(g, a, src, dst, gin, gout, tws, si, fs); break;
        case 4: mixed_stage<4, COLS, FIRST, LAST, FS>(g, a, src, dst, gin, gout, tws, si, fs); break;
        case 5: mixed_stage<5, COLS, FIRST, LAST, FS>(g, a, src, dst, gin, gout, tws, si, fs); break;
        case 6: mixed_stage<6, COLS, FIRST, LAST, FS>(g, a, src, dst, gin, gout, tws, si, fs); break;
        case 7: mixed_stage<7, COLS, FIRST, LAST, FS>(g, a, src, dst, gin, gout, tws, si, fs); break;
        case 8: mixed_stage<8, COLS, FIRST, LAST, FS>(g, a, src, dst, gin, gout, tws, si, fs); break;
        case 9: mixed_stage<9, COLS, FIRST, LAST, FS>(g, a, src, dst, gin, gout, tws, si, fs); break;
        case 10: mixed_stage<10, COLS, FIRST, LAST, FS>(g, a, src, dst, gin, gout, tws, si, fs); break;
        case 11: mixed_stage<11, COLS, FIRST, LAST, FS>(g, a, src, dst, gin, gout, tws, si, fs); break;
        case 12: mixed_stage<12, COLS, FIRST, LAST, FS>(g, a, src, dst, gin, gout, tws, si, fs); break;
        case 13: mixed_stage<13, COLS, FIRST, LAST, FS>(g, a, src, dst, gin, gout, tws, si, fs); break;
        case 14: mixed_stage<14, COLS, FIRST, LAST, FS>(g, a, src, dst, gin, gout, tws, si, fs); break;
        case 15: mixed_stage<15, COLS, FIRST, LAST, FS>(g, a, src, dst, gin, gout, tws, si, fs); break;
        default: mixed_stage<16, COLS, FIRST, LAST, FS>(g, a, src, dst, gin, gout, tws, si, fs); break;
    }
}

template <bool COLS, bool FS>
__global__ void __launch_bounds__(1024) k_mixed(const float2 *in, float2 *out, const float2 *__restrict__ tw,
                                                const MixedStages st, long long ntrans, int W, int nx, int conj,
                                                FourStepB fs) {
    extern __shared__ __align__(16) float2 mbuf[];
    MixedGeom g;
    g.n = st.n;
    g.W = W;
    const long long t0 = (long long)blockIdx.x * W;  // first transform of this CTA
    long long base;
    if (COLS) {
        // transform t: column t % nx of slice t / nx; W divides nx
        const long long b = t0 / nx;
        const int x0 = (int)(t0 - b * nx);
        g.nv = W;
        base = b * (long long)nx * st.n + x0;
        g.estride = nx;
        g.tstride = 1;
    } else {
        g.nv = (int)(ntrans - t0 < W ? ntrans - t0 : W);
        base = t0 * st.n;
        g.estride = 1;
        g.tstride = st.n;
    }
    const float2 *gin = in + base;
    float2 *gout = out + base;  // four-step rows: replaced below by the transposed output origin
    // the first stage reads the group's input in rounds of blockDim.x
    // butterflies: ask L2 for all of it now, so later rounds find it there
    if (!COLS) {
        if (threadIdx.x == 0) {
            // the group's rows are contiguous: one bulk prefetch of the
            // 16-byte-aligned interior
            const uintptr_t a0 = reinterpret_cast<uintptr_t>(gin);
            const uintptr_t a1 = a0 + (uintptr_t)g.nv * st.n * sizeof(float2);
            const uintptr_t p0 = (a0 + 15) & ~(uintptr_t)15, p1 = a1 & ~(uintptr_t)15;
            if (p1 > p0) bulk_prefetch_l2(reinterpret_cast<const void *>(p0), (uint32_t)(p1 - p0));
        }
    } else {
        for (int i = threadIdx.x; i < st.n; i += blockDim.x)
            asm volatile("prefetch.global.L2 [%0];" ::"l"(gin + (long long)i * nx));
    }
    if (FS) {
        // rows t0 .. t0 + W - 1 are rows k1 of one transform b (W divides n1)
        const long long b = t0 / fs.n1;
        fs.k1 = (int)(t0 - b * fs.n1);
        gout = out + b * (long long)fs.n1 * st.n + fs.k1;
    }
    const float si = conj ? -1.f : 1.f;
    float2 *A = mbuf, *B = mbuf + st.buf_elems;
    for (int s = 0; s < st.S; ++s) {
        StageArgs a;
        a.nb = st.nb[s];
        a.Ns = st.ns[s];
        a.mag_nb = st.mag_nb[s];
        a.mag_ns = st.mag_ns[s];
        a.wlog = st.wlog;
        a.pin = (s > 0 && st.pad[s - 1]) ? st.pad[s - 1] : 31;
        a.pout = st.pad[s] ? st.pad[s] : 31;
        const float2 *tws = tw + st.tw_off[s];
        const int R = st.radix[s];
        if (st.S == 1) mixed_dispatch<COLS, true, true, FS>(R, g, a, A, B, gin, gout, tws, si, fs);
        else if (s == 0) mixed_dispatch<COLS, true, false, FS>(R, g, a, A, B, gin, gout, tws, si, fs);
        else if (s == st.S - 1) mixed_dispatch<COLS, false, true, FS>(R, g, a, A, B, gin, gout, tws, si, fs);
        else mixed_dispatch<COLS, false, false, FS>(R, g, a, A, B, gin, gout, tws, si, fs);
        __syncthreads();
        float2 *tmp = A;
        A = B;
        B = tmp;
    }
}

// stage s's table, as 16-byte pairs: pair p of butterfly k (k < Ns) at
// pair index p Ns + k holds w_{Ns R}^{k r} for r = 2p + 1 and 2p + 2 (the
// second zero when R - 1 is odd), from the FP64 root, rounded once
__global__ void k_mixed_twiddles(float2 *t, int Ns, int R) {
    const int M = mixed_tw_stride(R);
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= Ns * M) return;
    const int q = e >> 1, p = q / Ns, k = q - p * Ns, r = 2 * p + 1 + (e & 1);
    if (r >= R) {
        t[e] = make_float2(0.f, 0.f);
        return;
    }
    const int L = Ns * R;
    double sv, cv;
    sincospi(2.0 * (double)((k * r) % L) / (double)L, &sv, &cv);
    t[e] = make_float2((float)cv, (float)(-sv));
}

const void *mixed_fn(bool cols, bool fs) {
    return cols ? (const void *)k_mixed<true, false>
                : fs ? (const void *)k_mixed<false, true> : (const void *)k_mixed<false, false>;
}

// One kernel serves every mixed length, each plan with its own shared
// memory size, so the kernel's dynamic shared-memory limit is raised to the
// largest any plan may ask for, the same value from every plan: a
// plan-sized limit would let a plan created later (or concurrently, on
// another thread) lower it below what an earlier plan launches with.
bool smem_ok(const void *fn, size_t smem) {
    if (smem > kMixedMaxSmem) return false;
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMixedMaxSmem) != cudaSuccess)
        return false;
    return true;
}

uint32_t magic(int d) { return d <= 1 ? 0u : (uint32_t)((((uint64_t)1 << 32) + (uint64_t)d - 1) / (uint64_t)d); }

// Threads for a group of W transforms of total length W n: a group longer
// than 8192 points fills one SM's shared memory alone, so it brings the
// most threads it can.
int mixed_threads(int elems) { return elems > 8192 ? 1024 : elems > 4096 ? 512 : 256; }

// Shared-memory wavefronts of one access pattern under the half-warp model
// for 8-byte words: the 16 lanes of a half-warp form one wavefront per
// distinct word sharing a bank pair, so the cost of a half-warp is the
// largest number of distinct words on one pair (1 when conflict free).
// `addr(lane)` gives the padded word index or -1 for an idle lane.
template <class F>
long long half_warp_cost(int lanes, F addr) {
    long long cost = 0;
    for (int h = 0; h < lanes; h += 16) {
        int words[16][16];
        int cnt[16] = {};
        for (int l = h; l < h + 16 && l < lanes; ++l) {
            const int a = addr(l);
            if (a < 0) continue;
            const int b = a & 15;
            bool seen = false;
            for (int q = 0; q < cnt[b]; ++q) seen = seen || words[b][q] == a;
            if (!seen) words[b][cnt[b]++] = a;
        }
        int worst = 0;
        for (int b = 0; b < 16; ++b) worst = cnt[b] > worst ? cnt[b] : worst;
        cost += worst;
    }
    return cost;
}

// Cost of the buffer written by stage s (with shift ps) and read by stage
// s + 1 (same shift), over the first warps of every round (the patterns
// repeat with the butterfly index).
long long boundary_cost(const MixedStages &st, int s, int W, bool cols, bool fs, int T, int ps) {
    auto pad = [ps](int x) { return ps ? x + (x >> ps) : x; };
    long long cost = 0;
    for (int side = 0; side < 2; ++side) {
        const int t = s + side;  // stage that writes (side 0) or reads (side 1)
        const int R = st.radix[t], nb = st.nb[t], Ns = st.ns[t];
        const int total = W * nb;
        for (int base = 0; base < total; base += T)
            for (int w0 = base; w0 < base + T && w0 < total && w0 < base + 4 * 32; w0 += 32)
                for (int r = 0; r < R; ++r)
                    cost += half_warp_cost(32, [&](int l) {
                        const int idx = w0 + l;
                        if (idx >= total || idx >= base + T) return -1;
                        // lane order of stage t (the four-step row pass's last
                        // stage takes the transforms fastest, like the columns)
                        const bool cfast = cols || (fs && t == st.S - 1);
                        const int c = cfast ? idx % W : idx / nb;
                        const int j = cfast ? idx / W : idx % nb;
                        const int k = j % Ns;
                        const int e = side ? j + r * nb : (j - k) * R + k + r * Ns;
                        return pad(cols ? e * W + c : c * st.n + e);
                    });
    }
    return cost;
}

// the stage constants the kernel reads for a group of W transforms, with a
// padding shift per stage boundary chosen by the bank model
MixedStages with_group(const MixedStages &st, int W, bool cols, bool fs, int T) {
    MixedStages m = st;
    m.wlog = ilog2(W);
    int elems = W * st.n;
    for (int s = 0; s < st.S; ++s) {
        m.mag_nb[s] = magic(st.nb[s]);
        m.mag_ns[s] = magic(st.ns[s]);
        m.pad[s] = 0;
        if (s + 1 < st.S) {
            long long best = boundary_cost(st, s, W, cols, fs, T, 0);
            for (int ps : {5, 4, 3}) {
                // both buffers, padded, within one CTA's shared memory
                if ((size_t)2 * (W * st.n + ((W * st.n - 1) >> ps)) * sizeof(float2) > kMixedMaxSmem) continue;
                const long long c = boundary_cost(st, s, W, cols, fs, T, ps);
                if (c < best) {
                    best = c;
                    m.pad[s] = ps;
                }
            }
            const int e = W * st.n + ((W * st.n - 1) >> (m.pad[s] ? m.pad[s] : 31));
            if (m.pad[s] && e > elems) elems = e;
        }
    }
    m.buf_elems = elems;
    return m;
}

// the compiled radices, largest first
constexpr int kMixedRadices[] = {16, 15, 14, 13, 12, 11, 10, 9, 8, 7, 6, 5, 4, 3, 2};

// rest as a product of exactly `left` compiled radices, none larger than
// `cap` (non-increasing, so each multiset is tried once), into out[]
bool factor_exact(int rest, int left, int cap, int *out) {
    if (left == 0) return rest == 1;
    long long reach = 1;
    for (int i = 0; i < left; ++i) reach *= cap;
    if (reach < rest) return false;
    for (int R : kMixedRadices) {
        if (R > cap || rest % R) continue;
        out[0] = R;
        if (factor_exact(rest / R, left - 1, R, out + 1)) return true;
    }
    return false;
}

}  // namespace

bool mixed_factor(int n, MixedStages *st) {
    if (n < 2 || n > kMixedMaxN) return false;
    MixedStages m;
    m.n = n;
    int rest = n, S = 0;
    auto push = [&](int R) {
        if (S >= kMixedMaxStages) return false;
        m.radix[S++] = R;
        rest /= R;
        return true;
    };
    // greedy: powers of two: 16s, then one 8, 4 or 2; odd part: 3 * 5 and 3 * 3
    // in one register stage each, then single 3, 5, 7, 11, 13 (a 25-point stage needs
    // twice the registers of a 16-point one and halves the CTAs per SM:
    // measured slower than two 5-point stages)
    int e3 = 0, e5 = 0;
    for (int t = rest; t % 3 == 0; t /= 3) ++e3;
    for (int t = rest; t % 5 == 0; t /= 5) ++e5;
    while (rest % 16 == 0)
        if (!push(16)) return false;
    for (int R : {8, 4, 2})
        if (rest % R == 0 && !push(R)) return false;
    for (; e5 >= 1 && e3 >= 1; --e5, --e3)
        if (!push(15)) return false;
    for (; e3 >= 2; e3 -= 2)
        if (!push(9)) return false;
    if (e3 == 1 && !push(3)) return false;
    for (; e5 >= 1; --e5)
        if (!push(5)) return false;
    for (int R : {7, 11, 13})
        while (rest % R == 0)
            if (!push(R)) return false;
    if (rest != 1) return false;
    // the greedy schedule above is kept where no schedule has fewer stages
    // (e.g. 3000 = 8 15 5 5); otherwise the first of the fewest, radices
    // non-increasing (1000 = 10 10 10 in place of 8 5 5 5, 1728 = 16 12 9 in
    // place of 16 4 9 3, 96 = 16 6 in place of 16 2 3)
    for (int d = 1; d < S; ++d) {
        int r[kMixedMaxStages];
        if (factor_exact(n, d, 16, r)) {
            for (int i = 0; i < d; ++i) m.radix[i] = r[i];
            S = d;
            break;
        }
    }
    m.S = S;
    int off = 0, Ns = 1;
    for (int s = 0; s < S; ++s) {
        m.tw_off[s] = off;
        m.ns[s] = Ns;
        m.nb[s] = n / m.radix[s];
        off += Ns * mixed_tw_stride(m.radix[s]);
        Ns *= m.radix[s];
    }
    m.tw_size = off;
    if (st) *st = m;
    return true;
}

cudaError_t build_mixed_twiddles(float2 *tw, const MixedStages &st, cudaStream_t s) {
    int Ns = 1;
    for (int i = 0; i < st.S; ++i) {
        const int R = st.radix[i], count = Ns * mixed_tw_stride(R);
        k_mixed_twiddles<<<(count + 255) / 256, 256, 0, s>>>(tw + st.tw_off[i], Ns, R);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        Ns *= R;
    }
    return cudaSuccess;
}

int mixed_rows_per_cta(int n) {
    int W = 1;
    while (W < 64 && (long long)2 * W * n <= 4096) W *= 2;
    return W;
}

int mixed_cols_width(int n, int nx) {
    // widest group of adjacent columns (a divisor of nx) whose two buffers
    // leave room for three CTAs per SM, else the widest that fits at all
    for (int W : {8, 4, 2})
        if (nx % W == 0 && (size_t)2 * W * n * sizeof(float2) <= 72 * 1024) return W;
    for (int W : {8, 4, 2})
        if (nx % W == 0 && (size_t)2 * W * n * sizeof(float2) <= kMixedMaxSmem) return W;
    return 1;
}

int mixed_prepare(const MixedStages &st, bool cols, int nx, MixedLaunch *out, int fs_n1) {
    MixedLaunch L;
    L.cols = cols;
    L.nx = cols ? nx : 0;
    const bool fs = !cols && fs_n1 > 0;
    if (fs) {
        // W rows of one transform per CTA (W divides n1); the last stage
        // stores W adjacent outputs of the result per row
        L.fs.n1 = fs_n1;
        L.W = 1;
        for (int W : {8, 4, 2})
            if (fs_n1 % W == 0 && (size_t)2 * W * st.n * sizeof(float2) <= 72 * 1024) {
                L.W = W;
                break;
            }
    } else {
        L.W = cols ? mixed_cols_width(st.n, nx) : mixed_rows_per_cta(st.n);
    }
    if (cols && (nx <= 0 || nx % L.W)) return -1;
    L.T = mixed_threads(L.W * st.n);
    // no more threads than the widest stage has butterflies: for short
    // transforms the idle ones would hold registers and block slots (measured
    // 100 x 100 x 2048: 0.259 -> 0.154 ms).  More threads than the default,
    // to run a stage in one round, measured slower where they cost resident
    // blocks (96-point rows 0.152 -> 0.194 ms, 1920 x 1080 x 8: 0.183 -> 0.197)
    int most = 0;
    for (int s = 0; s < st.S; ++s) most = L.W * st.nb[s] > most ? L.W * st.nb[s] : most;
    if (((most + 31) & ~31) < L.T) L.T = (most + 31) & ~31;
    L.m = with_group(st, L.W, cols, fs, L.T);
    L.smem = (size_t)2 * L.m.buf_elems * sizeof(float2);
    if (L.smem > kMixedMaxSmem) return -1;
    if (!smem_ok(mixed_fn(cols, fs), L.smem)) return -1;
    *out = L;
    return 0;
}

bool mixed_split(int n, int *n1, int *n2) {
    int best = 0;
    double bd = 1e30;
    for (int d = 2; d <= kMixedMaxN && d < n; ++d) {
        if (n % d || n / d > kMixedMaxN || !mixed_factor(d, nullptr) || !mixed_factor(n / d, nullptr)) continue;
        const double dist = fabs(log((double)d) - 0.5 * log((double)n));
        if (dist < bd) {
            bd = dist;
            best = d;
        }
    }
    if (!best) return false;
    *n2 = best;
    *n1 = n / best;
    return true;
}

cudaError_t launch_mixed(const MixedLaunch &L, const float2 *tw, const float2 *in, float2 *out, long long count,
                         int conj, cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    if (L.T <= 0) return cudaErrorInvalidValue;
    // rows: count transforms; columns: count slices of nx columns
    long long ntrans = L.cols ? count * L.nx : count;
    const long long grid = (ntrans + L.W - 1) / L.W;
    if (grid > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    const void *fn = mixed_fn(L.cols, L.fs.n1 > 0);
    int W = L.W, nx = L.nx;
    FourStepB fs = L.fs;
    void *args[] = {(void *)&in, (void *)&out, (void *)&tw, (void *)&L.m, (void *)&ntrans, (void *)&W,
                    (void *)&nx, (void *)&conj, (void *)&fs};
    return cudaLaunchKernel(fn, dim3((unsigned)grid), dim3(L.T), args, L.smem, s);
}

}  // namespace gb300fft

// The float constants the composite-radix DFTs multiply by, as the
// compiler evaluates them (host copy of the same constexpr functions).
extern "C" int fft_debug_root(int m, int r, float *c, float *s) {
    if (!c || !s || r < 1) return FFT_ERR_INVALID_ARG;
    *c = (float)gb300fft::cos_2pi(m, r);
    *s = (float)gb300fft::sin_2pi(m, r);
    return FFT_OK;
}
