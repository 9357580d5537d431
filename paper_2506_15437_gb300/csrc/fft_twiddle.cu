// Twiddle tables and small helper kernels.
//
// The paper computes its twiddle factors once at initialisation and keeps
// them on chip because they do not change from step to step (Section 4).
// Here each plan builds, once, one table per (length n, elements per thread
// E): stage s >= 1 of the schedule (radix E, span Ns) owns E*Ns float2
// entries holding, as float4 pairs at float4 index k*Ns + m,
//     (exp(-2*pi*i*(2k+1)*m/(Ns*E)), exp(-2*pi*i*(2k+2)*m/(Ns*E))),  k < E/2,
// so that the threads of a warp (consecutive m) read consecutive 16-byte
// words, two twiddles per load.  Values are computed in double precision with sincospi of the
// exact dyadic argument 2*r*m/(Ns*E) and rounded once to float -- the only
// place double precision runs on the GPU.
#include "fft_common.cuh"
#include "fft_internal.h"

namespace gb300fft {

__global__ void k_twiddles(float2 *tw, int r0, int e, int stages, int total) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= total) return;
    int off = 0;
    long long ns = r0;
    for (int s = 1; s < stages; ++s) {
        const long long sz = (long long)e * ns;
        if (idx < off + sz) {
            const long long k2 = idx - off;          // float2 index within the stage
            const long long f = k2 >> 1;             // float4 index = pair * Ns + m
            const long long r = 2 * (f / ns) + 1 + (k2 & 1);
            const long long m = f % ns;
            const long long K = ns * e;
            double sv, cv;
            sincospi(2.0 * (double)((r * m) % K) / (double)K, &sv, &cv);
            tw[idx] = make_float2((float)cv, (float)(-sv));
            return;
        }
        off += (int)sz;
        ns *= e;
    }
}

int twiddle_table_size(int n, int e) {
    int rad[16];
    const int S = schedule_radices(n, e, rad);
    if (S < 0) return -1;
    long long total = 0, ns = rad[0];
    for (int k = 1; k < S; ++k) {
        total += (long long)rad[k] * ns;
        ns *= rad[k];
    }
    return (int)total;
}

cudaError_t build_twiddles(float2 *tw, int n, int e, cudaStream_t s) {
    int rad[16];
    const int S = schedule_radices(n, e, rad);
    if (S < 0) return cudaErrorInvalidValue;
    long long total = 0, ns = rad[0];
    for (int k = 1; k < S; ++k) {
        total += (long long)rad[k] * ns;
        ns *= rad[k];
    }
    if (total == 0) return cudaSuccess;
    const int threads = 256;
    const int blocks = (int)((total + threads - 1) / threads);
    k_twiddles<<<blocks, threads, 0, s>>>(tw, rad[0], S > 1 ? rad[1] : 1, S, (int)total);
    return cudaGetLastError();
}

__global__ void k_roots(float2 *t, int n) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    double sv, cv;
    sincospi(2.0 * (double)k / (double)n, &sv, &cv);
    t[k] = make_float2((float)cv, (float)(-sv));
}

cudaError_t build_roots(float2 *t, int n, cudaStream_t s) {
    k_roots<<<(n + 255) / 256, 256, 0, s>>>(t, n);
    return cudaGetLastError();
}

// t[k] = exp(-2*pi*i*(k*stride mod n)/n) for k < count: the two factor tables
// of the four-step inter-pass twiddle (stride 1 and stride 8192).
__global__ void k_roots_strided(float2 *t, int count, long long n, long long stride) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= count) return;
    const long long a = ((long long)k * stride) % n;
    double sv, cv;
    sincospi(2.0 * (double)a / (double)n, &sv, &cv);
    t[k] = make_float2((float)cv, (float)(-sv));
}

cudaError_t build_roots_strided(float2 *t, int count, long long n, long long stride, cudaStream_t s) {
    if (count < 1 || n < 1 || stride < 0) return cudaErrorInvalidValue;
    k_roots_strided<<<(count + 255) / 256, 256, 0, s>>>(t, count, n, stride);
    return cudaGetLastError();
}

// Partial sums of sum_i w[i] * |X[i]|^2: one float partial per CTA.  Each
// thread keeps a compensated (Kahan) float sum over its grid-stride share,
// then the CTA adds its threads' sums as a tree.  The caller adds the
// partials (in double on the host side).
__global__ void __launch_bounds__(256) k_weighted_power(const float2 *__restrict__ X, const float *__restrict__ w,
                                                        long long n, float *partials) {
    float acc = 0.f, comp = 0.f;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const float2 x = __ldg(X + i);
        const float term = __ldg(w + i) * fmaf(x.x, x.x, x.y * x.y);
        const float y = term - comp;
        const float t = acc + y;
        comp = (t - acc) - y;
        acc = t;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    __shared__ float red[8];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int k = 0; k < 8; ++k) t += red[k];
        partials[blockIdx.x] = t;
    }
}

cudaError_t launch_weighted_power(const float2 *X, const float *w, long long n, float *partials,
                                  int parts, cudaStream_t s) {
    k_weighted_power<<<parts, 256, 0, s>>>(X, w, n, partials);
    return cudaGetLastError();
}

}  // namespace gb300fft
