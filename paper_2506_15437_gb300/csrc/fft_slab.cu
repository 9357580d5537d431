// Slab decomposition of a 2D transform over several GPUs: the exchange step.
//
// The paper scales its 2D FFT across cores by row FFTs, a global transpose
// and column FFTs (Section 5, Fig. 6), and leaves the multi-card version, with
// the transpose as the exchange between cards, as future work (Section 6).
// Here G ranks each hold `rows` = ny/G consecutive rows of every [ny][nx]
// slice.  After the local row FFTs, rank r sends rank s the (rows x w) block
// of its rows that lies in column slab s (w = nx/G columns); after the
// all-to-all, rank s holds all ny rows of its w columns and runs the column
// FFTs locally.  These two kernels lay the blocks out so that the exchange is
// one contiguous chunk per peer:
//   pack:   out[s][b][y][x'] = in[b][y][s*w + x']      (send buffer, by peer)
//   unpack: out[b][r*rows + y][x'] = in[r][b][y][x']   (receive buffer -> slab)
// Both are plain copies of complex64 elements: runs of w contiguous elements
// move as 16-byte pairs when w is even, else one element at a time.
#include "fft_common.cuh"
#include "fft_internal.h"

namespace gb300fft {

// V = float4 (two elements, w even) or float2 (one)
template <class V>
__global__ void __launch_bounds__(256) k_slab_pack(const V *__restrict__ in, V *__restrict__ out, int G, int batch,
                                                   int rows, int nxv, int wv) {
    const long long total = (long long)G * batch * rows * wv;
    for (long long o = (long long)blockIdx.x * blockDim.x + threadIdx.x; o < total;
         o += (long long)gridDim.x * blockDim.x) {
        const long long xq = o % wv;           // element pair within the block row
        const long long r1 = o / wv;           // (s, b, y) flattened
        const long long y = r1 % rows;
        const long long r2 = r1 / rows;        // (s, b)
        const long long b = r2 % batch;
        const long long s = r2 / batch;
        out[o] = in[(b * rows + y) * nxv + s * wv + xq];
    }
}

template <class V>
__global__ void __launch_bounds__(256) k_slab_unpack(const V *__restrict__ in, V *__restrict__ out, int G, int batch,
                                                     int rows, int wv) {
    const long long total = (long long)G * batch * rows * wv;
    for (long long o = (long long)blockIdx.x * blockDim.x + threadIdx.x; o < total;
         o += (long long)gridDim.x * blockDim.x) {
        const long long xq = o % wv;
        const long long r1 = o / wv;           // (b, Y) flattened, Y = r*rows + y
        const long long Y = r1 % ((long long)G * rows);
        const long long b = r1 / ((long long)G * rows);
        const long long r = Y / rows, y = Y % rows;
        out[o] = in[((r * batch + b) * rows + y) * wv + xq];
    }
}

static int slab_grid(long long total) {
    long long blocks = (total + 255) / 256;
    if (blocks > 152LL * 16) blocks = 152LL * 16;  // grid-stride beyond 16 CTAs per SM
    return blocks < 1 ? 1 : (int)blocks;
}

}  // namespace gb300fft

extern "C" {

int fft_slab_pack(const void *in, void *out, int parts, int batch, int rows, int nx, void *stream) {
    using namespace gb300fft;
    if (!in || !out || in == out) return FFT_ERR_INVALID_ARG;
    if (parts < 1 || batch < 1 || rows < 1 || nx < parts || nx % parts) return FFT_ERR_INVALID_SIZE;
    if ((long long)parts * batch * rows * (nx / parts) > (1LL << 31)) return FFT_ERR_INVALID_SIZE;
    if ((reinterpret_cast<uintptr_t>(in) & 15) || (reinterpret_cast<uintptr_t>(out) & 15)) return FFT_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int w = nx / parts;
    if (w % 2 == 0) {
        const long long total = (long long)parts * batch * rows * (w / 2);
        k_slab_pack<float4><<<slab_grid(total), 256, 0, s>>>(static_cast<const float4 *>(in), static_cast<float4 *>(out),
                                                             parts, batch, rows, nx / 2, w / 2);
    } else {
        const long long total = (long long)parts * batch * rows * w;
        k_slab_pack<float2><<<slab_grid(total), 256, 0, s>>>(static_cast<const float2 *>(in), static_cast<float2 *>(out),
                                                             parts, batch, rows, nx, w);
    }
    return cudaGetLastError() == cudaSuccess ? FFT_OK : FFT_ERR_CUDA;
}

int fft_slab_unpack(const void *in, void *out, int parts, int batch, int rows, int w, void *stream) {
    using namespace gb300fft;
    if (!in || !out || in == out) return FFT_ERR_INVALID_ARG;
    if (parts < 1 || batch < 1 || rows < 1 || w < 1) return FFT_ERR_INVALID_SIZE;
    if ((long long)parts * batch * rows * w > (1LL << 31)) return FFT_ERR_INVALID_SIZE;
    if ((reinterpret_cast<uintptr_t>(in) & 15) || (reinterpret_cast<uintptr_t>(out) & 15)) return FFT_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (w % 2 == 0) {
        const long long total = (long long)parts * batch * rows * (w / 2);
        k_slab_unpack<float4><<<slab_grid(total), 256, 0, s>>>(static_cast<const float4 *>(in),
                                                               static_cast<float4 *>(out), parts, batch, rows, w / 2);
    } else {
        const long long total = (long long)parts * batch * rows * w;
        k_slab_unpack<float2><<<slab_grid(total), 256, 0, s>>>(static_cast<const float2 *>(in),
                                                               static_cast<float2 *>(out), parts, batch, rows, w);
    }
    return cudaGetLastError() == cudaSuccess ? FFT_OK : FFT_ERR_CUDA;
}

}  // extern "C"
