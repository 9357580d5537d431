// Host-side declarations shared by the gb300fft translation units.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace gb300fft {

constexpr int kMaxLog2 = 13;  // n <= 8192 per axis

// Launch shape of one compiled row-pass variant (length n = 2^log2n).
struct RowVariant {
    const void *fn = nullptr;  // __global__ function
    int n = 0, e = 0;          // transform length, elements per thread
    int threads = 0;           // threads per CTA
    int rows_per_cta = 0;
    size_t smem = 0;           // dynamic shared memory bytes
    int tw_size = 0;           // twiddle table entries for (n, e)
};

// Launch shape of one compiled column-pass variant.
struct ColVariant {
    const void *fn = nullptr;
    int n = 0, e = 0, w = 0;   // column length, elements per thread, columns per tile
    int threads = 0;
    size_t smem = 0;
    int box_rows = 0;          // rows per TMA box
    int tw_size = 0;
};

// Variant tables (defined in fft_rows.cu / fft_cols.cu).
const RowVariant *row_variant(int log2n, int e);           // nullptr if not compiled
const ColVariant *col_variant(int log2n, int e, int w);    // nullptr if not compiled
int default_row_e(int n);
int default_col_e(int n);
int default_col_w(int n, int nx);

// Stage radices of the (n, e) schedule, first stage first; returns count.
int schedule_radices(int n, int e, int *radices);

// Twiddle tables (fft_twiddle.cu): fills `tw` (tw_size entries) for (n, e).
cudaError_t build_twiddles(float2 *tw, int n, int e, cudaStream_t s);

// Kernel launchers.
// Row pass over `nrows` rows of length v.n.  split = P in {1, 2}: with P = 2
// the rows form [.][ny][n] slices and the pass also applies the column
// pre-split (2-point DFT across rows y and y + ny/2, twiddle twp[q*kp]).
cudaError_t launch_rows(const RowVariant &v, const float2 *in, float2 *out, const float2 *tw,
                        const float2 *twp, long long nrows, int ny, int split, int conj_in,
                        int conj_out, const float *weight, float wscale, int grid, int pf_dist,
                        cudaStream_t s);
int row_grid(const RowVariant &v, long long nrows, int num_sms, bool weighted, int split, bool persistent);
// Long-row pass with a TMA landing ring (fft_rows_ring.cu), n in 2048..8192.
bool ring_rows_available(int n);
int ring_rows_grid(int n, long long nrows, int split, int num_sms, bool weighted);
cudaError_t launch_rows_ring(int n, const float2 *in, float2 *out, const float2 *tw, const float2 *twp,
                             long long nrows, int ny, int split, int conj_in, int conj_out, const float *weight,
                             float wscale, int *status, int grid, cudaStream_t s);
// Column pass of column length v.n over `batch` slices of P*v.n rows each.
cudaError_t launch_cols(const ColVariant &v, const CUtensorMap &map, float2 *out,
                        const float2 *tw, int nx, int batch, int split, int conj_out, int *status,
                        int grid, int pf_dist, cudaStream_t s);
// Table of exp(-2*pi*i*k/n) for k < n (FP64-generated, rounded once).
cudaError_t build_roots(float2 *t, int n, cudaStream_t s);
int col_ctas_per_sm(const ColVariant &v);

// Reorder-map debug launchers: write map[i] = output position of input i.
cudaError_t launch_rows_movemap(int log2n, int *map, cudaStream_t s);
cudaError_t launch_cols_movemap(int log2n, int *map, cudaStream_t s);

// Sets the calling thread's fft_last_error() value.
void set_last_error(int code);

// 3D tensor map over a complex64 buffer of `rows` rows of nx elements, seen
// as (float within row, kp < split, i) with row = kp + split * i; boxes of
// 2w floats x 1 x box_rows.
int encode_col_map(CUtensorMap *map, const void *base, int nx, long long rows, int split, int w,
                   int box_rows);

}  // namespace gb300fft
