// Host-side declarations shared by the gb300fft translation units.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <vector>

#include "../../include/gb300fft.h"

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
bool row_split_available(int n, int e);  // a column pre-split (P = 2) row kernel exists
// Launch shape of the compiled row kernel (n, e, split): threads per CTA,
// rows per CTA and shared-memory float2 elements per row; false if none.
bool row_variant_info(int n, int e, int split, int *threads, int *rows_per_cta, int *smem_elems);
int default_col_e(int n);
int preferred_col_e(int n, int w);
int default_col_w(int n, int nx);

// Stage radices of the (n, e) schedule, first stage first; returns count.
int schedule_radices(int n, int e, int *radices);

// Twiddle tables (fft_twiddle.cu): fills `tw` (tw_size entries) for (n, e).
cudaError_t build_twiddles(float2 *tw, int n, int e, cudaStream_t s);

// Kernel launchers.
// Row pass over `nrows` rows of length v.n.  split = P in {1, 2}: with P = 2
// the rows form [.][ny][n] slices and the pass also applies the column
// pre-split (2-point DFT across rows y and y + ny/2, twiddle twp[q*kp]).
// A weighted pass multiplies each input by wscale * weight[i], and by
// *wscale_dev too when that device pointer is not null.
cudaError_t launch_rows(const RowVariant &v, const float2 *in, float2 *out, const float2 *tw,
                        const float2 *twp, long long nrows, int ny, int split, int conj_in,
                        int conj_out, const float *weight, float wscale, const float *wscale_dev, int grid,
                        int pf_dist, int perm_t, int perm_g, int planar, cudaStream_t s);
int row_grid(const RowVariant &v, long long nrows, int num_sms, bool weighted, int split, bool persistent);
// Long-row pass with a TMA landing ring (fft_rows_ring.cu), n in 2048..8192.
bool ring_rows_available(int n);
int ring_rows_grid(int n, long long nrows, int split, int num_sms, bool weighted);
cudaError_t launch_rows_ring(int n, const float2 *in, float2 *out, const float2 *tw, const float2 *twp,
                             long long nrows, int ny, int split, int conj_in, int conj_out, const float *weight,
                             float wscale, const float *wscale_dev, int *status, int grid, cudaStream_t s);
// Split-FP16 tensor-core variants (fft_tc.cu), E = 16.
cudaError_t build_w16_table(void *t, cudaStream_t s);
bool tc_rows_available(int n);
int tc_col_width(int n, int nx);
int tc_col_box_rows(int n);
// tcg: 1 = tcgen05/TMEM butterfly, 0 = mma.sync butterfly
bool tcg_available(int rown, int coln, int colw);
int tc_cols_grid(int n, int w, int tcg, long long ntiles, int num_sms);
cudaError_t launch_rows_tc(int n, int tcg, const float2 *in, float2 *out, const float2 *tw, const float2 *twp,
                           const void *w16, long long nrows, int ny, int split, int conj_in, int conj_out, int *status,
                           cudaStream_t s);
cudaError_t launch_cols_tc(int n, int w, int tcg, const CUtensorMap &map, float2 *out, const float2 *tw,
                           const void *w16, int nx, int batch, int split, int conj_out, int *status, int grid,
                           cudaStream_t s);
// Split-FP16 tensor-core variants with radix-32 tcgen05 stages (fft_tc32.cu):
// rows and columns of 1024..8192 points; the plan owns the FP64-built B table.
cudaError_t build_w32_table(void *t, cudaStream_t s);
constexpr size_t kW32TableBytes = 4 * 64 * 64 * 2;  // two tables of B_hi, B_lo
bool tc32_rows_available(int n);
int tc32_col_width(int n, int nx);
int tc32_cols_grid(int n, int w, long long ntiles, int num_sms);
// tmem_a: the A operand in tensor memory (else staged in shared memory)
cudaError_t launch_rows_tc32(int n, int tmem_a, const float2 *in, float2 *out, const float2 *tw, const float2 *twp,
                             const void *w32, long long nrows, int ny, int split, int conj_in, int conj_out,
                             int *status, cudaStream_t s);
// Small square 2D transforms in one cooperative launch (fft_small2d.cu):
// n x n, n = 256..1024, at most 2^20 points, rows with E = 16 (the plan's row
// twiddle table).
bool small2d_available(int nx, int ny, int batch, int row_e);
int small2d_grid(int n, int batch, int num_sms);  // 0 if it cannot launch
cudaError_t launch_small2d(int n, const float2 *in, float2 *out, const float2 *tw, int batch, int conj,
                           unsigned *bar, int *status, int grid, cudaStream_t s);
// Streaming split-FP16 tensor-core column pass (fft_tc_stream.cu): 4096-point
// column blocks, tiles of tc_stream_width() columns, E = 64 twiddles; the
// row pass stores the permutation tc_stream_perm() gives.
bool tc_stream_available(int n, int nx);
int tc_stream_layout(long long *v);  // compile-time layout (host only)
void tc_stream_perm(int *perm_t, int *perm_g);
int tc_stream_width();
int tc_stream_twiddle_e();
cudaError_t launch_cols_tc_stream(const CUtensorMap &map, float2 *out, const float2 *tw, const void *w32, int nx,
                                  int batch, int split, int conj_out, int *status, int num_sms, cudaStream_t s);
// Landed-row form (persistent, 512 threads, all TMEM columns of the SM):
// rows per unit (0: not compiled), and whether a call is covered.
int tc32_land_rows(int n);
int tc32_land_layout(int n, int kind, long long *v);  // compile-time layout (host only)
bool tc32_land_available(int n, long long nrows, int ny, int split);
cudaError_t launch_rows_tc32_land(int n, const float2 *in, float2 *out, const float2 *tw, const float2 *twp,
                                  const void *w32, long long nrows, int ny, int split, int conj_in, int conj_out,
                                  int perm_t, int perm_g, int *status, int num_sms, cudaStream_t s);
cudaError_t launch_cols_tc32(int n, int w, int tmem_a, const CUtensorMap &map, float2 *out, const float2 *tw,
                             const void *w32, int nx, int batch, int split, int conj_out, int *status, int grid,
                             cudaStream_t s);
// Entries of the stage twiddle table of the (n, e) schedule (build_twiddles).
int twiddle_table_size(int n, int e);
// Column pass by 2-CTA clusters (fft_cols_pair.cu): block length n = 2 * N2.
int pair_cols_width(int n, int e, int nx);
int pair_cols_tw_size(int n, int e);
cudaError_t launch_cols_pair(int n, int e, float2 *data, const float2 *tw, const float2 *roots, int nx, int batch,
                             int split, int conj_out, cudaStream_t s);
// Column pass by C-CTA clusters sharing a block through DSMEM
// (fft_cols_cluster.cu): block length n = C * NQ, NQ in {1024, 2048}.
int cluster_cols_width(int n, int e, int C, int nx);
int cluster_cols_tw_size(int n, int e, int C);
int cluster_cols_box_rows(int n, int e, int C);
cudaError_t launch_cols_cluster(int n, int e, int C, const CUtensorMap &map, float2 *out, const float2 *tw,
                                const float2 *roots, int nx, int batch, int split, int conj_out, int *status,
                                cudaStream_t s);
// Column pass of column length v.n over `batch` slices of P*v.n rows each.
cudaError_t launch_cols(const ColVariant &v, const CUtensorMap &map, float2 *out,
                        const float2 *tw, int nx, int batch, int split, int conj_out, int *status,
                        int grid, int pf_dist, cudaStream_t s);
// Table of exp(-2*pi*i*k/n) for k < n (FP64-generated, rounded once).
cudaError_t build_roots(float2 *t, int n, cudaStream_t s);
int col_ctas_per_sm(const ColVariant &v);

// Four-step large 1D FFT.  Pass A is the plain column pass (launch_cols, out
// of place into the workspace); pass B (fft_fourstep.cu) is below: the
// variant for row length n2 = 2^log2n (128..8192), e elements per thread and
// w rows per CTA, or nullptr; fourstep_row_e / _w(n2) are the preferred ones.
const ColVariant *fourstep_row_variant(int log2n, int e, int w);
int fourstep_row_e(int n);
int fourstep_row_w(int n);
// Pass B: element i2 of row k1 of work [batch][n1][v.n] times w_n^{i2*k1}
// (from lohi = [w_n^k, k < 8192 | w_n^{8192 k}, k < n/8192]), length-v.n FFTs
// of the rows, element k2 of row k1 stored at out[b][k] with k = k1 + n1*k2,
// or at out[b][(n - k) mod n] if reverse (which turns the forward transform
// into the inverse).
cudaError_t launch_rows_fourstep(const ColVariant &v, const float2 *work, float2 *out, const float2 *tw,
                                 const float2 *lohi, int n1, int batch, int reverse, int *status, cudaStream_t s,
                                 int m = 1);  // m > 1: the three-pass form's last pass (no twiddle)
// middle pass of the three-pass form (m = 2 or 4), in place on the workspace
cudaError_t launch_fs_mid(float2 *work, const float2 *lohi, int n1, int m, int n3, int batch, cudaStream_t s);
// t[k] = exp(-2*pi*i*(k*stride mod n)/n), k < count, built in FP64.
cudaError_t build_roots_strided(float2 *t, int count, long long n, long long stride, cudaStream_t s);

// Pre-split row pass from a landed pair of rows (fft_rows_land.cu): one CTA
// per pair q, both output rows kp = 0, 1, stored like launch_rows stores them.
bool land_rows_available(int n, int e);
cudaError_t launch_rows_land(int e, const float2 *in, float2 *out, const float2 *tw, const float2 *twp, int ny,
                             int batch, int conj_in, int perm_t, int perm_g, int planar, int *status, int num_sms,
                             int pf, cudaStream_t s);

// Streaming column pass (fft_cols_stream.cu) over a row-permuted
// intermediate: the variant for column length n and row length nx, or
// nullptr; *perm_t / *perm_g receive the row permutation launch_rows must
// apply (perm_t = stage-0 butterflies T, perm_g = butterflies per warp G).
// tstore: the variant whose outputs leave through TMA stores (4D map from
// encode_stream_store_map); else plain global stores.
const ColVariant *stream_col_variant(int n, int nx, int *perm_t, int *perm_g, int tstore = 1);
bool stream_tstore(const ColVariant &v);
int encode_stream_store_map(CUtensorMap *map, const ColVariant &v, const void *base, int nx, long long rows,
                            int split);
cudaError_t launch_cols_stream(const ColVariant &v, const CUtensorMap &map, const CUtensorMap *omap, float2 *out,
                               const float2 *tw, int nx, int batch, int split, int conj_out, int *status, int grid,
                               int planar, cudaStream_t s);

// Reorder-map debug launchers: write map[i] = output position of input i.
cudaError_t launch_rows_movemap(int log2n, int *map, cudaStream_t s);
cudaError_t launch_cols_movemap(int log2n, int *map, cudaStream_t s);
// Differentiation form, fused column half (fft_cols.cu, P = 1, n <= 2048):
// forward column transform, per-tile partials of w |X|^2, and F_cols^H (w (.) X)
// stored in place; one partial per tile of v.w columns.
bool cols_wadj_available(const ColVariant &v);
int cols_wadj_ctas_per_sm(const ColVariant &v);
cudaError_t launch_cols_wadj(const ColVariant &v, const CUtensorMap &map, float2 *out, const float2 *tw,
                             const float *w, float *partials, int nx, int batch, int *status, int grid, int pf_dist,
                             cudaStream_t s);

// Sets the calling thread's fft_last_error() value.
void set_last_error(int code);

// 3D tensor map over a complex64 buffer of `rows` rows of nx elements, seen
// as (float within row, kp < split, i) with row = kp + split * i; boxes of
// 2w floats x 1 x box_rows.
int encode_col_map(CUtensorMap *map, const void *base, int nx, long long rows, int split, int w,
                   int box_rows);
// 4D tensor map over the same buffer seen as (float within row, kp < split,
// r mod t, r / t) with row = kp + split * r; boxes of 2w floats x 1 x
// box_rows x box_k.
int encode_map4(CUtensorMap *map, const void *base, int nx, long long rows, int split, int t, int w, int box_rows,
                int box_k);

// Tunable schedule of a dense plan (every field has a default).
enum { kColTile = 0, kColPair = 1, kColCluster = 2 };
struct Schedule {
    int row_e = 0;         // elements per thread of the row pass (0: default)
    int row_persist = -1;  // 1 persistent row grid, 0 one CTA per group, -1 persistent iff pre-split
    int row_pf = 1;        // persistent row pass: L2 prefetch distance (groups)
    int ring = 0;          // long rows through the TMA landing-ring kernel
    int split = 0;         // column pre-split P (0: default, 2 when ny >= 8192)
    int col_kind = kColTile;
    int col_e = 0;         // elements per thread of the column pass (0: default)
    int col_w = 0;         // TMA tile width (0: default)
    int col_c = 2;         // cluster size of the DSMEM column kernel
    int col_pf = 0;        // TMA column pass: L2 prefetch distance (tiles)
    int col_stream = 1;    // out-of-place calls: streaming column pass over row-permuted rows, where compiled
    int col_tstore = 1;    // streaming column pass through TMA stores: 1 unsplit blocks, 2 always, 0 never
    int planar = 1;        // pre-split plans with the streaming pass: blocks as planes of a workspace
    int row_land = 1;      // pre-split 8192-point rows: one CTA per landed pair of input rows
    int land_pf = 1;       // landed-pair rows: L2 prefetch distance in pairs
};

// One axis of a dense plan: a row-pass length (contiguous) or a column-pass
// length (strided), its kernel variant and its twiddle table.
struct AxisPlan {
    const RowVariant *row = nullptr;
    const ColVariant *col = nullptr;
    float2 *tw = nullptr;
    int n = 1;
    int grid = 0;  // column pass: persistent grid size
    int tc_w = 0;  // tensor-core column pass: tile width
    int tcg = 0;   // tensor-core column pass: 1 tcgen05 butterflies, 0 mma.sync
    int tc32 = 0;  // tensor-core pass with radix-32 tcgen05 stages (rows: the plan's rows axis)
    int tcs = 0;   // tensor-core column pass also available streaming (out-of-place calls; E = 64 twiddles)
    int pair_e = 0;  // >0: column pass by 2-CTA clusters with this E (length n/2 sub-FFTs)
    int cl_c = 0, cl_e = 0;  // >0: column pass by cl_c-CTA DSMEM clusters with E = cl_e
    float2 *roots = nullptr;  // pair column pass: exp(-2*pi*i*k/n), k < n
    // streaming column pass (out-of-place calls): kernel, the row permutation
    // the row pass applies for it, its grid and twiddle table
    const ColVariant *stream = nullptr;
    int perm_t = 0, perm_g = 0, stream_grid = 0;
    float2 *stream_tw = nullptr;
    // column pass: cached tensor map of the last output pointer
    CUtensorMap map;
    const void *map_base = nullptr;
    // streaming column pass with TMA stores: cached output map
    CUtensorMap omap;
    const void *omap_base = nullptr;
};


// A large 1D transform of length n = n1 * n2 > 8192 by the four-step
// decomposition: pass A (columns of [n1][n2], twiddled) into `work`, pass B
// (rows of work, stored transposed) into the output.
struct FourStepPlan {
    int n = 0, n1 = 0, n2 = 0;  // n1 == 0: not a four-step plan
    int m = 1;                  // > 1: three passes, rows of n2 / m after an m-point middle pass
    const ColVariant *a = nullptr;
    const ColVariant *b = nullptr;
    float2 *tw_a = nullptr, *tw_b = nullptr;  // stage twiddles of the two passes
    float2 *lohi = nullptr;                   // w_n^k (k < 8192), then w_n^{8192 k} (k < n / 8192)
    float2 *work = nullptr;                   // [batch][n1][n2] workspace
    int grid_a = 0;
    CUtensorMap map;  // pass A's view of the last input pointer
    const void *map_base = nullptr;
};

// Any-size transforms (fft_bluestein.cu kernels, fft_plan.cu logic).  One
// axis: `rows` transforms of length n along contiguous rows, by a
// power-of-two sub-plan (M == 0) or by Bluestein over a length-M sub-plan.
// Fused Bluestein kernels for one padded length M (fft_bluestein.cu).
struct BluVariant {
    // phase 0 (forward, chirp in, filter out), 1 (inverse, chirp out), 2 (both in one pass)
    const void *fn[3] = {nullptr, nullptr, nullptr};
    int n = 0, e = 0, threads = 0, rows_per_cta = 0;
    size_t smem = 0;
};
const BluVariant *blu_variant(int M);
cudaError_t launch_blu(const BluVariant &v, int phase, const float2 *src, float2 *dst, const float2 *tw,
                       const float2 *chirp, const float2 *H, int n, long long rows, cudaStream_t s);

// Mixed-radix stages of a 13-smooth length n <= kMixedMaxN (fft_mixed.cu).
constexpr int kMixedMaxN = 14336;           // two float2 buffers of n in one CTA's shared memory
constexpr size_t kMixedMaxSmem = 227 * 1024;
constexpr int kMixedMaxStages = 16;
struct MixedStages {
    int n = 0, S = 0, tw_size = 0;
    int wlog = 0;                      // log2 of the columns per CTA (column kernel)
    int buf_elems = 0;                 // elements of one padded shared-memory buffer
    int pad[kMixedMaxStages] = {};     // padding shift of the buffer stage s writes (0: none)
    int radix[kMixedMaxStages] = {};
    int ns[kMixedMaxStages] = {};      // product of the radices before stage s
    int nb[kMixedMaxStages] = {};      // butterflies per transform, n / radix
    uint32_t mag_nb[kMixedMaxStages] = {}, mag_ns[kMixedMaxStages] = {};  // ceil(2^32 / d) divisors
    int tw_off[kMixedMaxStages] = {};  // stage s's twiddles w_{Ns R}^{k r}, 16-byte pairs (r odd, r + 1) at pair (r - 1) / 2 * Ns + k
};
// Second pass of a mixed-radix four-step transform (n = n1 n2): row k1 of
// the first pass's output is multiplied by w_n^{i2 k1} as it is loaded and
// its outputs k2 are stored at k1 + n1 k2.
struct FourStepB {
    const float2 *hi = nullptr, *lo = nullptr;  // w_n^{t 2^lshift}, w_n^u (u < 2^lshift)
    int n1 = 0;      // rows per transform (0: not a four-step pass)
    int k1 = 0;      // set per CTA in the kernel
    int lshift = 0, lmask = 0;
};

// Launch configuration of the mixed-radix kernel for one axis, fixed at
// plan creation: transforms per CTA, threads, padded buffers.
struct MixedLaunch {
    MixedStages m;
    bool cols = false;
    int nx = 0;  // columns: row length of the [ny][nx] slices
    int W = 1, T = 0;
    size_t smem = 0;
    FourStepB fs;
};
bool mixed_factor(int n, MixedStages *st);  // false unless n = 2^a 3^b 5^c 7^d 11^e 13^f <= kMixedMaxN
cudaError_t build_mixed_twiddles(float2 *tw, const MixedStages &st, cudaStream_t s);
int mixed_rows_per_cta(int n);
int mixed_cols_width(int n, int nx);
// 0 on success; fs_n1 > 0: the second pass of a four-step transform with
// n1 rows per transform (rows layout)
int mixed_prepare(const MixedStages &st, bool cols, int nx, MixedLaunch *out, int fs_n1 = 0);
// n = n1 n2 with both factors mixed-radix lengths (<= kMixedMaxN), n1 and
// n2 as close as possible; false if none
bool mixed_split(int n, int *n1, int *n2);
// rows: `count` transforms along contiguous rows; columns: `count` [n][nx] slices
cudaError_t launch_mixed(const MixedLaunch &L, const float2 *tw, const float2 *in, float2 *out, long long count,
                         int conj, cudaStream_t s);

struct AnyAxis {
    bool mixed = false;                 // 13-smooth n: the mixed-radix kernel, no padding
    MixedStages mst;
    MixedLaunch ml;                     // rows, or (the y axis of a 2D plan) columns
    bool mfs = false;                   // 13-smooth n > kMixedMaxN: mixed-radix four-step
    int n1 = 0, n2 = 0;                 // n = n1 n2: columns of length n1, then rows of n2
    MixedLaunch mla, mlb;               // the two passes
    float2 *mtwa = nullptr, *mtwb = nullptr, *fs_hi = nullptr, *fs_lo = nullptr, *fs_work = nullptr;
    float2 *mtw = nullptr;              // mixed-radix twiddles (forward)
    const BluVariant *fused = nullptr;  // M <= 8192: fused kernels (same E as the sub-plan's row pass)
    bool fused_one = false;             // the fused transform in one pass (no padded workspace)
    int n = 1, M = 0;
    long long rows = 0;
    fft_plan_s *sub = nullptr;           // (n or M, 1, rows), run forward and inverse
    float2 *chirp[2] = {nullptr, nullptr};  // [0] forward exp(-pi i j^2/n), [1] its conjugate
    float2 *H[2] = {nullptr, nullptr};      // F(filter)/M for each direction
    float2 *A = nullptr;                    // rows * M workspace (not with the one-pass form)
};
// A plan whose sizes are not all powers of two: x axis over the rows, then
// (2D) transpose, y axis over the rows of the transposed array, transpose back.
struct AnyPlan {
    AnyAxis x, y;                // y.n == 1: a 1D batch
    bool y_cols = false;         // y axis by the mixed-radix column kernel, in place, no transposes
    float2 *t = nullptr;         // [batch][nx][ny] transposed workspace
};
cudaError_t build_chirp(float2 *c, int n, int sgn, cudaStream_t s);
cudaError_t build_chirp_filter(float2 *h, const float2 *c, int n, int M, cudaStream_t s);
cudaError_t launch_scale(float2 *a, long long count, float sc, cudaStream_t s);
cudaError_t launch_blu_pre(const float2 *x, float2 *A, const float2 *c, int n, int M, long long rows, cudaStream_t s);
cudaError_t launch_blu_mul(float2 *A, const float2 *H, int M, long long rows, cudaStream_t s);
cudaError_t launch_blu_post(const float2 *A, float2 *out, const float2 *c, int n, int M, long long rows,
                            cudaStream_t s);
cudaError_t launch_transpose(const float2 *in, float2 *out, int rows, int cols, long long batch, cudaStream_t s);

// Host-buffer execution (fft_execute_host): two staging buffers per
// direction, one copy stream per direction, events linking them to the
// caller's stream.
struct HostStage {
    float2 *din[2] = {nullptr, nullptr}, *dout[2] = {nullptr, nullptr};
    cudaStream_t cin = nullptr, cout = nullptr, comp = nullptr;
    cudaEvent_t in_ready[2] = {nullptr, nullptr}, computed[2] = {nullptr, nullptr},
                out_done[2] = {nullptr, nullptr}, entry = nullptr;
    unsigned long long calls = 0;
};

struct RaggedState;
void ragged_destroy(RaggedState *r);

}  // namespace gb300fft

// A plan (opaque to the C ABI): dense or ragged.
struct fft_plan_s {
    int kind = 0;  // 0 dense, 1 ragged
    int axes = 3;  // dense plans: transformed axes, bit 0 x (rows), bit 1 y (columns)
    gb300fft::RaggedState *ragged = nullptr;
    int nx = 1, ny = 1, batch = 1, dir = FFT_FORWARD, prec = FFT_PREC_FP32;
    int device = 0;
    int num_sms = 0;
    gb300fft::AxisPlan rows;        // length nx (or ny when nx == 1)
    gb300fft::AxisPlan cols;        // length ny, used when nx > 1 and ny > 1
    gb300fft::AxisPlan cols_split;  // length ny / split, for out-of-place calls when split > 1
    gb300fft::FourStepPlan fs;      // large 1D plans (n > 8192)
    gb300fft::AnyPlan *any = nullptr;  // sizes that are not all powers of two
    // pre-split plans: the row pass writes each column block as a plane of
    // this workspace (batch*ny*nx), read by the streaming column pass through
    // planar_map; any call, in place or not, then runs the split path
    float2 *planar_work = nullptr;
    CUtensorMap planar_map;
    gb300fft::HostStage *host = nullptr;  // fft_execute_host staging (first use)
    bool last_use_host = false;           // the plan's latest work was an fft_execute_host call
    int split = 1;        // column pre-split P done by the row pass (out of place only)
    float2 *twp = nullptr;  // exp(-2*pi*i*k/ny), k < ny: the pre-split twiddles
    int row_grid[2][2] = {{0, 0}, {0, 0}};  // persistent row grid [weighted][split > 1]
    bool ring = false;    // long rows: TMA landing-ring row kernel
    int row_persist = -1;  // row pass grid: 1 persistent, 0 one CTA per group, -1 persistent iff split
    int row_pf = 1;        // persistent row pass: L2 prefetch distance in groups
    int col_pf = 0;        // column pass: L2 prefetch distance in tiles (0: measured best)
    int *status = nullptr;  // device status word
    void *w16 = nullptr;    // split-FP16 plans: hi/lo W16 table (FP64-built)
    void *w32 = nullptr;    // split-FP16 plans with radix-32 stages: hi/lo B table (FP64-built)
    int tc_radix = 32;      // split-FP16 plans: largest tensor-core radix allowed (32, or 16)
    int tc_tmem_a = 1;      // radix-32 tensor-core stages: A operand in tensor memory (0: shared memory)
    int tc_land = 1;        // radix-32 tensor-core rows from landed rows where the shape allows (A in TMEM)
    int small_grid = 0;     // > 0: n x n FP32 plans of n <= 2048 run both passes in one cooperative launch
    unsigned *small_bar = nullptr;  // its grid barrier (arrivals, generation)
    int tc_stream = 1;      // tensor-core columns of 4096 points: streaming radix-64 pass where allowed
    int tcg = 1;            // split-FP16 plans: 1 tcgen05/TMEM butterflies, 0 mma.sync
    int wp_parts = 0;
    // the fused differentiation form's column map (over the caller's y)
    CUtensorMap wadj_map;
    const void *wadj_base = nullptr;
    float2 *wadj_tw = nullptr;  // its column twiddles (plan creation)
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};  // optional per-pass timing events
    gb300fft::Schedule sched;  // the schedule this plan was built with
    std::vector<void *> allocations;
};

namespace gb300fft {
// out = DFT_sign(in) of a dense plan (optionally weighted by wscale * w on
// load); returns an FFT_* code.  Defined in fft_plan.cu.
int run_dense(fft_plan_s *p, const void *in, void *out, int sign, const float *weight, float wscale,
              cudaStream_t s, const float *wscale_dev = nullptr);
// Frees a plan and everything it owns.
void free_plan(fft_plan_s *p);
}  // namespace gb300fft
