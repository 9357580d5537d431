/*
 * gb300fft -- 2D complex-to-complex Cooley-Tukey FFT for the NVIDIA GB300
 * (sm_103a).  C ABI of libgb300fft.so.
 *
 * What is computed.  For each [ny][nx] slice of a row-major complex64 array
 * (interleaved re, im float32; nx is the contiguous row length), the
 * unnormalised 2D DFT
 *
 *     X[ky][kx] = sum_{y<ny} sum_{x<nx} x[y][x] * exp(dir*2*pi*i*(ky*y/ny + kx*x/nx)),
 *
 * evaluated as the paper's Section 5 decomposition (Fig. 6): radix-2^k
 * Cooley-Tukey FFTs (Section 2.2, Fig. 2, Listing 1) along every row, then
 * along every column.  The twiddle multiply (Section 2.2) and the data
 * reordering between butterfly steps (Section 4, Figs. 4 and 5) are fused
 * into the kernels; the output is always in natural [ky][kx] order.  The
 * paper states neither a sign convention nor a normalisation: here
 * dir = -1 (FFT_FORWARD) is exp(-...), dir = +1 (FFT_INVERSE) is exp(+...),
 * and neither direction scales, so inverse(forward(x)) = nx*ny*x.
 *
 * Memory.  Every data pointer passed to an execute call is a caller-owned
 * DEVICE pointer to contiguous complex64 data, 16-byte aligned.  in == out
 * (in place) is allowed; partially overlapping buffers are not.  A plan owns
 * its device workspace (twiddle tables, status word, ragged work queue) and
 * allocates all of it at creation; execute calls allocate nothing and do
 * not synchronise, so they are stream-ordered and may be captured in a CUDA
 * graph.  A plan must not be used on two streams at the same time.
 * Different plans may be created, used and destroyed from several host
 * threads at once (the library's kernel tables are filled once, under
 * std::call_once, and each kernel's dynamic shared-memory limit is one fixed
 * value whichever plan sets it).
 *
 * Streams.  `stream` is a cudaStream_t passed as void* (NULL = the legacy
 * default stream).
 *
 * Errors.  Calls return FFT_OK (0) or a negative FFT_ERR_* code; plan
 * constructors return NULL and leave the reason in fft_last_error()
 * (per calling thread).  Launch failures map to FFT_ERR_CUDA.  Device-side
 * failures (a bounded wait that ran out) are recorded in the plan's device
 * status word, read back by fft_plan_status().  No kernel traps.
 */
#ifndef GB300FFT_H
#define GB300FFT_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fft_plan_s *fft_plan_t;

enum { FFT_FORWARD = -1, FFT_INVERSE = 1 };

/* Arithmetic of the butterflies.  FFT_PREC_FP32: every stage in float32 on
 * the CUDA cores.  FFT_PREC_SPLIT_FP16_TC: the radix-16 stages run as
 * 16x16 complex DFT-matrix products on the tensor cores with operands split
 * into a high and a low float16 part (3 products, float32 accumulation);
 * twiddles between stages stay float32. */
enum { FFT_PREC_FP32 = 0, FFT_PREC_SPLIT_FP16_TC = 1 };

enum {
    FFT_OK = 0,
    FFT_ERR_INVALID_SIZE = -1, /* a length out of range, batch < 1, count < 1 */
    FFT_ERR_INVALID_ARG = -2,  /* NULL / misaligned pointer, bad dir or precision, bad index */
    FFT_ERR_ALLOC = -3,        /* device or host allocation failed at plan creation */
    FFT_ERR_CUDA = -4,         /* a CUDA runtime call or kernel launch failed */
    FFT_ERR_UNSUPPORTED = -5,  /* valid request this build does not implement */
    FFT_ERR_TIMEOUT = -6       /* a device-side bounded wait ran out (status word) */
};

/*
 * fft_plan_create -- plan `batch` 2D transforms of size [ny][nx].
 *   nx, ny     >= 1 (nx = 1 or ny = 1 gives a batch of 1D transforms along
 *              the other axis).  Powers of two up to 8192 per axis run the
 *              dense two-pass path (Section 5).  A 1D length may go up to
 *              2^26 for a power of two and 2^24 otherwise; 2D axes up to
 *              65536.  Power-of-two 1D lengths above 8192 run as the
 *              four-step decomposition the paper leaves as its next step
 *              (Section 6) -- n = n1*n2, length-n1 FFTs down the columns of
 *              the [n1][n2] view, then the twiddle w_n^{i2*k1} applied as the
 *              rows are loaded and length-n2 FFTs along them, stored
 *              transposed -- two HBM passes through a plan-owned workspace
 *              of n*batch complex values (2^25 and 2^26: three passes,
 *              n = 4096*M*4096, with an M-point middle pass that applies the
 *              twiddles, so no pass works on a length-8192 axis).  Every
 *              other shape is planned axis
 *              by axis (the paper's uneven sizes, Sections 6 and 7):
 *              lengths 2^a 3^b 5^c 7^d 11^e 13^f up to 14336 by mixed-radix
 *              stages (every radix from 2 to 16, the fewest stages) in
 *              one pass, longer such
 *              lengths by a mixed-radix four-step, powers of two by the
 *              dense path, any other length by Bluestein's algorithm over a
 *              power-of-two length M >= 2n - 1; the y axis of a 2D plan runs
 *              down the columns in place when it is mixed-radix and between
 *              two transposes otherwise.  Plans other than the dense 2D
 *              ones are FFT_PREC_FP32 only (else FFT_ERR_UNSUPPORTED) and
 *              have no fft_backward_weighted.
 *   batch      >= 1; slices are stored back to back, nx*ny elements apart;
 *              nx*ny*batch <= 2^31.
 *   dir        FFT_FORWARD or FFT_INVERSE: the exponent sign of fft_execute.
 *   precision  FFT_PREC_FP32 or FFT_PREC_SPLIT_FP16_TC.  The split form needs
 *              every transformed length >= 16 (a radix-16 stage) and, for 2D,
 *              (ny / 16) * min(nx, 32) >= 32 (a column tile fills a warp);
 *              other sizes return NULL with FFT_ERR_UNSUPPORTED.
 * Returns NULL on failure (reason in fft_last_error()).  Must be called with
 * the device that will run the plan current; allocates device memory.
 */
fft_plan_t fft_plan_create(int nx, int ny, int batch, int dir, int precision);

/*
 * fft_plan_create_columns -- plan only the column half of Section 5's
 * decomposition: the length-ny transforms down every column of `batch`
 * [ny][nx] slices (no row FFTs).  This is the local step a rank runs after
 * the exchange of a slab-decomposed 2D transform (see fft_slab_pack).
 *   nx  power of two, 2..65536 (columns per slice); ny power of two, 2..8192.
 *   FFT_PREC_FP32 only (FFT_ERR_UNSUPPORTED otherwise).
 * fft_execute / fft_backward then take in and out of batch*ny*nx complex64
 * each; in == out is allowed (each column tile is read whole before it is
 * written).  Returns NULL on failure (reason in fft_last_error()).
 */
fft_plan_t fft_plan_create_columns(int nx, int ny, int batch, int dir, int precision);

/*
 * fft_slab_pack / fft_slab_unpack -- the data layout of the exchange step of
 * a slab-decomposed 2D transform over `parts` ranks (the multi-card form of
 * Section 5's global transpose, which the paper's Section 6 leaves as future
 * work).  Each rank holds `rows` = ny/parts consecutive rows of every slice.
 *   pack:   out[s][b][y][x'] = in[b][y][s*w + x'],  w = nx/parts: the block of
 *           rank s (its w columns of this rank's rows) made contiguous, so one
 *           all-to-all chunk goes to each rank.  in: batch*rows*nx elements,
 *           out: the same count; nx a multiple of parts.
 *   unpack: out[b][r*rows + y][x'] = in[r][b][y][x']: the chunks received from
 *           ranks r = 0..parts-1 assembled into this rank's column slab
 *           [batch][parts*rows][w].
 * Device pointers, complex64, 16-byte aligned, in != out; plain copies on
 * `stream`.  FFT_ERR_INVALID_SIZE for inconsistent sizes (or more than 2^31
 * elements), FFT_ERR_INVALID_ARG for NULL / misaligned / aliased pointers.
 */
int fft_slab_pack(const void *in, void *out, int parts, int batch, int rows, int nx, void *stream);
int fft_slab_unpack(const void *in, void *out, int parts, int batch, int rows, int w, void *stream);

/*
 * fft_execute -- out = DFT_dir(in) for the plan's batch (Section 5: row
 * FFTs, then column FFTs, natural-order output).  `in` and `out` are device
 * pointers to batch*ny*nx complex64 each, 16-byte aligned; in == out is
 * allowed.  Four-step plans read `in` whole before writing `out`.
 */
int fft_execute(fft_plan_t p, const void *in, void *out, void *stream);

/*
 * fft_execute_host -- fft_execute from and to host memory: host_in is copied
 * to a plan-owned device buffer, transformed, and the result copied back to
 * host_out.  Work issued on `stream` after this call sees host_out complete
 * (the stream waits for the device-to-host copy).  The copies run on the
 * plan's own copy streams through two staging buffers per direction and the
 * transform on the plan's own compute stream, so successive calls pipeline:
 * a call's host-to-device copy starts at once and overlaps the previous
 * call's device-to-host copy (the host link carries both directions at the
 * same time), and its transform overlaps that copy too.  Hence host_in is
 * read from the moment of the call on and must already hold the input then:
 * it may not be the output of earlier work on `stream`.  The plan's shared
 * workspaces stay ordered: after fft_execute / fft_backward on `stream` the
 * next host call's transform waits for that work.
 *   host_in, host_out  batch*ny*nx complex64 each; page-locked memory
 *                      (cudaHostAlloc, or torch's pin_memory) keeps the
 *                      copies asynchronous.  They may not overlap.
 * The first call allocates the staging buffers (four times the transform's
 * size) and the copy streams; later calls allocate nothing.  Not for ragged
 * plans (FFT_ERR_INVALID_ARG).
 */
int fft_execute_host(fft_plan_t p, const void *host_in, void *host_out, void *stream);

/*
 * fft_backward -- the adjoint (conjugate transpose) of the plan's transform:
 * grad_in = F^H grad_out, i.e. the unnormalised transform with the opposite
 * exponent sign.  This is the vector-Jacobian product of fft_execute for a
 * real loss under PyTorch's conjugate-Wirtinger convention.
 */
int fft_backward(fft_plan_t p, const void *grad_out, void *grad_in, void *stream);

/*
 * fft_backward_weighted -- grad_in = F^H (scale * w (.) X), with the
 * elementwise weighting fused into the first pass's load.  For the loss
 * L = sum w*|F x|^2, passing X = F x and scale = 2 gives dL/dx.
 *   X, grad_in  device complex64, batch*ny*nx elements (may alias).
 *   w           device float32, batch*ny*nx elements (must not alias X).
 * Returns FFT_ERR_UNSUPPORTED for split-FP16 plans and 1D plans longer than
 * 8192 (four-step).
 */
int fft_backward_weighted(fft_plan_t p, const void *X, const void *w, float scale,
                          void *grad_in, void *stream);

/*
 * fft_backward_weighted_dev -- fft_backward_weighted with the scale read on
 * the device: grad_in = F^H (scale * scale_dev[0] * w (.) X).  scale_dev is a
 * device pointer to one float32 (4-byte aligned), read by the adjoint's first
 * pass when it runs, so a scale produced by earlier work on `stream` (an
 * autograd output gradient, for instance) never has to be copied to the host.
 * For L = sum w*|F x|^2 with upstream gradient g = dOut/dL, passing X = F x,
 * scale = 2 and scale_dev = &g gives dOut/dx.  Same sizes, aliasing rules and
 * FFT_ERR_UNSUPPORTED cases as fft_backward_weighted; FFT_ERR_INVALID_ARG for
 * a NULL or misaligned scale_dev.
 */
int fft_backward_weighted_dev(fft_plan_t p, const void *X, const void *w, const void *scale_dev,
                              float scale, void *grad_in, void *stream);

/*
 * fft_weighted_power -- partial sums of L = sum w*|X|^2 over X, w of the
 * plan's full size: writes `nparts` float32 partial sums to the device array
 * `partials` (the caller adds them, preferably in double).  nparts is
 * fft_weighted_power_parts(p).  Each partial is a compensated float sum.
 */
int fft_weighted_power(fft_plan_t p, const void *X, const void *w, void *partials,
                       void *stream);
int fft_weighted_power_parts(fft_plan_t p);

/*
 * fft_weighted_power_adjoint -- the loss L = sum w*|X|^2 of X = F x and
 * the column half of its adjoint, y = F_cols^H (w (.) X), in two passes.
 * The gradient dL/dx = 2 F^H (w (.) X) = 2 F_rows^H y, since the 2D F^H is
 * F_rows^H F_cols^H; fft_backward_rows_scaled finishes it.  The row pass
 * writes F_rows x into y.  The column pass then runs, for each tile of
 * columns:
 *   - the forward column transform, giving X in registers;
 *   - the tile's partial sum of w*|X|^2 into `partials`;
 *   - F_cols^H of w (.) X, stored over the tile in y.
 * X itself is never stored.
 *   x, y       device complex64, batch*ny*nx elements (may alias).
 *   w          device float32, batch*ny*nx elements, the layout of X (must
 *              not alias x or y).
 *   partials   device float32, fft_weighted_power_adjoint_parts(p)
 *              entries: one float tree sum per tile, which the caller
 *              adds, preferably in double.
 * Covered: dense 2D FP32 forward plans whose column length is at most 2048.
 * Every other plan returns FFT_ERR_UNSUPPORTED, from both calls, and keeps
 * the unfused path: fft_execute, fft_weighted_power,
 * fft_backward_weighted_dev.  FFT_ERR_INVALID_ARG for NULL or misaligned
 * pointers (16 bytes for x, y, w; 4 for partials).
 */
int fft_weighted_power_adjoint(fft_plan_t p, const void *x, const void *w, void *partials, void *y,
                               void *stream);
int fft_weighted_power_adjoint_parts(fft_plan_t p);

/*
 * fft_backward_rows_scaled -- the row half of the adjoint, for the plans
 * fft_weighted_power_adjoint covers:
 *   grad_in = scale * scale_dev[0] * F_rows^H y,
 * the scale applied as the row pass loads.  scale_dev is a device float32
 * (4-byte aligned), read when the pass runs; NULL means 1.  With
 * y = fft_weighted_power_adjoint's output, scale = 2 and scale_dev =
 * &dOut/dL, this gives dOut/dx.  y and grad_in may alias.
 */
int fft_backward_rows_scaled(fft_plan_t p, const void *y, const void *scale_dev, float scale, void *grad_in,
                             void *stream);

/* Destroy a plan and free its device memory (synchronises the device).
 * NULL is a no-op returning FFT_OK. */
int fft_plan_destroy(fft_plan_t p);

/* Last error set on this thread by a plan constructor (FFT_OK if none). */
int fft_last_error(void);

/* Static description of an error code (never NULL). */
const char *fft_error_string(int code);

/*
 * Ragged batches (many independent 2D transforms of mixed sizes in one
 * persistent launch captured in a CUDA graph).
 *
 * fft_plan_create_ragged -- `count` instances, instance i of size
 * [ny[i]][nx[i]] with nx[i], ny[i] powers of two in 32..1024.  nx, ny are
 * host arrays read only during the call.  Instances are packed back to back
 * in the order given: instance i starts fft_ragged_offset(i) complex
 * elements into the buffer.
 */
fft_plan_t fft_plan_create_ragged(int count, const int *nx, const int *ny, int dir,
                                  int precision);

/* Element offset of instance i in the packed layout (i == count gives the
 * total number of elements). */
int fft_ragged_offset(fft_plan_t p, int i, long long *elem_offset);

/* Transform every instance of a ragged plan: one graph launch. */
int fft_execute_ragged(fft_plan_t p, const void *in, void *out, void *stream);

/* The same work as fft_execute_ragged, issued as one plain launch per
 * instance of the row/column kernels (the comparison baseline). */
int fft_execute_ragged_loop(fft_plan_t p, const void *in, void *out, void *stream);

/*
 * fft_execute_ragged_noalloc -- the ragged transform of fft_execute_ragged
 * (same persistent kernel, same packing: instance i starts at the sum of the
 * earlier nx*ny) for callers that cannot allocate device memory: a process
 * whose device memory belongs to a pool or framework allocator that it must
 * not go around (a cudaMalloc there would be memory the pool does not know
 * of), or a runtime that forbids device allocation once it has started (all
 * memory is reserved at start-up so that a long-running service cannot fail
 * later for lack of it).  The paper has no counterpart; it is an addition of
 * this library.
 *   count    1..1024 instances; nx[i], ny[i] powers of two in 32..1024 (host
 *            arrays, read during the call); at most 131072 work items (one
 *            item is 4096 elements of one pass; a 512 x 512 instance takes 128).
 *            Larger requests return FFT_ERR_INVALID_SIZE without launching.
 *   dir      FFT_FORWARD or FFT_INVERSE.
 *   in, out  caller-owned device buffers of the packed batch (may be equal).
 *   status   optional caller-owned device int: a kernel that times out on
 *            its bounded wait writes FFT_ERR_TIMEOUT there (NULL: not reported).
 * It allocates nothing.  Its scratch is one fixed array of about 2.1 MiB
 * inside the library, present on every GPU that loads the library until the
 * process exits.  The first call on each device looks up that array's address
 * and fills its twiddle tables (a short set-up, with the device current, that
 * synchronises `stream`), so that first call should come before any stream
 * capture.  Each call copies its small work list (about 16 bytes per work
 * item) from host memory into the array.  Every call reuses the same
 * array and it keeps the previous call's contents; the call clears what must
 * start at zero.  Calls that overlap on the GPU (different streams, or
 * concurrent host threads) race on the array: serialise them.
 */
int fft_execute_ragged_noalloc(int count, const int *nx, const int *ny, int dir, const void *in,
                               void *out, int *status, void *stream);

/*
 * fft_plan_status -- synchronise `stream`, return the plan's device status
 * word (FFT_OK, or the FFT_ERR_* a kernel recorded) and clear it.
 */
int fft_plan_status(fft_plan_t p, void *stream);

/*
 * fft_debug_reorder_map -- the index permutation realised by the kernels'
 * data movement alone.  Runs the row engine (axis 0) or the column engine
 * (axis 1) for length n with every butterfly replaced by the identity and an
 * integer payload, and writes map[i] = the output position of input i.
 * With the arithmetic removed, the fused Stockham movement of the kernels is
 * the mixed-radix digit reversal of the stage radices (Section 4's
 * reordering, here folded into the stage loads and stores).  `map` is a
 * device array of n int32.  Same n range as fft_plan_create.
 */
int fft_debug_reorder_map(int n, int axis, void *map, void *stream);

/*
 * fft_plan_set_pass_events -- profiling hook.  When set, every following
 * fft_execute / fft_backward on this dense plan records ev_start before the
 * row pass, ev_mid between the row and column passes and ev_end after the
 * column pass, on the call's stream (cudaEvent_t handles passed as void*,
 * created by the caller with timing enabled).  Passing three NULLs turns it
 * off.  The events' elapsed times are the per-pass kernel durations.
 */
int fft_plan_set_pass_events(fft_plan_t p, void *ev_start, void *ev_mid, void *ev_end);

/*
 * fft_plan_autotune -- time the plan's candidate schedules (row-pass elements
 * per thread and grid, column pre-split, column kernel: TMA tile or DSMEM
 * cluster) on scratch buffers of the plan's size and keep the fastest.  The
 * choice is appended to the tuning cache ($GB300FFT_TUNE_CACHE, default
 * ~/.cache/gb300fft/tune.jsonl), which later fft_plan_create calls for the
 * same shape and GPU read.  Allocates and frees two scratch buffers of the
 * plan's size; synchronises `stream`.  Creating a plan with the environment
 * variable GB300FFT_AUTOTUNE=1 runs it when the cache has no entry.  Split
 * tensor-core plans have a single schedule (no-op).
 */
int fft_plan_autotune(fft_plan_t p, void *stream);

/*
 * fft_plan_describe -- the schedule a plan runs, as a NUL-terminated JSON
 * object written to the host buffer `buf` of `len` bytes: kernel names,
 * elements per thread, tile widths, column pre-split, grids and stage radices
 * of each pass.  Returns the number of characters needed (excluding the NUL);
 * the output is truncated when that is >= len.
 */
int fft_plan_describe(fft_plan_t p, char *buf, int len);

/* Stage radices the kernels use for length n along an axis (0 rows, 1
 * columns), first stage first; returns the number of stages written to
 * `radices` (capacity 16) or a negative error. */
int fft_debug_radices(int n, int axis, int *radices);

/* The mixed-radix schedule of length n (2 <= n <= 2^24; Sections 6-7's
 * uneven sizes): for n = 2^a 3^b 5^c 7^d 11^e 13^f <= 14336 the stage radices of the
 * one-CTA kernel, first stage first, written to `radices` (capacity 16) and
 * their count returned, *n1 = *n2 = 0; for longer such n, 0 returned and the
 * four-step split n = n1 * n2 written (columns of length n1, then rows of
 * length n2); FFT_ERR_INVALID_SIZE when n has a prime factor above 13 or is
 * out of range, FFT_ERR_INVALID_ARG for NULL pointers.  Host only: no
 * device call. */
int fft_debug_mixed_plan(int n, int *radices, int *n1, int *n2);

/*
 * fft_debug_row_variant -- launch shape of the compiled row-pass kernel for
 * length n (a power of two, 2..8192), e elements per thread and column
 * pre-split `split` (1: none; 2: the row pass also applies the first radix-2
 * step of the column transform, Section 5's column FFTs split as 2 x ny/2).
 * Writes to the host array info[20]: threads per CTA, rows per CTA,
 * shared-memory float2 elements per row, the stage count S, then the S stage
 * radices (first stage first) and zeros.  FFT_ERR_UNSUPPORTED if that kernel
 * is not compiled, FFT_ERR_INVALID_SIZE for a bad n, FFT_ERR_INVALID_ARG for
 * a NULL info.  Host only: no device call (the tests model the kernel's
 * index arithmetic on the CPU from these shapes).
 */
int fft_debug_row_variant(int n, int e, int split, int *info);

/*
 * fft_debug_tc_layout -- compile-time layout of the split-FP16 tensor-core
 * kernels (the radix-32 stages of Section 2.2's butterflies on tcgen05),
 * written to the host array info[32] of long long:
 *   kind 0, the landed pre-split row-pair kernel for rows of n points
 *     (1024..8192): threads, threads per row T, output rows per unit L,
 *     exchange float2 elements per row, buffer bytes, B-table offset,
 *     barrier offset, dynamic shared-memory bytes, landing bytes per unit;
 *   kind 1, the landed unsplit sub-unit kernel: threads, T, rows per CTA L,
 *     exchange elements per row, rows per sub-unit RS, threads per sub-unit
 *     U, sub-units K, row-span stride SPAN (float2), buffer bytes, B-table
 *     offset, barrier offset, TMEM-slot offset, shared-memory bytes;
 *   kind 2 (n = 4096), the streaming column kernel: n, tile width W, ring
 *     slots S, threads, warps, MMA groups, butterflies per warp G, rows per
 *     segment, float2 per segment, rows per TMA box, bytes per segment,
 *     exchange float2 elements, ring offset, B-table offset, barrier offset,
 *     TMEM-slot offset, shared-memory bytes, then each warp's landing span
 *     offset in the exchange (float2).
 * FFT_ERR_UNSUPPORTED for a length or kind not compiled, FFT_ERR_INVALID_ARG
 * for a NULL info.  Host only: no device call (the tests check the spans,
 * offsets and barrier ids on the CPU from these values).
 */
int fft_debug_tc_layout(int n, int kind, long long *info);

/* cos(2 pi m / r) and sin(2 pi m / r) as the float constants the composite
 * mixed-radix DFTs use (evaluated at compile time from an integer quadrant
 * split and Taylor series in double, rounded once): written to *c and *s.
 * FFT_ERR_INVALID_ARG for NULL pointers or r < 1.  Host only. */
int fft_debug_root(int m, int r, float *c, float *s);

/* The library's CUDA runtime keeps its own per-thread last error (it is
 * linked statically): the text of the last CUDA error this thread met inside
 * the library, without clearing it ("no error" if none).  A call that
 * returned FFT_ERR_CUDA has left its cause here.  Never NULL. */
const char *fft_debug_last_cuda_error(void);

/* Library version string. */
const char *fft_version(void);

#ifdef __cplusplus
}
#endif

#endif /* GB300FFT_H */
