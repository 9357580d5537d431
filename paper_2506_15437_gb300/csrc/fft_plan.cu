// Plans and the C ABI of libgb300fft.so (declared in include/gb300fft.h).
//
// A dense plan runs the paper's Section 5 decomposition as two kernels on the
// caller's stream: the row pass (in -> out) and the TMA-staged column pass
// (out -> out, in place, no transpose).  The inverse and the adjoint reuse the
// forward tables through conj(F(conj(x))): the row pass conjugates on load,
// the column pass conjugates on store.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "../../include/gb300fft.h"
#include "fft_common.cuh"
#include "fft_internal.h"

namespace gb300fft {
cudaError_t launch_weighted_power(const float2 *X, const float *w, long long n, float *partials,
                                  int parts, cudaStream_t s);
}

using namespace gb300fft;

namespace {

thread_local int t_last_error = FFT_OK;

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *,
                                  CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                  CUtensorMapFloatOOBfill);

EncodeTiledFn get_encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    });
    return fn;
}

bool is_pow2(long long n) { return n >= 1 && (n & (n - 1)) == 0; }

int fail(int code) {
    t_last_error = code;
    return code;
}

template <class T>
T *dev_alloc(fft_plan_s *p, size_t count) {
    void *d = nullptr;
    if (count == 0) count = 1;
    if (cudaMalloc(&d, count * sizeof(T)) != cudaSuccess) return nullptr;
    p->allocations.push_back(d);
    return static_cast<T *>(d);
}


bool aligned16(const void *ptr) { return (reinterpret_cast<uintptr_t>(ptr) & 15u) == 0; }

int setup_row_axis(fft_plan_s *p, AxisPlan &ax, int n) {
    ax.n = n;
    if (n == 1) return FFT_OK;
    int e = default_row_e(n);
    if (p->prec == FFT_PREC_SPLIT_FP16_TC) {
        if (!tc_rows_available(n)) return FFT_ERR_UNSUPPORTED;
        e = 16;
    } else if (const char *ev = getenv("GB300FFT_ROW_E")) {
        const int forced = atoi(ev);
        if (row_variant(ilog2(n), forced)) e = forced;
    }
    ax.row = row_variant(ilog2(n), e);
    if (!ax.row) return FFT_ERR_UNSUPPORTED;
    if (ax.row->tw_size > 0) {
        ax.tw = dev_alloc<float2>(p, ax.row->tw_size);
        if (!ax.tw) return FFT_ERR_ALLOC;
        if (build_twiddles(ax.tw, n, ax.row->e, 0) != cudaSuccess) return FFT_ERR_CUDA;
    }
    if (ax.row->smem > 48 * 1024)
        cudaFuncSetAttribute(ax.row->fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ax.row->smem);
    // long rows may go through the TMA landing-ring kernel (same E = 16
    // schedule and twiddle table as the plain row kernel); off by default,
    // the plain persistent kernel measured faster
    p->ring = false;
    if (const char *ev = getenv("GB300FFT_ROW_PERSIST")) p->row_persist = atoi(ev);
    if (const char *ev = getenv("GB300FFT_ROW_PF")) p->row_pf = atoi(ev);
    if (const char *ev = getenv("GB300FFT_COL_PF")) p->col_pf = atoi(ev);
    if (const char *ev = getenv("GB300FFT_RING")) p->ring = ring_rows_available(n) && ax.row->e == 16 && atoi(ev) != 0;
    return FFT_OK;
}

int setup_col_axis(fft_plan_s *p, AxisPlan &ax, int n, int nx, long long tiles_per_w) {
    ax.n = n;
    if (p->prec == FFT_PREC_SPLIT_FP16_TC) {
        ax.tc_w = tc_col_width(n, nx);
        if (ax.tc_w == 0) return FFT_ERR_UNSUPPORTED;
        ax.col = col_variant(ilog2(n), 16 > n ? n : 16, 2);  // twiddle schedule (E = 16) and box rows
        if (!ax.col) return FFT_ERR_UNSUPPORTED;
        if (ax.col->tw_size > 0) {
            ax.tw = dev_alloc<float2>(p, ax.col->tw_size);
            if (!ax.tw) return FFT_ERR_ALLOC;
            if (build_twiddles(ax.tw, n, ax.col->e, 0) != cudaSuccess) return FFT_ERR_CUDA;
        }
        ax.grid = tc_cols_grid(n, ax.tc_w, tiles_per_w / ax.tc_w, p->num_sms);
        return ax.grid > 0 ? FFT_OK : FFT_ERR_UNSUPPORTED;
    }
    int w = default_col_w(n, nx);
    int e = default_col_e(n);
    if (const char *ev = getenv("GB300FFT_COL_E")) {
        const int forced = atoi(ev);
        if (col_variant(ilog2(n), forced, w)) e = forced;
    }
    if (const char *ev = getenv("GB300FFT_COL_W")) {
        const int forced = atoi(ev);
        if (forced >= 2 && forced <= nx && col_variant(ilog2(n), e, forced)) w = forced;
    }
    ax.col = col_variant(ilog2(n), e, w);
    if (!ax.col) return FFT_ERR_UNSUPPORTED;
    if (ax.col->tw_size > 0) {
        ax.tw = dev_alloc<float2>(p, ax.col->tw_size);
        if (!ax.tw) return FFT_ERR_ALLOC;
        if (build_twiddles(ax.tw, n, ax.col->e, 0) != cudaSuccess) return FFT_ERR_CUDA;
    }
    const long long ntiles = tiles_per_w / w;
    long long grid = (long long)p->num_sms * col_ctas_per_sm(*ax.col);
    if (grid > ntiles) grid = ntiles;
    if (grid < 1) grid = 1;
    ax.grid = (int)grid;
    return FFT_OK;
}

}  // namespace

namespace gb300fft {
void free_plan(fft_plan_s *p) {
    if (!p) return;
    if (p->ragged) ragged_destroy(p->ragged);
    for (void *d : p->allocations) cudaFree(d);
    delete p;
}

// out = DFT_{sign}(in) (optionally weighted by scale*w on load) for a dense plan.
int run_dense(fft_plan_s *p, const void *in, void *out, int sign, const float *weight, float wscale,
              cudaStream_t s) {
    const bool inv = sign > 0;
    const float2 *src = static_cast<const float2 *>(in);
    float2 *dst = static_cast<float2 *>(out);
    if (!src || !dst || !aligned16(src) || !aligned16(dst)) return FFT_ERR_INVALID_ARG;
    cudaSetDevice(p->device);
    const long long total = (long long)p->nx * p->ny * p->batch;
    if (p->rows.n == 1) {
        // 1x1 transforms are the identity (times the weight, if any)
        if (weight) return FFT_ERR_UNSUPPORTED;
        if (src != dst && cudaMemcpyAsync(dst, src, total * sizeof(float2), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            return FFT_ERR_CUDA;
        return FFT_OK;
    }
    const bool two_pass = p->cols.col != nullptr;
    // the pre-split pairs rows across CTAs, so an in-place call must not use it
    const int P = (two_pass && src != dst) ? p->split : 1;
    AxisPlan &cp = (P > 1) ? p->cols_split : p->cols;
    const long long nrows = total / p->rows.n;
    if (p->prec == FFT_PREC_SPLIT_FP16_TC) {
        if (weight) return FFT_ERR_UNSUPPORTED;
        if (p->ev[0] && cudaEventRecord(p->ev[0], s) != cudaSuccess) return FFT_ERR_CUDA;
        if (launch_rows_tc(p->rows.n, src, dst, p->rows.tw, p->twp, p->w16, nrows, p->ny, P, inv ? 1 : 0,
                           (inv && !two_pass) ? 1 : 0, s) != cudaSuccess)
            return FFT_ERR_CUDA;
        if (p->ev[1] && cudaEventRecord(p->ev[1], s) != cudaSuccess) return FFT_ERR_CUDA;
        if (two_pass) {
            if (cp.map_base != out) {
                if (encode_col_map(&cp.map, out, p->nx, (long long)p->ny * p->batch, P, cp.tc_w,
                                   tc_col_box_rows(cp.n)) != 0)
                    return FFT_ERR_CUDA;
                cp.map_base = out;
            }
            if (launch_cols_tc(cp.n, cp.tc_w, cp.map, dst, cp.tw, p->w16, p->nx, p->batch, P, inv ? 1 : 0, p->status,
                               cp.grid, s) != cudaSuccess)
                return FFT_ERR_CUDA;
        }
        if (p->ev[2] && cudaEventRecord(p->ev[2], s) != cudaSuccess) return FFT_ERR_CUDA;
        return FFT_OK;
    }
    int &grid = p->row_grid[weight ? 1 : 0][P > 1 ? 1 : 0];
    if (grid == 0)
        grid = p->ring ? ring_rows_grid(p->rows.n, nrows, P, p->num_sms, weight != nullptr)
                       : row_grid(*p->rows.row, nrows, p->num_sms, weight != nullptr, P,
                                  p->row_persist < 0 ? P > 1 : p->row_persist != 0);
    if (p->ev[0] && cudaEventRecord(p->ev[0], s) != cudaSuccess) return FFT_ERR_CUDA;
    const cudaError_t er =
        p->ring ? launch_rows_ring(p->rows.n, src, dst, p->rows.tw, p->twp, nrows, p->ny, P, inv ? 1 : 0,
                                   (inv && !two_pass) ? 1 : 0, weight, wscale, p->status, grid, s)
                : launch_rows(*p->rows.row, src, dst, p->rows.tw, p->twp, nrows, p->ny, P, inv ? 1 : 0,
                              (inv && !two_pass) ? 1 : 0, weight, wscale, grid, p->row_pf, s);
    if (er != cudaSuccess) return FFT_ERR_CUDA;
    if (p->ev[1] && cudaEventRecord(p->ev[1], s) != cudaSuccess) return FFT_ERR_CUDA;
    if (!two_pass) {
        if (p->ev[2] && cudaEventRecord(p->ev[2], s) != cudaSuccess) return FFT_ERR_CUDA;
        return FFT_OK;
    }
    if (cp.map_base != out) {
        if (encode_col_map(&cp.map, out, p->nx, (long long)p->ny * p->batch, P, cp.col->w, cp.col->box_rows) != 0)
            return FFT_ERR_CUDA;
        cp.map_base = out;
    }
    if (launch_cols(*cp.col, cp.map, dst, cp.tw, p->nx, p->batch, P, inv ? 1 : 0, p->status, cp.grid, p->col_pf,
                    s) != cudaSuccess)
        return FFT_ERR_CUDA;
    if (p->ev[2] && cudaEventRecord(p->ev[2], s) != cudaSuccess) return FFT_ERR_CUDA;
    return FFT_OK;
}

void set_last_error(int code) { t_last_error = code; }

int encode_col_map(CUtensorMap *map, const void *base, int nx, long long rows, int split, int w, int box_rows) {
    EncodeTiledFn enc = get_encode_fn();
    if (!enc || split < 1 || rows % split) return -1;
    // (float within a row, kp, row block index): row r = kp + split * i
    cuuint64_t dims[3] = {(cuuint64_t)2 * nx, (cuuint64_t)split, (cuuint64_t)(rows / split)};
    cuuint64_t strides[2] = {(cuuint64_t)nx * sizeof(float2), (cuuint64_t)split * nx * sizeof(float2)};
    cuuint32_t box[3] = {(cuuint32_t)(2 * w), 1, (cuuint32_t)box_rows};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void *>(base), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? 0 : -1;
}
}  // namespace gb300fft

extern "C" {

const char *fft_version(void) { return "gb300fft 0.1 (sm_103a)"; }

int fft_last_error(void) { return t_last_error; }

const char *fft_error_string(int code) {
    switch (code) {
        case FFT_OK: return "success";
        case FFT_ERR_INVALID_SIZE: return "invalid size (lengths must be powers of two in range, counts >= 1)";
        case FFT_ERR_INVALID_ARG: return "invalid argument (NULL or misaligned pointer, bad dir/precision/index)";
        case FFT_ERR_ALLOC: return "allocation failed";
        case FFT_ERR_CUDA: return "CUDA runtime or launch error";
        case FFT_ERR_UNSUPPORTED: return "unsupported by this build";
        case FFT_ERR_TIMEOUT: return "device-side bounded wait timed out";
        default: return "unknown error code";
    }
}

fft_plan_t fft_plan_create(int nx, int ny, int batch, int dir, int precision) {
    t_last_error = FFT_OK;
    if (!is_pow2(nx) || !is_pow2(ny) || nx > 8192 || ny > 8192 || batch < 1) {
        fail(FFT_ERR_INVALID_SIZE);
        return nullptr;
    }
    if (dir != FFT_FORWARD && dir != FFT_INVERSE) {
        fail(FFT_ERR_INVALID_ARG);
        return nullptr;
    }
    if (precision != FFT_PREC_FP32 && precision != FFT_PREC_SPLIT_FP16_TC) {
        fail(FFT_ERR_INVALID_ARG);
        return nullptr;
    }
    if ((long long)nx * ny * batch > (1LL << 31)) {
        fail(FFT_ERR_INVALID_SIZE);
        return nullptr;
    }
    fft_plan_s *p = new (std::nothrow) fft_plan_s();
    if (!p) {
        fail(FFT_ERR_ALLOC);
        return nullptr;
    }
    p->nx = nx;
    p->ny = ny;
    p->batch = batch;
    p->dir = dir;
    p->prec = precision;
    if (cudaGetDevice(&p->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, p->device) != cudaSuccess) {
        free_plan(p);
        fail(FFT_ERR_CUDA);
        return nullptr;
    }
    int rc = FFT_OK;
    if (precision == FFT_PREC_SPLIT_FP16_TC) {
        p->w16 = dev_alloc<unsigned char>(p, 4 * 256 * 2);
        if (!p->w16) rc = FFT_ERR_ALLOC;
        else if (build_w16_table(p->w16, 0) != cudaSuccess) rc = FFT_ERR_CUDA;
    }
    if (rc != FFT_OK) {
    } else if (nx == 1 || ny == 1) {
        rc = setup_row_axis(p, p->rows, nx == 1 ? ny : nx);
    } else {
        rc = setup_row_axis(p, p->rows, nx);
        if (rc == FFT_OK) rc = setup_col_axis(p, p->cols, ny, nx, (long long)nx * batch);
        // Column pre-split: a length-8192 column needs a 128 KiB tile (one CTA
        // per SM); splitting it as 2 x 4096 halves the tile.
        int split = ny >= 8192 ? 2 : 1;
        if (const char *ev = getenv("GB300FFT_SPLIT")) {
            const int forced = atoi(ev);
            if (forced == 1 || (forced == 2 && ny >= 4)) split = forced;
        }
        if (rc == FFT_OK && split > 1) {
            rc = setup_col_axis(p, p->cols_split, ny / split, nx, (long long)nx * batch * split);
            if (rc == FFT_OK) {
                p->twp = dev_alloc<float2>(p, ny);
                if (!p->twp) rc = FFT_ERR_ALLOC;
                else if (build_roots(p->twp, ny, 0) != cudaSuccess) rc = FFT_ERR_CUDA;
            }
            if (rc == FFT_OK) p->split = split;
        }
    }
    if (rc == FFT_OK) {
        p->status = dev_alloc<int>(p, 1);
        if (!p->status) rc = FFT_ERR_ALLOC;
        else if (cudaMemset(p->status, 0, sizeof(int)) != cudaSuccess) rc = FFT_ERR_CUDA;
    }
    p->wp_parts = p->num_sms * 4;
    if (rc == FFT_OK && cudaDeviceSynchronize() != cudaSuccess) rc = FFT_ERR_CUDA;
    if (rc != FFT_OK) {
        free_plan(p);
        fail(rc);
        return nullptr;
    }
    return p;
}

int fft_execute(fft_plan_t p, const void *in, void *out, void *stream) {
    if (!p || p->kind != 0) return FFT_ERR_INVALID_ARG;
    return run_dense(p, in, out, p->dir, nullptr, 1.f, static_cast<cudaStream_t>(stream));
}

int fft_backward(fft_plan_t p, const void *grad_out, void *grad_in, void *stream) {
    if (!p || p->kind != 0) return FFT_ERR_INVALID_ARG;
    return run_dense(p, grad_out, grad_in, -p->dir, nullptr, 1.f, static_cast<cudaStream_t>(stream));
}

int fft_backward_weighted(fft_plan_t p, const void *X, const void *w, float scale, void *grad_in, void *stream) {
    if (!p || p->kind != 0 || !w || !aligned16(w)) return FFT_ERR_INVALID_ARG;
    return run_dense(p, X, grad_in, -p->dir, static_cast<const float *>(w), scale,
                     static_cast<cudaStream_t>(stream));
}

int fft_weighted_power_parts(fft_plan_t p) { return p ? p->wp_parts : FFT_ERR_INVALID_ARG; }

int fft_weighted_power(fft_plan_t p, const void *X, const void *w, void *partials, void *stream) {
    if (!p || p->kind != 0 || !X || !w || !partials) return FFT_ERR_INVALID_ARG;
    cudaSetDevice(p->device);
    const long long total = (long long)p->nx * p->ny * p->batch;
    if (launch_weighted_power(static_cast<const float2 *>(X), static_cast<const float *>(w), total,
                              static_cast<float *>(partials), p->wp_parts,
                              static_cast<cudaStream_t>(stream)) != cudaSuccess)
        return FFT_ERR_CUDA;
    return FFT_OK;
}

int fft_plan_destroy(fft_plan_t p) {
    if (!p) return FFT_OK;
    cudaSetDevice(p->device);
    cudaDeviceSynchronize();
    free_plan(p);
    return FFT_OK;
}

int fft_plan_status(fft_plan_t p, void *stream) {
    if (!p || !p->status) return FFT_ERR_INVALID_ARG;
    cudaSetDevice(p->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int h = 0;
    if (cudaMemcpyAsync(&h, p->status, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) return FFT_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return FFT_ERR_CUDA;
    if (h != 0 && cudaMemsetAsync(p->status, 0, sizeof(int), s) != cudaSuccess) return FFT_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return FFT_ERR_CUDA;
    return h;
}

int fft_plan_set_pass_events(fft_plan_t p, void *ev_start, void *ev_mid, void *ev_end) {
    if (!p || p->kind != 0) return FFT_ERR_INVALID_ARG;
    const bool all = ev_start && ev_mid && ev_end;
    const bool none = !ev_start && !ev_mid && !ev_end;
    if (!all && !none) return FFT_ERR_INVALID_ARG;
    p->ev[0] = static_cast<cudaEvent_t>(ev_start);
    p->ev[1] = static_cast<cudaEvent_t>(ev_mid);
    p->ev[2] = static_cast<cudaEvent_t>(ev_end);
    return FFT_OK;
}

int fft_debug_radices(int n, int axis, int *radices) {
    if (!is_pow2(n) || n > 8192 || !radices || (axis != 0 && axis != 1)) return FFT_ERR_INVALID_ARG;
    const int e = axis == 0 ? default_row_e(n) : default_col_e(n);
    return schedule_radices(n, e, radices);
}

int fft_debug_reorder_map(int n, int axis, void *map, void *stream) {
    if (!is_pow2(n) || n > 8192 || !map || (axis != 0 && axis != 1)) return FFT_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (n == 1) {
        const int zero = 0;
        return cudaMemcpyAsync(map, &zero, sizeof(int), cudaMemcpyHostToDevice, s) == cudaSuccess ? FFT_OK
                                                                                                  : FFT_ERR_CUDA;
    }
    cudaError_t e = axis == 0 ? launch_rows_movemap(ilog2(n), static_cast<int *>(map), s)
                              : launch_cols_movemap(ilog2(n), static_cast<int *>(map), s);
    return e == cudaSuccess ? FFT_OK : FFT_ERR_CUDA;
}

// Ragged plans: provided by fft_ragged.cu.
}  // extern "C"
