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
#include <string>
#include <sys/stat.h>

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

// The differentiation form with the loss and the adjoint's column half fused
// into the forward's column pass: dense 2D FP32 forward plans whose column
// pass runs without a pre-split and has a compiled fused variant.
// Its tiles are the widest of at most 64 KiB (whole warps, W adjacent
// columns), not the narrowed tiles small plans use for their column pass:
// two CTAs per SM, one transforming while the other loads (measured against
// the column pass's own 128 KiB tiles: 8 x 2048^2 step 0.495 -> 0.483 ms,
// 32 x 1024^2 0.461 -> 0.452).
const ColVariant *wadj_variant(fft_plan_s *p) {
    if (!p || p->kind != 0 || p->prec != FFT_PREC_FP32 || p->dir != FFT_FORWARD) return nullptr;
    if (p->any || p->fs.n1 > 0 || p->axes == 2 || p->rows.n < 2 || !p->rows.row || !p->cols.col) return nullptr;
    // the whole column in one tile, up to 2048 points: at 4096 the fused
    // column pass (two transforms per tile at 8 warps per SM) made the
    // 2 x 4096^2 step slower than the unfused one
    const int n = p->ny;
    if (n > 2048 || !is_pow2(n)) return nullptr;
    int w = default_col_w(n, p->nx);
    while (w > 2 && (long long)n * w * sizeof(float2) > 65536) w >>= 1;
    const ColVariant *v = col_variant(ilog2(n), preferred_col_e(n, w), w);
    return v && p->nx % v->w == 0 && cols_wadj_available(*v) ? v : nullptr;
}


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

Schedule default_schedule(int nx, int ny) {
    Schedule sc;
    (void)nx;
    sc.split = ny >= 8192 ? 2 : 1;
    return sc;
}

// GB300FFT_* environment overrides (experiments and tests).
void apply_env_overrides(Schedule *sc) {
    auto geti = [](const char *name, int *dst) {
        if (const char *ev = getenv(name)) *dst = atoi(ev);
    };
    geti("GB300FFT_ROW_E", &sc->row_e);
    geti("GB300FFT_ROW_PERSIST", &sc->row_persist);
    geti("GB300FFT_ROW_PF", &sc->row_pf);
    geti("GB300FFT_RING", &sc->ring);
    geti("GB300FFT_SPLIT", &sc->split);
    geti("GB300FFT_COL_E", &sc->col_e);
    geti("GB300FFT_COL_W", &sc->col_w);
    geti("GB300FFT_COL_PF", &sc->col_pf);
    geti("GB300FFT_COL_STREAM", &sc->col_stream);
    geti("GB300FFT_COL_TSTORE", &sc->col_tstore);
    geti("GB300FFT_LAND_PF", &sc->land_pf);
    geti("GB300FFT_PLANAR", &sc->planar);
    geti("GB300FFT_ROW_LAND", &sc->row_land);
    if (const char *ev = getenv("GB300FFT_COL_CLUSTER")) {
        const int c = atoi(ev);
        if (c == 2 || c == 4) {
            sc->col_kind = kColCluster;
            sc->col_c = c;
        }
    }
    if (const char *ev = getenv("GB300FFT_COL_PAIR"))
        if (atoi(ev)) sc->col_kind = kColPair;
}

// ---------------------------------------------------------------------------
// Autotune cache: one JSON object per line,
//   {"key": "<nx>x<ny>x<batch>:<prec>:<gpu>:<sms>", "row_e": .., ...}
// in $GB300FFT_TUNE_CACHE (default ~/.cache/gb300fft/tune.jsonl).
// ---------------------------------------------------------------------------
std::string tune_cache_path() {
    if (const char *ev = getenv("GB300FFT_TUNE_CACHE")) return ev;
    const char *home = getenv("HOME");
    return std::string(home ? home : "/tmp") + "/.cache/gb300fft/tune.jsonl";
}

std::string tune_key(int nx, int ny, int batch, int prec) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceProp prop;
    std::string name = "gpu";
    if (cudaGetDeviceProperties(&prop, dev) == cudaSuccess) name = prop.name;
    for (char &ch : name)
        if (ch == '"' || ch == ':') ch = '_';
    char buf[256];
    snprintf(buf, sizeof buf, "%dx%dx%d:%d:%s:%d", nx, ny, batch, prec, name.c_str(), sms);
    return buf;
}

int json_int(const std::string &line, const char *field, int dflt) {
    const std::string pat = std::string("\"") + field + "\": ";
    const size_t pos = line.find(pat);
    if (pos == std::string::npos) return dflt;
    return atoi(line.c_str() + pos + pat.size());
}

bool tune_cache_lookup(int nx, int ny, int batch, int prec, Schedule *sc) {
    FILE *f = fopen(tune_cache_path().c_str(), "r");
    if (!f) return false;
    const std::string key = "\"key\": \"" + tune_key(nx, ny, batch, prec) + "\"";
    char line[1024];
    bool found = false;
    while (fgets(line, sizeof line, f)) {
        std::string l(line);
        if (l.find(key) == std::string::npos) continue;
        sc->row_e = json_int(l, "row_e", sc->row_e);
        sc->row_persist = json_int(l, "row_persist", sc->row_persist);
        sc->row_pf = json_int(l, "row_pf", sc->row_pf);
        sc->split = json_int(l, "split", sc->split);
        sc->col_kind = json_int(l, "col_kind", sc->col_kind);
        sc->col_e = json_int(l, "col_e", sc->col_e);
        sc->col_w = json_int(l, "col_w", sc->col_w);
        sc->col_c = json_int(l, "col_c", sc->col_c);
        sc->col_stream = json_int(l, "col_stream", sc->col_stream);
        sc->col_tstore = json_int(l, "col_tstore", sc->col_tstore);
        sc->planar = json_int(l, "planar", sc->planar);
        sc->row_land = json_int(l, "row_land", sc->row_land);
        found = true;  // the last matching line wins
    }
    fclose(f);
    return found;
}

void tune_cache_store(int nx, int ny, int batch, int prec, const Schedule &sc, float ms) {
    const std::string path = tune_cache_path();
    const size_t slash = path.rfind('/');
    if (slash != std::string::npos) {
        // create the directory chain (best effort)
        std::string dir = path.substr(0, slash);
        for (size_t i = 1; i <= dir.size(); ++i)
            if (i == dir.size() || dir[i] == '/') mkdir(dir.substr(0, i).c_str(), 0755);
    }
    FILE *f = fopen(path.c_str(), "a");
    if (!f) return;
    fprintf(f,
            "{\"key\": \"%s\", \"row_e\": %d, \"row_persist\": %d, \"row_pf\": %d, \"split\": %d, "
            "\"col_kind\": %d, \"col_e\": %d, \"col_w\": %d, \"col_c\": %d, \"col_stream\": %d, \"col_tstore\": %d, "
            "\"planar\": %d, "
            "\"row_land\": %d, \"ms\": %.5f}\n",
            tune_key(nx, ny, batch, prec).c_str(), sc.row_e, sc.row_persist, sc.row_pf, sc.split, sc.col_kind,
            sc.col_e, sc.col_w, sc.col_c, sc.col_stream, sc.col_tstore, sc.planar, sc.row_land, ms);
    fclose(f);
}

int setup_row_axis(fft_plan_s *p, AxisPlan &ax, int n, const Schedule &sc) {
    ax.n = n;
    if (n == 1) return FFT_OK;
    int e = default_row_e(n);
    if (p->prec == FFT_PREC_SPLIT_FP16_TC) {
        if (!tc_rows_available(n)) return FFT_ERR_UNSUPPORTED;
        e = 16;
        // radix-32 tensor-core stages (tcgen05 only) where compiled
        if (p->tcg && p->tc_radix >= 32 && p->w32 && tc32_rows_available(n)) {
            e = 32;
            ax.tc32 = 1;
        }
    } else if (sc.row_e > 0 && row_variant(ilog2(n), sc.row_e)) {
        e = sc.row_e;
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
    p->row_persist = sc.row_persist;
    p->row_pf = sc.row_pf;
    p->col_pf = sc.col_pf;
    // long rows may go through the TMA landing-ring kernel (same E = 16
    // schedule and twiddle table as the plain row kernel)
    p->ring = sc.ring && ring_rows_available(n) && ax.row->e == 16 && p->prec == FFT_PREC_FP32;
    return FFT_OK;
}

int setup_col_axis(fft_plan_s *p, AxisPlan &ax, int n, int nx, long long tiles_per_w, const Schedule &sc) {
    ax.n = n;
    if (p->prec == FFT_PREC_SPLIT_FP16_TC && p->tcg && p->tc_radix >= 32 && p->w32 && tc32_col_width(n, nx) > 0) {
        // radix-32 tcgen05 column pass: E = 32 twiddles, tiles of tc_w columns
        ax.tc32 = 1;
        ax.tcg = 1;
        ax.tc_w = tc32_col_width(n, nx);
        ax.col = col_variant(ilog2(n), 16 > n ? n : 16, 2);  // keeps ax.col non-null (the pass exists)
        if (!ax.col) return FFT_ERR_UNSUPPORTED;
        const int sz = twiddle_table_size(n, 32);
        if (sz < 0) return FFT_ERR_UNSUPPORTED;
        if (sz > 0) {
            ax.tw = dev_alloc<float2>(p, sz);
            if (!ax.tw) return FFT_ERR_ALLOC;
            if (build_twiddles(ax.tw, n, 32, 0) != cudaSuccess) return FFT_ERR_CUDA;
        }
        ax.grid = tc32_cols_grid(n, ax.tc_w, tiles_per_w / ax.tc_w, p->num_sms);
        if (ax.grid <= 0) return FFT_ERR_UNSUPPORTED;
        // streaming form for out-of-place calls (same tile width, its own
        // E = 64 twiddle table, a row permutation the row pass applies)
        if (p->tc_stream && p->tc_tmem_a && tc_stream_available(n, nx) && ax.tc_w == tc_stream_width()) {
            const int e64 = tc_stream_twiddle_e();
            const int sz64 = twiddle_table_size(n, e64);
            if (sz64 > 0) {
                ax.stream_tw = dev_alloc<float2>(p, sz64);
                if (!ax.stream_tw) return FFT_ERR_ALLOC;
                if (build_twiddles(ax.stream_tw, n, e64, 0) != cudaSuccess) return FFT_ERR_CUDA;
                tc_stream_perm(&ax.perm_t, &ax.perm_g);
                ax.tcs = 1;
            }
        }
        return FFT_OK;
    }
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
        ax.tcg = (p->tcg && tcg_available(p->rows.n, n, ax.tc_w)) ? 1 : 0;
        ax.grid = tc_cols_grid(n, ax.tc_w, ax.tcg, tiles_per_w / ax.tc_w, p->num_sms);
        return ax.grid > 0 ? FFT_OK : FFT_ERR_UNSUPPORTED;
    }
    if (sc.col_kind == kColCluster) {
        const int ce = sc.col_e > 0 ? sc.col_e : 16;
        const int ccl = sc.col_c;
        if (cluster_cols_width(n, ce, ccl, nx) > 0) {
            ax.cl_c = ccl;
            ax.cl_e = ce;
            const int sz = cluster_cols_tw_size(n, ce, ccl);
            ax.tw = dev_alloc<float2>(p, sz > 0 ? sz : 1);
            ax.roots = dev_alloc<float2>(p, n);
            if (!ax.tw || !ax.roots) return FFT_ERR_ALLOC;
            if ((sz > 0 && build_twiddles(ax.tw, n / ccl, ce, 0) != cudaSuccess) ||
                build_roots(ax.roots, n, 0) != cudaSuccess)
                return FFT_ERR_CUDA;
            ax.col = col_variant(ilog2(n), default_col_e(n), 2);  // keeps ax.col non-null
            return ax.col ? FFT_OK : FFT_ERR_UNSUPPORTED;
        }
    }
    if (sc.col_kind == kColPair) {
        const int pe = sc.col_e > 0 ? sc.col_e : 16;
        if (pair_cols_width(n, pe, nx) > 0) {
            ax.pair_e = pe;
            const int sz = pair_cols_tw_size(n, pe);
            ax.tw = dev_alloc<float2>(p, sz > 0 ? sz : 1);
            ax.roots = dev_alloc<float2>(p, n);
            if (!ax.tw || !ax.roots) return FFT_ERR_ALLOC;
            if ((sz > 0 && build_twiddles(ax.tw, n / 2, pe, 0) != cudaSuccess) || build_roots(ax.roots, n, 0) != cudaSuccess)
                return FFT_ERR_CUDA;
            ax.col = col_variant(ilog2(n), default_col_e(n), 2);  // unused by the pair kernel; keeps ax.col non-null
            return ax.col ? FFT_OK : FFT_ERR_UNSUPPORTED;
        }
    }
    int w = default_col_w(n, nx);
    // small arrays: narrower tiles (down to 32-byte tile rows) until there is
    // a tile per SM (1024^2: 0.0144 -> 0.0120 ms; 512^2: 0.0105 -> 0.0084)
    while (w > 4 && tiles_per_w / w < p->num_sms && col_variant(ilog2(n), preferred_col_e(n, w / 2), w / 2)) w /= 2;
    int e = preferred_col_e(n, w);
    if (sc.col_kind == kColTile && sc.col_e > 0 && col_variant(ilog2(n), sc.col_e, w)) e = sc.col_e;
    if (sc.col_kind == kColTile && sc.col_w >= 2 && sc.col_w <= nx && col_variant(ilog2(n), e, sc.col_w)) w = sc.col_w;
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
    int pt = 0, pg = 0;
    const ColVariant *sv = sc.col_stream ? stream_col_variant(n, nx, &pt, &pg, sc.col_tstore) : nullptr;
    if (sv && sv->w == ax.col->w && sv->box_rows == ax.col->box_rows) {
        ax.stream = sv;
        ax.perm_t = pt;
        ax.perm_g = pg;
        if (ax.col->e == sv->e) {
            ax.stream_tw = ax.tw;
        } else {
            ax.stream_tw = dev_alloc<float2>(p, sv->tw_size);
            if (!ax.stream_tw) return FFT_ERR_ALLOC;
            if (build_twiddles(ax.stream_tw, n, sv->e, 0) != cudaSuccess) return FFT_ERR_CUDA;
        }
        long long sg = (long long)p->num_sms * col_ctas_per_sm(*sv);
        ax.stream_grid = (int)(sg > ntiles ? ntiles : (sg < 1 ? 1 : sg));
    }
    return FFT_OK;
}

// A large 1D plan (n > 8192): row length n2 (pass B) and column length
// n1 = n / n2 (pass A), both <= 8192; both passes keep whole-sector tiles up
// to n = 2^24, above that one length is 8192 with 16-byte tile rows.
int setup_fourstep(fft_plan_s *p, int n) {
    const int L = ilog2(n);
    FourStepPlan &fs = p->fs;
    fs.n = n;
    // n2 = 2^ceil(L/2), except that a length-8192 row (16-byte store chunks)
    // is avoided while n1 stays <= 8192 (2^25: 8192 x 4096 measured faster)
    fs.n2 = 1 << ((L + 1) / 2);
    if (fs.n2 == 8192 && n / 4096 <= 8192) fs.n2 = 4096;
    // GB300FFT_FS_N2 / _FS_WA / _FS_EA / _FS_EB / _FS_WB: schedule
    // experiments (row length, tile width and elements per thread of pass A,
    // elements per thread and rows per CTA of pass B)
    if (const char *ev = getenv("GB300FFT_FS_N2")) {
        const int v = atoi(ev);
        if (is_pow2(v) && v >= 128 && v <= 8192 && n / v >= 128 && n / v <= 8192) fs.n2 = v;
    }
    fs.n1 = n / fs.n2;
    // 2^25 and 2^26: three passes (4096-point columns, an M-point middle pass,
    // 4096-point rows), every pass on 32-byte tiles; GB300FFT_FS_THREE=0 keeps
    // the two-pass split with its length-8192 axis
    const char *e3 = getenv("GB300FFT_FS_THREE");
    if (n >= (1 << 25) && !(e3 && atoi(e3) == 0)) {
        fs.n1 = 4096;
        fs.n2 = n / 4096;
        fs.m = fs.n2 / 4096;
    }
    // pass A tile width: 4 from 2048 up, 8 at 1024, 16 below (measured; the
    // 2D column pass's rule gives 8 at 2048, 0.31 vs 0.26 ms here)
    int wa = fs.n1 >= 8192 ? 2 : fs.n1 >= 2048 ? 4 : fs.n1 == 1024 ? 8 : 16;
    if (const char *ev = getenv("GB300FFT_FS_WA"))
        if (col_variant(ilog2(fs.n1), default_col_e(fs.n1), atoi(ev)) && atoi(ev) <= fs.n2) wa = atoi(ev);
    // E = 32 for the length-8192 column pass (measured 0.62 -> 0.52 ms at 2^26)
    const int rown = fs.n2 / fs.m;  // length of pass B's rows
    int ea = fs.n1 == 8192 ? 32 : preferred_col_e(fs.n1, wa), eb = fourstep_row_e(rown);
    int wb = fourstep_row_w(rown);
    if (const char *ev = getenv("GB300FFT_FS_EA"))
        if (col_variant(ilog2(fs.n1), atoi(ev), wa)) ea = atoi(ev);
    if (fs.m == 1) {
        if (const char *ev = getenv("GB300FFT_FS_EB"))
            if (fourstep_row_variant(ilog2(fs.n2), atoi(ev), wb)) eb = atoi(ev);
        if (const char *ev = getenv("GB300FFT_FS_WB"))
            if (fourstep_row_variant(ilog2(fs.n2), eb, atoi(ev))) wb = atoi(ev);
    }
    fs.a = col_variant(ilog2(fs.n1), ea, wa);
    fs.b = fourstep_row_variant(ilog2(rown), eb, wb);
    if (!fs.a || !fs.b || fs.a->w > fs.n2 || fs.b->w > fs.n1) return FFT_ERR_UNSUPPORTED;
    fs.tw_a = dev_alloc<float2>(p, fs.a->tw_size);
    fs.tw_b = dev_alloc<float2>(p, fs.b->tw_size);
    fs.lohi = dev_alloc<float2>(p, 8192 + n / 8192);
    fs.work = dev_alloc<float2>(p, (size_t)n * p->batch);
    if (!fs.tw_a || !fs.tw_b || !fs.lohi || !fs.work) return FFT_ERR_ALLOC;
    if (build_twiddles(fs.tw_a, fs.n1, fs.a->e, 0) != cudaSuccess ||
        build_twiddles(fs.tw_b, rown, fs.b->e, 0) != cudaSuccess ||
        build_roots_strided(fs.lohi, 8192, n, 1, 0) != cudaSuccess ||
        build_roots_strided(fs.lohi + 8192, n / 8192, n, 8192, 0) != cudaSuccess)
        return FFT_ERR_CUDA;
    const long long ntiles = (long long)p->batch * (fs.n2 / fs.a->w);
    long long grid = (long long)p->num_sms * col_ctas_per_sm(*fs.a);
    if (grid > ntiles) grid = ntiles;
    fs.grid_a = (int)(grid < 1 ? 1 : grid);
    p->rows.n = n;  // the transform length (no plain row variant)
    return FFT_OK;
}

// A dense plan for (nx, ny, batch, dir, prec) running schedule `sc`.
fft_plan_s *create_dense(int nx, int ny, int batch, int dir, int precision, const Schedule &sc, int *rc_out) {
    fft_plan_s *p = new (std::nothrow) fft_plan_s();
    if (!p) {
        *rc_out = FFT_ERR_ALLOC;
        return nullptr;
    }
    p->nx = nx;
    p->ny = ny;
    p->batch = batch;
    p->dir = dir;
    p->prec = precision;
    p->sched = sc;
    int rc = FFT_OK;
    if (cudaGetDevice(&p->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, p->device) != cudaSuccess)
        rc = FFT_ERR_CUDA;
    if (rc == FFT_OK && precision == FFT_PREC_SPLIT_FP16_TC) {
        if (const char *ev = getenv("GB300FFT_TC_MMA")) p->tcg = strcmp(ev, "sync") != 0;
        if (p->tcg && !tcg_available(nx > 1 ? nx : ny, 1, 0)) p->tcg = 0;
        if (const char *ev = getenv("GB300FFT_TC_RADIX")) p->tc_radix = atoi(ev) >= 32 ? 32 : 16;
        if (const char *ev = getenv("GB300FFT_TC_TMEM_A")) p->tc_tmem_a = atoi(ev) != 0;
        if (const char *ev = getenv("GB300FFT_TC_LAND")) p->tc_land = atoi(ev) != 0;
        if (const char *ev = getenv("GB300FFT_TC_STREAM")) p->tc_stream = atoi(ev) != 0;
        p->w16 = dev_alloc<unsigned char>(p, 4 * 256 * 2);
        if (!p->w16) rc = FFT_ERR_ALLOC;
        else if (build_w16_table(p->w16, 0) != cudaSuccess) rc = FFT_ERR_CUDA;
        if (rc == FFT_OK && p->tcg && p->tc_radix >= 32) {
            p->w32 = dev_alloc<unsigned char>(p, kW32TableBytes);
            if (!p->w32) rc = FFT_ERR_ALLOC;
            else if (build_w32_table(p->w32, 0) != cudaSuccess) rc = FFT_ERR_CUDA;
        }
    }
    if (rc != FFT_OK) {
    } else if ((nx == 1 || ny == 1) && (nx > 8192 || ny > 8192)) {
        rc = setup_fourstep(p, nx == 1 ? ny : nx);
    } else if (nx == 1 || ny == 1) {
        rc = setup_row_axis(p, p->rows, nx == 1 ? ny : nx, sc);
    } else {
        rc = setup_row_axis(p, p->rows, nx, sc);
        // the unsplit column pass serves in-place calls
        Schedule plain = sc;
        if (rc == FFT_OK) rc = setup_col_axis(p, p->cols, ny, nx, (long long)nx * batch, plain);
        // Column pre-split: a length-8192 column needs a 128 KiB tile (one CTA
        // per SM); splitting it as 2 x 4096 halves the tile.  Only row
        // schedules compiled with the pre-split take it.
        int split =
            (sc.split == 2 && ny >= 4 && p->rows.row && row_split_available(p->rows.n, p->rows.row->e)) ? 2 : 1;
        if (precision == FFT_PREC_SPLIT_FP16_TC && p->rows.tc32) {
            // radix-32 tensor-core rows: pre-split when ny = 8192 (as on the
            // FP32 path); GB300FFT_TC_SPLIT = 1 or 2 overrides
            split = ny >= 8192 ? 2 : 1;
            if (const char *ev = getenv("GB300FFT_TC_SPLIT")) {
                const int v = atoi(ev);
                if ((v == 1 || v == 2) && ny % v == 0 && ny / v >= 16) split = v;
            }
        }
        // small square FP32 arrays: one cooperative launch for both passes
        const char *esm = getenv("GB300FFT_SMALL2D");  // 0: separate row and column launches
        if (rc == FFT_OK && precision == FFT_PREC_FP32 && !(esm && atoi(esm) == 0) && p->rows.row &&
            small2d_available(nx, ny, batch, p->rows.row->e)) {
            const int grid = small2d_grid(nx, batch, p->num_sms);
            if (grid > 0) {
                p->small_bar = dev_alloc<unsigned>(p, 2);
                if (!p->small_bar) rc = FFT_ERR_ALLOC;
                else if (cudaMemset(p->small_bar, 0, 2 * sizeof(unsigned)) != cudaSuccess) rc = FFT_ERR_CUDA;
                else p->small_grid = grid;
            }
        }
        if (rc == FFT_OK && split > 1) {
            // TMA stores for the pre-split blocks only when asked for (2):
            // their output rows lie P apart and plain stores measured faster
            Schedule ss = sc;
            if (ss.col_tstore == 1) ss.col_tstore = 0;
            rc = setup_col_axis(p, p->cols_split, ny / split, nx, (long long)nx * batch * split, ss);
            if (rc == FFT_OK) {
                p->twp = dev_alloc<float2>(p, ny);
                if (!p->twp) rc = FFT_ERR_ALLOC;
                else if (build_roots(p->twp, ny, 0) != cudaSuccess) rc = FFT_ERR_CUDA;
            }
            if (rc == FFT_OK) p->split = split;
            // planar blocks in a workspace for the streaming column pass (FP32)
            const AxisPlan &cs = p->cols_split;
            if (rc == FFT_OK && sc.planar && precision == FFT_PREC_FP32 && cs.stream && cs.cl_c == 0 &&
                cs.pair_e == 0 && !p->ring) {
                p->planar_work = dev_alloc<float2>(p, (size_t)nx * ny * batch);
                if (!p->planar_work) rc = FFT_ERR_ALLOC;
                else if (encode_col_map(&p->planar_map, p->planar_work, nx, (long long)ny * batch, 1, cs.stream->w,
                                        cs.stream->box_rows) != 0)
                    rc = FFT_ERR_CUDA;
            }
        }
    }
    if (rc == FFT_OK) {
        p->status = dev_alloc<int>(p, 1);
        if (!p->status) rc = FFT_ERR_ALLOC;
        else if (cudaMemset(p->status, 0, sizeof(int)) != cudaSuccess) rc = FFT_ERR_CUDA;
    }
    p->wp_parts = p->num_sms * 4;
    if (rc == FFT_OK) {
        // the fused differentiation form's column twiddles, where it applies
        if (const ColVariant *wv = wadj_variant(p)) {
            p->wadj_tw = dev_alloc<float2>(p, wv->tw_size > 0 ? wv->tw_size : 1);
            if (!p->wadj_tw) rc = FFT_ERR_ALLOC;
            else if (wv->tw_size > 0 && build_twiddles(p->wadj_tw, wv->n, wv->e, 0) != cudaSuccess) rc = FFT_ERR_CUDA;
        }
    }
    if (rc == FFT_OK && cudaDeviceSynchronize() != cudaSuccess) rc = FFT_ERR_CUDA;
    if (rc != FFT_OK) {
        free_plan(p);
        *rc_out = rc;
        return nullptr;
    }
    *rc_out = FFT_OK;
    return p;
}

long long next_pow2(long long v) {
    long long m = 1;
    while (m < v) m <<= 1;
    return m;
}

// mixed-radix stages for this length, unless GB300FFT_MIXED=0 (tests and
// experiments compare against Bluestein).  A mixed-radix axis given
// `cols_nx` > 0 runs down the columns of [n][cols_nx] slices.
bool use_mixed(int n, MixedStages *st) {
    const char *ev = getenv("GB300FFT_MIXED");
    if (ev && atoi(ev) == 0) return false;
    return !is_pow2(n) && mixed_factor(n, st);
}

// a 13-smooth length beyond one CTA that splits into two mixed-radix lengths,
// unless GB300FFT_MIXED=0
bool use_mixed_fourstep(int n, int *n1, int *n2) {
    const char *ev = getenv("GB300FFT_MIXED");
    if (ev && atoi(ev) == 0) return false;
    return !is_pow2(n) && n > kMixedMaxN && mixed_split(n, n1, n2);
}

// One axis of an any-size plan: rows transforms of length n.  A power of two
// gets a dense sub-plan of its own; a 13-smooth n up to kMixedMaxN the
// mixed-radix kernel; any other n Bluestein over a length-M power-of-two
// sub-plan, M >= 2n - 1, with the chirps and the filter transforms built here.
int setup_any_axis(fft_plan_s *p, AnyAxis &ax, int n, long long rows, int cols_nx = 0) {
    ax.n = n;
    ax.rows = rows;
    int rc = FFT_OK;
    if (is_pow2(n)) {
        ax.sub = create_dense(n, 1, (int)rows, FFT_FORWARD, FFT_PREC_FP32, default_schedule(n, 1), &rc);
        return ax.sub ? FFT_OK : rc;
    }
    if (use_mixed(n, &ax.mst)) {
        ax.mixed = true;
        ax.mtw = dev_alloc<float2>(p, ax.mst.tw_size > 0 ? ax.mst.tw_size : 1);
        if (!ax.mtw) return FFT_ERR_ALLOC;
        if (mixed_prepare(ax.mst, cols_nx > 0, cols_nx, &ax.ml) != 0) return FFT_ERR_UNSUPPORTED;
        return build_mixed_twiddles(ax.mtw, ax.mst, 0) == cudaSuccess ? FFT_OK : FFT_ERR_CUDA;
    }
    // a longer smooth length: four-step over two mixed-radix passes (columns
    // of length n1 into a workspace, then rows of length n2 with the
    // inter-pass twiddle on load and a transposed store)
    if (use_mixed_fourstep(n, &ax.n1, &ax.n2)) {
        MixedStages sa, sb;
        if (!mixed_factor(ax.n1, &sa) || !mixed_factor(ax.n2, &sb)) return FFT_ERR_UNSUPPORTED;
        if (mixed_prepare(sa, true, ax.n2, &ax.mla) != 0 || mixed_prepare(sb, false, 0, &ax.mlb, ax.n1) != 0)
            return FFT_ERR_UNSUPPORTED;
        int lshift = 0;
        while ((1LL << (2 * lshift)) < n) ++lshift;  // 2^lshift >= sqrt(n)
        const int nlo = 1 << lshift, nhi = (int)((n + nlo - 1) / nlo);
        ax.mtwa = dev_alloc<float2>(p, sa.tw_size > 0 ? sa.tw_size : 1);
        ax.mtwb = dev_alloc<float2>(p, sb.tw_size > 0 ? sb.tw_size : 1);
        ax.fs_lo = dev_alloc<float2>(p, nlo);
        ax.fs_hi = dev_alloc<float2>(p, nhi);
        ax.fs_work = dev_alloc<float2>(p, (size_t)rows * n);
        if (!ax.mtwa || !ax.mtwb || !ax.fs_lo || !ax.fs_hi || !ax.fs_work) return FFT_ERR_ALLOC;
        if (build_mixed_twiddles(ax.mtwa, sa, 0) != cudaSuccess || build_mixed_twiddles(ax.mtwb, sb, 0) != cudaSuccess ||
            build_roots_strided(ax.fs_lo, nlo, n, 1, 0) != cudaSuccess ||
            build_roots_strided(ax.fs_hi, nhi, n, nlo, 0) != cudaSuccess)
            return FFT_ERR_CUDA;
        ax.mlb.fs.hi = ax.fs_hi;
        ax.mlb.fs.lo = ax.fs_lo;
        ax.mlb.fs.lshift = lshift;
        ax.mlb.fs.lmask = nlo - 1;
        ax.mfs = true;
        return FFT_OK;
    }
    ax.M = (int)next_pow2(2LL * n - 1);
    if (rows * ax.M > (1LL << 31)) return FFT_ERR_INVALID_SIZE;
    ax.sub = create_dense(ax.M, 1, (int)rows, FFT_FORWARD, FFT_PREC_FP32, default_schedule(ax.M, 1), &rc);
    if (!ax.sub) return rc;
    for (int d = 0; d < 2; ++d) {
        ax.chirp[d] = dev_alloc<float2>(p, n);
        ax.H[d] = dev_alloc<float2>(p, ax.M);
        if (!ax.chirp[d] || !ax.H[d]) return FFT_ERR_ALLOC;
    }
    float2 *filt = dev_alloc<float2>(p, ax.M);
    if (!filt) return FFT_ERR_ALLOC;
    // H[d] = F(filter of chirp d) / M through a one-row plan of length M
    fft_plan_s *one = create_dense(ax.M, 1, 1, FFT_FORWARD, FFT_PREC_FP32, default_schedule(ax.M, 1), &rc);
    if (!one) return rc;
    for (int d = 0; d < 2 && rc == FFT_OK; ++d) {
        if (build_chirp(ax.chirp[d], n, d == 0 ? -1 : 1, 0) != cudaSuccess ||
            build_chirp_filter(filt, ax.chirp[d], n, ax.M, 0) != cudaSuccess)
            rc = FFT_ERR_CUDA;
        if (rc == FFT_OK) rc = run_dense(one, filt, ax.H[d], FFT_FORWARD, nullptr, 1.f, 0);
        if (rc == FFT_OK && launch_scale(ax.H[d], ax.M, 1.0f / (float)ax.M, 0) != cudaSuccess) rc = FFT_ERR_CUDA;
    }
    if (rc == FFT_OK && cudaDeviceSynchronize() != cudaSuccess) rc = FFT_ERR_CUDA;
    free_plan(one);
    // fused kernels when the padded length is one row pass with the same E
    // (so they share the sub-plan's twiddle table)
    const char *ev = getenv("GB300FFT_BLUESTEIN_FUSED");  // 0: the five-pass form (tests, experiments)
    const BluVariant *fv = (ev && atoi(ev) == 0) ? nullptr : blu_variant(ax.M);
    if (rc == FFT_OK && fv && ax.sub->rows.row && ax.sub->fs.n1 == 0 && !ax.sub->any &&
        fv->e == ax.sub->rows.row->e && (ax.sub->rows.tw || ax.sub->rows.row->tw_size == 0))
        ax.fused = fv;
    // the one-pass fused kernel needs no padded workspace; it is the faster
    // form up to M = 2048 (measured: 0.37 against 0.43 ms for 65536 rows of
    // 500 points, M = 1024), the two-pass one from M = 4096 (0.96 against
    // 0.81 ms for 32768 rows of 2047 points)
    const char *e1 = getenv("GB300FFT_BLUESTEIN_ONEPASS");  // 0 / 1 forces the form
    ax.fused_one = ax.fused && ax.fused->fn[2] && (e1 ? atoi(e1) != 0 : ax.M <= 2048);
    if (rc == FFT_OK && !ax.fused_one) {
        ax.A = dev_alloc<float2>(p, (size_t)rows * ax.M);
        if (!ax.A) return FFT_ERR_ALLOC;
    }
    return rc;
}

// A plan axis by axis (FP32): sizes that are not all powers of two, and 2D
// power-of-two shapes with an axis above 8192.  nx == 1 or ny == 1 is a 1D
// batch; otherwise the x axis, then the y axis down the columns in place
// (mixed radix) or between two transposes.
fft_plan_s *create_any(int nx, int ny, int batch, int dir, int *rc_out) {
    fft_plan_s *p = new (std::nothrow) fft_plan_s();
    AnyPlan *ap = new (std::nothrow) AnyPlan();
    if (!p || !ap) {
        delete p;
        delete ap;
        *rc_out = FFT_ERR_ALLOC;
        return nullptr;
    }
    p->nx = nx;
    p->ny = ny;
    p->batch = batch;
    p->dir = dir;
    p->prec = FFT_PREC_FP32;
    p->any = ap;
    int rc = FFT_OK;
    if (cudaGetDevice(&p->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, p->device) != cudaSuccess)
        rc = FFT_ERR_CUDA;
    if (rc == FFT_OK) {
        if (nx == 1 || ny == 1) {
            rc = setup_any_axis(p, ap->x, nx == 1 ? ny : nx, batch);
        } else {
            rc = setup_any_axis(p, ap->x, nx, (long long)ny * batch);
            // a mixed-radix y axis runs down the columns in place
            if (rc == FFT_OK) rc = setup_any_axis(p, ap->y, ny, (long long)nx * batch, nx);
            ap->y_cols = rc == FFT_OK && ap->y.mixed;
            if (rc == FFT_OK && !ap->y_cols) {
                ap->t = dev_alloc<float2>(p, (size_t)nx * ny * batch);
                if (!ap->t) rc = FFT_ERR_ALLOC;
            }
        }
    }
    if (rc == FFT_OK) {
        p->status = dev_alloc<int>(p, 1);
        if (!p->status) rc = FFT_ERR_ALLOC;
        else if (cudaMemset(p->status, 0, sizeof(int)) != cudaSuccess) rc = FFT_ERR_CUDA;
    }
    // the sub-plans' kernels report into this plan's status word
    if (rc == FFT_OK) {
        if (ap->x.sub) ap->x.sub->status = p->status;
        if (ap->y.sub) ap->y.sub->status = p->status;
    }
    p->wp_parts = p->num_sms * 4;
    if (rc == FFT_OK && cudaDeviceSynchronize() != cudaSuccess) rc = FFT_ERR_CUDA;
    if (rc != FFT_OK) {
        free_plan(p);
        *rc_out = rc;
        return nullptr;
    }
    *rc_out = FFT_OK;
    return p;
}

}  // namespace

namespace gb300fft {
void free_plan(fft_plan_s *p) {
    if (!p) return;
    if (p->ragged) ragged_destroy(p->ragged);
    if (p->host) {
        HostStage &h = *p->host;
        for (int i = 0; i < 2; ++i) {
            if (h.in_ready[i]) cudaEventDestroy(h.in_ready[i]);
            if (h.computed[i]) cudaEventDestroy(h.computed[i]);
            if (h.out_done[i]) cudaEventDestroy(h.out_done[i]);
        }
        if (h.entry) cudaEventDestroy(h.entry);
        if (h.cin) cudaStreamDestroy(h.cin);
        if (h.cout) cudaStreamDestroy(h.cout);
        if (h.comp) cudaStreamDestroy(h.comp);
        delete p->host;  // the staging buffers are in p->allocations
    }
    if (p->any) {
        free_plan(p->any->x.sub);
        free_plan(p->any->y.sub);
        delete p->any;
    }
    for (void *d : p->allocations) cudaFree(d);
    delete p;
}

// rows transforms of length ax.n along contiguous rows, in -> out (may alias)
int run_any_axis(AnyAxis &ax, const float2 *in, float2 *out, int sign, cudaStream_t s) {
    if (ax.mfs) {
        const int cj = sign > 0 ? 1 : 0;  // conj(F(conj x)): each pass conjugates its loads and stores
        if (launch_mixed(ax.mla, ax.mtwa, in, ax.fs_work, ax.rows, cj, s) != cudaSuccess ||
            launch_mixed(ax.mlb, ax.mtwb, ax.fs_work, out, ax.rows * ax.n1, cj, s) != cudaSuccess)
            return FFT_ERR_CUDA;
        return FFT_OK;
    }
    if (ax.mixed)
        return launch_mixed(ax.ml, ax.mtw, in, out, ax.rows, sign > 0 ? 1 : 0, s) == cudaSuccess ? FFT_OK
                                                                                                : FFT_ERR_CUDA;
    if (!ax.M) return run_dense(ax.sub, in, out, sign, nullptr, 1.f, s);
    const int d = sign > 0 ? 1 : 0;
    if (ax.fused) {
        // one pass (each CTA reads its rows before it writes them, so in
        // place is fine), or the two-pass form through the padded rows
        if (ax.fused_one)
            return launch_blu(*ax.fused, 2, in, out, ax.sub->rows.tw, ax.chirp[d], ax.H[d], ax.n, ax.rows, s) ==
                           cudaSuccess
                       ? FFT_OK
                       : FFT_ERR_CUDA;
        if (launch_blu(*ax.fused, 0, in, ax.A, ax.sub->rows.tw, ax.chirp[d], ax.H[d], ax.n, ax.rows, s) != cudaSuccess ||
            launch_blu(*ax.fused, 1, ax.A, out, ax.sub->rows.tw, ax.chirp[d], nullptr, ax.n, ax.rows, s) != cudaSuccess)
            return FFT_ERR_CUDA;
        return FFT_OK;
    }
    if (launch_blu_pre(in, ax.A, ax.chirp[d], ax.n, ax.M, ax.rows, s) != cudaSuccess) return FFT_ERR_CUDA;
    int rc = run_dense(ax.sub, ax.A, ax.A, FFT_FORWARD, nullptr, 1.f, s);
    if (rc != FFT_OK) return rc;
    if (launch_blu_mul(ax.A, ax.H[d], ax.M, ax.rows, s) != cudaSuccess) return FFT_ERR_CUDA;
    rc = run_dense(ax.sub, ax.A, ax.A, FFT_INVERSE, nullptr, 1.f, s);
    if (rc != FFT_OK) return rc;
    if (launch_blu_post(ax.A, out, ax.chirp[d], ax.n, ax.M, ax.rows, s) != cudaSuccess) return FFT_ERR_CUDA;
    return FFT_OK;
}

// Records pass event i on s.  Under stream capture it is recorded as an
// event-record node (cudaEventRecordExternal), so a captured step still
// time-stamps its passes when the graph runs (a plain record there would only
// order work inside the graph); the flag is not accepted outside capture.
static cudaError_t pass_event(const fft_plan_s *p, int i, cudaStream_t s) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) return cudaErrorUnknown;
    return cs == cudaStreamCaptureStatusActive ? cudaEventRecordWithFlags(p->ev[i], s, cudaEventRecordExternal)
                                               : cudaEventRecord(p->ev[i], s);
}

// out = DFT_sign(in) for an any-size plan
int run_any(fft_plan_s *p, const float2 *src, float2 *dst, int sign, cudaStream_t s) {
    AnyPlan &ap = *p->any;
    if (p->ev[0] && pass_event(p, 0, s) != cudaSuccess) return FFT_ERR_CUDA;
    int rc = run_any_axis(ap.x, src, dst, sign, s);
    if (rc != FFT_OK) return rc;
    if (p->ev[1] && pass_event(p, 1, s) != cudaSuccess) return FFT_ERR_CUDA;
    if (ap.y_cols) {
        if (launch_mixed(ap.y.ml, ap.y.mtw, dst, dst, p->batch, sign > 0 ? 1 : 0, s) != cudaSuccess)
            return FFT_ERR_CUDA;
    } else if (p->nx > 1 && p->ny > 1) {
        const long long batch = p->batch;
        if (launch_transpose(dst, ap.t, p->ny, p->nx, batch, s) != cudaSuccess) return FFT_ERR_CUDA;
        rc = run_any_axis(ap.y, ap.t, ap.t, sign, s);
        if (rc != FFT_OK) return rc;
        if (launch_transpose(ap.t, dst, p->nx, p->ny, batch, s) != cudaSuccess) return FFT_ERR_CUDA;
    }
    if (p->ev[2] && pass_event(p, 2, s) != cudaSuccess) return FFT_ERR_CUDA;
    return FFT_OK;
}

// Large 1D transform: pass A (the plain column pass over the [n1][n2] view of
// `in`, out of place into the workspace), pass B (twiddle on load, rows of the
// workspace, stored transposed into `out`); with m > 1 (2^25, 2^26) an m-point
// middle pass between them carries the twiddles and pass B's rows are n2 / m
// long.  The inverse is the forward transform stored at the reflected index
// (n - k) mod n.
int run_fourstep(fft_plan_s *p, const float2 *src, float2 *dst, bool inv, cudaStream_t s) {
    FourStepPlan &fs = p->fs;
    if (fs.map_base != src) {
        if (encode_col_map(&fs.map, src, fs.n2, (long long)fs.n1 * p->batch, 1, fs.a->w, fs.a->box_rows) != 0)
            return FFT_ERR_CUDA;
        fs.map_base = src;
    }
    if (p->ev[0] && pass_event(p, 0, s) != cudaSuccess) return FFT_ERR_CUDA;
    if (launch_cols(*fs.a, fs.map, fs.work, fs.tw_a, fs.n2, p->batch, 1, 0, p->status, fs.grid_a, 0, s) !=
        cudaSuccess)
        return FFT_ERR_CUDA;
    if (p->ev[1] && pass_event(p, 1, s) != cudaSuccess) return FFT_ERR_CUDA;
    if (fs.m > 1 && launch_fs_mid(fs.work, fs.lohi, fs.n1, fs.m, fs.n2 / fs.m, p->batch, s) != cudaSuccess)
        return FFT_ERR_CUDA;
    if (launch_rows_fourstep(*fs.b, fs.work, dst, fs.tw_b, fs.lohi, fs.n1, p->batch, inv ? 1 : 0, p->status, s,
                             fs.m) != cudaSuccess)
        return FFT_ERR_CUDA;
    if (p->ev[2] && pass_event(p, 2, s) != cudaSuccess) return FFT_ERR_CUDA;
    return FFT_OK;
}

// Column-only plan: the column FFTs of each [ny][nx] slice, read through a
// tensor map over `in` (so in and out may differ or coincide: every tile is
// read whole before its columns are written).  The inverse conjugates on load
// and on store.
// The tensor-core row pass runs from landed rows when the plan allows it and
// the rows divide into whole units (A in TMEM only).
static bool tc32_land_used(const fft_plan_s *p, long long nrows, int P) {
    return p->tc_land && p->tc_tmem_a && tc32_land_available(p->rows.n, nrows, p->ny, P);
}

int run_columns(fft_plan_s *p, const float2 *src, float2 *dst, bool inv, cudaStream_t s) {
    AxisPlan &cp = p->cols;
    if (cp.map_base != src) {
        if (encode_col_map(&cp.map, src, p->nx, (long long)p->ny * p->batch, 1, cp.col->w, cp.col->box_rows) != 0)
            return FFT_ERR_CUDA;
        cp.map_base = src;
    }
    if (p->ev[0] && pass_event(p, 0, s) != cudaSuccess) return FFT_ERR_CUDA;
    if (p->ev[1] && pass_event(p, 1, s) != cudaSuccess) return FFT_ERR_CUDA;
    if (launch_cols(*cp.col, cp.map, dst, cp.tw, p->nx, p->batch, 1, inv ? 3 : 0, p->status, cp.grid, p->col_pf, s) !=
        cudaSuccess)
        return FFT_ERR_CUDA;
    if (p->ev[2] && pass_event(p, 2, s) != cudaSuccess) return FFT_ERR_CUDA;
    return FFT_OK;
}

// out = DFT_{sign}(in) (optionally weighted by scale*w on load) for a dense plan.
int run_dense(fft_plan_s *p, const void *in, void *out, int sign, const float *weight, float wscale,
              cudaStream_t s, const float *wscale_dev) {
    const bool inv = sign > 0;
    const float2 *src = static_cast<const float2 *>(in);
    float2 *dst = static_cast<float2 *>(out);
    if (!src || !dst || !aligned16(src) || !aligned16(dst)) return FFT_ERR_INVALID_ARG;
    cudaSetDevice(p->device);
    if (p->axes == 2) return weight ? FFT_ERR_UNSUPPORTED : run_columns(p, src, dst, inv, s);
    if (p->any) return weight ? FFT_ERR_UNSUPPORTED : run_any(p, src, dst, sign, s);
    if (p->fs.n1 > 0) return weight ? FFT_ERR_UNSUPPORTED : run_fourstep(p, src, dst, inv, s);
    const long long total = (long long)p->nx * p->ny * p->batch;
    if (p->rows.n == 1) {
        // 1x1 transforms are the identity (times the weight, if any)
        if (weight) return FFT_ERR_UNSUPPORTED;
        if (src != dst && cudaMemcpyAsync(dst, src, total * sizeof(float2), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            return FFT_ERR_CUDA;
        return FFT_OK;
    }
    const bool two_pass = p->cols.col != nullptr;
    // the pre-split pairs rows across CTAs, so an in-place call must not use
    // it -- unless the blocks go through the planar workspace
    const bool planar = two_pass && p->planar_work != nullptr && p->prec == FFT_PREC_FP32;
    const int P = (two_pass && (src != dst || planar)) ? p->split : 1;
    AxisPlan &cp = (P > 1) ? p->cols_split : p->cols;
    const long long nrows = total / p->rows.n;
    if (p->prec == FFT_PREC_SPLIT_FP16_TC) {
        if (weight) return FFT_ERR_UNSUPPORTED;
        if (p->ev[0] && pass_event(p, 0, s) != cudaSuccess) return FFT_ERR_CUDA;
        const bool land = p->rows.tc32 && tc32_land_used(p, nrows, P);
        // streaming tensor-core columns: out of place, rows from landed units
        // stored in the permuted order
        const bool tstream = two_pass && land && src != dst && cp.tcs;
        const cudaError_t er =
            land ? launch_rows_tc32_land(p->rows.n, src, dst, p->rows.tw, p->twp, p->w32, nrows, p->ny, P, inv ? 1 : 0,
                                         (inv && !two_pass) ? 1 : 0, tstream ? cp.perm_t : 0, tstream ? cp.perm_g : 0,
                                         p->status, p->num_sms, s)
            : p->rows.tc32 ? launch_rows_tc32(p->rows.n, p->tc_tmem_a, src, dst, p->rows.tw, p->twp, p->w32, nrows, p->ny, P,
                                            inv ? 1 : 0, (inv && !two_pass) ? 1 : 0, p->status, s)
                         : launch_rows_tc(p->rows.n, p->tcg, src, dst, p->rows.tw, p->twp, p->w16, nrows, p->ny, P,
                                          inv ? 1 : 0, (inv && !two_pass) ? 1 : 0, p->status, s);
        if (er != cudaSuccess) return FFT_ERR_CUDA;
        if (p->ev[1] && pass_event(p, 1, s) != cudaSuccess) return FFT_ERR_CUDA;
        if (two_pass) {
            if (cp.map_base != out) {
                if (encode_col_map(&cp.map, out, p->nx, (long long)p->ny * p->batch, P, cp.tc_w,
                                   tc_col_box_rows(cp.n)) != 0)
                    return FFT_ERR_CUDA;
                cp.map_base = out;
            }
            const cudaError_t ec =
                tstream ? launch_cols_tc_stream(cp.map, dst, cp.stream_tw, p->w32, p->nx, p->batch, P, inv ? 1 : 0,
                                                p->status, p->num_sms, s)
                : cp.tc32 ? launch_cols_tc32(cp.n, cp.tc_w, p->tc_tmem_a, cp.map, dst, cp.tw, p->w32, p->nx, p->batch, P, inv ? 1 : 0,
                                           p->status, cp.grid, s)
                        : launch_cols_tc(cp.n, cp.tc_w, cp.tcg, cp.map, dst, cp.tw, p->w16, p->nx, p->batch, P,
                                         inv ? 1 : 0, p->status, cp.grid, s);
            if (ec != cudaSuccess) return FFT_ERR_CUDA;
        }
        if (p->ev[2] && pass_event(p, 2, s) != cudaSuccess) return FFT_ERR_CUDA;
        return FFT_OK;
    }
    // small square arrays: both passes in one cooperative launch (the pass
    // events then time the whole transform as the row pass)
    if (p->small_grid > 0 && !weight && two_pass && P == 1) {
        if (p->ev[0] && pass_event(p, 0, s) != cudaSuccess) return FFT_ERR_CUDA;
        if (launch_small2d(p->nx, src, dst, p->rows.tw, p->batch, inv ? 1 : 0, p->small_bar, p->status, p->small_grid,
                           s) != cudaSuccess)
            return FFT_ERR_CUDA;
        if (p->ev[1] && (pass_event(p, 1, s) != cudaSuccess || pass_event(p, 2, s) != cudaSuccess))
            return FFT_ERR_CUDA;
        return FFT_OK;
    }
    // out of place: the row pass may store its rows permuted for the
    // streaming column pass (in place it must not: rows would overwrite rows
    // other CTAs have yet to read)
    const bool stream =
        planar || (two_pass && src != dst && cp.stream && !p->ring && cp.cl_c == 0 && cp.pair_e == 0);
    float2 *row_dst = planar ? p->planar_work : dst;
    int &grid = p->row_grid[weight ? 1 : 0][P > 1 ? 1 : 0];
    if (grid == 0)
        grid = p->ring ? ring_rows_grid(p->rows.n, nrows, P, p->num_sms, weight != nullptr)
                       : row_grid(*p->rows.row, nrows, p->num_sms, weight != nullptr, P,
                                  p->row_persist < 0 ? P > 1 : p->row_persist != 0);
    if (p->ev[0] && pass_event(p, 0, s) != cudaSuccess) return FFT_ERR_CUDA;
    const bool land = P == 2 && !weight && !p->ring && p->sched.row_land &&
                      land_rows_available(p->rows.n, p->rows.row->e);
    const cudaError_t er =
        land ? launch_rows_land(p->rows.row->e, src, row_dst, p->rows.tw, p->twp, p->ny, p->batch, inv ? 1 : 0,
                                stream ? cp.perm_t : 0, stream ? cp.perm_g : 0, planar ? 1 : 0, p->status,
                                p->num_sms, p->sched.land_pf, s)
        : p->ring ? launch_rows_ring(p->rows.n, src, dst, p->rows.tw, p->twp, nrows, p->ny, P, inv ? 1 : 0,
                                   (inv && !two_pass) ? 1 : 0, weight, wscale, wscale_dev, p->status, grid, s)
                : launch_rows(*p->rows.row, src, row_dst, p->rows.tw, p->twp, nrows, p->ny, P, inv ? 1 : 0,
                              (inv && !two_pass) ? 1 : 0, weight, wscale, wscale_dev, grid, p->row_pf,
                              stream ? cp.perm_t : 0,
                              stream ? cp.perm_g : 0, planar ? 1 : 0, s);
    if (er != cudaSuccess) return FFT_ERR_CUDA;
    if (p->ev[1] && pass_event(p, 1, s) != cudaSuccess) return FFT_ERR_CUDA;
    if (!two_pass) {
        if (p->ev[2] && pass_event(p, 2, s) != cudaSuccess) return FFT_ERR_CUDA;
        return FFT_OK;
    }
    if (cp.cl_c > 0) {
        if (cp.map_base != out) {
            if (encode_col_map(&cp.map, out, p->nx, (long long)p->ny * p->batch, P,
                               cluster_cols_width(cp.n, cp.cl_e, cp.cl_c, p->nx),
                               cluster_cols_box_rows(cp.n, cp.cl_e, cp.cl_c)) != 0)
                return FFT_ERR_CUDA;
            cp.map_base = out;
        }
        if (launch_cols_cluster(cp.n, cp.cl_e, cp.cl_c, cp.map, dst, cp.tw, cp.roots, p->nx, p->batch, P, inv ? 1 : 0,
                                p->status, s) != cudaSuccess)
            return FFT_ERR_CUDA;
        if (p->ev[2] && pass_event(p, 2, s) != cudaSuccess) return FFT_ERR_CUDA;
        return FFT_OK;
    }
    if (cp.pair_e > 0) {
        if (launch_cols_pair(cp.n, cp.pair_e, dst, cp.tw, cp.roots, p->nx, p->batch, P, inv ? 1 : 0, s) != cudaSuccess)
            return FFT_ERR_CUDA;
        if (p->ev[2] && pass_event(p, 2, s) != cudaSuccess) return FFT_ERR_CUDA;
        return FFT_OK;
    }
    if (stream && stream_tstore(*cp.stream) && cp.omap_base != out) {
        if (encode_stream_store_map(&cp.omap, *cp.stream, out, p->nx, (long long)p->ny * p->batch, P) != 0)
            return FFT_ERR_CUDA;
        cp.omap_base = out;
    }
    if (!planar && cp.map_base != out) {
        if (encode_col_map(&cp.map, out, p->nx, (long long)p->ny * p->batch, P, cp.col->w, cp.col->box_rows) != 0)
            return FFT_ERR_CUDA;
        cp.map_base = out;
    }
    const cudaError_t ec =
        stream ? launch_cols_stream(*cp.stream, planar ? p->planar_map : cp.map, &cp.omap, dst, cp.stream_tw, p->nx,
                                    p->batch, P,
                                    inv ? 1 : 0, p->status, cp.stream_grid, planar ? 1 : 0, s)
               : launch_cols(*cp.col, cp.map, dst, cp.tw, p->nx, p->batch, P, inv ? 1 : 0, p->status, cp.grid,
                             p->col_pf, s);
    if (ec != cudaSuccess) return FFT_ERR_CUDA;
    if (p->ev[2] && pass_event(p, 2, s) != cudaSuccess) return FFT_ERR_CUDA;
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

int encode_map4(CUtensorMap *map, const void *base, int nx, long long rows, int split, int t, int w, int box_rows,
                int box_k) {
    EncodeTiledFn enc = get_encode_fn();
    if (!enc || split < 1 || t < 1 || rows % ((long long)split * t)) return -1;
    // (float within a row, kp, r mod t, r / t): row = kp + split * r
    const cuuint64_t rs = (cuuint64_t)nx * sizeof(float2);
    cuuint64_t dims[4] = {(cuuint64_t)2 * nx, (cuuint64_t)split, (cuuint64_t)t,
                          (cuuint64_t)(rows / ((long long)split * t))};
    cuuint64_t strides[3] = {rs, rs * split, rs * split * t};
    cuuint32_t box[4] = {(cuuint32_t)(2 * w), 1, (cuuint32_t)box_rows, (cuuint32_t)box_k};
    cuuint32_t estr[4] = {1, 1, 1, 1};
    CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<void *>(base), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
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

fft_plan_t fft_plan_create_columns(int nx, int ny, int batch, int dir, int precision) {
    t_last_error = FFT_OK;
    if (nx < 2 || ny < 2 || batch < 1 || !is_pow2(nx) || !is_pow2(ny) || ny > 8192 || nx > 65536 ||
        (long long)nx * ny * batch > (1LL << 31)) {
        fail(FFT_ERR_INVALID_SIZE);
        return nullptr;
    }
    if (dir != FFT_FORWARD && dir != FFT_INVERSE) {
        fail(FFT_ERR_INVALID_ARG);
        return nullptr;
    }
    if (precision != FFT_PREC_FP32) {
        fail(precision == FFT_PREC_SPLIT_FP16_TC ? FFT_ERR_UNSUPPORTED : FFT_ERR_INVALID_ARG);
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
    p->axes = 2;
    Schedule sc = default_schedule(nx, ny);
    apply_env_overrides(&sc);
    sc.col_stream = 0;  // the streaming pass needs rows stored in its own order
    sc.col_kind = kColTile;
    p->sched = sc;
    p->col_pf = sc.col_pf;
    int rc = FFT_OK;
    if (cudaGetDevice(&p->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, p->device) != cudaSuccess)
        rc = FFT_ERR_CUDA;
    if (rc == FFT_OK) rc = setup_col_axis(p, p->cols, ny, nx, (long long)nx * batch, sc);
    if (rc == FFT_OK) {
        p->status = dev_alloc<int>(p, 1);
        if (!p->status) rc = FFT_ERR_ALLOC;
        else if (cudaMemset(p->status, 0, sizeof(int)) != cudaSuccess) rc = FFT_ERR_CUDA;
    }
    p->rows.n = 1;
    if (rc == FFT_OK && cudaDeviceSynchronize() != cudaSuccess) rc = FFT_ERR_CUDA;
    if (rc != FFT_OK) {
        free_plan(p);
        fail(rc);
        return nullptr;
    }
    return p;
}

fft_plan_t fft_plan_create(int nx, int ny, int batch, int dir, int precision) {
    t_last_error = FFT_OK;
    // a 1D length (the other axis 1) up to 2^26 for powers of two (the
    // four-step path above 8192), 2^24 otherwise; 2D axes up to 65536.  Dense
    // plans: powers of two, 2D axes up to 8192; everything else goes axis by
    // axis (mixed radix, four-step or Bluestein per axis, FP32 only)
    const bool pow2 = is_pow2(nx) && is_pow2(ny);
    const bool oned = nx == 1 || ny == 1;
    const bool large1d = pow2 && oned && (nx > 8192 || ny > 8192);
    const bool dense = pow2 && (oned || (nx <= 8192 && ny <= 8192));
    const int cap = oned ? (pow2 ? (1 << 26) : (1 << 24)) : 65536;
    if (nx < 1 || ny < 1 || batch < 1 || nx > cap || ny > cap) {
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
    if ((large1d || !dense) && precision != FFT_PREC_FP32) {
        fail(FFT_ERR_UNSUPPORTED);
        return nullptr;
    }
    if (!dense) {
        int rc = FFT_OK;
        fft_plan_s *p = create_any(nx, ny, batch, dir, &rc);
        if (!p) fail(rc);
        return p;
    }
    Schedule sc = default_schedule(nx, ny);
    const bool cached = precision == FFT_PREC_FP32 && tune_cache_lookup(nx, ny, batch, precision, &sc);
    apply_env_overrides(&sc);
    int rc = FFT_OK;
    fft_plan_s *p = create_dense(nx, ny, batch, dir, precision, sc, &rc);
    if (!p) {
        fail(rc);
        return nullptr;
    }
    const char *ev = getenv("GB300FFT_AUTOTUNE");
    if (!cached && ev && atoi(ev) != 0 && precision == FFT_PREC_FP32) {
        rc = fft_plan_autotune(p, nullptr);
        if (rc != FFT_OK) {
            free_plan(p);
            fail(rc);
            return nullptr;
        }
    }
    return p;
}

int fft_execute(fft_plan_t p, const void *in, void *out, void *stream) {
    if (!p || p->kind != 0) return FFT_ERR_INVALID_ARG;
    p->last_use_host = false;
    return run_dense(p, in, out, p->dir, nullptr, 1.f, static_cast<cudaStream_t>(stream));
}

int fft_execute_host(fft_plan_t p, const void *host_in, void *host_out, void *stream) {
    if (!p || p->kind != 0 || !host_in || !host_out || host_in == host_out) return FFT_ERR_INVALID_ARG;
    cudaSetDevice(p->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const size_t bytes = (size_t)p->nx * p->ny * p->batch * sizeof(float2);
    if (!p->host) {
        HostStage *h = new (std::nothrow) HostStage();
        if (!h) return FFT_ERR_ALLOC;
        p->host = h;
        const size_t count = bytes / sizeof(float2);
        for (int i = 0; i < 2; ++i) {
            h->din[i] = dev_alloc<float2>(p, count);
            h->dout[i] = dev_alloc<float2>(p, count);
            if (!h->din[i] || !h->dout[i]) return FFT_ERR_ALLOC;
            if (cudaEventCreateWithFlags(&h->in_ready[i], cudaEventDisableTiming) != cudaSuccess ||
                cudaEventCreateWithFlags(&h->computed[i], cudaEventDisableTiming) != cudaSuccess ||
                cudaEventCreateWithFlags(&h->out_done[i], cudaEventDisableTiming) != cudaSuccess)
                return FFT_ERR_CUDA;
        }
        if (cudaStreamCreateWithFlags(&h->cin, cudaStreamNonBlocking) != cudaSuccess ||
            cudaStreamCreateWithFlags(&h->cout, cudaStreamNonBlocking) != cudaSuccess ||
            cudaStreamCreateWithFlags(&h->comp, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&h->entry, cudaEventDisableTiming) != cudaSuccess)
            return FFT_ERR_CUDA;
    }
    HostStage &h = *p->host;
    const int i = (int)(h.calls & 1);
    // input staging buffer i is free once the transform of two calls ago ran
    if (cudaStreamWaitEvent(h.cin, h.computed[i], 0) != cudaSuccess ||
        cudaMemcpyAsync(h.din[i], host_in, bytes, cudaMemcpyHostToDevice, h.cin) != cudaSuccess ||
        cudaEventRecord(h.in_ready[i], h.cin) != cudaSuccess)
        return FFT_ERR_CUDA;
    // The transform runs on the plan's compute stream, so it can overlap the
    // previous call's copy-out.  It reads and writes only staging buffers and
    // the plan's workspaces; the workspaces were last used by a host call
    // (already ordered on this stream) unless the plan ran on the caller's
    // stream since, in which case the compute stream waits for that first.
    if (!p->last_use_host &&
        (cudaEventRecord(h.entry, s) != cudaSuccess || cudaStreamWaitEvent(h.comp, h.entry, 0) != cudaSuccess))
        return FFT_ERR_CUDA;
    // after its input arrived and after the copy-out of two calls ago left
    // output staging buffer i
    if (cudaStreamWaitEvent(h.comp, h.in_ready[i], 0) != cudaSuccess ||
        cudaStreamWaitEvent(h.comp, h.out_done[i], 0) != cudaSuccess)
        return FFT_ERR_CUDA;
    const int rc = run_dense(p, h.din[i], h.dout[i], p->dir, nullptr, 1.f, h.comp);
    if (rc != FFT_OK) return rc;
    p->last_use_host = true;
    if (cudaEventRecord(h.computed[i], h.comp) != cudaSuccess ||
        cudaStreamWaitEvent(h.cout, h.computed[i], 0) != cudaSuccess ||
        cudaMemcpyAsync(host_out, h.dout[i], bytes, cudaMemcpyDeviceToHost, h.cout) != cudaSuccess ||
        cudaEventRecord(h.out_done[i], h.cout) != cudaSuccess ||
        cudaStreamWaitEvent(s, h.out_done[i], 0) != cudaSuccess)  // the caller's stream sees host_out
        return FFT_ERR_CUDA;
    h.calls += 1;
    return FFT_OK;
}

int fft_backward(fft_plan_t p, const void *grad_out, void *grad_in, void *stream) {
    if (!p || p->kind != 0) return FFT_ERR_INVALID_ARG;
    p->last_use_host = false;
    return run_dense(p, grad_out, grad_in, -p->dir, nullptr, 1.f, static_cast<cudaStream_t>(stream));
}

int fft_backward_weighted(fft_plan_t p, const void *X, const void *w, float scale, void *grad_in, void *stream) {
    if (!p || p->kind != 0 || !w || !aligned16(w)) return FFT_ERR_INVALID_ARG;
    p->last_use_host = false;
    return run_dense(p, X, grad_in, -p->dir, static_cast<const float *>(w), scale,
                     static_cast<cudaStream_t>(stream));
}

int fft_backward_weighted_dev(fft_plan_t p, const void *X, const void *w, const void *scale_dev, float scale,
                              void *grad_in, void *stream) {
    if (!p || p->kind != 0 || !w || !aligned16(w) || !scale_dev ||
        (reinterpret_cast<uintptr_t>(scale_dev) & 3))
        return FFT_ERR_INVALID_ARG;
    p->last_use_host = false;
    return run_dense(p, X, grad_in, -p->dir, static_cast<const float *>(w), scale,
                     static_cast<cudaStream_t>(stream), static_cast<const float *>(scale_dev));
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

int fft_weighted_power_adjoint_parts(fft_plan_t p) {
    if (!p) return FFT_ERR_INVALID_ARG;
    const ColVariant *v = wadj_variant(p);
    if (!v) return FFT_ERR_UNSUPPORTED;
    const long long tiles = (long long)(p->nx / v->w) * p->batch;
    return tiles > 0x7fffffffLL ? FFT_ERR_UNSUPPORTED : (int)tiles;
}

int fft_weighted_power_adjoint(fft_plan_t p, const void *x, const void *w, void *partials, void *y, void *stream) {
    if (!p || !x || !w || !partials || !y || !aligned16(x) || !aligned16(y) || !aligned16(w) ||
        (reinterpret_cast<uintptr_t>(partials) & 3))
        return FFT_ERR_INVALID_ARG;
    const ColVariant *v = wadj_variant(p);
    if (!v || !p->wadj_tw) return FFT_ERR_UNSUPPORTED;
    cudaSetDevice(p->device);
    p->last_use_host = false;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    float2 *yd = static_cast<float2 *>(y);
    const long long nrows = (long long)p->ny * p->batch;
    // forward rows, x -> y
    const int rgrid = row_grid(*p->rows.row, nrows, p->num_sms, false, 1, p->row_persist > 0);
    if (launch_rows(*p->rows.row, static_cast<const float2 *>(x), yd, p->rows.tw, p->twp, nrows, p->ny, 1, 0, 0,
                    nullptr, 1.f, nullptr, rgrid, p->row_pf, 0, 0, 0, s) != cudaSuccess)
        return FFT_ERR_CUDA;
    // fused columns, in place on y
    if (p->wadj_base != y) {
        if (encode_col_map(&p->wadj_map, y, p->nx, (long long)p->ny * p->batch, 1, v->w, v->box_rows) != 0)
            return FFT_ERR_CUDA;
        p->wadj_base = y;
    }
    const long long tiles = (long long)(p->nx / v->w) * p->batch;
    int grid = p->num_sms * cols_wadj_ctas_per_sm(*v);
    if (grid > tiles) grid = (int)tiles;
    if (launch_cols_wadj(*v, p->wadj_map, yd, p->wadj_tw, static_cast<const float *>(w), static_cast<float *>(partials),
                         p->nx, p->batch, p->status, grid, p->col_pf, s) != cudaSuccess)
        return FFT_ERR_CUDA;
    return FFT_OK;
}

int fft_backward_rows_scaled(fft_plan_t p, const void *y, const void *scale_dev, float scale, void *grad_in,
                             void *stream) {
    if (!p || !y || !grad_in || !aligned16(y) || !aligned16(grad_in) ||
        (scale_dev && (reinterpret_cast<uintptr_t>(scale_dev) & 3)))
        return FFT_ERR_INVALID_ARG;
    if (!wadj_variant(p)) return FFT_ERR_UNSUPPORTED;
    cudaSetDevice(p->device);
    p->last_use_host = false;
    const long long nrows = (long long)p->ny * p->batch;
    // F_rows^H = conj F_rows conj, times scale (and *scale_dev) on load
    const int rgrid = row_grid(*p->rows.row, nrows, p->num_sms, true, 1, p->row_persist > 0);
    if (launch_rows(*p->rows.row, static_cast<const float2 *>(y), static_cast<float2 *>(grad_in), p->rows.tw, p->twp,
                    nrows, p->ny, 1, 1, 1, nullptr, scale, static_cast<const float *>(scale_dev), rgrid, p->row_pf, 0,
                    0, 0, static_cast<cudaStream_t>(stream)) != cudaSuccess)
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

int fft_plan_autotune(fft_plan_t p, void *stream) {
    if (!p || p->kind != 0) return FFT_ERR_INVALID_ARG;
    if (p->prec != FFT_PREC_FP32 || p->fs.n1 > 0 || p->any) return FFT_OK;  // one schedule only
    cudaSetDevice(p->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const long long total = (long long)p->nx * p->ny * p->batch;
    float2 *a = nullptr, *b = nullptr;
    if (cudaMalloc(&a, total * sizeof(float2)) != cudaSuccess) return FFT_ERR_ALLOC;
    if (cudaMalloc(&b, total * sizeof(float2)) != cudaSuccess) {
        cudaFree(a);
        return FFT_ERR_ALLOC;
    }
    cudaMemsetAsync(a, 0x3e, total * sizeof(float2), s);
    // candidates: row E, row persistence, column pre-split, column kernel
    std::vector<Schedule> cands;
    const bool twod = p->nx > 1 && p->ny > 1;
    const int rown = p->nx > 1 ? p->nx : p->ny;
    for (int re : {16, 32, 8}) {
        if (rown < re || !row_variant(ilog2(rown), re)) continue;
        for (int persist : {-1, 0, 1}) {
            if (!twod) {
                Schedule c;
                c.row_e = re;
                c.row_persist = persist < 0 ? 0 : persist;
                c.split = 1;
                cands.push_back(c);
                continue;
            }
            for (int split : {1, 2}) {
                if (split == 2 && (p->ny < 4 || !row_split_available(rown, re))) continue;
                Schedule c;
                c.row_e = re;
                c.row_persist = persist;
                c.split = split;
                const int cn = p->ny / split;
                c.col_kind = kColTile;
                cands.push_back(c);
                if (stream_col_variant(cn, p->nx, nullptr, nullptr)) {
                    Schedule d = c;
                    d.col_stream = 0;
                    cands.push_back(d);
                    Schedule t = c;
                    t.col_tstore = 0;
                    cands.push_back(t);
                    if (split == 2) {
                        Schedule e = c;
                        e.planar = 0;
                        cands.push_back(e);
                        Schedule f = c;
                        f.row_land = 0;
                        cands.push_back(f);
                    }
                }
                for (int ce : {16, 64}) {
                    if (!col_variant(ilog2(cn), ce, default_col_w(cn, p->nx)) || ce == preferred_col_e(cn, default_col_w(cn, p->nx)))
                        continue;
                    Schedule d = c;
                    d.col_e = ce;
                    cands.push_back(d);
                }
                if (cluster_cols_width(cn, 16, 2, p->nx) > 0) {
                    Schedule d = c;
                    d.col_kind = kColCluster;
                    d.col_c = 2;
                    d.col_e = 16;
                    cands.push_back(d);
                }
            }
        }
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    Schedule bestsc = p->sched;
    for (const Schedule &c : cands) {
        int rc = FFT_OK;
        fft_plan_s *q = create_dense(p->nx, p->ny, p->batch, p->dir, p->prec, c, &rc);
        if (!q) continue;
        bool ok = true;
        for (int w = 0; w < 2 && ok; ++w) ok = run_dense(q, a, b, q->dir, nullptr, 1.f, s) == FFT_OK;
        const int reps = total >= (1LL << 24) ? 5 : 20;
        cudaEventRecord(e0, s);
        for (int k = 0; k < reps && ok; ++k) ok = run_dense(q, a, b, q->dir, nullptr, 1.f, s) == FFT_OK;
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ok && cudaGetLastError() == cudaSuccess && ms / reps < best) {
            best = ms / reps;
            bestsc = c;
        }
        free_plan(q);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(a);
    cudaFree(b);
    // rebuild this plan with the winner, keeping its identity (handle)
    int rc = FFT_OK;
    fft_plan_s *q = create_dense(p->nx, p->ny, p->batch, p->dir, p->prec, bestsc, &rc);
    if (!q) return rc;
    std::swap(*p, *q);
    free_plan(q);
    tune_cache_store(p->nx, p->ny, p->batch, p->prec, bestsc, best);
    return FFT_OK;
}

int fft_plan_describe(fft_plan_t p, char *buf, int len) {
    if (!p || (len > 0 && !buf) || len < 0) return FFT_ERR_INVALID_ARG;
    char tmp[1024];
    int k = 0;
    auto rad = [](int n, int e, char *o, int cap) {
        int r[16];
        const int S = schedule_radices(n, e, r);
        int w = snprintf(o, cap, "[");
        for (int i = 0; i < S && w < cap; ++i) w += snprintf(o + w, cap - w, i ? ",%d" : "%d", r[i]);
        if (w < cap) w += snprintf(o + w, cap - w, "]");
        return w;
    };
    if (p->kind == 1) {
        k = snprintf(tmp, sizeof tmp, "{\"kind\": \"ragged\", \"kernel\": \"k_ragged\"}");
    } else if (p->any) {
        const gb300fft::AnyPlan &ap = *p->any;
        k = snprintf(tmp, sizeof tmp,
                     "{\"kind\": \"any\", \"precision\": \"fp32\", \"x\": {\"n\": %d, \"bluestein_m\": %d, "
                     "\"fused\": %d, \"mixed\": %d, \"mixed_fourstep\": [%d, %d]}, \"y\": {\"n\": %d, "
                     "\"bluestein_m\": %d, \"fused\": %d, \"mixed\": %d, \"mixed_fourstep\": [%d, %d]}, "
                     "\"transposes\": %d}",
                     ap.x.n, ap.x.M, ap.x.fused ? (ap.x.fused_one ? 2 : 1) : 0, ap.x.mixed ? 1 : 0, ap.x.n1, ap.x.n2,
                     ap.y.n, ap.y.M, ap.y.fused ? (ap.y.fused_one ? 2 : 1) : 0, ap.y.mixed ? 1 : 0, ap.y.n1, ap.y.n2,
                     (p->nx > 1 && p->ny > 1 && !ap.y_cols) ? 2 : 0);
    } else if (p->fs.n1 > 0) {
        const gb300fft::FourStepPlan &fs = p->fs;
        char ra[96], rb[96];
        rad(fs.n1, fs.a->e, ra, sizeof ra);
        rad(fs.n2 / fs.m, fs.b->e, rb, sizeof rb);
        k = snprintf(tmp, sizeof tmp,
                     "{\"kind\": \"dense\", \"precision\": \"fp32\", \"fourstep\": {\"n\": %d, \"n1\": %d, "
                     "\"n2\": %d, \"m\": %d, \"mid\": \"%s\"}, \"rows\": {\"kernel\": "
                     "\"k_rows_fourstep<%d,%d,%d>\", \"n\": %d, \"e\": %d, "
                     "\"w\": %d, \"radices\": %s, \"persistent\": 0}, \"cols\": {\"kernel\": "
                     "\"k_cols<%d,%d,%d>\", \"n\": %d, \"e\": %d, \"w\": %d, \"radices\": %s, "
                     "\"grid\": %d}, \"split\": 1}",
                     fs.n, fs.n1, fs.n2, fs.m, fs.m == 4 ? "k_fs_mid<4>" : fs.m == 2 ? "k_fs_mid<2>" : "",
                     fs.n2 / fs.m, fs.b->e, fs.b->w, fs.n2 / fs.m, fs.b->e, fs.b->w, rb, fs.n1, fs.a->e, fs.a->w,
                     fs.n1, fs.a->e, fs.a->w, ra, fs.grid_a);
    } else if (p->axes == 2) {
        char r2[96] = "[]";
        rad(p->cols.n, p->cols.col->e, r2, sizeof r2);
        k = snprintf(tmp, sizeof tmp,
                     "{\"kind\": \"dense\", \"precision\": \"fp32\", \"axes\": \"y\", \"rows\": {\"kernel\": "
                     "\"none\", \"n\": 1}, \"cols\": {\"kernel\": \"k_cols<%d,%d,%d>\", \"n\": %d, \"e\": %d, "
                     "\"w\": %d, \"radices\": %s, \"grid\": %d}, \"split\": 1}",
                     p->cols.n, p->cols.col->e, p->cols.col->w, p->cols.n, p->cols.col->e, p->cols.col->w, r2,
                     p->cols.grid);
    } else {
        const bool tc = p->prec == FFT_PREC_SPLIT_FP16_TC;
        char r1[96] = "[]", r2[96] = "[]";
        const int re = p->rows.row ? (tc ? (p->rows.tc32 ? 32 : 16) : p->rows.row->e) : 1;
        if (p->rows.row) rad(p->rows.n, re, r1, sizeof r1);
        const gb300fft::AxisPlan &cp = p->split > 1 ? p->cols_split : p->cols;
        // an out-of-place split-FP16 call streams the columns when the rows land
        const bool tcs = tc && cp.tcs && p->rows.tc32 &&
                         tc32_land_used(p, (long long)p->nx * p->ny * p->batch / p->rows.n, p->split);
        if (cp.cl_c > 0) {
            char r3[96];
            rad(cp.n / cp.cl_c, cp.cl_e, r3, sizeof r3);
            snprintf(r2, sizeof r2, "[%d,%s", cp.cl_c, r3 + 1);
        } else if (cp.pair_e > 0) {
            char r3[96];
            rad(cp.n / 2, cp.pair_e, r3, sizeof r3);
            snprintf(r2, sizeof r2, "[2,%s", r3 + 1);
        } else if (cp.col) {
            rad(cp.n, tc ? (tcs ? 64 : cp.tc32 ? 32 : 16) : cp.col->e, r2, sizeof r2);
        }
        k = snprintf(tmp, sizeof tmp,
                     "{\"kind\": \"dense\", \"precision\": \"%s\", \"rows\": {\"kernel\": \"%s<%d,%d,split%d>\", "
                     "\"n\": %d, \"e\": %d, \"radices\": %s, \"persistent\": %d}, "
                     "\"cols\": {\"kernel\": \"%s<%d,%d,%d>\", \"n\": %d, \"e\": %d, \"w\": %d, \"radices\": %s, "
                     "\"grid\": %d}, \"split\": %d, \"col_tma_store\": %d, \"one_launch\": %d}",
                     tc ? "split_fp16_tc" : "fp32", tc ? (p->rows.tc32 ? (tc32_land_used(p, (long long)p->nx * p->ny * p->batch / p->rows.n, p->split) ? "k_rows_tc32_land" : "k_rows_tc32") : p->tcg ? "k_rows_tcgen05" : "k_rows_mmasync") : (p->ring ? "k_rows_ring" : (p->split == 2 && p->sched.row_land && p->rows.row && land_rows_available(p->rows.n, p->rows.row->e)) ? "k_rows_land" : "k_rows"), p->rows.n, re,
                     p->split, p->rows.n, re, r1, p->row_persist < 0 ? (p->split > 1) : p->row_persist,
                     !cp.col ? "none" : tc ? (tcs ? "k_cols_tc_stream" : cp.tc32 ? "k_cols_tc32" : cp.tcg ? "k_cols_tcgen05" : "k_cols_mmasync") : (cp.cl_c > 0 ? "k_cols_cluster" : cp.pair_e > 0 ? "k_cols_pair" : (cp.stream && !p->ring) ? "k_cols_stream" : "k_cols"), cp.n,
                     cp.cl_c > 0 ? cp.cl_e : cp.pair_e > 0 ? cp.pair_e : cp.col ? (tc ? (tcs ? 64 : cp.tc32 ? 32 : 16) : cp.col->e) : 0,
                     cp.cl_c > 0 ? cp.cl_c : cp.pair_e > 0 ? pair_cols_width(cp.n, cp.pair_e, p->nx) : cp.col ? (tc ? cp.tc_w : cp.col->w) : 0,
                     cp.n, cp.cl_c > 0 ? cp.cl_e : cp.pair_e > 0 ? cp.pair_e : cp.col ? (tc ? (tcs ? 64 : cp.tc32 ? 32 : 16) : cp.col->e) : 0,
                     cp.pair_e > 0 ? pair_cols_width(cp.n, cp.pair_e, p->nx) : cp.col ? (tc ? cp.tc_w : cp.col->w) : 0, r2,
                     cp.grid, p->split, (!tc && cp.stream && !p->ring && stream_tstore(*cp.stream)) ? 1 : 0,
                     p->small_grid > 0 ? 1 : 0);
    }
    if (len > 0) {
        const int c = k < len - 1 ? k : len - 1;
        memcpy(buf, tmp, (size_t)c);
        buf[c] = 0;
    }
    return k;
}

int fft_debug_radices(int n, int axis, int *radices) {
    if (!is_pow2(n) || n > 8192 || !radices || (axis != 0 && axis != 1)) return FFT_ERR_INVALID_ARG;
    const int e = axis == 0 ? default_row_e(n) : default_col_e(n);
    return schedule_radices(n, e, radices);
}

int fft_debug_tc_layout(int n, int kind, long long *info) {
    if (!info) return FFT_ERR_INVALID_ARG;
    if (kind == 2) return n == 4096 && gb300fft::tc_stream_layout(info) == 0 ? FFT_OK : FFT_ERR_UNSUPPORTED;
    return gb300fft::tc32_land_layout(n, kind, info) == 0 ? FFT_OK : FFT_ERR_UNSUPPORTED;
}

int fft_debug_row_variant(int n, int e, int split, int *info) {
    if (!info) return FFT_ERR_INVALID_ARG;
    if (!is_pow2(n) || n < 2 || n > 8192) return FFT_ERR_INVALID_SIZE;
    int threads = 0, rows = 0, elems = 0;
    if (!gb300fft::row_variant_info(n, e, split, &threads, &rows, &elems)) return FFT_ERR_UNSUPPORTED;
    int rad[16];
    const int S = schedule_radices(n, e > n ? n : e, rad);
    if (S < 1) return FFT_ERR_UNSUPPORTED;
    info[0] = threads;
    info[1] = rows;
    info[2] = elems;
    info[3] = S;
    for (int k = 0; k < 16; ++k) info[4 + k] = k < S ? rad[k] : 0;
    return FFT_OK;
}

// The library links the CUDA runtime statically, so its last error is not
// the caller's runtime's: this reads it (without clearing it).
const char *fft_debug_last_cuda_error(void) { return cudaGetErrorString(cudaPeekAtLastError()); }

int fft_debug_mixed_plan(int n, int *radices, int *n1, int *n2) {
    if (!radices || !n1 || !n2) return FFT_ERR_INVALID_ARG;
    *n1 = *n2 = 0;
    if (n < 2 || n > (1 << 24)) return FFT_ERR_INVALID_SIZE;
    gb300fft::MixedStages st;
    if (n <= gb300fft::kMixedMaxN) {
        if (!gb300fft::mixed_factor(n, &st)) return FFT_ERR_INVALID_SIZE;
        for (int s = 0; s < st.S; ++s) radices[s] = st.radix[s];
        return st.S;
    }
    return gb300fft::mixed_split(n, n1, n2) ? 0 : FFT_ERR_INVALID_SIZE;
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
