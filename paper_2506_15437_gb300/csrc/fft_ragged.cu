// Ragged batches: many independent 2D transforms of mixed power-of-two sizes
// (each axis 32..1024) in ONE persistent launch, replayed from a CUDA graph.
//
// The paper's 2D transform (Section 5) runs row FFTs, then column FFTs, with
// the rows spread evenly over cores (it assumes an even decomposition).  A
// ragged batch has no even decomposition, so the work is cut into items of
// 4096 complex elements (32 KiB), executed by a 256-thread CTA each (four per
// SM; items of 8192 elements at two 512-thread CTAs per SM measured 2 %
// slower on the 512-instance batch):
//   * fused item  -- a whole instance with nx*ny <= 4096: its rows, then (same
//     CTA, through L2) its columns;
//   * row item    -- 4096/nx consecutive rows of a larger instance;
//   * column item -- 4096/ny adjacent columns of a larger instance; it may
//     start only when every row item of its instance has finished, which a
//     per-instance counter records (release: __threadfence + atomicAdd;
//     acquire: ld.acquire polled with a bounded wait).
// Persistent CTAs take items from a device-wide atomic queue head in queue
// order.  The host orders the queue so that an instance's column items come
// after all its row items (no circular wait: a waiting item depends only on
// earlier items, all of which are held by running CTAs) and a configurable
// lag behind them, so the rows are done by then and still sit in L2.
//
// Every wait is bounded (globaltimer): on expiry the kernel records
// FFT_ERR_TIMEOUT in the plan's status word and skips the item; it never traps
// or hangs.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <utility>
#include <vector>

#include "fft_common.cuh"
#include "fft_internal.h"

namespace gb300fft {

constexpr int kRagThreads = 256;
constexpr int kRagItem = 4096;  // complex elements per work item
constexpr int kRagCtasPerSm = 4;
constexpr int kRagE = 16;

enum : int { kItemFused = 0, kItemRows = 1, kItemCols = 2 };

struct RagTw {
    const float2 *p[11];  // per-stage twiddle tables for n = 2^k, k <= 10, E = 16
};

struct RagArgs {
    const int4 *items;       // {kind, instance, first, count}
    int nitems;
    const int4 *inst;        // {log2 nx, log2 ny, row items, 0}
    const long long *offs;   // element offset of each instance
    const float2 *in;
    float2 *out;
    int *head;               // queue head (zeroed before each launch)
    int *done;               // per-instance finished row items (zeroed)
    int *status;
    float si, so;            // conj multipliers for input / output
    int withhold;            // test hook: row items do not report completion
    long long spin_limit_ns; // bounded wait for column items
    RagTw tw;
};

struct SyncNamed {  // barrier over the first n threads of the CTA (n % 32 == 0)
    int n;
    __device__ __forceinline__ void operator()() const { asm volatile("bar.sync 1, %0;" ::"r"(n) : "memory"); }
};

__device__ __forceinline__ int ld_acquire(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// `count` rows (count * NX / 16 threads take part) of one instance, starting
// at row `first`: load, transform along x, store.
template <int NX>
__device__ __forceinline__ void rag_rows(const float2 *in, float2 *out, int first, int count, const float2 *tw,
                                         float si, float so, float2 *smem) {
    using Eng = Engine<NX, kRagE, 1, PadShift<kRagE>::value>;
    constexpr int T = NX / kRagE;
    constexpr int R0 = Eng::R0;
    const int active_threads = count * T;
    if ((int)threadIdx.x >= active_threads) return;
    const int g = threadIdx.x / T;
    const int tt = threadIdx.x - g * T;
    const long long row = first + g;
    const float2 *src = in + row * NX;
    float2 *dst = out + row * NX;
    float2 v[kRagE];
#pragma unroll
    for (int b = 0; b < kRagE / R0; ++b) {
        const int j = tt + b * T;
#pragma unroll
        for (int r = 0; r < R0; ++r) {
            float2 x = __ldg(src + j + r * (NX / R0));
            x.y *= si;
            v[b * R0 + r] = x;
        }
    }
    auto store = [&](int i, int, float2 x) { dst[i] = x; };
    auto none = [] {};
    if constexpr (T >= 32)
        Eng::template run<FftPolicy, false>(v, smem + g * Eng::SMEM_ELEMS, tw, tt, 0, SyncNamed{active_threads}, none,
                                            store);
    else
        Eng::template run<FftPolicy, false>(v, smem + g * Eng::SMEM_ELEMS, tw, tt, 0, SyncWarp{}, none, store);
    (void)so;
}

// W adjacent columns (first_col ..) of an [NY][nx] instance, in place in
// `data`: loads through L2 (the rows were written by other CTAs), transform
// along y, store with the output conjugation.
template <int NY, int W>
__device__ __forceinline__ void rag_cols(float2 *data, int nx, int first_col, const float2 *tw, float so,
                                         float2 *smem) {
    using Eng = Engine<NY, kRagE, W, PadShift<kRagE>::value>;
    constexpr int T = NY / kRagE;
    constexpr int NT = T * W;
    constexpr int R0 = Eng::R0;
    static_assert(NT <= kRagThreads && NT % 32 == 0, "column item shape");
    if ((int)threadIdx.x >= NT) return;
    const int c = threadIdx.x % W;
    const int tt = threadIdx.x / W;
    float2 *base = data + first_col;
    float2 v[kRagE];
#pragma unroll
    for (int b = 0; b < kRagE / R0; ++b) {
        const int j = tt + b * T;
#pragma unroll
        for (int r = 0; r < R0; ++r) v[b * R0 + r] = __ldcg(base + (long long)(j + r * (NY / R0)) * nx + c);
    }
    auto store = [&](int i, int cc, float2 x) {
        x.y *= so;
        base[(long long)i * nx + cc] = x;
    };
    auto none = [] {};
    Eng::template run<FftPolicy, false>(v, smem, tw, tt, c, SyncNamed{NT}, none, store);
}

// Item handlers are not inlined so that each item shape gets its own
// register allocation inside the one persistent kernel.
template <int LX>
__device__ __noinline__ void dispatch_rows(const float2 *tw, float si, const float2 *in, float2 *out, int first,
                                           int count, float2 *smem) {
    rag_rows<1 << LX>(in, out, first, count, tw, si, 1.f, smem);
}

template <int LY>
__device__ __noinline__ void dispatch_cols(const float2 *tw, float so, float2 *out, int nx, int first,
                                           float2 *smem) {
    constexpr int NY = 1 << LY;
    rag_cols<NY, kRagItem / NY>(out, nx, first, tw, so, smem);
}

template <int LX, int LY>
__device__ __noinline__ void fused_item(const float2 *twx, const float2 *twy, float si, float so, const float2 *in,
                                        float2 *out, float2 *smem) {
    constexpr int NX = 1 << LX, NY = 1 << LY;
    rag_rows<NX>(in, out, 0, NY, twx, si, 1.f, smem);
    __syncthreads();  // the CTA's row results are visible to the CTA
    rag_cols<NY, NX>(out, NX, 0, twy, so, smem);
}

__global__ void __launch_bounds__(kRagThreads, kRagCtasPerSm) k_ragged(const RagArgs a) {
    extern __shared__ __align__(16) float2 smem[];
    __shared__ int s_item;
    __shared__ int s_ok;
    for (;;) {
        __syncthreads();  // previous item finished with shared memory and s_item
        if (threadIdx.x == 0) s_item = atomicAdd(a.head, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= a.nitems) return;
        const int4 item = a.items[it];
        const int4 ins = a.inst[item.y];
        const long long off = a.offs[item.y];
        const float2 *in = a.in + off;
        float2 *out = a.out + off;
        const int lx = ins.x, ly = ins.y;
        if (item.x == kItemRows) {
            switch (lx) {
                case 5: dispatch_rows<5>(a.tw.p[5], a.si, in, out, item.z, item.w, smem); break;
                case 6: dispatch_rows<6>(a.tw.p[6], a.si, in, out, item.z, item.w, smem); break;
                case 7: dispatch_rows<7>(a.tw.p[7], a.si, in, out, item.z, item.w, smem); break;
                case 8: dispatch_rows<8>(a.tw.p[8], a.si, in, out, item.z, item.w, smem); break;
                case 9: dispatch_rows<9>(a.tw.p[9], a.si, in, out, item.z, item.w, smem); break;
                default: dispatch_rows<10>(a.tw.p[10], a.si, in, out, item.z, item.w, smem); break;
            }
            __syncthreads();
            if (threadIdx.x == 0 && !a.withhold) {
                __threadfence();  // release this item's stores before counting it
                atomicAdd(a.done + item.y, 1);
            }
        } else if (item.x == kItemCols) {
            if (threadIdx.x == 0) {
                const int need = ins.z;
                const uint64_t t0 = globaltimer_ns();
                int ok = 0;
                for (uint32_t k = 0; k < (1u << 30); ++k) {
                    if (ld_acquire(a.done + item.y) >= need) {
                        ok = 1;
                        break;
                    }
                    if ((k & 63) == 63 && globaltimer_ns() - t0 > (uint64_t)a.spin_limit_ns) break;
                    __nanosleep(64);
                }
                if (!ok) record_status(a.status, kStatusTimeout);
                s_ok = ok;
            }
            __syncthreads();
            if (!s_ok) continue;
            const int nx = 1 << lx;
            switch (ly) {
                case 5: dispatch_cols<5>(a.tw.p[5], a.so, out, nx, item.z, smem); break;
                case 6: dispatch_cols<6>(a.tw.p[6], a.so, out, nx, item.z, smem); break;
                case 7: dispatch_cols<7>(a.tw.p[7], a.so, out, nx, item.z, smem); break;
                case 8: dispatch_cols<8>(a.tw.p[8], a.so, out, nx, item.z, smem); break;
                case 9: dispatch_cols<9>(a.tw.p[9], a.so, out, nx, item.z, smem); break;
                default: dispatch_cols<10>(a.tw.p[10], a.so, out, nx, item.z, smem); break;
            }
        } else {
            switch (lx * 16 + ly) {  // lx + ly <= 12, both >= 5
                case 5 * 16 + 5: fused_item<5, 5>(a.tw.p[5], a.tw.p[5], a.si, a.so, in, out, smem); break;
                case 5 * 16 + 6: fused_item<5, 6>(a.tw.p[5], a.tw.p[6], a.si, a.so, in, out, smem); break;
                case 5 * 16 + 7: fused_item<5, 7>(a.tw.p[5], a.tw.p[7], a.si, a.so, in, out, smem); break;
                case 6 * 16 + 5: fused_item<6, 5>(a.tw.p[6], a.tw.p[5], a.si, a.so, in, out, smem); break;
                case 6 * 16 + 6: fused_item<6, 6>(a.tw.p[6], a.tw.p[6], a.si, a.so, in, out, smem); break;
                default: fused_item<7, 5>(a.tw.p[7], a.tw.p[5], a.si, a.so, in, out, smem); break;
            }
        }
    }
}

// Shared memory of the largest item: 4096/n rows (or W columns) of padded
// length-n exchange buffers.
constexpr size_t kRagSmem = sizeof(float2) * (size_t)(kRagItem + (kRagItem >> 4));

// ---------------------------------------------------------------------------
// Host side.
// ---------------------------------------------------------------------------
struct RaggedState {
    int count = 0;
    std::vector<int> nx, ny;
    std::vector<long long> offs;  // count + 1 entries
    long long total = 0;
    // device
    int4 *d_items = nullptr;
    int4 *d_inst = nullptr;
    long long *d_offs = nullptr;
    int *d_counters = nullptr;  // [0] head, [1..count] done
    float2 *d_tw[11] = {};
    int nitems = 0;
    int grid = 0;
    int lag = 0;
    // schedule knobs (autotuned)
    int small_last = 1;
    // graph
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    const void *g_in = nullptr;
    void *g_out = nullptr;
    int g_dir = 0;
    // loop baseline: one dense plan per distinct shape
    std::map<std::pair<int, int>, fft_plan_s *> shape_plans;
    std::vector<void *> allocs;
    int withhold = 0;
    long long spin_limit_ns = 1000000000LL;
};

void ragged_destroy(RaggedState *r) {
    if (!r) return;
    if (r->exec) cudaGraphExecDestroy(r->exec);
    if (r->graph) cudaGraphDestroy(r->graph);
    for (auto &kv : r->shape_plans) free_plan(kv.second);
    for (void *d : r->allocs) cudaFree(d);
    delete r;
}

namespace {

int ilog2_host(int n) {
    int l = 0;
    while ((1 << l) < n) ++l;
    return l;
}

// Queue order: large instances' row items in instance order, each instance's
// column items emitted once `lag` further row items have gone out (then the
// remaining ones), and the small fused items first or last.
std::vector<int4> build_items(const RaggedState &r, int lag, bool small_last, std::vector<int4> &inst) {
    std::vector<int4> items, smalls;
    inst.assign(r.count, make_int4(0, 0, 0, 0));
    struct Pending {
        int i;
        long long emitted_at;
    };
    std::vector<Pending> pending;
    long long rows_emitted = 0;
    auto emit_cols = [&](int i) {
        const int W = kRagItem / r.ny[i];
        for (int c = 0; c < r.nx[i]; c += W) items.push_back(make_int4(kItemCols, i, c, W));
    };
    for (int i = 0; i < r.count; ++i) {
        const int lx = ilog2_host(r.nx[i]), ly = ilog2_host(r.ny[i]);
        if ((long long)r.nx[i] * r.ny[i] <= kRagItem) {
            inst[i] = make_int4(lx, ly, 0, 0);
            smalls.push_back(make_int4(kItemFused, i, 0, r.ny[i]));
            continue;
        }
        const int R = kRagItem / r.nx[i];
        const int nrow_items = r.ny[i] / R;
        inst[i] = make_int4(lx, ly, nrow_items, 0);
        for (int y = 0; y < r.ny[i]; y += R) items.push_back(make_int4(kItemRows, i, y, R));
        rows_emitted += nrow_items;
        pending.push_back({i, rows_emitted});
        while (!pending.empty() && rows_emitted - pending.front().emitted_at >= lag) {
            emit_cols(pending.front().i);
            pending.erase(pending.begin());
        }
    }
    for (auto &pd : pending) emit_cols(pd.i);
    if (small_last)
        items.insert(items.end(), smalls.begin(), smalls.end());
    else
        items.insert(items.begin(), smalls.begin(), smalls.end());
    return items;
}

int upload_schedule(RaggedState &r) {
    std::vector<int4> inst;
    std::vector<int4> items = build_items(r, r.lag, r.small_last != 0, inst);
    r.nitems = (int)items.size();
    if (cudaMemcpy(r.d_items, items.data(), items.size() * sizeof(int4), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(r.d_inst, inst.data(), inst.size() * sizeof(int4), cudaMemcpyHostToDevice) != cudaSuccess)
        return FFT_ERR_CUDA;
    return FFT_OK;
}

RagArgs make_args(const RaggedState &r, const void *in, void *out, int dir, int *status) {
    RagArgs a;
    a.items = r.d_items;
    a.nitems = r.nitems;
    a.inst = r.d_inst;
    a.offs = r.d_offs;
    a.in = static_cast<const float2 *>(in);
    a.out = static_cast<float2 *>(out);
    a.head = r.d_counters;
    a.done = r.d_counters + 1;
    a.status = status;
    a.si = dir > 0 ? -1.f : 1.f;
    a.so = dir > 0 ? -1.f : 1.f;
    a.withhold = r.withhold;
    a.spin_limit_ns = r.spin_limit_ns;
    for (int k = 0; k < 11; ++k) a.tw.p[k] = r.d_tw[k];
    return a;
}

cudaError_t launch_ragged(const RaggedState &r, const RagArgs &a, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(r.d_counters, 0, sizeof(int) * (size_t)(r.count + 1), s);
    if (e != cudaSuccess) return e;
    void *args[] = {(void *)&a};
    return cudaLaunchKernel((const void *)k_ragged, dim3(r.grid), dim3(kRagThreads), args, kRagSmem, s);
}

// Captures memset + persistent launch into a graph for (in, out, dir).
int capture_graph(RaggedState &r, const void *in, void *out, int dir, int *status) {
    if (r.exec) {
        cudaGraphExecDestroy(r.exec);
        r.exec = nullptr;
    }
    if (r.graph) {
        cudaGraphDestroy(r.graph);
        r.graph = nullptr;
    }
    cudaStream_t cs;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return FFT_ERR_CUDA;
    const RagArgs a = make_args(r, in, out, dir, status);
    int rc = FFT_OK;
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) rc = FFT_ERR_CUDA;
    if (rc == FFT_OK) {
        const cudaError_t le = launch_ragged(r, a, cs);
        const cudaError_t ce = cudaStreamEndCapture(cs, &r.graph);
        if (le != cudaSuccess || ce != cudaSuccess) rc = FFT_ERR_CUDA;
    }
    if (rc == FFT_OK && cudaGraphInstantiate(&r.exec, r.graph, 0) != cudaSuccess) rc = FFT_ERR_CUDA;
    cudaStreamDestroy(cs);
    if (rc == FFT_OK) {
        r.g_in = in;
        r.g_out = out;
        r.g_dir = dir;
    }
    return rc;
}

}  // namespace

int ragged_run(fft_plan_s *p, const void *in, void *out, int dir, cudaStream_t s) {
    RaggedState &r = *p->ragged;
    if (!in || !out || (reinterpret_cast<uintptr_t>(in) & 15) || (reinterpret_cast<uintptr_t>(out) & 15))
        return FFT_ERR_INVALID_ARG;
    cudaSetDevice(p->device);
    if (!r.exec || r.g_in != in || r.g_out != out || r.g_dir != dir) {
        const int rc = capture_graph(r, in, out, dir, p->status);
        if (rc != FFT_OK) return rc;
    }
    return cudaGraphLaunch(r.exec, s) == cudaSuccess ? FFT_OK : FFT_ERR_CUDA;
}

int ragged_run_loop(fft_plan_s *p, const void *in, void *out, cudaStream_t s) {
    RaggedState &r = *p->ragged;
    if (!in || !out || (reinterpret_cast<uintptr_t>(in) & 15) || (reinterpret_cast<uintptr_t>(out) & 15))
        return FFT_ERR_INVALID_ARG;
    const float2 *src = static_cast<const float2 *>(in);
    float2 *dst = static_cast<float2 *>(out);
    for (int i = 0; i < r.count; ++i) {
        fft_plan_s *sp = r.shape_plans[{r.nx[i], r.ny[i]}];
        const int rc = run_dense(sp, src + r.offs[i], dst + r.offs[i], p->dir, nullptr, 1.f, s);
        if (rc != FFT_OK) return rc;
    }
    return FFT_OK;
}

// Times the graph launch for a few schedules and keeps the fastest.  Needs
// scratch buffers of the plan's size; runs at plan creation when asked for.
int ragged_autotune(fft_plan_s *p) {
    RaggedState &r = *p->ragged;
    float2 *a = nullptr, *b = nullptr;
    if (cudaMalloc(&a, r.total * sizeof(float2)) != cudaSuccess) return FFT_ERR_ALLOC;
    if (cudaMalloc(&b, r.total * sizeof(float2)) != cudaSuccess) {
        cudaFree(a);
        return FFT_ERR_ALLOC;
    }
    cudaMemset(a, 0, r.total * sizeof(float2));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int base_grid = r.grid;
    struct Cand {
        int lag, small_last, grid;
    };
    std::vector<Cand> cands;
    for (int lag : {0, base_grid / 2, base_grid, 2 * base_grid})
        for (int sl : {0, 1})
            for (int gdiv : {1, 2}) cands.push_back({lag, sl, base_grid / gdiv});
    float best = 1e30f;
    Cand bestc = {r.lag, r.small_last, r.grid};
    for (const Cand &c : cands) {
        r.lag = c.lag;
        r.small_last = c.small_last;
        r.grid = c.grid < 1 ? 1 : c.grid;
        if (upload_schedule(r) != FFT_OK) break;
        if (ragged_run(p, a, b, p->dir, 0) != FFT_OK) break;
        r.g_in = nullptr;  // force re-capture with the new schedule next time
        const RagArgs args = make_args(r, a, b, p->dir, p->status);
        for (int w = 0; w < 2; ++w) launch_ragged(r, args, 0);
        cudaEventRecord(e0, 0);
        for (int k = 0; k < 5; ++k) launch_ragged(r, args, 0);
        cudaEventRecord(e1, 0);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) {
            best = ms;
            bestc = c;
        }
    }
    r.lag = bestc.lag;
    r.small_last = bestc.small_last;
    r.grid = bestc.grid < 1 ? 1 : bestc.grid;
    const int rc = upload_schedule(r);
    r.g_in = nullptr;
    r.g_out = nullptr;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaDeviceSynchronize();
    cudaFree(a);
    cudaFree(b);
    int h = 0;
    cudaMemcpy(&h, p->status, sizeof(int), cudaMemcpyDeviceToHost);
    cudaMemset(p->status, 0, sizeof(int));
    return rc;
}

}  // namespace gb300fft

using namespace gb300fft;

extern "C" {

fft_plan_t fft_plan_create_ragged(int count, const int *nx, const int *ny, int dir, int precision) {
    set_last_error(FFT_OK);
    auto pow2_in = [](int n) { return n >= 32 && n <= 1024 && (n & (n - 1)) == 0; };
    if (count < 1) {
        set_last_error(FFT_ERR_INVALID_SIZE);
        return nullptr;
    }
    if (!nx || !ny || (dir != FFT_FORWARD && dir != FFT_INVERSE) ||
        (precision != FFT_PREC_FP32 && precision != FFT_PREC_SPLIT_FP16_TC)) {
        set_last_error(FFT_ERR_INVALID_ARG);
        return nullptr;
    }
    for (int i = 0; i < count; ++i)
        if (!pow2_in(nx[i]) || !pow2_in(ny[i])) {
            set_last_error(FFT_ERR_INVALID_SIZE);
            return nullptr;
        }
    if (precision != FFT_PREC_FP32) {
        set_last_error(FFT_ERR_UNSUPPORTED);
        return nullptr;
    }
    fft_plan_s *p = new (std::nothrow) fft_plan_s();
    RaggedState *r = new (std::nothrow) RaggedState();
    if (!p || !r) {
        delete p;
        delete r;
        set_last_error(FFT_ERR_ALLOC);
        return nullptr;
    }
    p->kind = 1;
    p->ragged = r;
    p->dir = dir;
    p->prec = precision;
    int rc = FFT_OK;
    if (cudaGetDevice(&p->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, p->device) != cudaSuccess)
        rc = FFT_ERR_CUDA;
    r->count = count;
    r->nx.assign(nx, nx + count);
    r->ny.assign(ny, ny + count);
    r->offs.resize(count + 1);
    r->offs[0] = 0;
    for (int i = 0; i < count; ++i) r->offs[i + 1] = r->offs[i] + (long long)nx[i] * ny[i];
    r->total = r->offs[count];
    if (const char *ev = getenv("GB300FFT_DEBUG_WITHHOLD")) r->withhold = atoi(ev);
    if (const char *ev = getenv("GB300FFT_SPIN_LIMIT_NS")) r->spin_limit_ns = atoll(ev);
    auto dalloc = [&](size_t bytes) -> void * {
        void *d = nullptr;
        if (cudaMalloc(&d, bytes) != cudaSuccess) return nullptr;
        r->allocs.push_back(d);
        return d;
    };
    if (rc == FFT_OK) {
        // upper bound on the item count: every instance split into rows + cols
        size_t max_items = 0;
        for (int i = 0; i < count; ++i) {
            const long long n = (long long)nx[i] * ny[i];
            max_items += n <= kRagItem ? 1 : (size_t)(ny[i] / (kRagItem / nx[i]) + nx[i] / (kRagItem / ny[i]));
        }
        r->d_items = static_cast<int4 *>(dalloc(max_items * sizeof(int4)));
        r->d_inst = static_cast<int4 *>(dalloc(count * sizeof(int4)));
        r->d_offs = static_cast<long long *>(dalloc((count + 1) * sizeof(long long)));
        r->d_counters = static_cast<int *>(dalloc((count + 1) * sizeof(int)));
        p->status = static_cast<int *>(dalloc(sizeof(int)));
        if (!r->d_items || !r->d_inst || !r->d_offs || !r->d_counters || !p->status) rc = FFT_ERR_ALLOC;
    }
    for (int l = 5; rc == FFT_OK && l <= 10; ++l) {
        int rad[16];
        const int S = schedule_radices(1 << l, kRagE, rad);
        long long sz = 0, ns = rad[0];
        for (int s2 = 1; s2 < S; ++s2) {
            sz += (long long)rad[s2] * ns;
            ns *= rad[s2];
        }
        r->d_tw[l] = static_cast<float2 *>(dalloc((size_t)(sz > 0 ? sz : 1) * sizeof(float2)));
        if (!r->d_tw[l]) rc = FFT_ERR_ALLOC;
        else if (build_twiddles(r->d_tw[l], 1 << l, kRagE, 0) != cudaSuccess) rc = FFT_ERR_CUDA;
    }
    if (rc == FFT_OK) {
        if (cudaMemcpy(r->d_offs, r->offs.data(), (count + 1) * sizeof(long long), cudaMemcpyHostToDevice) !=
                cudaSuccess ||
            cudaMemset(p->status, 0, sizeof(int)) != cudaSuccess)
            rc = FFT_ERR_CUDA;
    }
    if (rc == FFT_OK) {
        if (cudaFuncSetAttribute((const void *)k_ragged, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kRagSmem) != cudaSuccess)
            rc = FFT_ERR_CUDA;
        int per_sm = 0;
        if (rc == FFT_OK && (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void *)k_ragged,
                                                                           kRagThreads, kRagSmem) != cudaSuccess ||
                             per_sm < 1))
            rc = FFT_ERR_CUDA;
        r->grid = p->num_sms * per_sm;  // every CTA resident: required by the waits
        r->lag = r->grid;
        if (const char *ev = getenv("GB300FFT_RAGGED_LAG")) r->lag = atoi(ev);
    }
    if (rc == FFT_OK) rc = upload_schedule(*r);
    // the comparison baseline: one dense plan per distinct shape
    for (int i = 0; rc == FFT_OK && i < count; ++i) {
        auto key = std::make_pair(nx[i], ny[i]);
        if (r->shape_plans.count(key)) continue;
        fft_plan_t sp = fft_plan_create(nx[i], ny[i], 1, dir, FFT_PREC_FP32);
        if (!sp) rc = fft_last_error();
        else r->shape_plans[key] = sp;
    }
    if (rc == FFT_OK) {
        const char *ev = getenv("GB300FFT_AUTOTUNE");
        if (ev && atoi(ev) != 0) rc = ragged_autotune(p);
    }
    if (rc == FFT_OK && cudaDeviceSynchronize() != cudaSuccess) rc = FFT_ERR_CUDA;
    if (rc != FFT_OK) {
        free_plan(p);
        set_last_error(rc);
        return nullptr;
    }
    return p;
}

int fft_ragged_offset(fft_plan_t p, int i, long long *elem_offset) {
    if (!p || p->kind != 1 || !elem_offset || i < 0 || i > p->ragged->count) return FFT_ERR_INVALID_ARG;
    *elem_offset = p->ragged->offs[i];
    return FFT_OK;
}

int fft_execute_ragged(fft_plan_t p, const void *in, void *out, void *stream) {
    if (!p || p->kind != 1) return FFT_ERR_INVALID_ARG;
    return ragged_run(p, in, out, p->dir, static_cast<cudaStream_t>(stream));
}

int fft_execute_ragged_loop(fft_plan_t p, const void *in, void *out, void *stream) {
    if (!p || p->kind != 1) return FFT_ERR_INVALID_ARG;
    return ragged_run_loop(p, in, out, static_cast<cudaStream_t>(stream));
}

}  // extern "C"

namespace gb300fft {

// ---------------------------------------------------------------------------
// Ragged execution without any device allocation.
//
// Some callers cannot call cudaMalloc: processes whose device memory is
// owned by a pool or a framework allocator they must not bypass, and
// runtimes that forbid device allocation after start-up (everything is
// reserved up front so a long-running service cannot run out later).
// fft_execute_ragged_noalloc serves them: it runs
// the same persistent kernel as fft_execute_ragged, but its scratch (work
// queue, instance table, offsets, completion counters and twiddle tables)
// lives in the fixed array below instead of a plan.  The array is part of the
// library image, so every GPU that loads the library holds its
// kNoAllocBytes until the process exits.
// ---------------------------------------------------------------------------
constexpr int kNoAllocMaxCount = 1024;   // instances per call
constexpr int kNoAllocMaxItems = 131072;  // work items per call
constexpr size_t kNoAllocTwOffset = 0;   // twiddle tables, 4096 float2 (filled once per device)
constexpr size_t kNoAllocTwElems = 4096;
constexpr size_t kNoAllocItemsOffset = kNoAllocTwOffset + kNoAllocTwElems * sizeof(float2);
constexpr size_t kNoAllocInstOffset = kNoAllocItemsOffset + (size_t)kNoAllocMaxItems * sizeof(int4);
constexpr size_t kNoAllocOffsOffset = kNoAllocInstOffset + (size_t)kNoAllocMaxCount * sizeof(int4);
constexpr size_t kNoAllocCountersOffset = kNoAllocOffsOffset + (size_t)(kNoAllocMaxCount + 1) * sizeof(long long);
constexpr size_t kNoAllocBytes =
    (kNoAllocCountersOffset + (size_t)(kNoAllocMaxCount + 1) * sizeof(int) + 255) / 256 * 256;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

namespace {
constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mutex;
unsigned char *g_noalloc_ptr[kNoAllocMaxDevices] = {};  // device address of the array, per device
const float2 *g_noalloc_tw[kNoAllocMaxDevices][11] = {};

// Once per device, with that device current: look up the array's device
// address (the host-side symbol is only a stand-in) and fill the twiddle
// tables.  Returns FFT_OK or an error code.
int noalloc_setup(int dev, cudaStream_t s) {
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (g_noalloc_ptr[dev]) return FFT_OK;
    void *ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) return FFT_ERR_CUDA;
    unsigned char *base = static_cast<unsigned char *>(ptr);
    float2 *tw = reinterpret_cast<float2 *>(base + kNoAllocTwOffset);
    size_t used = 0;
    for (int l = 5; l <= 10; ++l) {
        int rad[16];
        const int S = schedule_radices(1 << l, kRagE, rad);
        long long sz = 0, ns = rad[0];
        for (int k = 1; k < S; ++k) {
            sz += (long long)rad[k] * ns;
            ns *= rad[k];
        }
        if (used + (size_t)sz > kNoAllocTwElems) return FFT_ERR_UNSUPPORTED;
        g_noalloc_tw[dev][l] = tw + used;
        if (sz > 0 && build_twiddles(tw + used, 1 << l, kRagE, s) != cudaSuccess) return FFT_ERR_CUDA;
        used += (size_t)sz;
    }
    if (cudaStreamSynchronize(s) != cudaSuccess) return FFT_ERR_CUDA;
    g_noalloc_ptr[dev] = base;
    return FFT_OK;
}
}  // namespace

}  // namespace gb300fft (no-alloc helpers)

extern "C" int fft_execute_ragged_noalloc(int count, const int *nx, const int *ny, int dir, const void *in, void *out,
                                          int *status, void *stream) {
    using namespace gb300fft;
    auto pow2_in = [](int n) { return n >= 32 && n <= 1024 && (n & (n - 1)) == 0; };
    if (count < 1 || count > kNoAllocMaxCount) return FFT_ERR_INVALID_SIZE;
    if (!nx || !ny || !in || !out || (dir != FFT_FORWARD && dir != FFT_INVERSE)) return FFT_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(in) & 15) || (reinterpret_cast<uintptr_t>(out) & 15)) return FFT_ERR_INVALID_ARG;
    for (int i = 0; i < count; ++i)
        if (!pow2_in(nx[i]) || !pow2_in(ny[i])) return FFT_ERR_INVALID_SIZE;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int dev = 0;
    int sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return FFT_ERR_CUDA;
    const int rc0 = noalloc_setup(dev, s);
    if (rc0 != FFT_OK) return rc0;
    unsigned char *base = g_noalloc_ptr[dev];

    // host-side schedule (same rules as a ragged plan)
    RaggedState r;
    r.count = count;
    r.nx.assign(nx, nx + count);
    r.ny.assign(ny, ny + count);
    r.offs.resize(count + 1);
    r.offs[0] = 0;
    for (int i = 0; i < count; ++i) r.offs[i + 1] = r.offs[i] + (long long)nx[i] * ny[i];
    int per_sm = 0;
    if (cudaFuncSetAttribute((const void *)k_ragged, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRagSmem) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void *)k_ragged, kRagThreads, kRagSmem) !=
            cudaSuccess ||
        per_sm < 1)
        return FFT_ERR_CUDA;
    r.grid = sms * per_sm;
    std::vector<int4> inst;
    const std::vector<int4> items = build_items(r, r.grid, true, inst);
    if (items.size() > (size_t)kNoAllocMaxItems) return FFT_ERR_INVALID_SIZE;

    int4 *d_items = reinterpret_cast<int4 *>(base + kNoAllocItemsOffset);
    int4 *d_inst = reinterpret_cast<int4 *>(base + kNoAllocInstOffset);
    long long *d_offs = reinterpret_cast<long long *>(base + kNoAllocOffsOffset);
    int *d_counters = reinterpret_cast<int *>(base + kNoAllocCountersOffset);
    // pageable sources: each copy returns once the host data has been staged
    if (cudaMemcpyAsync(d_items, items.data(), items.size() * sizeof(int4), cudaMemcpyHostToDevice, s) !=
            cudaSuccess ||
        cudaMemcpyAsync(d_inst, inst.data(), inst.size() * sizeof(int4), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(d_offs, r.offs.data(), (count + 1) * sizeof(long long), cudaMemcpyHostToDevice, s) !=
            cudaSuccess ||
        cudaMemsetAsync(d_counters, 0, (count + 1) * sizeof(int), s) != cudaSuccess)
        return FFT_ERR_CUDA;
    RagArgs a;
    a.items = d_items;
    a.nitems = (int)items.size();
    a.inst = d_inst;
    a.offs = d_offs;
    a.in = static_cast<const float2 *>(in);
    a.out = static_cast<float2 *>(out);
    a.head = d_counters;
    a.done = d_counters + 1;
    a.status = status;
    a.si = dir > 0 ? -1.f : 1.f;
    a.so = dir > 0 ? -1.f : 1.f;
    a.withhold = 0;
    a.spin_limit_ns = 1000000000LL;
    for (int k = 0; k < 11; ++k) a.tw.p[k] = g_noalloc_tw[dev][k];
    void *args[] = {(void *)&a};
    if (cudaLaunchKernel((const void *)k_ragged, dim3(r.grid), dim3(kRagThreads), args, kRagSmem, s) != cudaSuccess)
        return FFT_ERR_CUDA;
    return FFT_OK;
}
