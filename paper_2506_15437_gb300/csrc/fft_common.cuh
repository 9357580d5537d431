// Device building blocks shared by the gb300fft kernels (sm_103a).
//
// The transform is the radix-2^k Cooley-Tukey FFT of the paper's Section 2.2
// (Fig. 2, Listing 1) in its self-sorting (Stockham) arrangement: every
// butterfly stage reads its operands in the order that stage needs and writes
// its results straight into the order the NEXT stage needs.  That is the
// paper's "one reordering per step" idea (Section 4, Fig. 5) taken to its end
// point: the reordering is the address arithmetic of the stage's loads and
// stores, the intermediate orders live only in shared memory and registers,
// and no separate bit-reversal pass or HBM round trip exists.
//
// Twiddle tables: stage s >= 1 (radix R, span Ns) stores, for pair k < R/2
// and m < Ns, the float4 (w^{(2k+1) m}, w^{(2k+2) m}) with w = w_{Ns*R}, at
// float4 index k*Ns + m, so a warp's threads (consecutive m) load adjacent
// 16-byte words.
//
// Stage s of a length-N transform has radix R and span Ns = R_0 * ... * R_{s-1}.
// Butterfly j (0 <= j < N/R), with m = j mod Ns, reads a_r = d[j + r*N/R],
// multiplies a_r by w_{Ns*R}^{r*m} (w_K = exp(-2*pi*i/K)), takes the length-R
// DFT b_k = sum_r a_r w_R^{r*k}, and writes b_k to d'[(j - m)*R + m + k*Ns].
// The first stage (Ns = 1) needs no twiddles; the last one (Ns*R = N) writes
// natural order.  The inverse direction is computed as conj(F(conj(x))), so
// all tables and constants are for the forward sign only.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace gb300fft {

// Device status word codes (same values as the C ABI's FFT_ERR_*).
constexpr int kStatusOk = 0;
constexpr int kStatusTimeout = -6;

__host__ __device__ constexpr int ilog2(int n) { return n <= 1 ? 0 : 1 + ilog2(n >> 1); }
__host__ __device__ constexpr int ipow(int b, int e) { return e == 0 ? 1 : b * ipow(b, e - 1); }

// ---------------------------------------------------------------------------
// Complex arithmetic on float2 (x = re, y = im).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

// sin(2*pi*q/64) for 0 <= q <= 16, rounded to float (compile-time constants).
__host__ __device__ constexpr float qsin64(int q) {
    return q == 0    ? 0.0f
           : q == 1  ? 0.0980171403295606f
           : q == 2  ? 0.19509032201612825f
           : q == 3  ? 0.29028467725446233f
           : q == 4  ? 0.3826834323650898f
           : q == 5  ? 0.47139673682599764f
           : q == 6  ? 0.5555702330196022f
           : q == 7  ? 0.6343932841636455f
           : q == 8  ? 0.7071067811865475f
           : q == 9  ? 0.773010453362737f
           : q == 10 ? 0.8314696123025452f
           : q == 11 ? 0.8819212643483549f
           : q == 12 ? 0.9238795325112867f
           : q == 13 ? 0.9569403357322089f
           : q == 14 ? 0.9807852804032304f
           : q == 15 ? 0.9951847266721968f
                     : 1.0f;
}
// sin and cos of 2*pi*q/64 for any integer q, by quadrant symmetry.
__host__ __device__ constexpr float sin64(int q) {
    return (q & 63) < 16   ? qsin64(q & 63)
           : (q & 63) < 32 ? qsin64(32 - (q & 63))
           : (q & 63) < 48 ? -qsin64((q & 63) - 32)
                           : -qsin64(64 - (q & 63));
}
__host__ __device__ constexpr float cos64(int q) { return sin64(q + 16); }

// z * exp(-2*pi*i*q/64).  q is a compile-time constant after unrolling, so the
// branches fold: multiples of pi/2 become swaps and sign flips, odd multiples
// of pi/4 cost two adds and two multiplies, the rest a complex multiply by
// immediate constants.
__device__ __forceinline__ float2 mul_root64(float2 z, int q) {
    q &= 63;
    if (q == 0) return z;
    if (q == 16) return make_float2(z.y, -z.x);
    if (q == 32) return make_float2(-z.x, -z.y);
    if (q == 48) return make_float2(-z.y, z.x);
    if ((q & 15) == 8) {
        const float h = 0.7071067811865475f;
        if (q == 8) return make_float2((z.x + z.y) * h, (z.y - z.x) * h);
        if (q == 24) return make_float2((z.y - z.x) * h, (-z.x - z.y) * h);
        if (q == 40) return make_float2((-z.x - z.y) * h, (z.x - z.y) * h);
        return make_float2((z.x - z.y) * h, (z.x + z.y) * h);
    }
    const float c = cos64(q), s = sin64(q);
    return make_float2(fmaf(z.x, c, z.y * s), fmaf(z.y, c, -z.x * s));
}

__host__ __device__ constexpr int bitrev(int k, int bits) {
    return bits == 0 ? 0 : ((k & 1) << (bits - 1)) | bitrev(k >> 1, bits - 1);
}

// One radix-2 decimation-in-frequency level of span H over R registers:
// (u, v) -> (u + v, (u - v) * w_{2H}^k).  Levels recurse at compile time so
// every register index and twiddle is a constant.
template <int R, int H>
__device__ __forceinline__ void dif_level(float2 *a) {
    if constexpr (H >= 1) {
#pragma unroll
        for (int blk = 0; blk < R; blk += 2 * H) {
#pragma unroll
            for (int k = 0; k < H; ++k) {
                const float2 u = a[blk + k], v = a[blk + k + H];
                a[blk + k] = cadd(u, v);
                a[blk + k + H] = mul_root64(csub(u, v), k * (64 / (2 * H)));
            }
        }
        dif_level<R, H / 2>(a);
    }
}

// a[K] = t[bitrev(K)] for K = 0..R-1, every index a constant expression.
template <int R, int K>
__device__ __forceinline__ void bitrev_gather(float2 *a, const float2 *t) {
    if constexpr (K < R) {
        constexpr int src = bitrev(K, ilog2(R));
        a[K] = t[src];
        bitrev_gather<R, K + 1>(a, t);
    }
}

// In-register length-R DFT (forward sign), natural order in and out,
// R a power of two <= 64: radix-2 DIF levels, then a compile-time
// bit-reversal of register names.
template <int R>
__device__ __forceinline__ void dft(float2 *a) {
    if constexpr (R > 1) {
        dif_level<R, R / 2>(a);
        float2 t[R];
#pragma unroll
        for (int k = 0; k < R; ++k) t[k] = a[k];
        bitrev_gather<R, 0>(a, t);
    }
}

// ---------------------------------------------------------------------------
// Stage schedule of a length-N transform with E elements held per thread:
// first stage radix R0 = N / E^(S-1) (absorbs the remainder), then S-1
// stages of radix E.  Requires E <= N, both powers of two.
// ---------------------------------------------------------------------------
template <int N, int E>
struct Sched {
    static_assert(E <= N, "E must not exceed N");
    static constexpr int L = ilog2(N);
    static constexpr int LE = ilog2(E);
    static constexpr int S = (L + LE - 1) / LE > 0 ? (L + LE - 1) / LE : 1;
    static constexpr int R0 = N >> (LE * (S - 1));
    // span Ns of stage s
    static constexpr int ns(int s) { return s == 0 ? 1 : R0 * ipow(E, s - 1); }
    // offset of stage s's twiddle table in float2 units (stage 1 starts at
    // 0); a stage of radix R and span Ns holds R/2 float4 pairs per m
    static constexpr int tw_off(int s) { return s <= 1 ? 0 : tw_off(s - 1) + E * ns(s - 1); }
    static constexpr int tw_size = tw_off(S);
};

// ---------------------------------------------------------------------------
// Payload policies.  The FFT moves float2 and runs DFTs; the reorder-map debug
// path moves integer tags through exactly the same addresses with identity
// butterflies, which exposes the permutation the data movement realises.
// ---------------------------------------------------------------------------
struct FftPolicy {
    using T = float2;
    static constexpr bool kUsesTwiddles = true;
    template <int R>
    __device__ __forceinline__ void butterfly(T *a) const { dft<R>(a); }
    __device__ __forceinline__ T twiddle(T a, float2 w) const { return cmul(a, w); }
};
struct MovePolicy {
    using T = float2;  // integer tags carried bit-for-bit in the .x lane
    static constexpr bool kUsesTwiddles = false;
    template <int R>
    __device__ __forceinline__ void butterfly(T *) const {}
    __device__ __forceinline__ T twiddle(T a, float2) const { return a; }
};

struct SyncBlock {
    __device__ __forceinline__ void operator()() const { __syncthreads(); }
};
struct SyncWarp {
    __device__ __forceinline__ void operator()() const { __syncwarp(); }
};

// ---------------------------------------------------------------------------
// The Stockham engine.  A group of NT = W*N/E threads transforms W
// interleaved length-N vectors held in shared memory at element (i, c) ->
// padded flat index pad(i*W + c).  Thread t of the group owns column
// c = t % W and butterfly index tt = t / W.
//
// Caller contract: v[] holds the stage-0 inputs, v[b*R0 + r] = x[j + r*N/R0]
// for j = tt + b*(N/E).  `after_reads()` runs once every thread has issued its
// last shared-memory read (it must synchronise the group if it reuses the
// buffer); `store(i, c, value)` receives the natural-order outputs.
// SRC_IN_SMEM: stage-0 inputs were read from `sm` itself, so the first
// shared-memory write must wait for every thread's reads.
// ---------------------------------------------------------------------------
template <int N, int E, int W, int PADSH, int PADSH1 = PADSH>
struct Engine {
    using Sc = Sched<N, E>;
    static constexpr int T = N / E;   // threads per column
    static constexpr int NT = T * W;  // threads per group
    static constexpr int R0 = Sc::R0;
    static constexpr int S = Sc::S;
    static constexpr int RL = (S == 1) ? R0 : E;  // radix of the last stage
    // padded index of the exchange after stage s - 1: the first exchange may
    // use its own shift (PADSH1), since its write pattern follows radix R0
    __host__ __device__ static constexpr int pad(int f) { return f + (f >> PADSH); }
    __host__ __device__ static constexpr int pad_s(int f, int s) { return f + (f >> (s == 1 ? PADSH1 : PADSH)); }
    static constexpr int SMEM_ELEMS =
        (S > 1) ? (pad_s(N * W - 1, 1) > pad(N * W - 1) ? pad_s(N * W - 1, 1) : pad(N * W - 1)) + 1 : 0;

    template <class Pol, bool SRC_IN_SMEM, class Sync, class AfterReads, class Store>
    __device__ static __forceinline__ void run(typename Pol::T (&v)[E], typename Pol::T *sm,
                                               const float2 *__restrict__ tw, int tt, int c,
                                               Sync sync, AfterReads after_reads, Store store) {
        run_with<Pol, SRC_IN_SMEM>(Pol{}, v, sm, tw, tt, c, sync, after_reads, store);
    }

    // Same, with a policy object (a stateful butterfly, e.g. the tensor-core one).
    template <class Pol, bool SRC_IN_SMEM, class Sync, class AfterReads, class Store>
    __device__ static __forceinline__ void run_with(const Pol &pol, typename Pol::T (&v)[E], typename Pol::T *sm,
                                                    const float2 *__restrict__ tw, int tt, int c, Sync sync,
                                                    AfterReads after_reads, Store store) {
        using V = typename Pol::T;
        // stage 0: butterflies in registers, no twiddles
#pragma unroll
        for (int b = 0; b < E / R0; ++b) pol.template butterfly<R0>(&v[b * R0]);
        if constexpr (S == 1) {
            after_reads();
        } else {
#pragma unroll
            for (int s = 1; s < S; ++s) {
                const int Rp = (s == 1) ? R0 : E;  // radix of stage s-1
                const int Nsp = Sc::ns(s - 1);     // span of stage s-1
                if (s > 1 || SRC_IN_SMEM) sync();
#pragma unroll
                for (int b = 0; b < E / Rp; ++b) {
                    const int j = tt + b * T;
                    const int m = j & (Nsp - 1);
#pragma unroll
                    for (int k = 0; k < Rp; ++k) sm[pad_s(((j - m) * Rp + m + k * Nsp) * W + c, s)] = v[b * Rp + k];
                }
                sync();
                const int Ns = Sc::ns(s);
                const int m = tt & (Ns - 1);
#pragma unroll
                for (int r = 0; r < E; ++r) v[r] = sm[pad_s((tt + r * T) * W + c, s)];
                if (s == S - 1) after_reads();
                if constexpr (Pol::kUsesTwiddles) {
                    // twiddles r = 2k+1, 2k+2 of this butterfly in one 16-byte load
                    const float4 *tws = reinterpret_cast<const float4 *>(tw + Sc::tw_off(s)) + m;
#pragma unroll
                    for (int k = 0; k < E / 2; ++k) {
                        const float4 w2 = __ldg(tws + k * Ns);
                        v[2 * k + 1] = pol.twiddle(v[2 * k + 1], make_float2(w2.x, w2.y));
                        if (2 * k + 2 < E) v[2 * k + 2] = pol.twiddle(v[2 * k + 2], make_float2(w2.z, w2.w));
                    }
                }
                pol.template butterfly<E>(v);
            }
        }
        // natural-order outputs of the last stage: position j + k*N/RL
#pragma unroll
        for (int b = 0; b < E / RL; ++b) {
            const int j = tt + b * T;
#pragma unroll
            for (int k = 0; k < RL; ++k) store(j + k * (N / RL), c, v[b * RL + k]);
        }
    }
};

// Shared-memory padding shift used by every kernel for a given E: chosen so
// that the stage loads and stores of the common shapes hit each bank pair at
// most once per half-warp (checked by a bank model on the CPU).
template <int E>
struct PadShift {
    static constexpr int value = (E >= 64) ? 6 : (E >= 32) ? 5 : 4;
};
// First-exchange shift of the one-row engines (W = 1): with E = 32 the write
// after the radix-4/8 first stage puts 16 lanes 8 or 4 float2 apart, which
// a shift of 4 spreads over all banks (half-warp bank model; shift 5 leaves
// 2-way conflicts there).
template <int E>
struct RowPadShift1 {
    static constexpr int value = (E == 32) ? 4 : PadShift<E>::value;
};

// ---------------------------------------------------------------------------
// TMA / mbarrier helpers (inline PTX).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}
// Bounded wait on an mbarrier phase: gives up after ~`limit_ns` nanoseconds
// (or 2^26 polls) and returns false.  Never spins forever.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity,
                                                  uint64_t limit_ns = 2000000000ull) {
    const uint64_t t0 = globaltimer_ns();
    for (uint32_t it = 0; it < (1u << 26); ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 255) == 255 && globaltimer_ns() - t0 > limit_ns) break;
    }
    return false;
}
// 2D tiled TMA load of one box into shared memory, completing on `bar`.
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y,
                                            uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}
// 3D tiled TMA load (coordinates innermost first).
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int x, int y, int z,
                                            uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void tma_prefetch_3d(const CUtensorMap *map, int x, int y, int z) {
    asm volatile("cp.async.bulk.prefetch.tensor.3d.L2.global.tile [%0, {%1, %2, %3}];" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(x), "r"(y), "r"(z)
                 : "memory");
}
// 1D bulk copy global -> shared (16-byte aligned, size a multiple of 16),
// completing on `bar`.
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
// 4D tiled TMA store of one box from shared memory (coordinates innermost
// first), tracked in the issuing thread's bulk async-group.
__device__ __forceinline__ void tma_store_4d(const CUtensorMap *map, const void *src, int x, int y, int z, int w) {
    asm volatile(
        "cp.async.bulk.tensor.4d.global.shared::cta.bulk_group [%0, {%1, %2, %3, %4}], [%5];" ::"l"(
            reinterpret_cast<uint64_t>(map)),
        "r"(x), "r"(y), "r"(z), "r"(w), "r"(smem_u32(src))
        : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// Wait until at most one of this thread's bulk groups still reads shared memory.
__device__ __forceinline__ void bulk_wait_read_1() { asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory"); }
// Wait until every bulk group this thread issued has completed.
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// Prefetch of one box into L2 (no shared memory involved).
__device__ __forceinline__ void tma_prefetch_2d(const CUtensorMap *map, int x, int y) {
    asm volatile("cp.async.bulk.prefetch.tensor.2d.L2.global.tile [%0, {%1, %2}];" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(x), "r"(y)
                 : "memory");
}

// Bulk prefetch of a contiguous byte range into L2 (16-byte aligned address,
// size a multiple of 16).
__device__ __forceinline__ void bulk_prefetch_l2(const void *p, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(reinterpret_cast<uint64_t>(p)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void record_status(int *status, int code) {
    if (status) atomicCAS(status, kStatusOk, code);
}

}  // namespace gb300fft
