// Precision policies, float-float arithmetic and the row-tile machinery shared
// by the per-step kernels.
//
// On GB300 a float64 warp instruction occupies the FP64 pipe of an SM
// sub-partition for ~64 cycles (about 1/64 of the float32 rate), so the mixed
// path issues no float64 instructions per matrix entry or per vector element:
// quantities that need more than float32 (state vectors, float64-quality
// residuals, dot products) are carried as unevaluated sums of two floats
// ("float-float", ~48 significant bits) with the error-free transformations of
// Dekker (1971) and Knuth (TAOCP vol. 2, 4.2.2): two_sum, two_prod.
#pragma once

#include <cuda_runtime.h>

#include <type_traits>

#include "internal.cuh"

namespace oasis {

// ------------------------------------------------------------------ float-float
struct __align__(8) ff {
    float hi, lo;
};

// s + e == a + b exactly (Knuth).  No multiplications, so no FMA contraction.
__device__ __forceinline__ ff two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    const float e = (a - (s - bb)) + (b - bb);
    return {s, e};
}
// requires |a| >= |b| (Dekker)
__device__ __forceinline__ ff fast_two_sum(float a, float b) {
    const float s = a + b;
    const float e = b - (s - a);
    return {s, e};
}
// p + e == a * b exactly (the FMA gives the rounding error of the product)
__device__ __forceinline__ ff two_prod(float a, float b) {
    const float p = a * b;
    const float e = __fmaf_rn(a, b, -p);
    return {p, e};
}
__device__ __forceinline__ ff ff_add(ff a, ff b) {
    ff s = two_sum(a.hi, b.hi);
    const ff t = two_sum(a.lo, b.lo);
    s.lo += t.hi;
    s = fast_two_sum(s.hi, s.lo);
    s.lo += t.lo;
    return fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ ff ff_neg(ff a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ ff ff_sub(ff a, ff b) { return ff_add(a, ff_neg(b)); }
__device__ __forceinline__ ff ff_mul_f(ff a, float b) {
    ff p = two_prod(a.hi, b);
    p.lo = __fmaf_rn(a.lo, b, p.lo);
    return fast_two_sum(p.hi, p.lo);
}
// a + b * c with b * c formed exactly
__device__ __forceinline__ ff ff_fma_f(ff a, float b, float c) { return ff_add(a, two_prod(b, c)); }
__device__ __forceinline__ double ff_to_double(ff a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ ff ff_from_double(double d) {
    const float hi = (float)d;
    return {hi, (float)(d - (double)hi)};
}

// ------------------------------------------------------------------ policies
// S: storage/arithmetic type of the state and of float64-quality quantities
// V: type of matrix values and inner Krylov vectors
// Acc: dot-product accumulator
struct Fp64 {
    using V = double;
    using S = double;
    using Acc = double;
    static constexpr bool mixed = false;
};
struct Mixed {
    using V = float;
    using S = float2;      // (hi, lo) float-float
    using Acc = ff;
    static constexpr bool mixed = true;
};

// state arithmetic (double or float-float stored as float2)
__device__ __forceinline__ double s_add(double a, double b) { return a + b; }
__device__ __forceinline__ float2 s_add(float2 a, float2 b) {
    const ff r = ff_add({a.x, a.y}, {b.x, b.y});
    return make_float2(r.hi, r.lo);
}
__device__ __forceinline__ double s_sub(double a, double b) { return a - b; }
__device__ __forceinline__ float2 s_sub(float2 a, float2 b) {
    const ff r = ff_sub({a.x, a.y}, {b.x, b.y});
    return make_float2(r.hi, r.lo);
}
__device__ __forceinline__ double s_mul(double a, double b) { return a * b; }
__device__ __forceinline__ float2 s_mul(float2 a, float b) {
    const ff r = ff_mul_f({a.x, a.y}, b);
    return make_float2(r.hi, r.lo);
}
__device__ __forceinline__ double s_addv(double a, double v) { return a + v; }   // a + V
__device__ __forceinline__ float2 s_addv(float2 a, float v) {
    const ff r = ff_add({a.x, a.y}, {v, 0.f});
    return make_float2(r.hi, r.lo);
}
__device__ __forceinline__ double s_v(double a) { return a; }                    // round to V
__device__ __forceinline__ float s_v(float2 a) { return a.x + a.y; }
template <class S> __device__ __forceinline__ S s_zero();
template <> __device__ __forceinline__ double s_zero<double>() { return 0.0; }
template <> __device__ __forceinline__ float2 s_zero<float2>() { return make_float2(0.f, 0.f); }
__device__ __forceinline__ double s_from(double v) { return v; }                 // V -> S
__device__ __forceinline__ float2 s_from(float v) { return make_float2(v, 0.f); }
// S <-> float64 (used only at the API boundary and in once-per-solve scalars)
__device__ __forceinline__ double s_to_double(double a) { return a; }
__device__ __forceinline__ double s_to_double(float2 a) { return (double)a.x + (double)a.y; }
template <class S> __device__ __forceinline__ S s_of_double(double d);
template <> __device__ __forceinline__ double s_of_double<double>(double d) { return d; }
template <> __device__ __forceinline__ float2 s_of_double<float2>(double d) {
    const ff r = ff_from_double(d);
    return make_float2(r.hi, r.lo);
}
// product of two S values rounded to V (for norms of S quantities)
__device__ __forceinline__ ff s_ff(float2 a) { return {a.x, a.y}; }
// S * S (float-float product to ~float-float accuracy)
__device__ __forceinline__ double s_mul_s(double a, double b) { return a * b; }
__device__ __forceinline__ float2 s_mul_s(float2 a, float2 b) {
    ff p = two_prod(a.x, b.x);
    p.lo = __fmaf_rn(a.x, b.y, __fmaf_rn(a.y, b.x, p.lo));
    p = fast_two_sum(p.hi, p.lo);
    return make_float2(p.hi, p.lo);
}

// accumulators
__device__ __forceinline__ void acc_zero(double& a) { a = 0.0; }
__device__ __forceinline__ void acc_zero(ff& a) { a = {0.f, 0.f}; }
__device__ __forceinline__ void acc_prod(double& a, double x, double y) { a = fma(x, y, a); }
__device__ __forceinline__ void acc_prod(ff& a, float x, float y) { a = ff_fma_f(a, x, y); }
__device__ __forceinline__ void acc_add(double& a, double b) { a += b; }
__device__ __forceinline__ void acc_add(ff& a, ff b) { a = ff_add(a, b); }
__device__ __forceinline__ void acc_addv(double& a, double b) { a += b; }
__device__ __forceinline__ void acc_addv(ff& a, float b) { a = ff_add(a, {b, 0.f}); }
__device__ __forceinline__ double acc_double(double a) { return a; }
__device__ __forceinline__ double acc_double(ff a) { return ff_to_double(a); }
__device__ __forceinline__ double acc_shfl(double a, int o) { return __shfl_xor_sync(0xffffffffu, a, o); }
__device__ __forceinline__ ff acc_shfl(ff a, int o) {
    return {__shfl_xor_sync(0xffffffffu, a.hi, o), __shfl_xor_sync(0xffffffffu, a.lo, o)};
}

// Block-wide sum of NV accumulators (float-float or double), valid in thread 0.
// Fixed shuffle/shared-memory tree: deterministic.  Any block size up to 1024.
template <int NV, class A>
__device__ __forceinline__ void block_reduce(A (&v)[NV]) {
    static_assert(NV <= 8, "too many reduction values");
    __shared__ A sh[NV][32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (int)(blockDim.x >> 5);
#pragma unroll
    for (int k = 0; k < NV; ++k) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc_add(v[k], acc_shfl(v[k], o));
        if (lane == 0) sh[k][wid] = v[k];
    }
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            A x;
            acc_zero(x);
            if (lane < nw) x = sh[k][lane];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc_add(x, acc_shfl(x, o));
            v[k] = x;
        }
    }
    __syncthreads();
}

// The block's ticket of a last-block reduction, taken by the thread that wrote
// the block's partials: an atomic increment with release semantics (those
// writes become visible no later than the ticket) and acquire semantics.  True
// in the block that takes the last ticket; that block still fences before it
// reads the other blocks' partials.
__device__ __forceinline__ bool take_last_ticket(uint32_t* ticket) {
    uint32_t old;
    asm volatile("atom.add.acq_rel.gpu.u32 %0, [%1], 1;" : "=r"(old) : "l"(ticket) : "memory");
    return old == gridDim.x - 1;
}

// Deterministic grid reduction: every block publishes its NV partial sums; the
// block taking the last ticket sums them in block order.  Returns true in that
// block; its thread 0 then holds the totals (converted to double) in `tot`.
// The ticket is reset for the next launch.  `partial` holds gridDim.x * NV
// accumulators.
template <int NV, class A>
__device__ __forceinline__ bool grid_sum(A (&v)[NV], double (&tot)[NV], void* partial_raw, uint32_t* ticket) {
    A* partial = reinterpret_cast<A*>(partial_raw);
    block_reduce<NV, A>(v);
    __shared__ bool last;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) partial[(size_t)blockIdx.x * NV + k] = v[k];
        last = take_last_ticket(ticket);
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
    A s[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) acc_zero(s[k]);
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            A x;
            if constexpr (std::is_same<A, double>::value) {
                x = __ldcg(reinterpret_cast<const double*>(&partial[(size_t)b * NV + k]));
            } else {
                const float2 f = __ldcg(reinterpret_cast<const float2*>(&partial[(size_t)b * NV + k]));
                x = *reinterpret_cast<const A*>(&f);
            }
            acc_add(s[k], x);
        }
    }
    block_reduce<NV, A>(s);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) tot[k] = acc_double(s[k]);
        *ticket = 0u;
    }
    return true;
}

// Deterministic grid sum for the per-iteration Krylov scalars (dot products of
// the inner solves).  T is the kernel's value type: double in the float64 path;
// float in the mixed path, where each thread's products and its running sum over
// its rows stay float32 and the 32 lanes of a warp are summed by a float32
// shuffle tree (pairwise), while every sum above the warp -- the block's partial
// over its warps and the sum of the blocks' partials -- is carried in
// float-float (~48 bits), so the totals reach float64 quality however many
// blocks there are.  A float-float partial costs a few dozen float
// instructions per value in one warp per block (a float64 instruction is ~1/64
// of the float32 rate on GB300 and would cost microseconds per reduction).
// Partial storage per value: double (T = double) or float2 (hi, lo).
template <class T>
struct LiteAcc {
    using type = double;
};
template <>
struct LiteAcc<float> {
    using type = ff;
};
__device__ __forceinline__ double lite_of(double x) { return x; }
__device__ __forceinline__ ff lite_of(float x) { return {x, 0.f}; }
__device__ __forceinline__ double lite_load(const double* p) { return __ldcg(p); }
__device__ __forceinline__ ff lite_load(const ff* p) {
    const float2 f = __ldcg(reinterpret_cast<const float2*>(p));
    return {f.x, f.y};
}

// Stage 1: the block's sum of v stored as partial[index][0..NV) (type
// LiteAcc<T>::type).  Every thread of the block calls it; on return the shared
// scratch may be reused.
template <int NV, class T>
__device__ __forceinline__ void block_partial_lite(T (&v)[NV], void* partial_raw, int64_t index) {
    using A = typename LiteAcc<T>::type;
    A* partial = reinterpret_cast<A*>(partial_raw);
    __shared__ T sh[NV][32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (int)(blockDim.x >> 5);
#pragma unroll
    for (int k = 0; k < NV; ++k) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
        if (lane == 0) sh[k][wid] = v[k];
    }
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            A x = lite_of(lane < nw ? sh[k][lane] : (T)0);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc_add(x, acc_shfl(x, o));
            if (lane == 0) partial[(size_t)index * NV + k] = x;
        }
    }
    __syncthreads();
}

// Stage 2: after the block has stored its partials, the block that takes the
// last ticket sums all `count` partials in LiteAcc precision (order fixed by the
// block size) and returns true with the totals; the ticket is reset for the
// next use.
template <int NV, class T>
__device__ __forceinline__ bool grid_finish_lite(double (&tot)[NV], const void* partial_raw, int64_t count,
                                                 uint32_t* ticket) {
    using A = typename LiteAcc<T>::type;
    const A* partial = reinterpret_cast<const A*>(partial_raw);
    __shared__ A sh[NV][32];
    __shared__ bool last;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (int)(blockDim.x >> 5);
    if (threadIdx.x == 0) last = take_last_ticket(ticket);
    __syncthreads();
    if (!last) return false;
    __threadfence();
    A s[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) acc_zero(s[k]);
    // the partials are read 4 per thread at a time (independent loads in
    // flight) and added in the same order as a plain strided loop would
    const int64_t G = count, B = (int64_t)blockDim.x;
    int64_t b = threadIdx.x;
    for (; b + 3 * B < G; b += 4 * B) {
        A x[4][NV];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int k = 0; k < NV; ++k) x[u][k] = lite_load(&partial[(size_t)(b + u * B) * NV + k]);
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int k = 0; k < NV; ++k) acc_add(s[k], x[u][k]);
    }
    for (; b < G; b += B) {
#pragma unroll
        for (int k = 0; k < NV; ++k) acc_add(s[k], lite_load(&partial[(size_t)b * NV + k]));
    }
#pragma unroll
    for (int k = 0; k < NV; ++k) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc_add(s[k], acc_shfl(s[k], o));
        if (lane == 0) sh[k][wid] = s[k];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            A x;
            acc_zero(x);
            for (int w = 0; w < nw; ++w) acc_add(x, sh[k][w]);
            tot[k] = acc_double(x);
        }
        *ticket = 0u;
    }
    return true;
}

// One partial per block, then the last block sums them.
template <int NV, class T>
__device__ __forceinline__ bool grid_sum_lite(T (&v)[NV], double (&tot)[NV], void* partial_raw, uint32_t* ticket) {
    block_partial_lite<NV, T>(v, partial_raw, blockIdx.x);
    return grid_finish_lite<NV, T>(tot, partial_raw, gridDim.x, ticket);
}

// Limit of every bounded device-side wait (~2 s at 2 GHz).
constexpr long long kBarrierLimitCycles = 4000000000LL;

// ------------------------------------------------------------------ TMA bulk copies
// 1D bulk copies global -> shared (cp.async.bulk, the Blackwell/Hopper TMA engine)
// completing on an mbarrier.  Source and destination must be 16-byte aligned and
// the size a multiple of 16 bytes; callers copy aligned supersets of their ranges.
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_barrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Wait for the phase with the given parity to complete, for at most ~2 s.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > kBarrierLimitCycles) return false;
    return true;
}

// ------------------------------------------------------------------ row tiles
// A tile is kTile consecutive rows; its pattern entries [e0, e1) are
// contiguous.  Sparse kernels run in two phases per tile: an entry-parallel
// phase (coalesced reads of values and columns, one product per entry, results
// in shared memory) and a row-parallel phase (one thread per row sums its
// entries from shared memory and runs the row's epilogue with every lane busy).

struct TileRange {
    int64_t r0;
    int nr;
    int32_t e0, e1;
};

// Loads the tile's row pointers into s_rp[0..nr] and returns its range (R rows
// per tile).
template <int R = kTile>
__device__ __forceinline__ TileRange load_tile(int64_t tile, int64_t n, const int32_t* __restrict__ rp,
                                               int32_t* s_rp) {
    TileRange t;
    t.r0 = tile * R;
    t.nr = (int)min((int64_t)R, n - t.r0);
    for (int k = threadIdx.x; k <= t.nr; k += blockDim.x) s_rp[k] = rp[t.r0 + k];
    __syncthreads();
    t.e0 = s_rp[0];
    t.e1 = s_rp[t.nr];
    return t;
}

// Row of a tile entry (binary search in the tile's row pointers).
__device__ __forceinline__ int tile_row_of(const int32_t* s_rp, int nr, int32_t e) {
    int lo = 0, hi = nr;  // s_rp[lo] <= e < s_rp[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (s_rp[mid] <= e) lo = mid;
        else hi = mid;
    }
    return lo;
}

template <class T, int N>
struct Vec {
    T v[N];
};

// Four values loaded or stored as one aligned vector access.
template <class T>
struct alignas(4 * sizeof(T)) Vec4A {
    T v[4];
};

// Entry phase of a tile with U entries per thread in flight: `load(e)` reads
// everything an entry needs (its value, column and gathered vector entries) into
// an Item, `use(e, item)` consumes it.  All U loads of a thread are issued
// before any use, so a block does not wait on U serialised load chains.  Out of
// range slots load entry e0 (always valid) and are not used.
template <int U, class Item, class LoadF, class UseF>
__device__ __forceinline__ void tile_entries(const TileRange& T, LoadF&& load, UseF&& use) {
    for (int32_t base = T.e0 + (int32_t)threadIdx.x; base < T.e1; base += kTile * U) {
        Item it[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int32_t e = base + u * kTile;
            it[u] = load(e < T.e1 ? e : T.e0);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int32_t e = base + u * kTile;
            if (e < T.e1) use(e, it[u]);
        }
    }
}

}  // namespace oasis
