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
// Fixed shuffle/shared-memory tree: deterministic.
template <int NV, class A>
__device__ __forceinline__ void block_reduce(A (&v)[NV]) {
    static_assert(NV <= 8, "too many reduction values");
    __shared__ A sh[NV][kBlock / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
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
            if (lane < kBlock / 32) x = sh[k][lane];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc_add(x, acc_shfl(x, o));
            v[k] = x;
        }
    }
    __syncthreads();
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
        __threadfence();
        last = atomicAdd(ticket, 1u) == gridDim.x - 1;
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

// ------------------------------------------------------------------ row tiles
// A tile is kTile consecutive rows; its pattern entries [e0, e1) are
// contiguous.  Sparse kernels run in two phases per tile: an entry-parallel
// phase (coalesced reads of values and columns, one product per entry, results
// in shared memory) and a row-parallel phase (one thread per row sums its
// entries from shared memory and runs the row's epilogue with every lane busy).
constexpr int kTile = kBlock;

struct TileRange {
    int64_t r0;
    int nr;
    int32_t e0, e1;
};

// Loads the tile's row pointers into s_rp[0..nr] and returns its range.
__device__ __forceinline__ TileRange load_tile(int64_t tile, int64_t n, const int32_t* __restrict__ rp,
                                               int32_t* s_rp) {
    TileRange t;
    t.r0 = tile * kTile;
    t.nr = (int)min((int64_t)kTile, n - t.r0);
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

}  // namespace oasis
