// Device helpers: row-group reductions, deterministic block / grid reductions.
#pragma once

#include <cuda_runtime.h>

#include "internal.cuh"

namespace oasis {

// Sum over the L lanes of a row group (L divides 32).  Every lane of the warp
// must call it (full mask); lanes of other groups reduce their own values.
template <int L, class T>
__device__ __forceinline__ T group_sum(T v) {
#pragma unroll
    for (int o = L / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <class T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide sum of NV doubles; the totals are valid in thread 0.  Fixed
// summation tree, hence deterministic.  blockDim.x == kBlock.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV]) {
    __shared__ double sh[NV][kBlock / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        double x = warp_sum(v[k]);
        if (lane == 0) sh[k][wid] = x;
    }
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double x = lane < kBlock / 32 ? sh[k][lane] : 0.0;
            v[k] = warp_sum(x);
        }
    }
    __syncthreads();
}

// Grid-wide sum of NV doubles with a deterministic "last block finishes"
// reduction: every block writes its partials, takes a ticket, and the block
// that takes the last ticket sums all partials in block order.  Returns true
// in the last block only; there thread 0 holds the totals in v.  The ticket is
// reset for the next launch.  `partial` holds gridDim.x * NV doubles.
template <int NV>
__device__ __forceinline__ bool grid_sum(double (&v)[NV], double* partial, uint32_t* ticket) {
    block_sum<NV>(v);
    __shared__ bool last;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) partial[(size_t)blockIdx.x * NV + k] = v[k];
        __threadfence();
        const uint32_t t = atomicAdd(ticket, 1u);
        last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
    double s[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) s[k] = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
#pragma unroll
        for (int k = 0; k < NV; ++k) s[k] += __ldcg(&partial[(size_t)b * NV + k]);
    }
    block_sum<NV>(s);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) v[k] = s[k];
        *ticket = 0u;
    }
    return true;
}

template <class V>
__device__ __forceinline__ V ldg(const V* p) { return __ldg(p); }

}  // namespace oasis
