// Learned pressure guess: network object and kernels' argument block (net.cu).
#pragma once

#include <cuda_bf16.h>

#include <memory>

#include "internal.cuh"

namespace oasis {

constexpr int kNetParams = 2339;                 // see net.cu for the order
constexpr int kNetPartial = kNetParams - 224 + 1; // layer-2/readout gradient slots + loss
constexpr int kNetPartialStride = 2344;          // per-block partial row (>= kNetParams + 1)

struct NetArgs {
    const int32_t *rp, *col;
    int64_t n;
    const __nv_bfloat16* p16;
    const float* img;    // the weights as the kernels' shared-memory image (floats)
    const float* x;      // [n][3] features
    float* y;            // [n] output
    const float* t;      // [n] target
    float *h1, *dz2, *g; // [n][32] work
    float* partial;      // [blocks][kNetPartialStride]
    const __nv_bfloat16* bop;  // [W2a | W2b] as the tensor-core B operand (net.cu)
    float* rec;          // [n][8] inference records (x, mean x, 0, 0)
    int32_t* err;        // set when a bounded device-side wait ran out
};

struct Net {
    const Mesh* m = nullptr;
    int64_t n = 0;
    int grid = 1;
    DBuf<float> p32, mom, var, grad, loss;
    DBuf<__nv_bfloat16> p16;
    DBuf<float> img;     // bfloat16 weights widened to float, in shared-memory layout
    DBuf<float> h1, dz2, g, partial;
    DBuf<__nv_bfloat16> bop;  // layer-2 weights in the tensor-core operand layout
    DBuf<float> rec;          // inference records [n][8]
    DBuf<int32_t> err;
    int grid_fwd = 1;    // one resident wave of the forward kernels
    int grid_tc = 1;     // blocks of the tensor-core layer-2 kernel
};

Net* net_create(const Mesh& m);
void net_forward(Net& N, const float* x, float* y, cudaStream_t s);
// waits for `s`; OASIS_EWAIT if a forward's bounded device-side wait ran out
void net_check(Net& N, cudaStream_t s);
void net_backward(Net& N, const float* x, const float* t, float* grad, float* loss, cudaStream_t s);
void net_adam(Net& N, const float* grad, float lr, float b1, float b2, float eps, int step, cudaStream_t s);
void net_set_params(Net& N, const float* host);

}  // namespace oasis
