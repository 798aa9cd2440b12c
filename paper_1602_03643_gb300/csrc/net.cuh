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
};

struct Net {
    const Mesh* m = nullptr;
    int64_t n = 0;
    int grid = 1;
    DBuf<float> p32, mom, var, grad, loss;
    DBuf<__nv_bfloat16> p16;
    DBuf<float> img;     // bfloat16 weights widened to float, in shared-memory layout
    DBuf<float> h1, dz2, g, partial;
    int grid_fwd = 1;    // one resident wave of the forward kernels
};

Net* net_create(const Mesh& m);
void net_forward(Net& N, const float* x, float* y, cudaStream_t s);
void net_backward(Net& N, const float* x, const float* t, float* grad, float* loss, cudaStream_t s);
void net_adam(Net& N, const float* grad, float lr, float b1, float b2, float eps, int step, cudaStream_t s);
void net_set_params(Net& N, const float* host);

}  // namespace oasis
