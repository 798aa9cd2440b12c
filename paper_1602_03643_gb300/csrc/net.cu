// Learned initial guess for the pressure-correction solve: a two-layer
// message-passing network on the P1 sparsity graph (width 32), bfloat16 weights
// with float32 accumulation, and its hand-written training kernels.
//
// Network (per dof i; N(i) the pattern neighbours j != i, deg_i = |N(i)|):
//   x_i  = (b_i / s_b, phi1_i / s_phi, phi2_i / s_phi)
//   h1_i = relu(W1a x_i + W1b mean_{N(i)} x + c1)                   3 -> 32
//   h2_i = relu(W2a h1_i + W2b mean_{N(i)} h1 + c2)                 32 -> 32
//   y_i  = w3 . h2_i + c3 + a0 x_i,2 + a1 x_i,3,      guess phi0 = s_phi y
// Loss L = (1/N) sum_i (y_i - t_i)^2 with t = phi / s_phi.
// Parameter order: W1a[32][3], W1b[32][3], c1[32], W2a[32][32], W2b[32][32],
// c2[32], w3[32], c3, a[2]  (2339 values).
//
// Kernels run one warp per row with lane k owning channel k: neighbour means of
// h1 are 128-byte coalesced loads, the 32x32 products go through shuffles.
// Weight gradients are summed per lane over a warp's rows, then per block in
// warp order, then over blocks in block order (deterministic).
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "internal.cuh"
#include "net.cuh"

namespace oasis {

namespace {
constexpr int kH = 32;
constexpr int oW1a = 0, oW1b = 96, oC1 = 192, oW2a = 224, oW2b = 1248, oC2 = 2272, oW3 = 2304, oC3 = 2336, oA = 2337;
constexpr int kWarps = kBlock / 32;

// all weights as float in shared memory; W2a and W2b also transposed for
// conflict-free per-lane reads of a column
struct alignas(16) SW {
    float w1a[kH * 3], w1b[kH * 3], c1[kH];
    float w2a[kH * kH], w2b[kH * kH];     // [k][l] (row k = output channel)
    float w2aT[kH * kH], w2bT[kH * kH];   // [l][k]
    float c2[kH], w3[kH], c3, a0, a1, pad_;
};

// The shared-memory image of the weights (bfloat16 values widened to float,
// plus transposed copies of W2a and W2b) is built once per parameter update;
// every block then copies it with coalesced 16-byte loads.
__global__ void k_net_image(const __nv_bfloat16* __restrict__ p, float* __restrict__ img) {
    SW& s = *reinterpret_cast<SW*>(img);
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < kH * kH; q += gridDim.x * blockDim.x) {
        const int k = q / kH, l = q % kH;
        const float a = __bfloat162float(p[oW2a + q]), b = __bfloat162float(p[oW2b + q]);
        s.w2a[q] = a;
        s.w2b[q] = b;
        s.w2aT[l * kH + k] = a;
        s.w2bT[l * kH + k] = b;
        if (q < kH * 3) {
            s.w1a[q] = __bfloat162float(p[oW1a + q]);
            s.w1b[q] = __bfloat162float(p[oW1b + q]);
        }
        if (q < kH) {
            s.c1[q] = __bfloat162float(p[oC1 + q]);
            s.c2[q] = __bfloat162float(p[oC2 + q]);
            s.w3[q] = __bfloat162float(p[oW3 + q]);
        }
        if (q == 0) {
            s.c3 = __bfloat162float(p[oC3]);
            s.a0 = __bfloat162float(p[oA]);
            s.a1 = __bfloat162float(p[oA + 1]);
            s.pad_ = 0.f;
        }
    }
}

__device__ void load_weights(SW& s, const float* __restrict__ img) {
    static_assert(sizeof(SW) % 16 == 0, "weight image copied as 16-byte vectors");
    const float4* src = reinterpret_cast<const float4*>(img);
    float4* dst = reinterpret_cast<float4*>(&s);
    for (int q = threadIdx.x; q < (int)(sizeof(SW) / 16); q += blockDim.x) dst[q] = src[q];
    __syncthreads();
}

__device__ __forceinline__ float wsum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// mean of the features over the neighbours (lanes stride over the row)
__device__ __forceinline__ void mean3(const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                                      const float* __restrict__ x, int64_t i, int lane, float (&m)[3], float& invdeg) {
    const int32_t b = rp[i], e = rp[i + 1];
    float s0 = 0.f, s1 = 0.f, s2 = 0.f;
    int cnt = 0;
    for (int32_t q = b + lane; q < e; q += 32) {
        const int32_t j = col[q];
        if (j != i) {
            s0 += x[(size_t)j * 3];
            s1 += x[(size_t)j * 3 + 1];
            s2 += x[(size_t)j * 3 + 2];
            ++cnt;
        }
    }
    cnt = (int)wsum((float)cnt);
    invdeg = cnt > 0 ? 1.f / (float)cnt : 0.f;
    m[0] = wsum(s0) * invdeg;
    m[1] = wsum(s1) * invdeg;
    m[2] = wsum(s2) * invdeg;
}

// Sum over the neighbours j != i of v[j][lane] (rows of 32 floats): the row's
// column indices are loaded once, 32 at a time, by the lanes of the warp and
// broadcast with shuffles, and 8 neighbour rows are requested before any of
// them is added, so that the warp has 8 independent 128-byte loads in flight.
// The additions run in the row's column order (skipped entries add 0).
__device__ __forceinline__ float neighbour_sum(const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                                               const float* __restrict__ v, int64_t i, int lane) {
    constexpr int kU = 8;
    const int32_t b = rp[i], e = rp[i + 1];
    float s = 0.f;
    for (int32_t c0 = b; c0 < e; c0 += 32) {
        const int cnt = min(32, (int)(e - c0));
        const int32_t mine = lane < cnt ? col[c0 + lane] : -1;
        for (int t = 0; t < cnt; t += kU) {
            float x[kU];
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                const int32_t j = __shfl_sync(0xffffffffu, mine, (t + u) & 31);
                x[u] = (t + u < cnt && j != i) ? v[(size_t)j * kH + lane] : 0.f;
            }
#pragma unroll
            for (int u = 0; u < kU; ++u) s += x[u];
        }
    }
    return s;
}

// mean of h1 over the neighbours, channel = lane
__device__ __forceinline__ float mean_h(const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                                        const float* __restrict__ h, int64_t i, int lane, float invdeg) {
    return neighbour_sum(rp, col, h, i, lane) * invdeg;
}

// ------------------------------------------------------------------ forward
// The forward layers run 4 rows per warp: a row is served by a group of 8
// lanes, lane g of the group owning channels 4g..4g+3, so that a neighbour's
// h1 row is one 16-byte load per lane and a warp keeps 4 rows' loads in flight.
constexpr int kGroup = 8, kRowsPerWarp = 4;

__device__ __forceinline__ float gsum8(float v) {
    v += __shfl_xor_sync(0xffffffffu, v, 1);
    v += __shfl_xor_sync(0xffffffffu, v, 2);
    v += __shfl_xor_sync(0xffffffffu, v, 4);
    return v;
}

__global__ void __launch_bounds__(kBlock) k_net_l1(NetArgs a) {
    __shared__ SW s;
    load_weights(s, a.img);
    const int lane = threadIdx.x & 31, lg = lane & (kGroup - 1);
    const int64_t w0 = ((int64_t)blockIdx.x * kBlock + threadIdx.x) >> 5, nw = ((int64_t)gridDim.x * kBlock) >> 5;
    for (int64_t r0 = w0 * kRowsPerWarp; r0 < a.n; r0 += nw * kRowsPerWarp) {
        const int64_t i = r0 + (lane >> 3);
        const bool ok = i < a.n;
        float m0 = 0.f, m1 = 0.f, m2 = 0.f, cnt = 0.f;
        float xi[3] = {0.f, 0.f, 0.f};
        if (ok) {
            const int32_t b = a.rp[i], e = a.rp[i + 1];
            for (int32_t q = b + lg; q < e; q += kGroup) {
                const int32_t j = a.col[q];
                if (j != i) {
                    m0 += a.x[(size_t)j * 3];
                    m1 += a.x[(size_t)j * 3 + 1];
                    m2 += a.x[(size_t)j * 3 + 2];
                    cnt += 1.f;
                }
            }
#pragma unroll
            for (int c = 0; c < 3; ++c) xi[c] = a.x[(size_t)i * 3 + c];
        }
        cnt = gsum8(cnt);
        const float invdeg = cnt > 0.f ? 1.f / cnt : 0.f;
        const float mm[3] = {gsum8(m0) * invdeg, gsum8(m1) * invdeg, gsum8(m2) * invdeg};
        if (ok) {
            float h[4];
#pragma unroll
            for (int c4 = 0; c4 < 4; ++c4) {
                const int k = 4 * lg + c4;
                float z = s.c1[k];
#pragma unroll
                for (int c = 0; c < 3; ++c) z += s.w1a[k * 3 + c] * xi[c] + s.w1b[k * 3 + c] * mm[c];
                h[c4] = fmaxf(z, 0.f);
            }
            reinterpret_cast<float4*>(a.h1)[(size_t)i * (kH / 4) + lg] = make_float4(h[0], h[1], h[2], h[3]);
        }
    }
}

__global__ void __launch_bounds__(kBlock) k_net_l2(NetArgs a) {
    __shared__ SW s;
    load_weights(s, a.img);
    const int lane = threadIdx.x & 31, lg = lane & (kGroup - 1), gb = lane & ~(kGroup - 1);
    const float4* __restrict__ h4 = reinterpret_cast<const float4*>(a.h1);
    const int64_t w0 = ((int64_t)blockIdx.x * kBlock + threadIdx.x) >> 5, nw = ((int64_t)gridDim.x * kBlock) >> 5;
    for (int64_t r0 = w0 * kRowsPerWarp; r0 < a.n; r0 += nw * kRowsPerWarp) {
        const int64_t i = r0 + (lane >> 3);
        const bool ok = i < a.n;
        const int32_t b = ok ? a.rp[i] : 0, e = ok ? a.rp[i + 1] : 0;
        const int cnt = (int)(e - b);
        const int maxcnt = __reduce_max_sync(0xffffffffu, cnt);
        float4 hk = ok ? h4[(size_t)i * (kH / 4) + lg] : make_float4(0.f, 0.f, 0.f, 0.f);
        // neighbour sum of h1 (entries in column order, 8 loads in flight per lane)
        float4 ms = make_float4(0.f, 0.f, 0.f, 0.f);
        float deg = 0.f;
        for (int c0 = 0; c0 < maxcnt; c0 += kGroup) {
            const int32_t mine = c0 + lg < cnt ? a.col[b + c0 + lg] : -1;
            float4 x[kGroup];
#pragma unroll
            for (int u = 0; u < kGroup; ++u) {
                const int32_t j = __shfl_sync(0xffffffffu, mine, gb + u);
                const bool use = j >= 0 && j != i;
                x[u] = use ? h4[(size_t)j * (kH / 4) + lg] : make_float4(0.f, 0.f, 0.f, 0.f);
                deg += use ? 1.f : 0.f;
            }
#pragma unroll
            for (int u = 0; u < kGroup; ++u) {
                ms.x += x[u].x;
                ms.y += x[u].y;
                ms.z += x[u].z;
                ms.w += x[u].w;
            }
        }
        const float invdeg = deg > 0.f ? 1.f / deg : 0.f;
        const float hv[4] = {hk.x, hk.y, hk.z, hk.w};
        const float mv[4] = {ms.x * invdeg, ms.y * invdeg, ms.z * invdeg, ms.w * invdeg};
        float z[4];
#pragma unroll
        for (int c4 = 0; c4 < 4; ++c4) z[c4] = s.c2[4 * lg + c4];
#pragma unroll
        for (int l = 0; l < kH; ++l) {
            const float hl = __shfl_sync(0xffffffffu, hv[l & 3], gb + (l >> 2));
            const float ml = __shfl_sync(0xffffffffu, mv[l & 3], gb + (l >> 2));
            const float4 wa = reinterpret_cast<const float4*>(s.w2aT)[l * (kH / 4) + lg];
            const float4 wb = reinterpret_cast<const float4*>(s.w2bT)[l * (kH / 4) + lg];
            z[0] += wa.x * hl + wb.x * ml;
            z[1] += wa.y * hl + wb.y * ml;
            z[2] += wa.z * hl + wb.z * ml;
            z[3] += wa.w * hl + wb.w * ml;
        }
        float y = 0.f;
#pragma unroll
        for (int c4 = 0; c4 < 4; ++c4) y += s.w3[4 * lg + c4] * fmaxf(z[c4], 0.f);
        y = gsum8(y);
        if (ok && lg == 0) {
            const float* xi = a.x + (size_t)i * 3;
            a.y[i] = y + s.c3 + s.a0 * xi[1] + s.a1 * xi[2];
        }
    }
}

// layer 2 for row i: z2 (lane's channel), the neighbour mean m2 and h1_i of the lane
__device__ __forceinline__ float layer2(const SW& s, const NetArgs& a, int64_t i, int lane, float invdeg, float& hk,
                                        float& m2k) {
    hk = a.h1[(size_t)i * kH + lane];
    m2k = mean_h(a.rp, a.col, a.h1, i, lane, invdeg);
    float z = s.c2[lane];
#pragma unroll
    for (int l = 0; l < kH; ++l) {
        const float hl = __shfl_sync(0xffffffffu, hk, l);
        const float ml = __shfl_sync(0xffffffffu, m2k, l);
        z += s.w2aT[l * kH + lane] * hl + s.w2bT[l * kH + lane] * ml;
    }
    return z;
}

__device__ __forceinline__ float inv_degree(const int32_t* __restrict__ rp, const int32_t* __restrict__ col, int64_t i,
                                            int lane) {
    const int32_t b = rp[i], e = rp[i + 1];
    int cnt = 0;
    for (int32_t q = b + lane; q < e; q += 32) cnt += col[q] != i;
    cnt = (int)wsum((float)cnt);
    return cnt > 0 ? 1.f / (float)cnt : 0.f;
}

// ------------------------------------------------------------------ backward
// Layer-2 and readout gradients; stores dz2 and g = W2b^T dz2 / deg per row.
// Block partials: [oW2a..oW2b+1024) (dW2a, dW2b), c2, w3, c3, a, and the loss.
__global__ void __launch_bounds__(kBlock) k_net_bwd2(NetArgs a) {
    __shared__ SW s;
    __shared__ float red[kNetPartial];
    load_weights(s, a.img);
    for (int q = threadIdx.x; q < kNetPartial; q += blockDim.x) red[q] = 0.f;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t w0 = ((int64_t)blockIdx.x * kBlock + threadIdx.x) >> 5, nw = ((int64_t)gridDim.x * kBlock) >> 5;
    float gw2a[kH], gw2b[kH];
#pragma unroll
    for (int l = 0; l < kH; ++l) gw2a[l] = gw2b[l] = 0.f;
    float gc2 = 0.f, gw3 = 0.f, gc3 = 0.f, ga0 = 0.f, ga1 = 0.f, loss = 0.f;
    const float scale = 2.f / (float)a.n;
    for (int64_t i = w0; i < a.n; i += nw) {
        const float invdeg = inv_degree(a.rp, a.col, i, lane);
        float hk, m2k;
        const float z = layer2(s, a, i, lane, invdeg, hk, m2k);
        const float h2 = fmaxf(z, 0.f);
        const float* xi = a.x + (size_t)i * 3;
        const float y = wsum(s.w3[lane] * h2) + s.c3 + s.a0 * xi[1] + s.a1 * xi[2];
        const float r = y - a.t[i];
        const float dy = scale * r;
        loss += lane == 0 ? r * r : 0.f;
        gc3 += lane == 0 ? dy : 0.f;
        ga0 += lane == 0 ? dy * xi[1] : 0.f;
        ga1 += lane == 0 ? dy * xi[2] : 0.f;
        gw3 += dy * h2;
        const float dz = z > 0.f ? dy * s.w3[lane] : 0.f;
        gc2 += dz;
#pragma unroll
        for (int l = 0; l < kH; ++l) {
            gw2a[l] += dz * __shfl_sync(0xffffffffu, hk, l);
            gw2b[l] += dz * __shfl_sync(0xffffffffu, m2k, l);
        }
        a.dz2[(size_t)i * kH + lane] = dz;
        float g = 0.f;
#pragma unroll
        for (int l = 0; l < kH; ++l) g += s.w2b[l * kH + lane] * __shfl_sync(0xffffffffu, dz, l);
        a.g[(size_t)i * kH + lane] = g * invdeg;
    }
    // per-block sums in warp order (deterministic)
    for (int w = 0; w < kWarps; ++w) {
        if (wib == w) {
#pragma unroll
            for (int l = 0; l < kH; ++l) {
                red[(oW2a - oW2a) + lane * kH + l] += gw2a[l];
                red[(oW2b - oW2a) + lane * kH + l] += gw2b[l];
            }
            red[(oC2 - oW2a) + lane] += gc2;
            red[(oW3 - oW2a) + lane] += gw3;
            if (lane == 0) {
                red[oC3 - oW2a] += gc3;
                red[oA - oW2a] += ga0;
                red[oA + 1 - oW2a] += ga1;
                red[kNetPartial - 1] += loss;
            }
        }
        __syncthreads();
    }
    float* out = a.partial + (size_t)blockIdx.x * kNetPartialStride;
    for (int q = threadIdx.x; q < kNetPartial; q += blockDim.x) out[oW2a + q] = red[q];
}

// Layer-1 gradients: dh1 = W2a^T dz2 + sum_{j in N(i)} g_j, dz1 = dh1 [z1 > 0].
__global__ void __launch_bounds__(kBlock) k_net_bwd1(NetArgs a) {
    __shared__ SW s;
    __shared__ float red[oW2a];
    load_weights(s, a.img);
    for (int q = threadIdx.x; q < oW2a; q += blockDim.x) red[q] = 0.f;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t w0 = ((int64_t)blockIdx.x * kBlock + threadIdx.x) >> 5, nw = ((int64_t)gridDim.x * kBlock) >> 5;
    float gw1a[3] = {0.f, 0.f, 0.f}, gw1b[3] = {0.f, 0.f, 0.f}, gc1 = 0.f;
    for (int64_t i = w0; i < a.n; i += nw) {
        float m[3], invdeg;
        mean3(a.rp, a.col, a.x, i, lane, m, invdeg);
        const float* xi = a.x + (size_t)i * 3;
        float z = s.c1[lane];
#pragma unroll
        for (int c = 0; c < 3; ++c) z += s.w1a[lane * 3 + c] * xi[c] + s.w1b[lane * 3 + c] * m[c];
        const float dzi = a.dz2[(size_t)i * kH + lane];
        float dh = 0.f;
#pragma unroll
        for (int l = 0; l < kH; ++l) dh += s.w2a[l * kH + lane] * __shfl_sync(0xffffffffu, dzi, l);
        dh += neighbour_sum(a.rp, a.col, a.g, i, lane);
        const float dz = z > 0.f ? dh : 0.f;
        gc1 += dz;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            gw1a[c] += dz * xi[c];
            gw1b[c] += dz * m[c];
        }
    }
    for (int w = 0; w < kWarps; ++w) {
        if (wib == w) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                red[oW1a + lane * 3 + c] += gw1a[c];
                red[oW1b + lane * 3 + c] += gw1b[c];
            }
            red[oC1 + lane] += gc1;
        }
        __syncthreads();
    }
    float* out = a.partial + (size_t)blockIdx.x * kNetPartialStride;
    for (int q = threadIdx.x; q < oW2a; q += blockDim.x) out[q] = red[q];
}

// grad[p] = sum over blocks (in block order) of the partials; loss likewise.
__global__ void k_net_reduce(const float* __restrict__ partial, int blocks, float* __restrict__ grad,
                             float* __restrict__ loss, int n) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p > kNetParams) return;
    const int col = p < kNetParams ? p : oW2a + kNetPartial - 1;
    float acc = 0.f;
    for (int b = 0; b < blocks; ++b) acc += partial[(size_t)b * kNetPartialStride + col];
    if (p < kNetParams) grad[p] = acc;
    else *loss = acc / (float)n;
}

// Adam (Kingma & Ba 2015) on the float32 master copy; refreshes the bf16 copy.
__global__ void k_net_adam(float* __restrict__ p32, __nv_bfloat16* __restrict__ p16, float* __restrict__ m,
                           float* __restrict__ v, const float* __restrict__ g, float lr, float b1, float b2, float eps,
                           float c1, float c2) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= kNetParams) return;
    const float gq = g[q];
    const float mq = b1 * m[q] + (1.f - b1) * gq;
    const float vq = b2 * v[q] + (1.f - b2) * gq * gq;
    m[q] = mq;
    v[q] = vq;
    const float w = p32[q] - lr * (mq / c1) / (sqrtf(vq / c2) + eps);
    p32[q] = w;
    p16[q] = __float2bfloat16_rn(w);
}

__global__ void k_net_to_bf16(const float* __restrict__ p32, __nv_bfloat16* __restrict__ p16) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q < kNetParams) p16[q] = __float2bfloat16_rn(p32[q]);
}

int net_grid(int64_t rows) {
    const int64_t want = (rows + kWarps - 1) / kWarps;
    return (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)num_sms() * 8));
}
}  // namespace

Net* net_create(const Mesh& m) {
    OASIS_CHECK(m.assembled, OASIS_EINVAL, "mesh not assembled");
    auto N = std::make_unique<Net>();
    N->m = &m;
    N->n = m.n;
    N->p32.alloc(kNetParams);
    N->p16.alloc(kNetParams);
    N->mom.alloc(kNetParams);
    N->var.alloc(kNetParams);
    N->grad.alloc(kNetParams);
    N->loss.alloc(1);
    for (auto* b : {&N->p32, &N->mom, &N->var, &N->grad})
        OASIS_CUDA(cudaMemset(b->p, 0, b->bytes()));
    OASIS_CUDA(cudaMemset(N->p16.p, 0, N->p16.bytes()));
    N->h1.alloc((size_t)m.n * kH);
    N->dz2.alloc((size_t)m.n * kH);
    N->g.alloc((size_t)m.n * kH);
    N->grid = net_grid(m.n);
    N->img.alloc(sizeof(SW) / sizeof(float));
    k_net_image<<<4, 256>>>(N->p16.p, N->img.p);
    OASIS_CUDA(cudaGetLastError());
    int per_sm = 0;
    OASIS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_net_l2, kBlock, 0));
    const int64_t groups = (m.n + kRowsPerWarp - 1) / kRowsPerWarp;
    N->grid_fwd = (int)std::max<int64_t>(
        1, std::min<int64_t>((groups + kWarps - 1) / kWarps, (int64_t)std::max(per_sm, 1) * num_sms()));
    N->partial.alloc((size_t)N->grid * kNetPartialStride);
    OASIS_CUDA(cudaDeviceSynchronize());
    return N.release();
}

NetArgs net_args(Net& N, const float* x, float* y, const float* t) {
    NetArgs a{};
    a.rp = N.m->row_ptr.p;
    a.col = N.m->col.p;
    a.n = N.n;
    a.p16 = N.p16.p;
    a.img = N.img.p;
    a.x = x;
    a.y = y;
    a.t = t;
    a.h1 = N.h1.p;
    a.dz2 = N.dz2.p;
    a.g = N.g.p;
    a.partial = N.partial.p;
    return a;
}

void net_forward(Net& N, const float* x, float* y, cudaStream_t s) {
    const NetArgs a = net_args(N, x, y, nullptr);
    k_net_l1<<<N.grid_fwd, kBlock, 0, s>>>(a);
    k_net_l2<<<N.grid_fwd, kBlock, 0, s>>>(a);
    OASIS_CUDA(cudaGetLastError());
}

void net_backward(Net& N, const float* x, const float* t, float* grad, float* loss, cudaStream_t s) {
    const NetArgs a = net_args(N, x, nullptr, t);
    k_net_l1<<<N.grid_fwd, kBlock, 0, s>>>(a);
    k_net_bwd2<<<N.grid, kBlock, 0, s>>>(a);
    k_net_bwd1<<<N.grid, kBlock, 0, s>>>(a);
    k_net_reduce<<<(kNetParams + 1 + 255) / 256, 256, 0, s>>>(N.partial.p, N.grid, grad ? grad : N.grad.p,
                                                             loss ? loss : N.loss.p, (int)N.n);
    OASIS_CUDA(cudaGetLastError());
}

void net_adam(Net& N, const float* grad, float lr, float b1, float b2, float eps, int step, cudaStream_t s) {
    const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
    k_net_adam<<<(kNetParams + 255) / 256, 256, 0, s>>>(N.p32.p, N.p16.p, N.mom.p, N.var.p, grad ? grad : N.grad.p, lr,
                                                       b1, b2, eps, c1, c2);
    k_net_image<<<4, 256, 0, s>>>(N.p16.p, N.img.p);
    OASIS_CUDA(cudaGetLastError());
}

void net_set_params(Net& N, const float* host) {
    OASIS_CUDA(cudaMemcpy(N.p32.p, host, kNetParams * sizeof(float), cudaMemcpyHostToDevice));
    k_net_to_bf16<<<(kNetParams + 255) / 256, 256>>>(N.p32.p, N.p16.p);
    k_net_image<<<4, 256>>>(N.p16.p, N.img.p);
    OASIS_CUDA(cudaGetLastError());
    OASIS_CUDA(cudaMemset(N.mom.p, 0, N.mom.bytes()));
    OASIS_CUDA(cudaMemset(N.var.p, 0, N.var.bytes()));
    OASIS_CUDA(cudaDeviceSynchronize());
}

}  // namespace oasis
