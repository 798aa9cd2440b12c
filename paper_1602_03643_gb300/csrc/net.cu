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
// Inference: layer 1 on CUDA cores (3 -> 32), layer 2's dense product on the
// tensor cores (tcgen05, below).  Training kernels run one warp per row with
// lane k owning channel k: neighbour means of h1 are 128-byte coalesced loads,
// the 32x32 products go through shuffles.
// Weight gradients are summed per lane over a warp's rows, then per block in
// warp order, then over blocks in block order (deterministic).
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "internal.cuh"
#include "kern.cuh"
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

// ------------------------------------------------------------------ inference
// Two forms of inference (kInferStoredH1 picks one).  Stored (in use): layer 1
// writes h1 of every row ([n][32] float32, k_net_l1, as training does) and
// layer 2 gathers each neighbour's h1.  Records: layer 1 only forms each row's
// record (x_i, mean_{N(i)} x, 0, 0) (32 bytes, k_net_rec), and layer 2
// recomputes h1_j of every neighbour from its record (6 inputs, 32 channels),
// which moves 32 bytes per neighbour instead of h1's 128 but costs more
// arithmetic and shuffles than it saves (723 against 594 us per forward at
// 128^3 for records against stored h1 with its layer 1).  Layer 2's dense
// product then runs on the
// 5th-generation tensor cores: per tile of 128 rows, A = [h1_i | mean h1]
// (128 x 64), B = [W2a | W2b] (32 x 64, the bfloat16 weights), D = A B^T
// (128 x 32, float32 in tensor memory) by tcgen05.mma kind::f16 with M = 128,
// N = 32, K = 16.  A holds float32 activations: each is split into three
// bfloat16 terms (hi + mid + lo, ~24 significant bits), so that the products
// accumulated in float32 reproduce the float32 layer (the weights are bfloat16
// already).  Operands sit in shared memory in the canonical no-swizzle K-major
// layout: 8 x 16-byte core matrices, the two of a 16-wide K slab 128 bytes apart
// (LBO), consecutive 8-row groups 256 bytes apart (SBO).  One thread issues the
// MMAs and commits them to an mbarrier; warp w then reads rows 32 (w % 4) ..
// +31, columns 16 (w / 4) .. +15 of the accumulator (tcgen05.ld 32x32b) for the
// epilogue (relu, readout, skip terms), the two column halves added in a fixed
// order.
constexpr int kRec = 8;                            // floats per inference record
// Inference path: layer 1 stores h1 and layer 2 gathers it (true), or layer 1
// writes the 32-byte records and layer 2 rebuilds h1 of every neighbour (false).
constexpr bool kInferStoredH1 = true;

__global__ void __launch_bounds__(kBlock) k_net_rec(NetArgs a) {
    const int lane = threadIdx.x & 31, lg = lane & (kGroup - 1);
    const int64_t w0 = ((int64_t)blockIdx.x * kBlock + threadIdx.x) >> 5, nw = ((int64_t)gridDim.x * kBlock) >> 5;
    for (int64_t r0 = w0 * kRowsPerWarp; r0 < a.n; r0 += nw * kRowsPerWarp) {
        const int64_t i = r0 + (lane >> 3);
        const bool ok = i < a.n;
        float m0 = 0.f, m1 = 0.f, m2 = 0.f, cnt = 0.f;
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
        }
        cnt = gsum8(cnt);
        const float invdeg = cnt > 0.f ? 1.f / cnt : 0.f;
        const float mm[3] = {gsum8(m0) * invdeg, gsum8(m1) * invdeg, gsum8(m2) * invdeg};
        if (ok && lg == 0) {
            float4* rec = reinterpret_cast<float4*>(a.rec) + (size_t)i * 2;
            rec[0] = make_float4(a.x[(size_t)i * 3], a.x[(size_t)i * 3 + 1], a.x[(size_t)i * 3 + 2], mm[0]);
            rec[1] = make_float4(mm[1], mm[2], 0.f, 0.f);
        }
    }
}

constexpr int kTcRows = 128;                       // rows per tile (MMA M)
constexpr int kTcK = 2 * kH;                       // [h | m]
constexpr int kTcSlab = 16;                        // K per MMA
constexpr int kTcSplits = 3;                       // bfloat16 terms per activation
constexpr int kTcASlabBytes = kTcRows / 8 * 256;   // 4096
constexpr int kTcASplitBytes = kTcK / kTcSlab * kTcASlabBytes;   // 16384
constexpr int kTcBSlabBytes = kH / 8 * 256;        // 1024
constexpr int kTcBBytes = kTcK / kTcSlab * kTcBSlabBytes;        // 4096
constexpr int kTcThreads = 256;
constexpr int kTcWarps = kTcThreads / 32;
constexpr uint32_t kTcTmemCols = 32;
constexpr size_t kTcSmem = (size_t)kTcSplits * kTcASplitBytes + kTcBBytes + 2048;   // + alignment room

// byte offset of element (row, k) of an operand slab layout (rows a multiple of 8)
__host__ __device__ constexpr int tc_off(int row, int k, int slab_bytes) {
    return (k / kTcSlab) * slab_bytes + (row / 8) * 256 + ((k % kTcSlab) / 8) * 128 + (row % 8) * 16 + (k % 8) * 2;
}

// B operand image: B[n][k] = W2a[n][k] (k < 32), W2b[n][k - 32] (k >= 32)
__global__ void k_net_bop(const __nv_bfloat16* __restrict__ p, __nv_bfloat16* __restrict__ bop) {
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < kH * kTcK; q += gridDim.x * blockDim.x) {
        const int n = q / kTcK, k = q % kTcK;
        const __nv_bfloat16 v = k < kH ? p[oW2a + n * kH + k] : p[oW2b + n * kH + (k - kH)];
        bop[tc_off(n, k, kTcBSlabBytes) / 2] = v;
    }
}

// shared-memory matrix descriptor: start >> 4, LBO >> 4 at bit 16, SBO >> 4 at
// bit 32, descriptor version 1 at bit 46, no swizzle (layout 0 at bits 61-63)
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)(128u >> 4) << 16) | ((uint64_t)(256u >> 4) << 32) |
           (1ull << 46);
}
// instruction descriptor, kind::f16: D float32 (bits 4-5 = 1), A and B bfloat16
// (bits 7-9 = 1, 10-12 = 1), both K-major, N >> 3 at bit 17, M >> 4 at bit 24
constexpr uint32_t kTcIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kH >> 3) << 17) |
                              ((uint32_t)(kTcRows >> 4) << 24);

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tc_mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(kTcIdesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void tc_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
                 : "memory");
}

// 16 consecutive float32 columns of this warp's 32 lanes (one row per thread)
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = __uint_as_float(r[q]);
}

// four float32 values -> three 8-byte rows of bfloat16 terms (hi, mid, lo)
__device__ __forceinline__ void tc_split_store(unsigned char* a, int off, const float (&v)[4]) {
    __nv_bfloat16 t[kTcSplits][4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const __nv_bfloat16 hi = __float2bfloat16_rn(v[c]);
        const float r1 = v[c] - __bfloat162float(hi);
        const __nv_bfloat16 mid = __float2bfloat16_rn(r1);
        const float r2 = r1 - __bfloat162float(mid);
        t[0][c] = hi;
        t[1][c] = mid;
        t[2][c] = __float2bfloat16_rn(r2);
    }
#pragma unroll
    for (int sp = 0; sp < kTcSplits; ++sp)
        *reinterpret_cast<uint2*>(a + sp * kTcASplitBytes + off) = *reinterpret_cast<const uint2*>(t[sp]);
}

// layer-1 channels 4 lg .. 4 lg + 3 of a row from its record (x, mean x)
struct L1Lane {
    float wa[4][3], wb[4][3], c[4];
    __device__ __forceinline__ void h(const float (&in)[6], float (&out)[4]) const {
#pragma unroll
        for (int c4 = 0; c4 < 4; ++c4) {
            float z = c[c4];
#pragma unroll
            for (int q = 0; q < 3; ++q) z += wa[c4][q] * in[q] + wb[c4][q] * in[3 + q];
            out[c4] = fmaxf(z, 0.f);
        }
    }
};

// STORED: h1 of every row was written by k_net_l1 ([n][32] float32); a row's
// group loads its own h1 and each neighbour's as one 16-byte load per lane (the
// lane's 4 channels), the neighbour's index broadcast by one shuffle.  Else h1
// of the row and of each neighbour is rebuilt from the 32-byte records.
template <bool STORED>
__global__ void __launch_bounds__(kTcThreads, 4) k_net_l2_tc(NetArgs a) {
    extern __shared__ __align__(1024) unsigned char tc_dsm[];
    unsigned char* base = tc_dsm + ((1024 - (smem_addr(tc_dsm) & 1023)) & 1023);
    unsigned char* sa = base;                                        // [split][slab][rows]
    unsigned char* sb = base + kTcSplits * kTcASplitBytes;           // [slab][32 rows]
    __shared__ uint64_t bar;
    __shared__ uint32_t tmem_base;
    __shared__ float s_half[kTcRows];                                // readout of columns 16..31
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, lg = lane & (kGroup - 1), gb = lane & ~(kGroup - 1);
    const SW* gw = reinterpret_cast<const SW*>(a.img);
    L1Lane w1;
#pragma unroll
    for (int c4 = 0; c4 < 4; ++c4) {
        const int k = 4 * lg + c4;
        w1.c[c4] = gw->c1[k];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            w1.wa[c4][q] = gw->w1a[k * 3 + q];
            w1.wb[c4][q] = gw->w1b[k * 3 + q];
        }
    }
    // B operand: 4 KB, 16-byte copies
    for (int q = threadIdx.x; q < kTcBBytes / 16; q += kTcThreads)
        reinterpret_cast<uint4*>(sb)[q] = reinterpret_cast<const uint4*>(a.bop)[q];
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_base)),
                     "r"(kTcTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_barrier_init();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;
    const float4* __restrict__ rec4 = reinterpret_cast<const float4*>(a.rec);
    uint32_t phase = 0;
    bool ok_wait = true;
    const int64_t tiles = (a.n + kTcRows - 1) / kTcRows;
    for (int64_t tile = blockIdx.x; tile < tiles && ok_wait; tile += gridDim.x) {
        // A = [h1_i | mean h1] of the tile's rows, 4 rows per warp at a time;
        // a row's group of 8 lanes loads 8 neighbour records at once (one per
        // lane) and shares them with shuffles, in column order
        for (int it = 0; it < kTcRows / kTcWarps / kRowsPerWarp; ++it) {
            const int r = (kTcRows / kTcWarps) * warp + kRowsPerWarp * it + (lane >> 3);
            const int64_t i = tile * kTcRows + r;
            const bool ok = i < a.n;
            const int32_t b = ok ? a.rp[i] : 0, e = ok ? a.rp[i + 1] : 0;
            const int cnt = (int)(e - b);
            const int maxcnt = __reduce_max_sync(0xffffffffu, cnt);
            float hv[4] = {0.f, 0.f, 0.f, 0.f};
            float ms[4] = {0.f, 0.f, 0.f, 0.f};
            float deg = 0.f;
            if constexpr (STORED) {
                const float4* __restrict__ h4 = reinterpret_cast<const float4*>(a.h1);
                if (ok) {
                    const float4 hi = h4[(size_t)i * (kH / 4) + lg];
                    hv[0] = hi.x;
                    hv[1] = hi.y;
                    hv[2] = hi.z;
                    hv[3] = hi.w;
                }
                for (int c0 = 0; c0 < maxcnt; c0 += kGroup) {
                    const int32_t jl = c0 + lg < cnt ? a.col[b + c0 + lg] : -1;
                    float4 v[kGroup];
                    int use[kGroup];
#pragma unroll
                    for (int u = 0; u < kGroup; ++u) {
                        const int32_t j = __shfl_sync(0xffffffffu, jl, gb + u);
                        use[u] = j >= 0 && j != i;
                        v[u] = use[u] ? h4[(size_t)j * (kH / 4) + lg] : make_float4(0.f, 0.f, 0.f, 0.f);
                    }
#pragma unroll
                    for (int u = 0; u < kGroup; ++u) {
                        if (use[u]) {
                            ms[0] += v[u].x;
                            ms[1] += v[u].y;
                            ms[2] += v[u].z;
                            ms[3] += v[u].w;
                            deg += 1.f;
                        }
                    }
                }
            } else {
            if (ok) {
                const float4 r0 = rec4[(size_t)i * 2], r1 = rec4[(size_t)i * 2 + 1];
                const float in[6] = {r0.x, r0.y, r0.z, r0.w, r1.x, r1.y};
                w1.h(in, hv);
            }
            for (int c0 = 0; c0 < maxcnt; c0 += kGroup) {
                const int32_t j = c0 + lg < cnt ? a.col[b + c0 + lg] : -1;
                const bool use = j >= 0 && j != i;
                const float4 ra = use ? rec4[(size_t)j * 2] : make_float4(0.f, 0.f, 0.f, 0.f);
                const float4 rb = use ? rec4[(size_t)j * 2 + 1] : make_float4(0.f, 0.f, 0.f, 0.f);
                const int usei = use ? 1 : 0;
#pragma unroll
                for (int u = 0; u < kGroup; ++u) {
                    const int src = gb + u;
                    const int uu = __shfl_sync(0xffffffffu, usei, src);
                    const float in[6] = {__shfl_sync(0xffffffffu, ra.x, src), __shfl_sync(0xffffffffu, ra.y, src),
                                         __shfl_sync(0xffffffffu, ra.z, src), __shfl_sync(0xffffffffu, ra.w, src),
                                         __shfl_sync(0xffffffffu, rb.x, src), __shfl_sync(0xffffffffu, rb.y, src)};
                    if (uu) {
                        float h[4];
                        w1.h(in, h);
#pragma unroll
                        for (int c4 = 0; c4 < 4; ++c4) ms[c4] += h[c4];
                        deg += 1.f;
                    }
                }
            }
            }
            const float invdeg = deg > 0.f ? 1.f / deg : 0.f;
            const float mv[4] = {ms[0] * invdeg, ms[1] * invdeg, ms[2] * invdeg, ms[3] * invdeg};
            tc_split_store(sa, tc_off(r, 4 * lg, kTcASlabBytes), hv);
            tc_split_store(sa, tc_off(r, kH + 4 * lg, kTcASlabBytes), mv);
        }
        // make the generic-proxy stores visible to the tensor core, then one
        // thread issues the 3 x 4 MMAs and commits them to the barrier
        fence_proxy_async();
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (threadIdx.x == 0) {
            const uint32_t a0 = smem_addr(sa), b0 = smem_addr(sb);
            uint32_t acc = 0;
#pragma unroll
            for (int sp = 0; sp < kTcSplits; ++sp)
#pragma unroll
                for (int sl = 0; sl < kTcK / kTcSlab; ++sl) {
                    tc_mma(tmem, tc_desc(a0 + sp * kTcASplitBytes + sl * kTcASlabBytes), tc_desc(b0 + sl * kTcBSlabBytes),
                           acc);
                    acc = 1;
                }
            tc_commit(&bar);
        }
        const bool arrived = mbar_wait_bounded(&bar, phase);
        phase ^= 1u;
        ok_wait = __syncthreads_and(arrived) != 0;
        if (!ok_wait) break;
        tc_fence_after();
        const int quarter = warp & 3, half = warp >> 2;
        float z[16];
        tc_ld16(tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)(16 * half), z);
        float y = 0.f;
#pragma unroll
        for (int k = 0; k < 16; ++k) y += gw->w3[16 * half + k] * fmaxf(z[k] + gw->c2[16 * half + k], 0.f);
        const int row = 32 * quarter + lane;
        if (half == 1) s_half[row] = y;
        tc_fence_before();
        __syncthreads();
        const int64_t i = tile * kTcRows + row;
        if (half == 0 && i < a.n) {
            const float* xi = a.x + (size_t)i * 3;
            a.y[i] = (y + s_half[row]) + gw->c3 + gw->a0 * xi[1] + gw->a1 * xi[2];
        }
        // s_half, A and D are reused by the next tile
        __syncthreads();
    }
    if (!ok_wait) {
        if (lane == 0) atomicExch(a.err, 1);
        // the MMAs may still be in flight: wait for them (bounded) before freeing
        mbar_wait_bounded(&bar, phase ^ 1u);
    }
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcTmemCols) : "memory");
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
    N->bop.alloc((size_t)kH * kTcK);
    k_net_bop<<<8, 256>>>(N->p16.p, N->bop.p);
    N->err.alloc(1);
    N->rec.alloc((size_t)m.n * kRec);
    OASIS_CUDA(cudaMemset(N->err.p, 0, sizeof(int32_t)));
    OASIS_CUDA(cudaGetLastError());
    OASIS_CUDA(cudaFuncSetAttribute(k_net_l2_tc<kInferStoredH1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)kTcSmem));
    OASIS_CUDA(cudaFuncSetAttribute(k_net_l2_tc<kInferStoredH1>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                    (int)cudaSharedmemCarveoutMaxShared));
    // resident blocks per SM from the kernel's registers, shared memory, threads
    // and tensor-memory columns (the runtime's occupancy query reports one block
    // for this kernel, while the hardware holds three)
    int per_sm_tc = 0;
    {
        cudaFuncAttributes fa{};
        OASIS_CUDA(cudaFuncGetAttributes(&fa, k_net_l2_tc<kInferStoredH1>));
        int dev = 0, regs_sm = 0, smem_sm = 0, thr_sm = 0, resv = 0;
        OASIS_CUDA(cudaGetDevice(&dev));
        OASIS_CUDA(cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev));
        OASIS_CUDA(cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
        OASIS_CUDA(cudaDeviceGetAttribute(&thr_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev));
        OASIS_CUDA(cudaDeviceGetAttribute(&resv, cudaDevAttrReservedSharedMemoryPerBlock, dev));
        const int warp_regs = (fa.numRegs * 32 + 255) / 256 * 256;          // allocation unit: 256 per warp
        const int by_regs = regs_sm / std::max(1, warp_regs * kTcWarps);
        const int by_smem = smem_sm / (int)(kTcSmem + fa.sharedSizeBytes + (size_t)resv);
        const int by_thr = thr_sm / kTcThreads;
        per_sm_tc = std::min({by_regs, by_smem, by_thr, (int)(512 / kTcTmemCols)});
    }
    OASIS_CHECK(per_sm_tc > 0, OASIS_EINVAL, "tensor-core layer does not fit on an SM");
    const int64_t tc_tiles = (m.n + kTcRows - 1) / kTcRows;
    N->grid_tc = (int)std::max<int64_t>(1, std::min<int64_t>(tc_tiles, (int64_t)per_sm_tc * num_sms()));
    int per_sm = 0;
    OASIS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_net_l1, kBlock, 0));
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
    a.bop = N.bop.p;
    a.rec = N.rec.p;
    a.err = N.err.p;
    return a;
}

void net_forward(Net& N, const float* x, float* y, cudaStream_t s) {
    const NetArgs a = net_args(N, x, y, nullptr);
    if (kInferStoredH1) {
        k_net_l1<<<N.grid_fwd, kBlock, 0, s>>>(a);
        k_net_l2_tc<true><<<N.grid_tc, kTcThreads, kTcSmem, s>>>(a);
    } else {
        k_net_rec<<<N.grid_fwd, kBlock, 0, s>>>(a);
        k_net_l2_tc<false><<<N.grid_tc, kTcThreads, kTcSmem, s>>>(a);
    }
    OASIS_CUDA(cudaGetLastError());
}

void net_check(Net& N, cudaStream_t s) {
    int32_t e = 0;
    OASIS_CUDA(cudaMemcpyAsync(&e, N.err.p, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    OASIS_CUDA(cudaStreamSynchronize(s));
    if (e) {
        OASIS_CUDA(cudaMemsetAsync(N.err.p, 0, sizeof(int32_t), s));
        throw Error(OASIS_EWAIT, "tensor-core layer: a bounded wait ran out");
    }
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
    k_net_bop<<<8, 256, 0, s>>>(N.p16.p, N.bop.p);
    OASIS_CUDA(cudaGetLastError());
}

void net_set_params(Net& N, const float* host) {
    OASIS_CUDA(cudaMemcpy(N.p32.p, host, kNetParams * sizeof(float), cudaMemcpyHostToDevice));
    k_net_to_bf16<<<(kNetParams + 255) / 256, 256>>>(N.p32.p, N.p16.p);
    k_net_image<<<4, 256>>>(N.p16.p, N.img.p);
    k_net_bop<<<8, 256>>>(N.p16.p, N.bop.p);
    OASIS_CUDA(cudaGetLastError());
    OASIS_CUDA(cudaMemset(N.mom.p, 0, N.mom.bytes()));
    OASIS_CUDA(cudaMemset(N.var.p, 0, N.var.bytes()));
    OASIS_CUDA(cudaDeviceSynchronize());
}

}  // namespace oasis
