// One IPCS time step on the device: convection assembly fused with the
// Algorithm 2 combination, the tentative-velocity BiCGStab (d right-hand sides
// sharing one matrix), the pressure-correction CG, normalisation and the
// lumped-mass velocity update.  Every Krylov loop is device-driven: the
// scalars live in a KrylovState on the device, and the loops run either as
// CUDA-graph conditional WHILE nodes or, in eager mode, as host loops that
// poll the state.
//
// Unknowns are written in "delta form": the tentative solve is run for
// Delta = u^I - u^{n-1} with right-hand side r_0 = b - A u^{n-1}, and the
// pressure solve for phi = p - p* with right-hand side
// b_phi = -(1/dt) sum_k dP^k u_k^I (the K p* term of the algebraic pressure
// equation of Sec. 5 cancels).  The systems and their solutions are those of
// Sec. 5; only the initial residual is formed without the O(1/dt) cancellation
// of b - A u^{n-1}, which keeps float32 inner solves accurate.
//
// Sparse kernels use row tiles (kern.cuh): an entry-parallel phase with
// coalesced reads writes one product per pattern entry to shared memory, and a
// row-parallel phase sums each row and runs its epilogue.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <type_traits>

#include "kern.cuh"
#include "net.cuh"
#include "solver.cuh"

namespace oasis {

// Upper bound on refinement sweeps of one solve (each sweep also does at least
// one counted iteration, so max_it bounds them as well).
constexpr int kMaxSweeps = 1000;

__device__ __forceinline__ void set_cond(int use, cudaGraphConditionalHandle h, int v) {
    if (use) cudaGraphSetConditional(h, v ? 1u : 0u);
}

// A solver coefficient in the kernel's value type, read from its float64 value
// (float64 path) or its float mirror (mixed path).
template <class P>
__device__ __forceinline__ typename P::V coef(double d, float f) {
    if constexpr (P::mixed) return f;
    else return d;
}

__device__ __forceinline__ double acc_of_s(double a) { return a; }
__device__ __forceinline__ ff acc_of_s(float2 a) { return {a.x, a.y}; }
__device__ __forceinline__ double s_of_acc(double a) { return a; }
__device__ __forceinline__ float2 s_of_acc(ff a) { return make_float2(a.hi, a.lo); }
// S * V as an accumulator
__device__ __forceinline__ double acc_mul_sv(double s, double v) { return s * v; }
__device__ __forceinline__ ff acc_mul_sv(float2 s, float v) { return ff_mul_f({s.x, s.y}, v); }

// Scalar constants of a step in the kernel value type (computed on the host so
// that float32 kernels never touch float64 arithmetic).
template <class V>
struct Consts {
    V rdt, dt, nu, hnu, f[3];
};

// ================================================================ assembly
// The convecting velocity ubar = 1.5 u^{n-1} - 0.5 u^{n-2} (Eq. 22) once per dof
// in the value type (Sec. 5 precomputes it before the assembly), so that the
// cell pass gathers D values per vertex instead of both float64-quality states.
template <class P, int D>
__global__ void __launch_bounds__(kBlock) k_ubar(StepData<P> a) {
    using V = typename P::V;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < a.n * D; t += (int64_t)gridDim.x * blockDim.x)
        a.ubar[t] = (V)1.5 * s_v(a.u1[t]) - (V)0.5 * s_v(a.u2[t]);
}

// beta[c][m] = w_T grad lambda_m . sum_l ubar_l, ubar = 1.5 u^{n-1} - 0.5 u^{n-2}
// (Eq. 22), w_T = |T| / ((d+1)(d+2)).  With it the P1 convection element matrix is
//   C^T_im = w_T grad lambda_m . (sum_l ubar_l + ubar_i) = beta[T][m] + ubar_i . w_T grad lambda_m;
// the second term summed over the cells sharing an edge is ubar_i . dP_im / (d+2)
// and is added in the row pass.
// ABE (explicit Adams-Bashforth convection, Eq. 21): the same cell terms for
// the two convecting velocities u^{n-1} (into beta) and u^{n-2} (into beta2).
template <class P, int D, bool ABE>
__global__ void __launch_bounds__(kBlock) k_cell_beta(StepData<P> a) {
    using V = typename P::V;
    constexpr int NB = ABE ? 2 : 1;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < a.nc; c += (int64_t)gridDim.x * blockDim.x) {
        V S[NB][D];
#pragma unroll
        for (int b = 0; b < NB; ++b)
#pragma unroll
            for (int k = 0; k < D; ++k) S[b][k] = 0;
#pragma unroll
        for (int m = 0; m <= D; ++m) {
            const size_t j = (size_t)__ldg(&a.cell_dof[c * (D + 1) + m]) * D;
#pragma unroll
            for (int k = 0; k < D; ++k) {
                if constexpr (ABE) {
                    S[0][k] += s_v(a.u1[j + k]);
                    S[NB - 1][k] += s_v(a.u2[j + k]);
                } else {
                    S[0][k] += a.ubar[j + k];
                }
            }
        }
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            V out[4];
#pragma unroll
            for (int m = 0; m <= D; ++m) {
                V acc = 0;
#pragma unroll
                for (int k = 0; k < D; ++k) acc += __ldg(&a.gw[((size_t)c * (D + 1) + m) * D + k]) * S[b][k];
                out[m] = acc;
            }
            if (D == 2) out[3] = 0;
            V* dst = b == 0 ? a.beta : a.beta2;
#pragma unroll
            for (int m = 0; m < 4; ++m) dst[c * 4 + m] = out[m];
        }
    }
}

// Row pass of the convection assembly fused with Algorithm 2.  Per tile:
//  A (thread per row): the cell terms beta of the incident cells are summed
//    into a per-row, per-slot buffer in shared memory (increasing cell order,
//    no atomics).  (Splitting a row's cells over two threads, with a second
//    buffer, was measured slower at 128^3: 1.18 against 0.82 ms);
//  B (entry-parallel): C_ij = t1 + ubar_i . dP_ij / (d+2),
//    A_ij = M_ij/dt + C_ij/2 + nu K_ij/2 (Eq. 34), and the entry's share of
//    -(C_ij + nu K_ij) u_j^{n-1} - dP^k_ij p*_j;
//  C (thread per row): r0_i = f_k ML_i + sum of the shares, which is
//    b_k - A u_k^{n-1} for b_k = f_k ML + (2M/dt - A) u^{n-1} - dP^k p*, the
//    right-hand side formed by Algorithm 2.
// Dirichlet rows become unit rows of A with r0 = g - u^{n-1}.
// ABE: A = M/dt + nu K/2 and the shares -(nu K_ij u_j^{n-1} + 1.5 C1_ij u_j^{n-1}
// - 0.5 C2_ij u_j^{n-2} + dP_ij p*_j), C1 from u^{n-1}, C2 from u^{n-2} (Eq. 21):
// b - A u^{n-1} for b = (M/dt - nu K/2) u^{n-1} - 1.5 C1 u^{n-1} + 0.5 C2 u^{n-2}
// + f ML - dP p*.
template <class P, int D, bool ABE, int R>
__global__ void __launch_bounds__(kBlock) k_assemble(StepData<P> a, Consts<typename P::V> k_) {
    using V = typename P::V;
    using S = typename P::S;
    using Acc = typename P::Acc;
    constexpr int NB = ABE ? 2 : 1;
    extern __shared__ __align__(16) unsigned char dsm[];
    V* s_t1 = reinterpret_cast<V*>(dsm);                       // [NB][max_row][R]
    V* s_con = s_t1 + (size_t)NB * a.max_row * R;          // [tile_cap][D]
    __shared__ int32_t s_rp[R + 1];
    __shared__ V s_ub[NB][D][R];
    __shared__ int32_t s_dir[R];
    Acc part[D];
#pragma unroll
    for (int k = 0; k < D; ++k) acc_zero(part[k]);
    const V inv_d2 = (V)1 / (V)(D + 2);
    const int r = threadIdx.x;
    for (int64_t tile = blockIdx.x; tile * R < a.n; tile += gridDim.x) {
        const TileRange T = load_tile<R>(tile, a.n, a.rp, s_rp);
        if (r < T.nr) {
            const int64_t i = T.r0 + r;
            const int32_t len = s_rp[r + 1] - s_rp[r];
            for (int32_t sl = 0; sl < len; ++sl)
#pragma unroll
                for (int b = 0; b < NB; ++b) s_t1[((size_t)b * a.max_row + sl) * R + r] = 0;
            // incident cells 8 at a time: their indices and slots, then their
            // beta rows (one aligned 4-vector each), then the additions in cell
            // order (the same order as one at a time)
            constexpr int kU = 8;
            const int32_t q0 = a.inc_ptr[i], q1 = a.inc_ptr[i + 1];
            for (int32_t qb = q0; qb < q1; qb += kU) {
                int32_t c[kU];
                uint32_t w[kU];
#pragma unroll
                for (int u = 0; u < kU; ++u) {
                    const bool ok = qb + u < q1;
                    c[u] = ok ? a.inc_cell[qb + u] : 0;
                    w[u] = ok ? a.inc_slots[qb + u] : 0u;
                }
#pragma unroll
                for (int b = 0; b < NB; ++b) {
                    const V* bsrc = b == 0 ? a.beta : a.beta2;
                    V* t = s_t1 + (size_t)b * a.max_row * R;
                    Vec4A<V> bt[kU];
#pragma unroll
                    for (int u = 0; u < kU; ++u) bt[u] = reinterpret_cast<const Vec4A<V>*>(bsrc)[c[u]];
#pragma unroll
                    for (int u = 0; u < kU; ++u) {
                        if (qb + u >= q1) break;
#pragma unroll
                        for (int m = 0; m <= D; ++m) t[((w[u] >> (8 * m)) & 0xffu) * R + r] += bt[u].v[m];
                    }
                }
            }
#pragma unroll
            for (int k = 0; k < D; ++k) {
                if constexpr (ABE) {
                    s_ub[0][k][r] = s_v(a.u1[i * D + k]);
                    s_ub[NB - 1][k][r] = s_v(a.u2[i * D + k]);
                } else {
                    s_ub[0][k][r] = a.ubar[i * D + k];
                }
            }
            s_dir[r] = a.dir_index[i];
        }
        __syncthreads();
        for (int32_t e = T.e0 + r; e < T.e1; e += kBlock) {
            const int rr = tile_row_of(s_rp, T.nr, e);
            const int32_t sl = e - s_rp[rr];
            const int64_t ii = T.r0 + rr;
            const int32_t j = a.col[e];
            V gv[D], gdot[NB] = {};
#pragma unroll
            for (int k = 0; k < D; ++k) {
                gv[k] = a.G[(size_t)k * a.nnz + e];
#pragma unroll
                for (int b = 0; b < NB; ++b) gdot[b] += s_ub[b][k][rr] * gv[k];
            }
            V cb[NB];
#pragma unroll
            for (int b = 0; b < NB; ++b) cb[b] = s_t1[((size_t)b * a.max_row + sl) * R + rr] + gdot[b] * inv_d2;
            const V kv = a.K[e];
            // passive scalars: C(ubar), linear in the convecting velocity
            if (a.cbar) a.cbar[e] = ABE ? (V)1.5 * cb[0] - (V)0.5 * cb[NB - 1] : cb[0];
            V av = ABE ? a.M[e] * k_.rdt + k_.hnu * kv : a.M[e] * k_.rdt + (V)0.5 * cb[0] + k_.hnu * kv;
            if (s_dir[rr] >= 0) av = (j == ii) ? (V)1 : (V)0;
            a.A[e] = av;
            if (j == ii) a.dinvA[ii] = (V)1 / av;
            const V ps = s_v(a.pstar[j]);
            if constexpr (ABE) {
                const V c1 = (V)1.5 * cb[0] + k_.nu * kv, c2 = (V)0.5 * cb[NB - 1];
#pragma unroll
                for (int k = 0; k < D; ++k)
                    s_con[(size_t)(e - T.e0) * D + k] =
                        -(c1 * s_v(a.u1[(size_t)j * D + k]) - c2 * s_v(a.u2[(size_t)j * D + k]) + gv[k] * ps);
            } else {
                const V ck = cb[0] + k_.nu * kv;
#pragma unroll
                for (int k = 0; k < D; ++k)
                    s_con[(size_t)(e - T.e0) * D + k] = -(ck * s_v(a.u1[(size_t)j * D + k]) + gv[k] * ps);
            }
        }
        __syncthreads();
        if (r < T.nr) {
            const int64_t i = T.r0 + r;
            const int32_t b0 = s_rp[r] - T.e0, b1 = s_rp[r + 1] - T.e0;
            const int dir = s_dir[r];
#pragma unroll
            for (int k = 0; k < D; ++k) {
                V acc = 0;
                for (int32_t q = b0; q < b1; ++q) acc += s_con[(size_t)q * D + k];
                S r0v;
                if (dir >= 0) r0v = s_sub(a.g[(size_t)dir * D + k], a.u1[i * D + k]);
                else r0v = s_addv(s_from(k_.f[k] * a.ML[i]), acc);
                a.r0[i * D + k] = r0v;
                // initial guess of the solve: u^I_0 = 2 u^{n-1} - u^{n-2} (Delta_0 =
                // u^{n-1} - u^{n-2}); Dirichlet rows exact.  The stopping test stays
                // relative to r0 = b - A u^{n-1}, so the guess changes only the count.
                a.du[i * D + k] = dir >= 0 ? r0v : s_sub(a.u1[i * D + k], a.u2[i * D + k]);
                const V rv = s_v(r0v);
                acc_prod(part[k], rv, rv);
            }
        }
        __syncthreads();
    }
    double tot[D];
    if (grid_sum<D, Acc>(part, tot, a.partial, &a.stu->ticket) && threadIdx.x == 0) {
        KrylovState* st = a.stu;
        for (int k = 0; k < 3; ++k) {
            st->bb[k] = k < D ? tot[k] : 0.0;
            st->col_done[k] = k < D ? 0 : 1;
            st->in_done[k] = 1;
            st->it_total[k] = 0;
            st->rr[k] = k < D ? tot[k] : 0.0;
        }
        st->sweeps = 0;
        st->it_in = 0;
        st->status = OASIS_OK;
        st->first = 1;
    }
}

// ================================================================ BiCGStab
// Right-preconditioned BiCGStab (van der Vorst 1992) with Jacobi M = diag(A),
// per column k on A Delta_k = r0_k, inside refinement sweeps: every sweep starts
// from the float64-quality residual r = r0 - A Delta and ends with Delta += delta.
template <int NR>
__device__ __forceinline__ bool load_active(const KrylovState* st, int k0, int (&act)[NR]) {
    bool any = false;
#pragma unroll
    for (int c = 0; c < NR; ++c) {
        act[c] = !st->col_done[k0 + c] && !st->in_done[k0 + c];
        any |= act[c] != 0;
    }
    return any;
}

template <int NR>
__device__ __forceinline__ int any_inner(const KrylovState* st, int k0) {
    int any = 0;
    for (int c = 0; c < NR; ++c) any |= (!st->col_done[k0 + c] && !st->in_done[k0 + c]);
    return any;
}

__device__ __forceinline__ void mirror_coefs(KrylovState* st, int k) {
    st->alpha_f[k] = (float)st->alpha[k];
    st->omega_f[k] = (float)st->omega[k];
    st->beta_f[k] = (float)st->beta[k];
}

// Convergence test of an outer sweep and start of a new inner solve (last
// block, thread 0), from the squared norms of the float64-quality residuals.
template <int NR>
__device__ __forceinline__ void bicg_outer_finish(KrylovState* st, int k0, const double* tot, const Ctl& ctl) {
    int outer = 0;
    for (int c = 0; c < NR; ++c) {
        const int k = k0 + c;
        if (st->col_done[k]) continue;
        const double rr = tot[c];
        st->rr[k] = rr;
        if (!isfinite(rr)) {
            st->status = OASIS_ENAN;
            st->col_done[k] = 1;
        } else if (rr <= ctl.rtol2 * st->bb[k]) {
            st->col_done[k] = 1;
        } else if (st->it_total[k] >= ctl.max_it || st->sweeps >= kMaxSweeps) {
            st->status = OASIS_ENOTCONV;
            st->col_done[k] = 1;
        } else {
            st->in_done[k] = 0;
            st->rho[k] = 1.0;
            st->alpha[k] = 1.0;
            st->omega[k] = 1.0;
            st->beta[k] = 0.0;
            mirror_coefs(st, k);
            st->rho_new[k] = rr;
            st->rr0_in[k] = rr;
            st->rr_in[k] = rr;
            outer = 1;
        }
    }
    st->sweeps += 1;
    st->it_in = 0;
    set_cond(ctl.use_cond, ctl.h_outer, outer);
    set_cond(ctl.use_cond, ctl.h_inner, any_inner<NR>(st, k0));
}

// Outer sweep: r = r0 - A Delta with float64-quality products (float-float in
// the mixed path), convergence test, start of a new inner solve.
template <class P, int D, int NR, int R>
__global__ void __launch_bounds__(kBlock) k_bicg_outer(StepData<P> a, int k0, Ctl ctl) {
    using V = typename P::V;
    using S = typename P::S;
    using Acc = typename P::Acc;
    extern __shared__ __align__(16) unsigned char dsm[];
    Acc* s_prod = reinterpret_cast<Acc*>(dsm);                 // [tile_cap][NR]
    __shared__ int32_t s_rp[R + 1];
    int live[NR];
#pragma unroll
    for (int c = 0; c < NR; ++c) live[c] = !a.stu->col_done[k0 + c];
    Acc part[NR];
#pragma unroll
    for (int c = 0; c < NR; ++c) acc_zero(part[c]);
    const int r = threadIdx.x;
    for (int64_t tile = blockIdx.x; tile * R < a.n; tile += gridDim.x) {
        const TileRange T = load_tile<R>(tile, a.n, a.rp, s_rp);
        tile_entries<4, Vec<Acc, NR>>(
            T,
            [&](int32_t e) {
                const V av = a.A[e];
                const size_t j = (size_t)a.col[e] * D + k0;
                Vec<Acc, NR> it;
#pragma unroll
                for (int c = 0; c < NR; ++c) it.v[c] = acc_mul_sv(a.du[j + c], av);
                return it;
            },
            [&](int32_t e, const Vec<Acc, NR>& it) {
#pragma unroll
                for (int c = 0; c < NR; ++c) s_prod[(size_t)(e - T.e0) * NR + c] = it.v[c];
            });
        __syncthreads();
        if (r < T.nr) {
            const int64_t i = T.r0 + r;
            const int32_t b0 = s_rp[r] - T.e0, b1 = s_rp[r + 1] - T.e0;
#pragma unroll
            for (int c = 0; c < NR; ++c) {
                if (!live[c]) continue;
                Acc ax;
                acc_zero(ax);
                for (int32_t q = b0; q < b1; ++q) acc_add(ax, s_prod[(size_t)q * NR + c]);
                const size_t o = (size_t)i * D + k0 + c;
                const S rs = s_sub(a.r0[o], s_of_acc(ax));
                const V rv = s_v(rs);
                a.r[o] = rv;
                a.rh[o] = rv;
                a.p[o] = 0;
                a.v[o] = 0;
                a.dl[o] = 0;
                acc_prod(part[c], rv, rv);
            }
        }
        __syncthreads();
    }
    double tot[NR];
    if (grid_sum<NR, Acc>(part, tot, a.partial, &a.stu->ticket) && threadIdx.x == 0)
        bicg_outer_finish<NR>(a.stu, k0, tot, ctl);
}

// A product S * V added to an accumulator with the product's rounding error kept:
// float64 exactly as before; float-float lazily (the high parts summed by an
// error-free two-sum, every low part and error added in float, normalised once
// by lazy_norm), about 11 float operations instead of a full float-float add's 26.
__device__ __forceinline__ void lazy_add_prod(double& acc, double x, double v) { acc = fma(x, v, acc); }
__device__ __forceinline__ void lazy_add_prod(ff& acc, float2 x, float v) {
    const float p = x.x * v;
    const float e = __fmaf_rn(x.y, v, __fmaf_rn(x.x, v, -p));
    const ff t = two_sum(acc.hi, p);
    acc.hi = t.hi;
    acc.lo += t.lo + e;
}
__device__ __forceinline__ double lazy_norm(double a) { return a; }
__device__ __forceinline__ ff lazy_norm(ff a) { return two_sum(a.hi, a.lo); }

// The outer sweep in row-split form (G lanes per row, U rows in flight, as the
// row-split product): r = r0 - A Delta with float64-quality products, each
// lane's entries accumulated lazily, the group's lanes summed in a float-float
// shuffle tree; no shared-memory staging.
template <class P, int D, int NR, int G, int U>
__global__ void __launch_bounds__(kBlock) k_bicg_outer_rows(StepData<P> a, int k0, Ctl ctl) {
    using V = typename P::V;
    using S = typename P::S;
    using Acc = typename P::Acc;
    constexpr int RPW = 32 / G;
    int live[NR];
#pragma unroll
    for (int c = 0; c < NR; ++c) live[c] = !a.stu->col_done[k0 + c];
    Acc part[NR];
#pragma unroll
    for (int c = 0; c < NR; ++c) acc_zero(part[c]);
    const int32_t* __restrict__ rp = a.rp;
    const int32_t* __restrict__ col = a.col;
    const V* __restrict__ A = a.A;
    const S* __restrict__ du = a.du;
    const int lane = threadIdx.x & 31, lg = lane & (G - 1), grp = lane / G;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t base = w0 * RPW * U; base < a.n; base += nw * RPW * U) {
        int64_t i[U];
        int32_t q[U], e[U];
        Acc acc[U][NR];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            i[u] = base + u * RPW + grp;
            const bool ok = i[u] < a.n;
            q[u] = ok ? rp[i[u]] + lg : 0;
            e[u] = ok ? rp[i[u] + 1] : 0;
#pragma unroll
            for (int c = 0; c < NR; ++c) acc_zero(acc[u][c]);
        }
        bool more = false;
#pragma unroll
        for (int u = 0; u < U; ++u) more |= q[u] < e[u];
        while (more) {
            size_t j[U];
            V av[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const bool has = q[u] < e[u];
                j[u] = has ? (size_t)col[q[u]] * D + k0 : (size_t)k0;
                av[u] = has ? A[q[u]] : V(0);
            }
            S g[U][NR];
#pragma unroll
            for (int u = 0; u < U; ++u)
#pragma unroll
                for (int c = 0; c < NR; ++c) g[u][c] = du[j[u] + c];
            more = false;
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (q[u] < e[u]) {
#pragma unroll
                    for (int c = 0; c < NR; ++c) lazy_add_prod(acc[u][c], g[u][c], av[u]);
                    q[u] += G;
                }
                more |= q[u] < e[u];
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
#pragma unroll
            for (int c = 0; c < NR; ++c) {
                acc[u][c] = lazy_norm(acc[u][c]);
#pragma unroll
                for (int o = G / 2; o > 0; o >>= 1) acc_add(acc[u][c], acc_shfl(acc[u][c], o));
            }
            if (i[u] < a.n && lg == 0) {
#pragma unroll
                for (int c = 0; c < NR; ++c) {
                    if (!live[c]) continue;
                    const size_t o = (size_t)i[u] * D + k0 + c;
                    const S rs = s_sub(a.r0[o], s_of_acc(acc[u][c]));
                    const V rv = s_v(rs);
                    a.r[o] = rv;
                    a.rh[o] = rv;
                    a.p[o] = 0;
                    a.v[o] = 0;
                    a.dl[o] = 0;
                    acc_prod(part[c], rv, rv);
                }
            }
        }
    }
    double tot[NR];
    if (grid_sum<NR, Acc>(part, tot, a.partial, &a.stu->ticket) && threadIdx.x == 0)
        bicg_outer_finish<NR>(a.stu, k0, tot, ctl);
}

// p = r + beta (p - omega v),  ph = D^{-1} p
template <class P, int D, int NR>
__global__ void __launch_bounds__(kBlock) k_bicg_dir(StepData<P> a, int k0) {
    using V = typename P::V;
    int act[NR];
    if (!load_active<NR>(a.stu, k0, act)) return;
    V beta[NR], omega[NR];
#pragma unroll
    for (int c = 0; c < NR; ++c) {
        beta[c] = coef<P>(a.stu->beta[k0 + c], a.stu->beta_f[k0 + c]);
        omega[c] = coef<P>(a.stu->omega[k0 + c], a.stu->omega_f[k0 + c]);
    }
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.n; i += (int64_t)gridDim.x * blockDim.x) {
        const V di = a.dinvA[i];
#pragma unroll
        for (int c = 0; c < NR; ++c) {
            if (!act[c]) continue;
            const size_t o = (size_t)i * D + k0 + c;
            const V pv = a.r[o] + beta[c] * (a.p[o] - omega[c] * a.v[o]);
            a.p[o] = pv;
            a.ph[o] = di * pv;
        }
    }
}

// Coefficients from the product's dot products (last block, thread 0).
template <int MODE, int NR>
__device__ __forceinline__ void bicg_spmm_finish(KrylovState* st, int k0, const int (&act)[NR],
                                                 const double* tot, const Ctl& ctl) {
    for (int c = 0; c < NR; ++c) {
        if (!act[c]) continue;
        const int k = k0 + c;
        if (MODE == 0) {
            const double rv = tot[c];
            if (rv == 0.0 || !isfinite(rv)) {
                st->in_done[k] = 1;      // breakdown: restart from the float64-quality residual
                st->it_total[k] += 1;    // counted, so that restarts end at the cap
                st->alpha[k] = 0.0;
            } else {
                st->alpha[k] = st->rho_new[k] / rv;
            }
        } else {
            const double ts = tot[c], tt = tot[NR + c];
            st->omega[k] = (tt > 0.0 && isfinite(tt)) ? ts / tt : 0.0;
        }
        mirror_coefs(st, k);
    }
    if (MODE == 0) set_cond(ctl.use_cond, ctl.h_inner, any_inner<NR>(st, k0));
}

// y = A x with the dot products needed next:
//   MODE 0: v = A ph, <rhat, v>          -> alpha = rho / <rhat, v>
//   MODE 1: t = A sh, <t, s>, <t, t>     -> omega = <t, s> / <t, t>
template <class P, int D, int NR, int MODE, int R>
__global__ void __launch_bounds__(kBlock) k_bicg_spmm(StepData<P> a, int k0, Ctl ctl) {
    using V = typename P::V;
    using Acc = typename P::Acc;
    int act[NR];
    if (!load_active<NR>(a.stu, k0, act)) return;
    constexpr int NV = MODE == 0 ? NR : 2 * NR;
    extern __shared__ __align__(16) unsigned char dsm[];
    V* s_prod = reinterpret_cast<V*>(dsm);                     // [tile_cap][NR]
    __shared__ int32_t s_rp[R + 1];
    const V* __restrict__ x = MODE == 0 ? a.ph : a.sh;
    V* __restrict__ y = MODE == 0 ? a.v : a.t;
    V part[NV] = {};
    const int r = threadIdx.x;
    for (int64_t tile = blockIdx.x; tile * R < a.n; tile += gridDim.x) {
        const TileRange T = load_tile<R>(tile, a.n, a.rp, s_rp);
        tile_entries<8, Vec<V, NR>>(
            T,
            [&](int32_t e) {
                const V av = a.A[e];
                const size_t j = (size_t)a.col[e] * D + k0;
                Vec<V, NR> it;
#pragma unroll
                for (int c = 0; c < NR; ++c) it.v[c] = av * x[j + c];
                return it;
            },
            [&](int32_t e, const Vec<V, NR>& it) {
#pragma unroll
                for (int c = 0; c < NR; ++c) s_prod[(size_t)(e - T.e0) * NR + c] = it.v[c];
            });
        __syncthreads();
        if (r < T.nr) {
            const int64_t i = T.r0 + r;
            const int32_t b0 = s_rp[r] - T.e0, b1 = s_rp[r + 1] - T.e0;
#pragma unroll
            for (int c = 0; c < NR; ++c) {
                if (!act[c]) continue;
                V acc = 0;
                for (int32_t q = b0; q < b1; ++q) acc += s_prod[(size_t)q * NR + c];
                const size_t o = (size_t)i * D + k0 + c;
                y[o] = acc;
                if (MODE == 0) {
                    part[c] += a.rh[o] * acc;
                } else {
                    part[c] += acc * a.s[o];
                    part[NR + c] += acc * acc;
                }
            }
        }
        __syncthreads();
    }
    double tot[NV];
    if (grid_sum_lite<NV, V>(part, tot, a.partial, &a.stu->ticket) && threadIdx.x == 0)
        bicg_spmm_finish<MODE, NR>(a.stu, k0, act, tot, ctl);
}

// The same product and dots in row-split form: rows are served by groups of G
// lanes (lane lg takes the row's entries lg, lg + G, ...), and every group keeps
// U rows in flight (row pointers, then per round one entry of each unfinished
// row: value and column, then the NR gathered values), with no shared-memory
// staging; the lanes' sums meet in a fixed shuffle tree.  MINB: resident blocks
// per SM the registers are capped for (1 = no cap).  C16: columns read as the
// pattern's modular 16-bit offsets from the row (csr_dcol), 6 bytes per entry
// instead of 8.  Grid: one resident wave, rows walked grid-stride.
template <class P, int D, int NR, int MODE, int G, int U, int MINB, bool C16>
__global__ void __launch_bounds__(kBlock, MINB) k_bicg_spmm_rows(StepData<P> a, int k0, Ctl ctl) {
    using V = typename P::V;
    int act[NR];
    if (!load_active<NR>(a.stu, k0, act)) return;
    constexpr int NV = MODE == 0 ? NR : 2 * NR;
    constexpr int RPW = 32 / G;
    const V* __restrict__ x = MODE == 0 ? a.ph : a.sh;
    V* __restrict__ y = MODE == 0 ? a.v : a.t;
    const int32_t* __restrict__ rp = a.rp;
    const int32_t* __restrict__ col = a.col;
    const int16_t* __restrict__ dcol = a.csr_dcol;
    const V* __restrict__ A = a.A;
    const int lane = threadIdx.x & 31, lg = lane & (G - 1), grp = lane / G;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    V part[NV] = {};
    // row and entry offsets fit 32 bits (the mesh holds fewer than 2^31 dofs and
    // pattern entries; D n stays below 2^32), which keeps the kernel's registers
    // down: the product runs latency bound, so resident warps matter
    const uint32_t n32 = (uint32_t)a.n;
    for (int64_t base = w0 * RPW * U; base < a.n; base += nw * RPW * U) {
        uint32_t i[U];
        int32_t q[U], e[U];
        V acc[U][NR];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            i[u] = (uint32_t)(base + u * RPW + grp);
            const bool ok = i[u] < n32;
            q[u] = ok ? rp[i[u]] + lg : 0;
            e[u] = ok ? rp[i[u] + 1] : 0;
#pragma unroll
            for (int c = 0; c < NR; ++c) acc[u][c] = 0;
        }
        bool more = false;
#pragma unroll
        for (int u = 0; u < U; ++u) more |= q[u] < e[u];
        while (more) {
            uint32_t j[U];
            V av[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const bool has = q[u] < e[u];
                uint32_t jc;
                if constexpr (C16) {
                    // row + offset, wrapped once into [0, n)
                    int32_t jj = (int32_t)i[u] + (int32_t)(has ? dcol[q[u]] : (int16_t)0);
                    jj = jj < 0 ? jj + (int32_t)n32 : jj;
                    jc = (uint32_t)jj >= n32 ? (uint32_t)jj - n32 : (uint32_t)jj;
                } else {
                    jc = has ? (uint32_t)col[q[u]] : 0u;
                }
                j[u] = has ? jc * D + k0 : (uint32_t)k0;
                av[u] = has ? A[q[u]] : V(0);
            }
            V g[U][NR];
#pragma unroll
            for (int u = 0; u < U; ++u)
#pragma unroll
                for (int c = 0; c < NR; ++c) g[u][c] = x[j[u] + c];
            more = false;
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (q[u] < e[u]) {
#pragma unroll
                    for (int c = 0; c < NR; ++c) acc[u][c] += av[u] * g[u][c];
                    q[u] += G;
                }
                more |= q[u] < e[u];
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
#pragma unroll
            for (int c = 0; c < NR; ++c) {
#pragma unroll
                for (int o = G / 2; o > 0; o >>= 1) acc[u][c] += __shfl_xor_sync(0xffffffffu, acc[u][c], o);
            }
            if (i[u] < n32 && lg == 0) {
#pragma unroll
                for (int c = 0; c < NR; ++c) {
                    if (!act[c]) continue;
                    const uint32_t o = i[u] * D + k0 + c;
                    y[o] = acc[u][c];
                    if (MODE == 0) {
                        part[c] += a.rh[o] * acc[u][c];
                    } else {
                        part[c] += acc[u][c] * a.s[o];
                        part[NR + c] += acc[u][c] * acc[u][c];
                    }
                }
            }
        }
    }
    double tot[NV];
    if (grid_sum_lite<NV, V>(part, tot, a.partial, &a.stu->ticket) && threadIdx.x == 0)
        bicg_spmm_finish<MODE, NR>(a.stu, k0, act, tot, ctl);
}

// Candidate shapes of the d-RHS BiCGStab product for the autotuner: the row-tile
// form (lanes = 0) and row-split forms (G lanes per row, U rows in flight).  The
// shapes add a row's products in different orders, so the candidates agree to
// rounding, not bitwise; a solver keeps one shape for its whole life (and a
// caller may force one with bicg_variant).
// A row-split shape also runs the sweeps' outer residual in row-split form
// (same lanes per row, two rows in flight), the row-tile shape in tile form.
// Shapes with c16 = 1 read the columns as 16-bit offsets (meshes whose ordering
// keeps every neighbour within 2^15 of its row, modulo n); the tuner skips them
// elsewhere.
template <class P, int D>
struct BicgVariant {
    void (*fn0)(StepData<P>, int, Ctl);
    void (*fn1)(StepData<P>, int, Ctl);
    void (*outer)(StepData<P>, int, Ctl);   // row-split outer residual (null: tile form)
    int lanes, rows, minb, c16;
};
constexpr int kBicgVariants = 8;
template <class P, int D>
static const BicgVariant<P, D>* bicg_variant_table() {
#define OASIS_BICGV(G, U, B, C)                                                                              \
    {k_bicg_spmm_rows<P, D, D, 0, G, U, B, C>, k_bicg_spmm_rows<P, D, D, 1, G, U, B, C>,                    \
     k_bicg_outer_rows<P, D, D, G, 2>, G, U, B, C}
    static const BicgVariant<P, D> t[kBicgVariants] = {
        {k_bicg_spmm<P, D, D, 0, kTileN>, k_bicg_spmm<P, D, D, 1, kTileN>, nullptr, 0, kTileN, 1, 0},
        OASIS_BICGV(4, 4, 1, false), OASIS_BICGV(4, 4, 5, false), OASIS_BICGV(2, 4, 1, false),
        OASIS_BICGV(2, 4, 5, false), OASIS_BICGV(4, 4, 1, true), OASIS_BICGV(4, 4, 5, true),
        OASIS_BICGV(2, 4, 1, true)};
#undef OASIS_BICGV
    return t;
}

// s = r - alpha v,  sh = D^{-1} s
template <class P, int D, int NR>
__global__ void __launch_bounds__(kBlock) k_bicg_s(StepData<P> a, int k0) {
    using V = typename P::V;
    int act[NR];
    if (!load_active<NR>(a.stu, k0, act)) return;
    V alpha[NR];
#pragma unroll
    for (int c = 0; c < NR; ++c) alpha[c] = coef<P>(a.stu->alpha[k0 + c], a.stu->alpha_f[k0 + c]);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.n; i += (int64_t)gridDim.x * blockDim.x) {
        const V di = a.dinvA[i];
#pragma unroll
        for (int c = 0; c < NR; ++c) {
            if (!act[c]) continue;
            const size_t o = (size_t)i * D + k0 + c;
            const V sv = a.r[o] - alpha[c] * a.v[o];
            a.s[o] = sv;
            a.sh[o] = di * sv;
        }
    }
}

// delta += alpha ph + omega sh,  r = s - omega t,  <rhat, r>, <r, r>
template <class P, int D, int NR>
__global__ void __launch_bounds__(kBlock) k_bicg_xr(StepData<P> a, int k0, Ctl ctl) {
    using V = typename P::V;
    using Acc = typename P::Acc;
    int act[NR];
    if (!load_active<NR>(a.stu, k0, act)) return;
    V alpha[NR], omega[NR];
#pragma unroll
    for (int c = 0; c < NR; ++c) {
        alpha[c] = coef<P>(a.stu->alpha[k0 + c], a.stu->alpha_f[k0 + c]);
        omega[c] = coef<P>(a.stu->omega[k0 + c], a.stu->omega_f[k0 + c]);
    }
    V part[2 * NR] = {};
    // distinct arrays: restrict lets the loads of later rows start early
    V* __restrict__ dl = a.dl;
    V* __restrict__ rr_ = a.r;
    const V* __restrict__ ph = a.ph;
    const V* __restrict__ sh = a.sh;
    const V* __restrict__ sv_ = a.s;
    const V* __restrict__ tv = a.t;
    const V* __restrict__ rh = a.rh;
#pragma unroll 4
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.n; i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int c = 0; c < NR; ++c) {
            if (!act[c]) continue;
            const size_t o = (size_t)i * D + k0 + c;
            dl[o] += alpha[c] * ph[o] + omega[c] * sh[o];
            const V rv = sv_[o] - omega[c] * tv[o];
            rr_[o] = rv;
            part[c] += rh[o] * rv;
            part[NR + c] += rv * rv;
        }
    }
    double tot[2 * NR];
    if (grid_sum_lite<2 * NR, V>(part, tot, a.partial, &a.stu->ticket) && threadIdx.x == 0) {
        KrylovState* st = a.stu;
        for (int c = 0; c < NR; ++c) {
            if (!act[c]) continue;
            const int k = k0 + c;
            const double rho_new = tot[c], rr = tot[NR + c];
            st->it_total[k] += 1;
            const double om = st->omega[k];
            st->beta[k] = (st->rho_new[k] != 0.0 && om != 0.0) ? (rho_new / st->rho_new[k]) * (st->alpha[k] / om) : 0.0;
            st->rho[k] = st->rho_new[k];
            st->rho_new[k] = rho_new;
            st->rr_in[k] = rr;
            mirror_coefs(st, k);
            const bool stop = !isfinite(rr) || rr <= ctl.inner2 * st->rr0_in[k] || rr <= ctl.abs2 * st->bb[k] ||
                              om == 0.0 || rho_new == 0.0 || st->it_total[k] >= ctl.max_it ||
                              st->it_in + 1 >= ctl.sweep_cap;
            if (stop) st->in_done[k] = 1;
        }
        st->it_in += 1;
        set_cond(ctl.use_cond, ctl.h_inner, any_inner<NR>(st, k0));
    }
}

// Delta += delta for the columns refined in this sweep.
template <class P, int D, int NR>
__global__ void __launch_bounds__(kBlock) k_bicg_correct(StepData<P> a, int k0) {
    int live[NR];
    bool any = false;
#pragma unroll
    for (int c = 0; c < NR; ++c) {
        live[c] = !a.stu->col_done[k0 + c];
        any |= live[c] != 0;
    }
    if (!any) return;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.n; i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int c = 0; c < NR; ++c) {
            if (!live[c]) continue;
            const size_t o = (size_t)i * D + k0 + c;
            a.du[o] = s_addv(a.du[o], a.dl[o]);
        }
    }
}

// ================================================================ pressure
// u^I = u^{n-1} + Delta rounded to the value type (for the divergence products).

// The mean of the right-hand side (for the projection on sum_i b_i = 0) and a
// reset of the pressure solve's state (last block, thread 0).
__device__ __forceinline__ void pressure_rhs_finish(KrylovState* st, double total, int64_t n) {
    st->mean = total / (double)n;
    const float mh = (float)st->mean;
    st->mean_hi = mh;
    st->mean_lo = (float)(st->mean - (double)mh);
    for (int k = 0; k < 3; ++k) {
        st->col_done[k] = k == 0 ? 0 : 1;
        st->in_done[k] = 1;
        st->it_total[k] = 0;
    }
    st->sweeps = 0;
    st->it_in = 0;
    st->status = OASIS_OK;
    st->first = 1;
}

// u^I = u^{n-1} + Delta once per dof (float64 quality), for the pressure
// right-hand side
template <class P, int D>
__global__ void __launch_bounds__(kBlock) k_tentative_velocity(StepData<P> a) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < a.n * D; t += (int64_t)gridDim.x * blockDim.x)
        a.uI[t] = s_add(a.u1[t], a.du[t]);
}

// S * S added lazily to an accumulator (the product's rounding error and the
// cross terms kept, the high parts summed by an error-free two-sum, the low
// parts in float; normalised once by lazy_norm): float64 exactly as before
__device__ __forceinline__ void lazy_add_prod_s(double& acc, double x, double y) { acc = fma(x, y, acc); }
__device__ __forceinline__ void lazy_add_prod_s(ff& acc, float2 x, float2 y) {
    const float p = x.x * y.x;
    float e = __fmaf_rn(x.x, y.x, -p);
    e = __fmaf_rn(x.x, y.y, e);
    e = __fmaf_rn(x.y, y.x, e);
    const ff t = two_sum(acc.hi, p);
    acc.hi = t.hi;
    acc.lo += t.lo + e;
}

// The pressure right-hand side in row-split form (G lanes per row, U rows in
// flight): b_phi_i = -(1/dt) sum_k sum_j dP^k_ij u_k,j^I with float-float dP^k
// and u^I, each lane's products accumulated lazily, the group's lanes summed in
// a float-float shuffle tree, then the projection's mean as before.
template <class P, int D, int G, int U>
__global__ void __launch_bounds__(kBlock) k_pressure_rhs_rows(StepData<P> a) {
    using S = typename P::S;
    using Acc = typename P::Acc;
    constexpr int RPW = 32 / G;
    const int32_t* __restrict__ rp = a.rp;
    const int32_t* __restrict__ col = a.col;
    const S* __restrict__ Gout = a.Gout;
    const S* __restrict__ uI = a.uI;
    S* __restrict__ bo = a.b;
    const S mrdt = s_of_double<S>(-1.0 / a.dt);
    const int64_t nnz = a.nnz;
    const int lane = threadIdx.x & 31, lg = lane & (G - 1), grp = lane / G;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    Acc part[1];
    acc_zero(part[0]);
    for (int64_t base = w0 * RPW * U; base < a.n; base += nw * RPW * U) {
        int64_t i[U];
        int32_t q[U], e[U];
        Acc acc[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            i[u] = base + u * RPW + grp;
            const bool ok = i[u] < a.n;
            q[u] = ok ? rp[i[u]] + lg : 0;
            e[u] = ok ? rp[i[u] + 1] : 0;
            acc_zero(acc[u]);
        }
        bool more = false;
#pragma unroll
        for (int u = 0; u < U; ++u) more |= q[u] < e[u];
        while (more) {
            int64_t j[U];
            S gk[U][D], xk[U][D];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const bool has = q[u] < e[u];
                j[u] = has ? (int64_t)col[q[u]] * D : 0;
#pragma unroll
                for (int k = 0; k < D; ++k) gk[u][k] = has ? Gout[(size_t)k * nnz + q[u]] : s_zero<S>();
            }
#pragma unroll
            for (int u = 0; u < U; ++u)
#pragma unroll
                for (int k = 0; k < D; ++k) xk[u][k] = uI[j[u] + k];
            more = false;
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (q[u] < e[u]) {
#pragma unroll
                    for (int k = 0; k < D; ++k) lazy_add_prod_s(acc[u], gk[u][k], xk[u][k]);
                    q[u] += G;
                }
                more |= q[u] < e[u];
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            acc[u] = lazy_norm(acc[u]);
#pragma unroll
            for (int o = G / 2; o > 0; o >>= 1) acc_add(acc[u], acc_shfl(acc[u], o));
            if (i[u] < a.n && lg == 0) {
                const S bi = s_mul_s(s_of_acc(acc[u]), mrdt);
                bo[i[u]] = bi;
                acc_add(part[0], acc_of_s(bi));
            }
        }
    }
    double tot[1];
    if (grid_sum<1, Acc>(part, tot, a.partial, &a.stp->ticket) && threadIdx.x == 0)
        pressure_rhs_finish(a.stp, tot[0], a.n);
}

// mean of the pressure right-hand side (of_p = false) or of p = p* + phi
// (of_p = true) as a state value
template <class S>
__device__ __forceinline__ S mean_s(const KrylovState* st, bool of_p);
template <>
__device__ __forceinline__ double mean_s<double>(const KrylovState* st, bool of_p) {
    return of_p ? st->psum : st->mean;
}
template <>
__device__ __forceinline__ float2 mean_s<float2>(const KrylovState* st, bool of_p) {
    return of_p ? make_float2(st->meanp_hi, st->meanp_lo) : make_float2(st->mean_hi, st->mean_lo);
}

// Grid-stride walk over the SELL-32 slices, one warp per slice at a time: the
// reduction kernels run on a grid of one resident wave, so that their last
// block sums few partials.  body(i, len, base, lane) is called per slice with
// the lane's row i, the slice length and the lane's first SELL position.
template <class P, class F>
__device__ __forceinline__ void sell_slices(const StepData<P>& a, F&& body) {
    const int lane = (int)(threadIdx.x & 31);
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t sl = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; sl < a.n_slices; sl += nw)
        body(sl * 32 + lane, a.sell_len[sl], (int64_t)a.sell_ptr[sl] + lane, lane);
}

template <class P>
__device__ __forceinline__ bool sell_lane(const StepData<P>& a, int64_t& i, int& len, int64_t& base, int& lane) {
    lane = threadIdx.x & 31;
    const int64_t sl = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (sl >= a.n_slices) return false;
    i = sl * 32 + lane;
    len = a.sell_len[sl];
    base = (int64_t)a.sell_ptr[sl] + lane;
    return true;
}

// ---------------------------------------------------------------- learned guess
// Scales of the network inputs: s_b = rms(b - mean b), s_phi = rms(phi^{n-1})
// (1 where zero).
template <class P>
__global__ void __launch_bounds__(kBlock) k_guess_scales(StepData<P> a) {
    using V = typename P::V;
    using S = typename P::S;
    const S mean = mean_s<S>(a.stp, false);
    V part[2] = {};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.n; i += (int64_t)gridDim.x * blockDim.x) {
        const V bv = s_v(s_sub(a.b[i], mean)), f1 = s_v(a.phi_h1[i]);
        part[0] += bv * bv;
        part[1] += f1 * f1;
    }
    double tot[2];
    if (grid_sum_lite<2, V>(part, tot, a.partial, &a.stp->ticket) && threadIdx.x == 0) {
        for (int k = 0; k < 2; ++k) {
            const double r = sqrt(tot[k] / (double)a.n);
            a.stp->gscale[k] = r > 0.0 ? r : 1.0;
            a.stp->gscale_f[k] = (float)a.stp->gscale[k];
        }
    }
}

template <class P>
__global__ void __launch_bounds__(kBlock) k_guess_features(StepData<P> a) {
    using S = typename P::S;
    const S mean = mean_s<S>(a.stp, false);
    const float ib = 1.f / a.stp->gscale_f[0], ip = 1.f / a.stp->gscale_f[1];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.n; i += (int64_t)gridDim.x * blockDim.x) {
        a.feat[i * 3] = (float)s_v(s_sub(a.b[i], mean)) * ib;
        a.feat[i * 3 + 1] = (float)s_v(a.phi_h1[i]) * ip;
        a.feat[i * 3 + 2] = (float)s_v(a.phi_h2[i]) * ip;
    }
}

// The residual is the judge: ||(b - mean) - K phi0|| of the learned guess
// phi0 = s_phi y against that of the fallback phi^{n-1}; the smaller one is used.
template <class P>
__global__ void __launch_bounds__(kBlock) k_guess_judge(StepData<P> a) {
    using V = typename P::V;
    using S = typename P::S;
    const S mean = mean_s<S>(a.stp, false);
    const V sp = (V)a.stp->gscale_f[1];
    V part[2] = {};
    sell_slices(a, [&](int64_t i, int len, int64_t base, int) {
        V kl = 0, kp = 0;
        for (int k = 0; k < len; ++k) {
            const int64_t q = base + 32 * (int64_t)k;
            const int32_t j = a.sell_col[q];
            const V kv = a.Ks[q];
            kl += kv * (sp * (V)a.gy[j]);
            kp += kv * s_v(a.phi_h1[j]);
        }
        if (i < a.n) {
            const V bv = s_v(s_sub(a.b[i], mean));
            part[0] += (bv - kl) * (bv - kl);
            part[1] += (bv - kp) * (bv - kp);
        }
    });
    double tot[2];
    if (grid_sum_lite<2, V>(part, tot, a.partial, &a.stp->ticket) && threadIdx.x == 0) {
        a.stp->guess_rr[0] = tot[0];
        a.stp->guess_rr[1] = tot[1];
        a.stp->guess_used = (isfinite(tot[0]) && tot[0] < tot[1]) ? OASIS_GUESS_LEARNED : OASIS_GUESS_PREV_PHI;
    }
}

// Initial guess for phi: 0, the previous step's correction, or (mode LEARNED)
// the candidate the judge chose.
template <class P>
__global__ void k_phi_guess(StepData<P> a, int mode) {
    using S = typename P::S;
    const bool learned = mode == OASIS_GUESS_LEARNED && a.stp->guess_used == OASIS_GUESS_LEARNED;
    const float sp = a.stp->gscale_f[1];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.n; i += (int64_t)gridDim.x * blockDim.x) {
        if (learned) a.x[i] = s_from((typename P::V)(sp * a.gy[i]));
        else if (mode == OASIS_GUESS_ZERO) a.x[i] = s_zero<S>();
        else a.x[i] = a.phi_h1[i];
    }
}

// Training target of the last step: t = phi / s_phi.
template <class P>
__global__ void k_guess_target(StepData<P> a, float* t) {
    const float ip = 1.f / a.stp->gscale_f[1];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.n; i += (int64_t)gridDim.x * blockDim.x)
        t[i] = (float)s_v(a.phi[i]) * ip;
}


// ---------------------------------------------------------------- SELL-32 CG
// The pressure CG kernels on K stored as SELL-32 (one warp per slice of 32 rows,
// lane l owns row 32 s + l): every load of a column index or value is one
// 128-byte line per warp, the gathers of consecutive rows' k-th neighbours are
// consecutive for structured orderings, and row sums stay in registers.

// Outer sweep: r = (b - mean b) - K x with float64-quality products.
template <class P>
__global__ void __launch_bounds__(kBlock) k_pcg_outer_sell(StepData<P> a, Ctl ctl) {
    using V = typename P::V;
    using S = typename P::S;
    using Acc = typename P::Acc;
    const bool live = !a.stp->col_done[0];
    const S mean = mean_s<S>(a.stp, false);
    Acc part[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) acc_zero(part[k]);
    // restrict-qualified locals: the stores of one slice do not hold back the
    // next slice's loads
    const S* __restrict__ Kouts = a.Kouts;
    const S* __restrict__ xs = a.x;
    const int32_t* __restrict__ scol = a.sell_col;
    sell_slices(a, [&](int64_t i, int len, int64_t base, int) {
        Acc kx;
        acc_zero(kx);
        // four entries' column, value and gathered operand loads issued together,
        // then their products added in entry order
        constexpr int C = 4;
        for (int k = 0; k < len; k += C) {
            S kv[C], xv[C];
#pragma unroll
            for (int u = 0; u < C; ++u) {
                const int64_t q = base + 32 * (int64_t)(k + u);
                const bool ok = k + u < len;
                const int32_t j = ok ? scol[q] : 0;
                kv[u] = ok ? Kouts[q] : s_zero<S>();
                xv[u] = xs[j];
            }
#pragma unroll
            for (int u = 0; u < C; ++u)
                if (k + u < len) acc_add(kx, acc_of_s(s_mul_s(kv[u], xv[u])));
        }
        if (i < a.n) {
            const S bi = s_sub(a.b[i], mean);
            const V rv = s_v(s_sub(bi, s_of_acc(kx)));
            const V xv = s_v(a.x[i]);
            if (live) {
                CgQuad<V> q0;
                q0.r = rv;
                q0.w = 0;
                q0.s = 0;
                q0.d = a.dinvK[i];
                a.pq0[i] = q0;
                a.pp[i] = 0;
                a.pdl[i] = 0;
            }
            a.xv[i] = xv;
            acc_prod(part[0], rv, rv);
            const V bv = s_v(bi);
            acc_prod(part[1], bv, bv);
            acc_addv(part[2], s_v(a.pstar[i]));
            acc_addv(part[2], xv);
        }
    });
    double tot[3];
    if (grid_sum<3, Acc>(part, tot, a.partial, &a.stp->ticket) && threadIdx.x == 0) {
        KrylovState* st = a.stp;
        if (st->first) {
            st->bb[0] = tot[1];
            st->first = 0;
        }
        const double meanp = tot[2] / (double)a.n;
        st->psum = meanp;
        st->meanp_hi = (float)meanp;
        st->meanp_lo = (float)(meanp - (double)(float)meanp);
        int outer = 0;
        if (st->status != OASIS_OK) st->col_done[0] = 1;
        if (!st->col_done[0]) {
            const double rr = tot[0];
            st->rr[0] = rr;
            if (!isfinite(rr)) {
                st->status = OASIS_ENAN;
                st->col_done[0] = 1;
            } else if (rr <= ctl.rtol2 * st->bb[0]) {
                st->col_done[0] = 1;
            } else if (st->it_total[0] >= ctl.max_it || st->sweeps >= kMaxSweeps) {
                st->status = OASIS_ENOTCONV;
                st->col_done[0] = 1;
            } else {
                st->in_done[0] = 0;
                st->rr0_in[0] = rr;
                outer = 1;
            }
        }
        st->sweeps += 1;
        st->it_in = 0;
        set_cond(ctl.use_cond, ctl.h_outer, outer);
        set_cond(ctl.use_cond, ctl.h_inner, outer);
    }
}

// Start of an inner CG: w_0 = K M^{-1} r_0, gamma_0, delta_0, alpha_0.  Reads
// the quads {r_0, 0, 0, M^-1} of pq0 and writes {r_0, w_0, 0, M^-1} to pq1,
// where the first iteration reads them.
template <class P>
__global__ void __launch_bounds__(kBlock, P::mixed ? 8 : 4) k_pcg_init_sell(StepData<P> a, Ctl ctl) {
    using V = typename P::V;
    using Q = CgQuad<V>;
    if (a.stp->col_done[0] || a.stp->in_done[0]) return;
    const Q* __restrict__ q0 = a.pq0;
    V part[2] = {};
    int64_t i, base;
    int len, lane;
    if (sell_lane(a, i, len, base, lane)) {
        V w = 0;
        for (int k = 0; k < len; ++k) {
            const int64_t q = base + 32 * (int64_t)k;
            const Q g = q0[a.sell_col[q]];
            w += a.Ks[q] * (g.d * g.r);
        }
        if (i < a.n) {
            Q qi = q0[i];
            qi.w = w;
            a.pq1[i] = qi;
            const V u = qi.d * qi.r;
            part[0] += qi.r * u;
            part[1] += w * u;
        }
    }
    double tot[2];
    if (grid_sum_lite<2, V>(part, tot, a.partial, &a.stp->ticket) && threadIdx.x == 0) {
        KrylovState* st = a.stp;
        const double g0 = tot[0], d0 = tot[1];
        if (!(d0 > 0.0) || !isfinite(d0) || !isfinite(g0)) {
            st->in_done[0] = 1;
            st->it_total[0] += 1;
            st->alpha[0] = 0.0;
            set_cond(ctl.use_cond, ctl.h_inner, 0);
        } else {
            st->rho[0] = g0;
            st->alpha[0] = g0 / d0;
        }
        st->beta[0] = 0.0;
        mirror_coefs(st, 0);
    }
}

// Last block of a CG iteration: beta, alpha of the next iteration from the
// three reduced dot products (gamma = <r, u>, delta = <w, u>, <r, r>), the
// inner stopping test, and the loop condition.
template <class P>
__device__ __forceinline__ void pcg_iter_finish(const StepData<P>& a, const Ctl& ctl, const double (&tot)[3]) {
    KrylovState* st = a.stp;
    const double g = tot[0], dl = tot[1], rr = tot[2];
    st->it_total[0] += 1;
    const double g_old = st->rho[0], a_old = st->alpha[0];
    const double b_new = g_old != 0.0 ? g / g_old : 0.0;
    const double den = a_old != 0.0 ? dl - b_new * g / a_old : 0.0;
    const bool brk = !(den > 0.0) || !isfinite(den) || !isfinite(g) || g_old == 0.0;
    st->beta[0] = b_new;
    st->alpha[0] = brk ? 0.0 : g / den;
    st->rho[0] = g;
    st->rr_in[0] = rr;
    mirror_coefs(st, 0);
    const bool stop = brk || st->status != OASIS_OK || !isfinite(rr) || rr <= ctl.inner2 * st->rr0_in[0] ||
                      rr <= ctl.abs2 * st->bb[0] || st->it_total[0] >= ctl.max_it || st->it_in + 1 >= ctl.sweep_cap;
    if (stop) st->in_done[0] = 1;
    st->it_in += 1;
    set_cond(ctl.use_cond, ctl.h_inner, !stop);
}

// Column of SELL entry q of row `row`: the int32 index, or the 16-bit offset
// from the row taken modulo n.
template <bool D16, class P>
__device__ __forceinline__ int32_t sell_j(const StepData<P>& a, int64_t q, int32_t row) {
    if constexpr (D16) {
        int32_t j = row + (int32_t)a.sell_dcol[q];
        const int32_t n = (int32_t)a.n;
        j = j < 0 ? j + n : j;
        return j >= n ? j - n : j;
    } else {
        return a.sell_col[q];
    }
}

// Fused Chronopoulos-Gear iteration on SELL-32.  With the coefficients of the
// last reduction, every row forms s = w + beta s, r' = r - alpha s and
// u' = M^-1 r'; w' = K u' needs u' of the neighbours, which each lane rebuilds
// from the neighbour's gathered quad instead of waiting for a grid-wide sync.
// Iteration it_in reads the quads of one buffer and writes the other (parity).
// Shape parameters (chosen by the autotuner): C entries per lane have their
// column and value loads issued together, then their C gathers, then the C
// products; PF also issues the next chunk's column and value loads before the
// current products; D16 reads 16-bit column offsets.  C and PF trade registers
// (and so resident warps, MINB blocks per SM) for loads in flight per warp.
// The products are summed in entry order for every shape: same bits.
template <class P, int C, int MINB, bool PF, bool D16>
__global__ void __launch_bounds__(kBlock, MINB) k_pcg_iter_sell(StepData<P> a, Ctl ctl) {
    using V = typename P::V;
    using Q = CgQuad<V>;
    if (a.stp->col_done[0] || a.stp->in_done[0]) return;
    const int par = a.stp->it_in & 1;
    const Q* __restrict__ qo = par ? a.pq0 : a.pq1;
    Q* __restrict__ qn = par ? a.pq1 : a.pq0;
    const V alpha = coef<P>(a.stp->alpha[0], a.stp->alpha_f[0]);
    const V beta = coef<P>(a.stp->beta[0], a.stp->beta_f[0]);
    V part[3] = {};
    int64_t i, base;
    int len, lane;
    if (sell_lane(a, i, len, base, lane)) {
        const int32_t row = (int32_t)i;
        V w = 0;
        int32_t j[C];
        V kv[C];
        auto fetch = [&](int k, int32_t (&jj)[C], V (&kk)[C]) {
#pragma unroll
            for (int u = 0; u < C; ++u) {
                const int64_t q = base + 32 * (int64_t)(k + u);
                const bool ok = k + u < len;
                jj[u] = ok ? sell_j<D16>(a, q, row) : 0;
                kk[u] = ok ? a.Ks[q] : V(0);
            }
        };
        if constexpr (PF) fetch(0, j, kv);
        for (int k = 0; k < len; k += C) {
            if constexpr (!PF) fetch(k, j, kv);
            Q g[C];
#pragma unroll
            for (int u = 0; u < C; ++u) g[u] = qo[j[u]];
            V kc[C];
            if constexpr (PF) {
#pragma unroll
                for (int u = 0; u < C; ++u) kc[u] = kv[u];
                if (k + C < len) fetch(k + C, j, kv);
            } else {
#pragma unroll
                for (int u = 0; u < C; ++u) kc[u] = kv[u];
            }
#pragma unroll
            for (int u = 0; u < C; ++u)
                if (k + u < len) w += kc[u] * (g[u].d * (g[u].r - alpha * (g[u].w + beta * g[u].s)));
        }
        if (i < a.n) {
            const Q qi = qo[i];
            const V pv = qi.d * qi.r + beta * a.pp[i];
            const V sv = qi.w + beta * qi.s;
            a.pp[i] = pv;
            a.pdl[i] += alpha * pv;
            Q out;
            out.r = qi.r - alpha * sv;
            out.w = w;
            out.s = sv;
            out.d = qi.d;
            qn[i] = out;
            const V un = qi.d * out.r;
            part[0] += out.r * un;
            part[1] += w * un;
            part[2] += out.r * out.r;
        }
    }
    double tot[3];
    if (grid_sum_lite<3, V>(part, tot, a.partial, &a.stp->ticket) && threadIdx.x == 0) pcg_iter_finish<P>(a, ctl, tot);
}

// The same iteration with K streamed into shared memory by the bulk-copy
// (TMA) engine, in a persistent grid.  The slices are grouped in "virtual
// blocks" of 8 consecutive slices — exactly the rows one 256-thread block
// covers in k_pcg_iter_sell — and block b takes virtual blocks b, b + G, ...
// (G blocks), warp w the slice 8 vb + w of each.  Every warp owns a two-stage
// ring in shared memory: while it works on one slice, the values and columns
// of its next slice (contiguous in SELL order) are in flight as two
// cp.async.bulk copies completing on the stage's mbarrier; the lanes then read
// columns and values from shared memory, so the only global round trips left
// in the chain are the C gathers of the quads and the row's own loads, which
// are issued before the wait.  One partial per virtual block is stored with the
// same trees as the one-block-per-8-slices kernels, so every shape gives the
// same bits.  Every wait is bounded: on time-out the warp records OASIS_EWAIT,
// stops issuing and processing, waits (bounded) for its copies in flight, and
// the last block ends the solve.
template <class P, int WPB, int C, int MINB, bool D16>
__global__ void __launch_bounds__(WPB * 32, MINB) k_pcg_iter_tma(StepData<P> a, Ctl ctl) {
    using V = typename P::V;
    using Q = CgQuad<V>;
    using Col = typename std::conditional<D16, int16_t, int32_t>::type;
    static_assert(P::mixed, "the streamed CG iteration is built for float32 values");
    static_assert(WPB * 32 == kBlock, "virtual blocks are the 8-slice blocks of k_pcg_iter_sell");
    extern __shared__ __align__(128) unsigned char dsm[];
    __shared__ __align__(8) uint64_t bars[WPB][2];
    if (a.stp->col_done[0] || a.stp->in_done[0]) return;
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int par = a.stp->it_in & 1;
    const Q* __restrict__ qo = par ? a.pq0 : a.pq1;
    Q* __restrict__ qn = par ? a.pq1 : a.pq0;
    const V alpha = coef<P>(a.stp->alpha[0], a.stp->alpha_f[0]);
    const V beta = coef<P>(a.stp->beta[0], a.stp->beta_f[0]);
    const Col* __restrict__ cols = D16 ? reinterpret_cast<const Col*>(a.sell_dcol)
                                       : reinterpret_cast<const Col*>(a.sell_col);
    // stage layout: [max_row * 32] values, then [max_row * 32] columns (128-byte aligned)
    const size_t vbytes = (size_t)a.max_row * 32 * sizeof(V);
    const size_t sbytes = (vbytes + (size_t)a.max_row * 32 * sizeof(Col) + 127) & ~(size_t)127;
    unsigned char* wbase = dsm + (size_t)wib * 2 * sbytes;
    auto stage_v = [&](int st) { return reinterpret_cast<V*>(wbase + st * sbytes); };
    auto stage_c = [&](int st) { return reinterpret_cast<Col*>(wbase + st * sbytes + vbytes); };
    if (lane == 0) {
        mbar_init(&bars[wib][0], 1);
        mbar_init(&bars[wib][1], 1);
        fence_barrier_init();
    }
    __syncwarp();
    uint32_t issued[2] = {0u, 0u}, used[2] = {0u, 0u};     // copies per stage (same in every lane)
    auto issue = [&](int64_t sl, int st) {
        if (lane == 0) {
            const int64_t p0 = a.sell_ptr[sl];
            const uint32_t len = (uint32_t)a.sell_len[sl];
            const uint32_t vb = len * 32 * (uint32_t)sizeof(V), cb = len * 32 * (uint32_t)sizeof(Col);
            fence_proxy_async();
            mbar_expect_tx(&bars[wib][st], vb + cb);
            bulk_copy_g2s(stage_v(st), a.Ks + p0, vb, &bars[wib][st]);
            bulk_copy_g2s(stage_c(st), cols + p0, cb, &bars[wib][st]);
        }
        ++issued[st];
    };
    const int64_t n_vb = (a.n_slices + WPB - 1) / WPB;
    const int64_t G = gridDim.x;
    bool timed_out = false;
    int k = 0;
    int64_t vb = blockIdx.x;
    if (vb < n_vb && vb * WPB + wib < a.n_slices) issue(vb * WPB + wib, 0);
    for (; vb < n_vb; vb += G, ++k) {
        const int st = k & 1;
        const int64_t sl = vb * WPB + wib;
        const int64_t nsl = (vb + G) * WPB + wib;
        if (!timed_out && vb + G < n_vb && nsl < a.n_slices) issue(nsl, st ^ 1);
        V part[3] = {};
        if (!timed_out && sl < a.n_slices) {
            const int64_t i = sl * 32 + lane;
            const int32_t row = (int32_t)i;
            const bool own = i < a.n;
            Q qi{};
            V ppi = 0, pdli = 0;
            if (own) {
                qi = qo[i];
                ppi = a.pp[i];
                pdli = a.pdl[i];
            }
            const int len = a.sell_len[sl];
            if (!mbar_wait_bounded(&bars[wib][st], used[st] & 1u)) {
                timed_out = true;
            } else {
                ++used[st];
                const V* __restrict__ sv = stage_v(st);
                const Col* __restrict__ sc = stage_c(st);
                V w = 0;
                for (int k0 = 0; k0 < len; k0 += C) {
                    int32_t j[C];
                    V kv[C];
#pragma unroll
                    for (int u = 0; u < C; ++u) {
                        const bool ok = k0 + u < len;
                        const int e = (k0 + u) * 32 + lane;
                        int32_t jj = 0;
                        if (ok) {
                            if constexpr (D16) {
                                const int32_t n = (int32_t)a.n;
                                jj = row + (int32_t)sc[e];
                                jj = jj < 0 ? jj + n : jj;
                                jj = jj >= n ? jj - n : jj;
                            } else {
                                jj = sc[e];
                            }
                        }
                        j[u] = jj;
                        kv[u] = ok ? sv[e] : V(0);
                    }
                    Q g[C];
#pragma unroll
                    for (int u = 0; u < C; ++u) g[u] = qo[j[u]];
#pragma unroll
                    for (int u = 0; u < C; ++u)
                        if (k0 + u < len) w += kv[u] * (g[u].d * (g[u].r - alpha * (g[u].w + beta * g[u].s)));
                }
                if (own) {
                    const V pv = qi.d * qi.r + beta * ppi;
                    const V sv2 = qi.w + beta * qi.s;
                    a.pp[i] = pv;
                    a.pdl[i] = pdli + alpha * pv;
                    Q out;
                    out.r = qi.r - alpha * sv2;
                    out.w = w;
                    out.s = sv2;
                    out.d = qi.d;
                    qn[i] = out;
                    const V un = qi.d * out.r;
                    part[0] += out.r * un;
                    part[1] += w * un;
                    part[2] += out.r * out.r;
                }
            }
            __syncwarp();
        }
        block_partial_lite<3, V>(part, a.partial, vb);
    }
    if (timed_out) {
        // record the failure; let the copies this warp started finish (bounded)
        if (lane == 0) {
            a.stp->status = OASIS_EWAIT;
            for (int st = 0; st < 2; ++st)
                if (issued[st] > used[st]) mbar_wait_bounded(&bars[wib][st], (issued[st] - 1u) & 1u);
        }
        __syncwarp();
    }
    double tot[3];
    if (grid_finish_lite<3, V>(tot, a.partial, n_vb, &a.stp->ticket) &&
        threadIdx.x == 0)
        pcg_iter_finish<P>(a, ctl, tot);
}

// Candidate shapes of the CG iteration for the autotuner.
template <class P>
struct IterVariant {
    void (*fn)(StepData<P>, Ctl);
    int chunk, minb, pf, d16, tma, wpb;
};

#define OASIS_ITER(C, B, PF, D16) {k_pcg_iter_sell<P, C, B, PF, D16>, C, B, PF, D16, 0, kBlock / 32}
#define OASIS_ITER_TMA(W, C, B, D16) {k_pcg_iter_tma<P, W, C, B, D16>, C, B, 0, D16, 1, W}
template <class P>
static const IterVariant<P>* iter_variant_table(int& count) {
    if constexpr (P::mixed) {
        static const IterVariant<P> t[] = {
            OASIS_ITER(2, 8, false, false),   OASIS_ITER(4, 8, false, false),   OASIS_ITER(4, 6, false, false),
            OASIS_ITER(8, 4, false, false),   OASIS_ITER(8, 3, false, false),   OASIS_ITER(16, 2, false, false),
            OASIS_ITER(2, 6, true, false),    OASIS_ITER(4, 6, true, false),    OASIS_ITER(2, 8, false, true),
            OASIS_ITER(4, 8, false, true),    OASIS_ITER(2, 6, true, true),     OASIS_ITER(4, 6, true, true),
            OASIS_ITER_TMA(8, 8, 4, false),   OASIS_ITER_TMA(8, 8, 4, true),    OASIS_ITER_TMA(8, 16, 3, true),
            OASIS_ITER_TMA(8, 4, 4, true)};
        count = (int)(sizeof(t) / sizeof(t[0]));
        return t;
    } else {
        static const IterVariant<P> t[] = {OASIS_ITER(2, 4, false, false), OASIS_ITER(4, 4, false, false),
                                           OASIS_ITER(4, 3, false, false), OASIS_ITER(8, 2, false, false),
                                           OASIS_ITER(4, 3, true, false),  OASIS_ITER(4, 4, false, true)};
        count = (int)(sizeof(t) / sizeof(t[0]));
        return t;
    }
}
#undef OASIS_ITER_TMA
#undef OASIS_ITER

// ---------------------------------------------------------------- multigrid CG
// Chronopoulos-Gear CG with a general preconditioner u = M r (one multigrid
// V-cycle, amg.cu): per iteration the vector updates, the V-cycle, then
// w = K u with the three dot products in one reduction.

// Start of an inner solve: r from the sweep's residual (the quads written by
// k_pcg_outer_sell, which also cleared p and the update); s = 0.
template <class P>
__global__ void __launch_bounds__(kBlock) k_amg_cg_start(StepData<P> a) {
    if (a.stp->col_done[0] || a.stp->in_done[0]) return;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.n; i += (int64_t)gridDim.x * blockDim.x) {
        a.ar[i] = a.pq0[i].r;
        a.as[i] = 0;
    }
}

// p = u + beta p, s = w + beta s, delta += alpha p, r -= alpha s, and ||r||^2:
// when the new residual already meets the inner stopping test the inner solve
// ends here (counted; the loop's condition is cleared, so no V-cycle follows).
template <class P>
__global__ void __launch_bounds__(kBlock) k_amg_cg_update(StepData<P> a, Ctl ctl) {
    using V = typename P::V;
    if (a.stp->col_done[0] || a.stp->in_done[0]) return;
    const V alpha = coef<P>(a.stp->alpha[0], a.stp->alpha_f[0]);
    const V beta = coef<P>(a.stp->beta[0], a.stp->beta_f[0]);
    V part[1] = {};
    const V* __restrict__ au = a.au;
    const V* __restrict__ aw = a.aw;
    V* __restrict__ pp = a.pp;
    V* __restrict__ as_ = a.as;
    V* __restrict__ pdl = a.pdl;
    V* __restrict__ ar = a.ar;
#pragma unroll 4
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.n; i += (int64_t)gridDim.x * blockDim.x) {
        const V u = au[i], w = aw[i];
        const V pv = beta == V(0) ? u : u + beta * pp[i];
        const V sv = beta == V(0) ? w : w + beta * as_[i];
        pp[i] = pv;
        as_[i] = sv;
        pdl[i] += alpha * pv;
        const V r = ar[i] - alpha * sv;
        ar[i] = r;
        part[0] += r * r;
    }
    double tot[1];
    if (grid_sum_lite<1, V>(part, tot, a.partial, &a.stp->ticket) && threadIdx.x == 0) {
        KrylovState* st = a.stp;
        const double rr = tot[0];
        const bool stop = st->status != OASIS_OK || !isfinite(rr) || rr <= ctl.inner2 * st->rr0_in[0] ||
                          rr <= ctl.abs2 * st->bb[0] || st->it_total[0] + 1 >= ctl.max_it ||
                          st->it_in + 1 >= ctl.sweep_cap;
        if (stop) {
            st->it_total[0] += 1;
            st->it_in += 1;
            st->rr_in[0] = rr;
            st->in_done[0] = 1;
            set_cond(ctl.use_cond, ctl.h_inner, 0);
        }
    }
}

// End of the multigrid CG product: the three dots over the grid; START: first
// iteration of a sweep (alpha = gamma / delta, beta = 0); else the
// Chronopoulos-Gear update of alpha, beta and the inner stopping test.
template <class P, bool START>
__device__ __forceinline__ void amg_cg_spmv_finish(const StepData<P>& a, const Ctl& ctl,
                                                   typename P::V (&part)[3]) {
    using V = typename P::V;
    double tot[3];
    if (grid_sum_lite<3, V>(part, tot, a.partial, &a.stp->ticket) && threadIdx.x == 0) {
        if constexpr (START) {
            KrylovState* st = a.stp;
            const double g0 = tot[0], d0 = tot[1];
            if (!(d0 > 0.0) || !isfinite(d0) || !isfinite(g0)) {
                st->in_done[0] = 1;
                st->it_total[0] += 1;
                st->alpha[0] = 0.0;
                set_cond(ctl.use_cond, ctl.h_inner, 0);
            } else {
                st->rho[0] = g0;
                st->alpha[0] = g0 / d0;
            }
            st->beta[0] = 0.0;
            mirror_coefs(st, 0);
        } else {
            pcg_iter_finish<P>(a, ctl, tot);
        }
    }
}

// w = K u on SELL-32 with gamma = <r, u>, delta = <w, u> and <r, r>, then
// amg_cg_spmv_finish.
template <class P, bool START, bool D16, int C = 4, int MINB = 1>
__global__ void __launch_bounds__(kBlock, MINB) k_amg_cg_spmv(StepData<P> a, Ctl ctl) {
    using V = typename P::V;
    if (a.stp->col_done[0] || a.stp->in_done[0]) return;
    V part[3] = {};
    // the arrays through restrict-qualified locals: w is stored between slices,
    // and without them the next slice's loads could not move above that store
    // nor use the read-only path
    const V* __restrict__ Ks = a.Ks;
    const V* __restrict__ au = a.au;
    const V* __restrict__ ar = a.ar;
    V* __restrict__ aw = a.aw;
    const int16_t* __restrict__ dcol = a.sell_dcol;
    const int32_t* __restrict__ scol = a.sell_col;
    const int32_t n32 = (int32_t)a.n;
    sell_slices(a, [&](int64_t i, int len, int64_t base, int) {
        const int32_t row = (int32_t)i;
        V w = 0;
        for (int k = 0; k < len; k += C) {
            int32_t j[C];
            V kv[C];
#pragma unroll
            for (int u = 0; u < C; ++u) {
                const int64_t q = base + 32 * (int64_t)(k + u);
                const bool ok = k + u < len;
                int32_t jj = 0;
                if (ok) {
                    if constexpr (D16) {
                        jj = row + (int32_t)dcol[q];
                        jj = jj < 0 ? jj + n32 : jj;
                        jj = jj >= n32 ? jj - n32 : jj;
                    } else {
                        jj = scol[q];
                    }
                }
                j[u] = jj;
                kv[u] = ok ? Ks[q] : V(0);
            }
            V g[C];
#pragma unroll
            for (int u = 0; u < C; ++u) g[u] = au[j[u]];
#pragma unroll
            for (int u = 0; u < C; ++u)
                if (k + u < len) w += kv[u] * g[u];
        }
        if (i < a.n) {
            aw[i] = w;
            const V u = au[i], r = ar[i];
            part[0] += r * u;
            part[1] += w * u;
            part[2] += r * r;
        }
    });
    amg_cg_spmv_finish<P, START>(a, ctl, part);
}

// The same product on the pair-packed copy of K (float32 mixed path): per round
// C2 words of values (two entries each, 8 bytes) and C2 words of offsets are
// loaded, then their 2 C2 gathers; a row's products are added in entry order,
// as in k_amg_cg_spmv (the padding entry adds 0 times a valid operand).
template <class P, bool START, int C2, int MINB>
__global__ void __launch_bounds__(kBlock, MINB) k_amg_cg_spmv_pairs(StepData<P> a, Ctl ctl) {
    using V = typename P::V;
    static_assert(sizeof(V) == 4, "the pair-packed copy holds float32 values");
    if (a.stp->col_done[0] || a.stp->in_done[0]) return;
    V part[3] = {};
    const float2* __restrict__ kp = a.kpair;
    const uint32_t* __restrict__ cp = a.cpair;
    const V* __restrict__ au = a.au;
    const V* __restrict__ ar = a.ar;
    V* __restrict__ aw = a.aw;
    const int32_t n32 = (int32_t)a.n;
    const int lane = (int)(threadIdx.x & 31);
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t sl = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; sl < a.n_slices; sl += nw) {
        const int64_t i = sl * 32 + lane;
        const int32_t row = (int32_t)i;
        const int words = (a.sell_len[sl] + 1) >> 1;
        // 32-bit word offsets (the copy holds fewer than 2^31 entries)
        const uint32_t base = (uint32_t)(a.ptr2[sl] >> 1) + (uint32_t)lane;
        V w = 0;
        for (int k = 0; k < words; k += C2) {
            float2 kv[C2];
            uint32_t cw[C2];
#pragma unroll
            for (int u = 0; u < C2; ++u) {
                const uint32_t q = base + 32u * (uint32_t)(k + u);
                const bool ok = k + u < words;
                kv[u] = ok ? kp[q] : make_float2(0.f, 0.f);
                cw[u] = ok ? cp[q] : 0u;
            }
            V g[2 * C2];
#pragma unroll
            for (int e = 0; e < 2 * C2; ++e) {
                const uint32_t half = (e & 1) ? (cw[e >> 1] >> 16) : (cw[e >> 1] & 0xFFFFu);
                int32_t j = row + (int32_t)(int16_t)half;
                j = j < 0 ? j + n32 : j;
                j = j >= n32 ? j - n32 : j;
                g[e] = au[j];
            }
#pragma unroll
            for (int u = 0; u < C2; ++u)
                if (k + u < words) {
                    w += kv[u].x * g[2 * u];
                    w += kv[u].y * g[2 * u + 1];
                }
        }
        if (i < a.n) {
            aw[i] = w;
            const V u = au[i], r = ar[i];
            part[0] += r * u;
            part[1] += w * u;
            part[2] += r * r;
        }
    }
    amg_cg_spmv_finish<P, START>(a, ctl, part);
}

// Candidate shapes of the multigrid CG product: entries per lane whose column
// and value loads are issued together (C) and the blocks per SM the registers
// are sized for.  Every shape adds a row's products in entry order (same w);
// each runs one resident wave of its own, so on large meshes the dot products'
// partials can fall into other blocks and differ in the last bits, while every
// mesh small enough for one grid of a warp per slice gets the same bits.
template <class P>
struct AmgVariant {
    void (*fn16)(StepData<P>, Ctl);    // 16-bit offsets
    void (*fn32)(StepData<P>, Ctl);    // 32-bit columns
    void (*fnp)(StepData<P>, Ctl);     // pair-packed copy (float32 path with a multigrid hierarchy)
    int chunk, minb;                   // entries per round, blocks per SM the registers are sized for
    // the kernel for the layout at hand, or null where the shape does not apply
    void (*pick(const StepData<P>& a) const)(StepData<P>, Ctl) {
        if (fnp) return a.kpair ? fnp : nullptr;
        return a.sell_dcol ? fn16 : fn32;
    }
};
#define OASIS_AMGV(C, B) {k_amg_cg_spmv<P, false, true, C, B>, k_amg_cg_spmv<P, false, false, C, B>, nullptr, C, B}
#define OASIS_AMGP(C2, B) {nullptr, nullptr, k_amg_cg_spmv_pairs<P, false, C2, B>, 2 * C2, B}
constexpr int kAmgVariants = 7;                        // room for the longest table
template <class P>
static const AmgVariant<P>* amg_variant_table(int& count) {
    if constexpr (P::mixed) {
        static const AmgVariant<P> t[] = {OASIS_AMGV(4, 1), OASIS_AMGV(2, 8), OASIS_AMGV(4, 8), OASIS_AMGV(8, 4),
                                          OASIS_AMGP(2, 8), OASIS_AMGP(4, 6), OASIS_AMGP(4, 4)};
        count = (int)(sizeof(t) / sizeof(t[0]));
        return t;
    } else {
        static const AmgVariant<P> t[] = {OASIS_AMGV(4, 1), OASIS_AMGV(2, 8), OASIS_AMGV(4, 8), OASIS_AMGV(8, 4)};
        count = (int)(sizeof(t) / sizeof(t[0]));
        return t;
    }
}
#undef OASIS_AMGV
#undef OASIS_AMGP

template <class P>
__global__ void __launch_bounds__(kBlock) k_pcg_correct(StepData<P> a) {
    if (a.stp->col_done[0]) return;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.n; i += (int64_t)gridDim.x * blockDim.x)
        a.x[i] = s_addv(a.x[i], a.pdl[i]);
}

// Between inner repetitions (Algorithm 1): p* <- p* + phi, normalised to zero
// mean as in the update (the mean of p* + x comes from the last outer sweep);
// the velocities and the correction history are left as they are.
template <class P>
__global__ void __launch_bounds__(kBlock) k_pressure_advance(StepData<P> a) {
    using S = typename P::S;
    const S meanp = mean_s<S>(a.stp, true);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.n; i += (int64_t)gridDim.x * blockDim.x)
        a.pstar[i] = s_sub(s_add(a.pstar[i], a.x[i]), meanp);
}

// ================================================================ passive scalars
// Scalar equation of Sec. 3 for one scalar.  The fields of `a` point at that
// scalar's buffers: u1 = c^{n-1} [n], A / dinvA / r0 / du = its system, and
// dir_index / g = the scalars' Dirichlet set and this scalar's values;
// k_.nu = D_a, k_.hnu = D_a / 2, k_.f[0] = f_a.  With C(ubar) from the velocity
// assembly: A_a = M/dt + C/2 + D_a K/2 and r0 = f_a ML - (C + D_a K) c^{n-1},
// which is b_a - A_a c^{n-1} for b_a = (M/dt - C/2 - D_a K/2) c^{n-1} + f_a ML;
// Dirichlet rows are unit rows with r0 = g - c^{n-1}.  Resets the solve's
// scalars as the velocity assembly does.
template <class P>
__global__ void __launch_bounds__(kBlock) k_scalar_assemble(StepData<P> a, Consts<typename P::V> k_) {
    using V = typename P::V;
    using S = typename P::S;
    using Acc = typename P::Acc;
    extern __shared__ __align__(16) unsigned char dsm[];
    V* s_sh = reinterpret_cast<V*>(dsm);                       // [tile_cap]
    __shared__ int32_t s_rp[kTile + 1];
    __shared__ int32_t s_dir[kTile];
    Acc part[1];
    acc_zero(part[0]);
    const int r = threadIdx.x;
    for (int64_t tile = blockIdx.x; tile * kTile < a.n; tile += gridDim.x) {
        const TileRange T = load_tile(tile, a.n, a.rp, s_rp);
        if (r < T.nr) s_dir[r] = a.dir_index[T.r0 + r];
        __syncthreads();
        for (int32_t e = T.e0 + r; e < T.e1; e += kTile) {
            const int rr = tile_row_of(s_rp, T.nr, e);
            const int64_t ii = T.r0 + rr;
            const int32_t j = a.col[e];
            const V cv = a.cbar[e], kv = a.K[e];
            V av = a.M[e] * k_.rdt + (V)0.5 * cv + k_.hnu * kv;
            if (s_dir[rr] >= 0) av = (j == ii) ? (V)1 : (V)0;
            a.A[e] = av;
            if (j == ii) a.dinvA[ii] = (V)1 / av;
            s_sh[e - T.e0] = -(cv + k_.nu * kv) * s_v(a.u1[j]);
        }
        __syncthreads();
        if (r < T.nr) {
            const int64_t i = T.r0 + r;
            const int32_t b0 = s_rp[r] - T.e0, b1 = s_rp[r + 1] - T.e0;
            V acc = 0;
            for (int32_t q = b0; q < b1; ++q) acc += s_sh[q];
            const int dir = s_dir[r];
            const S r0v = dir >= 0 ? s_sub(a.g[dir], a.u1[i]) : s_addv(s_from(k_.f[0] * a.ML[i]), acc);
            a.r0[i] = r0v;
            a.du[i] = s_zero<S>();
            const V rv = s_v(r0v);
            acc_prod(part[0], rv, rv);
        }
        __syncthreads();
    }
    double tot[1];
    if (grid_sum<1, Acc>(part, tot, a.partial, &a.stu->ticket) && threadIdx.x == 0) {
        KrylovState* st = a.stu;
        for (int k = 0; k < 3; ++k) {
            st->bb[k] = k == 0 ? tot[0] : 0.0;
            st->col_done[k] = k == 0 ? 0 : 1;
            st->in_done[k] = 1;
            st->it_total[k] = 0;
            st->rr[k] = k == 0 ? tot[0] : 0.0;
        }
        st->sweeps = 0;
        st->it_in = 0;
        st->status = OASIS_OK;
        st->first = 1;
    }
}

// c^n = c^{n-1} + delta, Dirichlet rows = g.
template <class P>
__global__ void __launch_bounds__(kBlock) k_scalar_finish(StepData<P> a) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.n; i += (int64_t)gridDim.x * blockDim.x) {
        const int dir = a.dir_index[i];
        a.u1[i] = dir >= 0 ? a.g[dir] : s_add(a.u1[i], a.du[i]);
    }
}

// ================================================================ consistent-mass update
// Sec. 5 without lumping: M u^n = M u^I - dt dP^k phi with Dirichlet rows
// u^n = g, solved for the increment delta = u^n - u^I (the d components as d
// right-hand sides of one CG).  Dirichlet rows hold delta = g - u^I and stay out
// of the Krylov space (r = z = p = q = 0 there), so the CG runs on the interior
// block of M, which is symmetric positive definite.  The preconditioner is the
// lumped mass: for P1 elements every row sum of M is (d + 2) / 2 times its
// diagonal, so this is Jacobi.  Start: delta_0 = -dt dP^k phi / ML (the lumped
// update), stopping test ||r|| <= tol ||dt dP^k phi|| over the interior rows.
// Per iteration two kernels: q = M z + beta q, p = z + beta p with <p, q>, then
// delta += alpha p, r -= alpha q, z = r / ML with <r, z> and <r, r>; a converged
// component is frozen (its coefficients are no longer updated).

// delta_0 and -dt dP^k phi (kept in q until the residual kernel); block 0
// resets the solve's scalars (nothing else in this kernel reads them).
template <class P, int D>
__global__ void __launch_bounds__(kBlock) k_mass_guess(StepData<P> a, Consts<typename P::V> k_) {
    using V = typename P::V;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        KrylovState* st = a.stm;
        for (int k = 0; k < 3; ++k) {
            st->bb[k] = st->rr[k] = st->rho[k] = 0.0;
            st->alpha[k] = st->beta[k] = st->omega[k] = 0.0;
            mirror_coefs(st, k);
            st->col_done[k] = 1;
            st->it_total[k] = 0;
        }
        st->in_done[0] = 1;
        st->status = OASIS_OK;
    }
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.n; i += (int64_t)gridDim.x * blockDim.x) {
        const int dir = a.dir_index[i];
        if (dir >= 0) {
#pragma unroll
            for (int k = 0; k < D; ++k) {
                const size_t o = (size_t)i * D + k;
                a.mx[o] = s_v(s_sub(a.g[(size_t)dir * D + k], s_add(a.u1[o], a.du[o])));
                a.mq[o] = V(0);
            }
            continue;
        }
        V gp[D] = {};
        for (int32_t e = a.rp[i]; e < a.rp[i + 1]; ++e) {
            const V ph = a.xv[a.col[e]];
#pragma unroll
            for (int k = 0; k < D; ++k) gp[k] += a.G[(size_t)k * a.nnz + e] * ph;
        }
        const V iml = a.invML[i];
#pragma unroll
        for (int k = 0; k < D; ++k) {
            const size_t o = (size_t)i * D + k;
            const V b = -k_.dt * gp[k];
            a.mq[o] = b;
            a.mx[o] = b * iml;
        }
    }
}

// Interior rows: b = -dt dP^k phi - sum over Dirichlet columns of M_ij delta_j
// (the right-hand side of the interior system), r = b - M delta_0 over the
// interior columns; Dirichlet rows r = 0.  z = r / ML.  <r, z>, <r, r> and
// <b, b> per component, the stopping test ||r|| <= tol ||b||, beta = 0.  p and
// q are written by the first iteration (beta = 0 there).
template <class P, int D>
__global__ void __launch_bounds__(kBlock) k_mass_residual(StepData<P> a, Ctl ctl) {
    using V = typename P::V;
    V part[3 * D] = {};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.n; i += (int64_t)gridDim.x * blockDim.x) {
        V r[D] = {};
        if (a.dir_index[i] < 0) {
            V b[D], mi[D] = {};
#pragma unroll
            for (int k = 0; k < D; ++k) b[k] = a.mq[(size_t)i * D + k];
            for (int32_t e = a.rp[i]; e < a.rp[i + 1]; ++e) {
                const int32_t j = a.col[e];
                const V mv = a.M[e];
                const size_t oj = (size_t)j * D;
                if (a.dir_index[j] >= 0) {
#pragma unroll
                    for (int k = 0; k < D; ++k) b[k] -= mv * a.mx[oj + k];
                } else {
#pragma unroll
                    for (int k = 0; k < D; ++k) mi[k] += mv * a.mx[oj + k];
                }
            }
#pragma unroll
            for (int k = 0; k < D; ++k) {
                r[k] = b[k] - mi[k];
                part[2 * D + k] += b[k] * b[k];
            }
        }
        const V iml = a.invML[i];
#pragma unroll
        for (int k = 0; k < D; ++k) {
            const size_t o = (size_t)i * D + k;
            const V z = r[k] * iml;
            a.mr[o] = r[k];
            a.mz[o] = z;
            part[k] += r[k] * z;
            part[D + k] += r[k] * r[k];
        }
    }
    double tot[3 * D];
    if (grid_sum_lite<3 * D, V>(part, tot, a.partial, &a.stm->ticket) && threadIdx.x == 0) {
        KrylovState* st = a.stm;
        bool live = false;
        for (int k = 0; k < D; ++k) {
            st->rho[k] = tot[k];
            st->rr[k] = tot[D + k];
            st->bb[k] = tot[2 * D + k];
            st->beta[k] = 0.0;
            mirror_coefs(st, k);
            if (!isfinite(tot[k]) || !isfinite(tot[D + k]) || !isfinite(tot[2 * D + k])) st->status = OASIS_ENAN;
            const bool done = !(tot[D + k] > ctl.rtol2 * tot[2 * D + k]);
            st->col_done[k] = done ? 1 : 0;
            live |= !done;
        }
        if (st->status != OASIS_OK) live = false;
        st->in_done[0] = live ? 0 : 1;
        set_cond(ctl.use_cond, ctl.h_inner, live ? 1 : 0);
    }
}

// q = M z + beta q, p = z + beta p (interior rows; beta = 0 also clears what
// the start left there), alpha = <r, z> / <p, q> per live component.  Row
// tiles: the tile's entries M_ij z_j are formed with coalesced loads of M and
// the columns (8 in flight per thread), staged in shared memory and summed per
// row in entry order.
template <class P, int D>
__global__ void __launch_bounds__(kBlock) k_mass_spmv(StepData<P> a, Ctl ctl) {
    using V = typename P::V;
    extern __shared__ __align__(16) unsigned char dsm[];
    V* s_prod = reinterpret_cast<V*>(dsm);                     // [tile_cap][D]
    __shared__ int32_t s_rp[kTile + 1];
    const KrylovState* sc = a.stm;
    if (sc->in_done[0]) return;
    bool live[D];
    V beta[D];
#pragma unroll
    for (int k = 0; k < D; ++k) {
        live[k] = !sc->col_done[k];
        beta[k] = coef<P>(sc->beta[k], sc->beta_f[k]);
    }
    V part[D] = {};
    const int r = threadIdx.x;
    for (int64_t tile = blockIdx.x; tile * kTile < a.n; tile += gridDim.x) {
        const TileRange T = load_tile(tile, a.n, a.rp, s_rp);
        tile_entries<8, Vec<V, D>>(
            T,
            [&](int32_t e) {
                const V mv = a.M[e];
                const size_t oj = (size_t)a.col[e] * D;
                Vec<V, D> it;
#pragma unroll
                for (int k = 0; k < D; ++k) it.v[k] = mv * a.mz[oj + k];
                return it;
            },
            [&](int32_t e, const Vec<V, D>& it) {
#pragma unroll
                for (int k = 0; k < D; ++k) s_prod[(size_t)(e - T.e0) * D + k] = it.v[k];
            });
        __syncthreads();
        if (r < T.nr) {
            const int64_t i = T.r0 + r;
            const int32_t b0 = s_rp[r] - T.e0, b1 = s_rp[r + 1] - T.e0;
            const bool dir = a.dir_index[i] >= 0;
#pragma unroll
            for (int k = 0; k < D; ++k) {
                const size_t o = (size_t)i * D + k;
                if (dir) {
                    a.mp[o] = V(0);
                    a.mq[o] = V(0);
                    continue;
                }
                if (!live[k]) continue;
                V w = 0;
                for (int32_t q = b0; q < b1; ++q) w += s_prod[(size_t)q * D + k];
                const V p = beta[k] == V(0) ? a.mz[o] : a.mz[o] + beta[k] * a.mp[o];
                const V qv = beta[k] == V(0) ? w : w + beta[k] * a.mq[o];
                a.mp[o] = p;
                a.mq[o] = qv;
                part[k] += p * qv;
            }
        }
        __syncthreads();
    }
    double tot[D];
    if (grid_sum_lite<D, V>(part, tot, a.partial, &a.stm->ticket) && threadIdx.x == 0) {
        KrylovState* st = a.stm;
        for (int k = 0; k < D; ++k) {
            if (st->col_done[k]) continue;
            if (tot[k] > 0.0 && isfinite(tot[k])) {
                st->alpha[k] = st->rho[k] / tot[k];
            } else {
                // <p, q> = 0 with r != 0 cannot happen for SPD M: a breakdown
                st->alpha[k] = 0.0;
                st->col_done[k] = 1;
                st->status = isfinite(tot[k]) ? OASIS_EBREAKDOWN : OASIS_ENAN;
            }
            mirror_coefs(st, k);
        }
    }
}

// delta += alpha p, r -= alpha q, z = r / ML; <r, z>, <r, r>; beta = <r, z>_new /
// <r, z>_old, the stopping test per component and of the loop.
template <class P, int D>
__global__ void __launch_bounds__(kBlock) k_mass_update(StepData<P> a, Ctl ctl) {
    using V = typename P::V;
    const KrylovState* sc = a.stm;
    if (sc->in_done[0]) return;
    bool live[D];
    V alpha[D];
#pragma unroll
    for (int k = 0; k < D; ++k) {
        live[k] = !sc->col_done[k];
        alpha[k] = coef<P>(sc->alpha[k], sc->alpha_f[k]);
    }
    V part[2 * D] = {};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.n; i += (int64_t)gridDim.x * blockDim.x) {
        const V iml = a.invML[i];
#pragma unroll
        for (int k = 0; k < D; ++k) {
            if (!live[k]) continue;
            const size_t o = (size_t)i * D + k;
            a.mx[o] += alpha[k] * a.mp[o];
            const V r = a.mr[o] - alpha[k] * a.mq[o];
            const V z = r * iml;
            a.mr[o] = r;
            a.mz[o] = z;
            part[k] += r * z;
            part[D + k] += r * r;
        }
    }
    double tot[2 * D];
    if (grid_sum_lite<2 * D, V>(part, tot, a.partial, &a.stm->ticket) && threadIdx.x == 0) {
        KrylovState* st = a.stm;
        const int it = ++st->it_total[0];
        bool any = false;
        for (int k = 0; k < D; ++k) {
            if (st->col_done[k]) continue;
            const double rz = tot[k], rr = tot[D + k];
            st->rr[k] = rr;
            if (!isfinite(rz) || !isfinite(rr)) {
                st->status = OASIS_ENAN;
                st->col_done[k] = 1;
                continue;
            }
            if (!(rr > ctl.rtol2 * st->bb[k])) {
                st->col_done[k] = 1;
                continue;
            }
            st->beta[k] = st->rho[k] > 0.0 ? rz / st->rho[k] : 0.0;
            st->rho[k] = rz;
            mirror_coefs(st, k);
            any = true;
        }
        if (any && it >= ctl.max_it) {
            st->status = OASIS_ENOTCONV;
            any = false;
        }
        if (!any) {
            st->in_done[0] = 1;
            set_cond(ctl.use_cond, ctl.h_inner, 0);
        }
    }
}

// ================================================================ update
// u_k^n = u_k^I - dt (dP^k phi)_i / ML_i (Sec. 5, lumping), Dirichlet rows = g;
// p = p* + phi normalised to zero mean; rotation u^{n-2} <- u^{n-1} <- u^n,
// p* <- p, and the history of normalised corrections.
// CONS: u_k^n = u_k^I + delta_k, delta from the consistent-mass solve above.
template <class P, int D, bool CONS>
__global__ void __launch_bounds__(kBlock) k_update(StepData<P> a, Consts<typename P::V> k_) {
    using V = typename P::V;
    using S = typename P::S;
    extern __shared__ __align__(16) unsigned char dsm[];
    V* s_prod = reinterpret_cast<V*>(dsm);                     // [tile_cap][D]
    __shared__ int32_t s_rp[kTile + 1];
    const S meanp = mean_s<S>(a.stp, true);
    const int r = threadIdx.x;
    for (int64_t tile = blockIdx.x; tile * kTile < a.n; tile += gridDim.x) {
        const TileRange T = load_tile(tile, a.n, a.rp, s_rp);
        if constexpr (!CONS) tile_entries<8, Vec<V, D>>(
            T,
            [&](int32_t e) {
                const V ph = a.xv[a.col[e]];
                Vec<V, D> it;
#pragma unroll
                for (int k = 0; k < D; ++k) it.v[k] = a.G[(size_t)k * a.nnz + e] * ph;
                return it;
            },
            [&](int32_t e, const Vec<V, D>& it) {
#pragma unroll
                for (int k = 0; k < D; ++k) s_prod[(size_t)(e - T.e0) * D + k] = it.v[k];
            });
        __syncthreads();
        if (r < T.nr) {
            const int64_t i = T.r0 + r;
            const int32_t b0 = s_rp[r] - T.e0, b1 = s_rp[r + 1] - T.e0;
            const int dir = a.dir_index[i];
            const V iml = a.invML[i];
#pragma unroll
            for (int k = 0; k < D; ++k) {
                const size_t o = (size_t)i * D + k;
                const S u1 = a.u1[o];
                S un;
                if constexpr (CONS) {
                    un = s_addv(s_add(u1, a.du[o]), a.mx[o]);
                } else {
                    V gp = 0;
                    for (int32_t q = b0; q < b1; ++q) gp += s_prod[(size_t)q * D + k];
                    un = s_sub(s_add(u1, a.du[o]), s_from(k_.dt * gp * iml));
                }
                if (dir >= 0) un = a.g[(size_t)dir * D + k];
                a.u2[o] = u1;
                a.u1[o] = un;
            }
            const S ps = a.pstar[i];
            const S pn = s_sub(s_add(ps, a.x[i]), meanp);
            const S ph = s_sub(pn, ps);
            a.pstar[i] = pn;
            a.phi[i] = ph;
            a.phi_h2[i] = a.phi_h1[i];
            a.phi_h1[i] = ph;
        }
        __syncthreads();
    }
}

// ================================================================ conversions
// Internal index of caller index i under a renumbering of period pn (arrays of
// several fields of pn dofs each are renumbered field by field).
__device__ __forceinline__ int64_t renumbered(int64_t i, const int32_t* __restrict__ perm, int64_t pn) {
    if (!perm) return i;
    const int64_t f = i / pn;
    return f * pn + perm[i - f * pn];
}
// [comps][n] float64, caller order -> state [n][comps], internal order
template <class P>
__global__ void k_to_state(const double* __restrict__ src, typename P::S* __restrict__ dst, int64_t n, int comps,
                           const int32_t* __restrict__ perm, int64_t pn) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n * comps; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / comps;
        const int k = (int)(t - i * comps);
        dst[renumbered(i, perm, pn) * comps + k] = s_of_double<typename P::S>(src[(int64_t)k * n + i]);
    }
}
template <class P>
__global__ void k_from_state(const typename P::S* __restrict__ src, double* __restrict__ dst, int64_t n, int comps,
                             const int32_t* __restrict__ perm, int64_t pn) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n * comps; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / comps;
        const int k = (int)(t - i * comps);
        dst[(int64_t)k * n + i] = s_to_double(src[renumbered(i, perm, pn) * comps + k]);
    }
}
template <class V>
__global__ void k_v_to_double(const V* __restrict__ a, double* __restrict__ b, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        b[i] = (double)a[i];
}

// ================================================================ driver
// The kernel's dynamic shared memory limit is raised to the device maximum (the
// attribute is per kernel, shared by every solver of the process), and the
// occupancy for this solver's actual size gives the grid.
static int smem_optin() {
    static int v = 0;
    if (!v) {
        int dev = 0;
        OASIS_CUDA(cudaGetDevice(&dev));
        OASIS_CUDA(cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    }
    return v;
}

template <class K>
static int tile_grid(K kernel, size_t smem, int64_t tiles) {
    cudaFuncAttributes fa{};
    OASIS_CUDA(cudaFuncGetAttributes(&fa, kernel));
    const size_t room = (size_t)smem_optin() - fa.sharedSizeBytes;
    OASIS_CHECK(smem <= room, OASIS_EINVAL, "a row tile needs more shared memory than the device offers");
    OASIS_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)room));
    int per_sm = 0;
    OASIS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kBlock, smem));
    OASIS_CHECK(per_sm > 0, OASIS_EINVAL, "a row tile does not fit in shared memory");
    return (int)std::max<int64_t>(1, std::min<int64_t>(tiles, (int64_t)per_sm * num_sms()));
}

static int elem_grid(int64_t items) {
    const int64_t want = (items + kBlock - 1) / kBlock;
    return (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)num_sms() * 8));
}

// Elementwise kernels that end in a last-block reduction: two blocks per SM
// while the vectors fit in L2 (fewer partials and tickets; measured faster than
// one row per thread at 275k rows), a full resident wave of eight blocks per SM
// for larger systems, whose HBM streams need every warp's loads in flight
// (measured at 1.4M rows: 16 warps per SM left the CG update at 8 % of the DRAM
// bandwidth, stalled on latency).
static int red_grid(int64_t items) {
    const int64_t want = (items + kBlock - 1) / kBlock;
    const int per_sm = items >= (int64_t(1) << 20) ? 8 : 2;
    return (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)num_sms() * per_sm));
}

template <class P, int D>
struct StepImplT final : StepImpl {
    using V = typename P::V;
    using S = typename P::S;
    using Acc = typename P::Acc;
    Solver& Sv;
    StepData<P> a{};
    Consts<V> k_{};
    int64_t tiles = 0, tiles_n = 0;
    size_t sm_asm = 0, sm_asm2 = 0, sm_out_u = 0, sm_out_u1 = 0, sm_spmm = 0, sm_spmm1 = 0, sm_v1 = 0, sm_vd = 0;
    int g_asm = 1, g_asm2 = 1, g_out_u = 1, g_out_u1 = 1, g_spmm0 = 1, g_spmm1 = 1, g_spmm0_1 = 1, g_spmm1_1 = 1,
        g_rhs = 1, g_upd = 1, g_upd_c = 1, g_mspmv = 1, g_out_s = 1, g_spmm0_s = 1, g_spmm1_s = 1, g_sasm = 1;
    int ge_n = 1, ge_nd = 1, ge_c = 1, ge_red = 1;
    int g_sell = 1;
    // grid-stride SELL kernels ending in a reduction: one resident wave of each
    // kernel (its registers set the blocks per SM; a grid of 8 blocks per SM for a
    // kernel that fits 5 or 6 ran its latency-bound second wave nearly empty)
    int g_outer_sell = 1, g_judge = 1, g_cg_first = 1;
    int n_amg_v = 0;                                  // multigrid CG product shapes for this precision
    int amg_grid_v[kAmgVariants] = {};                // per shape, for the layout at hand
    int iter_v = 0;                                   // chosen CG iteration shape
    int amg_v = 0;                                    // chosen multigrid CG product shape
    int bicg_v = 0;                                   // chosen d-RHS BiCGStab product shape
    double bicg_us[kBicgVariants] = {0};
    int bicg_grid[kBicgVariants][2] = {};             // per product (v = A ph, t = A sh)
    int bicg_outer_grid[kBicgVariants] = {0};
    double amg_us[kAmgVariants] = {0};
    double tune_us[OASIS_MAX_VARIANTS] = {0};
    int it_grid[OASIS_MAX_VARIANTS] = {0}, it_block[OASIS_MAX_VARIANTS] = {0};
    size_t it_smem[OASIS_MAX_VARIANTS] = {0};


    // first multigrid CG product of a sweep, in the layout at hand
    void (*cg_first_fn() const)(StepData<P>, Ctl) {
        if constexpr (P::mixed) {
            if (a.kpair) return k_amg_cg_spmv_pairs<P, true, 4, 1>;
        }
        return a.sell_dcol ? k_amg_cg_spmv<P, true, true> : k_amg_cg_spmv<P, true, false>;
    }

    // one resident wave of a grid-stride SELL kernel (kBlock threads, no shared memory)
    template <class K>
    int sell_wave(K kernel) const {
        int per_sm = 0;
        OASIS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kBlock, 0));
        return (int)std::max<int64_t>(1, std::min<int64_t>(g_sell, (int64_t)std::max(per_sm, 1) * num_sms()));
    }

    template <class T>
    static T* mat(const DBuf<double>& d, const DBuf<float>& f) {
        if constexpr (sizeof(T) == 8) return (T*)(void*)d.p;
        else return (T*)(void*)f.p;
    }

    explicit StepImplT(Solver& s) : Sv(s) {
        Mesh& m = *Sv.m;
        a.rp = m.row_ptr.p;
        a.col = m.col.p;
        a.diag = m.diag.p;
        a.inc_ptr = m.inc_ptr.p;
        a.inc_cell = m.inc_cell.p;
        a.cell_dof = m.cell_dof.p;
        a.inc_slots = m.inc_slots.p;
        a.M = mat<V>(m.M64, m.M32);
        a.K = mat<V>(m.K64, m.K32);
        a.G = mat<V>(m.G64, m.G32);
        a.gw = mat<V>(m.gw64, m.gw32);
        a.ML = mat<V>(m.ML64, m.ML32);
        a.dinvK = mat<V>(m.dinvK64, m.dinvK32);
        a.invML = mat<V>(m.invML64, m.invML32);
        if constexpr (P::mixed) a.Kout = reinterpret_cast<const S*>(m.Kff.p);
        else a.Kout = reinterpret_cast<const S*>(m.K64.p);
        if constexpr (P::mixed) a.Gout = reinterpret_cast<const S*>(m.Gff.p);
        else a.Gout = reinterpret_cast<const S*>(m.G64.p);
        a.u1 = Sv.u1.as<S>();
        a.u2 = Sv.u2.as<S>();
        a.du = Sv.du.as<S>();
        a.r0 = Sv.r0.as<S>();
        a.pstar = Sv.pstar.as<S>();
        a.x = Sv.x.as<S>();
        a.b = Sv.b.as<S>();
        a.phi = Sv.phi.as<S>();
        a.phi_h1 = Sv.phi_h1.as<S>();
        a.phi_h2 = Sv.phi_h2.as<S>();
        a.g = Sv.g.as<S>();
        a.dir_index = Sv.dir_index.p;
        a.A = Sv.A.as<V>();
        a.dinvA = Sv.dinvA.as<V>();
        a.beta = Sv.beta.as<V>();
        a.beta2 = Sv.beta2.as<V>();
        a.ubar = Sv.ubar.as<V>();
        a.uI = Sv.uI.as<S>();
        V** w[9] = {&a.r, &a.rh, &a.p, &a.v, &a.s, &a.t, &a.ph, &a.sh, &a.dl};
        for (int q = 0; q < 9; ++q) *w[q] = Sv.w[q].as<V>();
        V** pw[3] = {&a.pp, &a.pdl, &a.xv};
        for (int q = 0; q < 3; ++q) *pw[q] = Sv.pw[q].as<V>();
        a.pq0 = Sv.pq[0].as<CgQuad<V>>();
        a.pq1 = Sv.pq[1].as<CgQuad<V>>();
        V** av[4] = {&a.ar, &a.as, &a.aw, &a.au};
        for (int q = 0; q < 4; ++q) *av[q] = Sv.amg_vec[q].as<V>();
        a.feat = Sv.feat.p;
        a.gy = Sv.gy.p;
        a.stu = Sv.st.p;
        a.stp = Sv.st.p + 1;
        a.stm = Sv.st.p + 2;
        V** mv[5] = {&a.mx, &a.mr, &a.mz, &a.mp, &a.mq};
        for (int q = 0; q < 5; ++q) *mv[q] = Sv.mw[q].as<V>();
        a.partial = Sv.partial.p;
        for (int k = 0; k < 3; ++k) a.f[k] = Sv.prm.f[k];
        a.dt = Sv.prm.dt;
        a.nu = Sv.prm.nu;
        a.n = m.n;
        a.nnz = m.nnz;
        a.nc = m.nc;
        a.max_row = m.max_row;
        a.tile_cap = m.tile_cap;
        a.n_slices = (m.n + 31) / 32;
        a.sell_ptr = m.sell_ptr.p;
        a.sell_len = m.sell_len.p;
        a.sell_col = m.sell_col.p;
        a.sell_dcol = m.sell_dcol.p;
        a.csr_dcol = m.csr_dcol.p;
        a.Ks = mat<V>(m.K64s, m.K32s);
        if constexpr (P::mixed) {
            if (Sv.prm.pressure_pc == OASIS_PC_AMG && m.amg && m.amg->fine.kp) {
                a.kpair = m.amg->fine.kp;
                a.cpair = m.amg->fine.cp;
                a.ptr2 = m.amg->fine.ptr2;
            }
        }
        if constexpr (P::mixed) a.Kouts = reinterpret_cast<const S*>(m.Kffs.p);
        else a.Kouts = reinterpret_cast<const S*>(m.K64s.p);
        k_.rdt = (V)(1.0 / Sv.prm.dt);
        k_.dt = (V)Sv.prm.dt;
        k_.nu = (V)Sv.prm.nu;
        k_.hnu = (V)(0.5 * Sv.prm.nu);
        for (int k = 0; k < 3; ++k) k_.f[k] = (V)Sv.prm.f[k];

        tiles = (m.n + kTile - 1) / kTile;
        tiles_n = (m.n + kTileN - 1) / kTileN;
        const size_t cap = (size_t)std::max(1, m.tile_cap);
        const size_t cap_n = (size_t)std::max(1, m.tile_cap_n);
        // assembly and BiCGStab products: narrow tiles (their per-entry staging)
        sm_asm = (size_t)m.max_row * kTileN * sizeof(V) + cap_n * D * sizeof(V);
        sm_asm2 = 2 * (size_t)m.max_row * kTileN * sizeof(V) + cap_n * D * sizeof(V);
        sm_out_u = cap_n * D * sizeof(Acc);
        sm_out_u1 = cap_n * sizeof(Acc);
        sm_spmm = cap_n * D * sizeof(V);
        sm_spmm1 = cap_n * sizeof(V);
        sm_v1 = cap * sizeof(V);
        sm_vd = cap * D * sizeof(V);
        g_asm = tile_grid(k_assemble<P, D, false, kTileN>, sm_asm, tiles_n);
        if (Sv.prm.convection == OASIS_CONV_ABE) g_asm2 = tile_grid(k_assemble<P, D, true, kTileN>, sm_asm2, tiles_n);
        g_out_u = tile_grid(k_bicg_outer<P, D, D, kTileN>, sm_out_u, tiles_n);
        g_out_u1 = tile_grid(k_bicg_outer<P, D, 1, kTileN>, sm_out_u1, tiles_n);
        g_spmm0 = tile_grid(k_bicg_spmm<P, D, D, 0, kTileN>, sm_spmm, tiles_n);
        g_spmm1 = tile_grid(k_bicg_spmm<P, D, D, 1, kTileN>, sm_spmm, tiles_n);
        g_spmm0_1 = tile_grid(k_bicg_spmm<P, D, 1, 0, kTileN>, sm_spmm1, tiles_n);
        g_spmm1_1 = tile_grid(k_bicg_spmm<P, D, 1, 1, kTileN>, sm_spmm1, tiles_n);
        g_sell = (int)std::max<int64_t>(1, ((m.n + 31) / 32 + kBlock / 32 - 1) / (kBlock / 32));
        g_outer_sell = sell_wave(k_pcg_outer_sell<P>);
        g_judge = sell_wave(k_guess_judge<P>);
        g_cg_first = sell_wave(cg_first_fn());
        {
            const AmgVariant<P>* t = amg_variant_table<P>(n_amg_v);
            for (int v = 0; v < n_amg_v; ++v) {
                const auto fn = t[v].pick(a);
                amg_grid_v[v] = fn ? sell_wave(fn) : 1;
            }
        }
        {
            int per_sm = 0;
            OASIS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pressure_rhs_rows<P, D, 4, 2>, kBlock, 0));
            const int64_t per_block = (int64_t)kBlock / 4 * 2;
            g_rhs = (int)std::max<int64_t>(
                1, std::min<int64_t>((m.n + per_block - 1) / per_block, (int64_t)std::max(per_sm, 1) * num_sms()));
        }
        g_upd = tile_grid(k_update<P, D, false>, sm_vd, tiles);
        g_upd_c = tile_grid(k_update<P, D, true>, 0, tiles);
        g_mspmv = tile_grid(k_mass_spmv<P, D>, sm_vd, tiles);
        g_out_s = tile_grid(k_bicg_outer<P, 1, 1, kTileN>, sm_out_u1, tiles_n);
        g_spmm0_s = tile_grid(k_bicg_spmm<P, 1, 1, 0, kTileN>, sm_spmm1, tiles_n);
        g_spmm1_s = tile_grid(k_bicg_spmm<P, 1, 1, 1, kTileN>, sm_spmm1, tiles_n);
        g_sasm = tile_grid(k_scalar_assemble<P>, sm_v1, tiles);
        ge_n = elem_grid(m.n);
        ge_red = red_grid(m.n);
        ge_nd = elem_grid(m.n * D);
        ge_c = elem_grid(m.nc);
    }

    void assemble(cudaStream_t s) override {
        const int pa = Sv.prof_begin(s, OASIS_PROF_ASSEMBLE);
        if (Sv.prm.convection == OASIS_CONV_ABE) {
            k_cell_beta<P, D, true><<<ge_c, kBlock, 0, s>>>(a);
            k_assemble<P, D, true, kTileN><<<g_asm2, kBlock, sm_asm2, s>>>(a, k_);
        } else {
            k_ubar<P, D><<<ge_nd, kBlock, 0, s>>>(a);
            k_cell_beta<P, D, false><<<ge_c, kBlock, 0, s>>>(a);
            k_assemble<P, D, false, kTileN><<<g_asm, kBlock, sm_asm, s>>>(a, k_);
        }
        Sv.prof_end(s, pa);
        OASIS_CUDA(cudaGetLastError());
    }

    Ctl ctl_u(const Loop& lp) const {
        Ctl c{};
        c.rtol2 = Sv.prm.rtol_u * Sv.prm.rtol_u;
        c.inner2 = P::mixed ? Sv.prm.inner_rtol * Sv.prm.inner_rtol : 0.0;
        c.abs2 = 0.25 * c.rtol2;
        c.max_it = Sv.prm.max_it_u;
        c.sweep_cap = P::mixed ? 400 : (1 << 30);
        c.use_cond = lp.graph;
        c.h_outer = lp.h_outer;
        c.h_inner = lp.h_inner;
        return c;
    }

    // Launch shapes of the BiCGStab kernels for NR right-hand sides of a [n][DD]
    // system (DD = D: velocity; DD = 1: a scalar).
    struct BicgGrids {
        int go, gs0, gs1;
        size_t so, ss;
    };
    template <int DD, int NR>
    BicgGrids bicg_grids() const {
        if constexpr (DD == 1) return {g_out_s, g_spmm0_s, g_spmm1_s, sm_out_u1, sm_spmm1};
        else if constexpr (NR == 1) return {g_out_u1, g_spmm0_1, g_spmm1_1, sm_out_u1, sm_spmm1};
        else return {g_out_u, g_spmm0, g_spmm1, sm_out_u, sm_spmm};
    }

    // BiCGStab with refinement sweeps on the system of q (state index `which`).
    template <int DD, int NR>
    void bicg_run(const StepData<P>& q, cudaStream_t s, int which, int k0, bool graph) {
        const BicgGrids G = bicg_grids<DD, NR>();
        Sv.run_loops(
            s, graph, which,
            [&](cudaStream_t ss_, const Loop& lp) {
                const int po = Sv.prof_begin(ss_, OASIS_PROF_OUTER);
                if constexpr (DD == D && NR == D) launch_bicg_outer(q, k0, ctl_u(lp), ss_);
                else k_bicg_outer<P, DD, NR, kTileN><<<G.go, kBlock, G.so, ss_>>>(q, k0, ctl_u(lp));
                Sv.prof_end(ss_, po);
                OASIS_CUDA(cudaGetLastError());
            },
            [&](cudaStream_t ss_, const Loop& lp) {
                const Ctl c = ctl_u(lp);
                int pv = Sv.prof_begin(ss_, OASIS_PROF_BICG_VEC);
                k_bicg_dir<P, DD, NR><<<ge_n, kBlock, 0, ss_>>>(q, k0);
                Sv.prof_end(ss_, pv);
                int pb = Sv.prof_begin(ss_, OASIS_PROF_BICG_SPMM);
                if constexpr (DD == D && NR == D) launch_bicg_spmm(0, q, k0, c, ss_);
                else k_bicg_spmm<P, DD, NR, 0, kTileN><<<G.gs0, kBlock, G.ss, ss_>>>(q, k0, c);
                Sv.prof_end(ss_, pb);
                pv = Sv.prof_begin(ss_, OASIS_PROF_BICG_VEC);
                k_bicg_s<P, DD, NR><<<ge_n, kBlock, 0, ss_>>>(q, k0);
                Sv.prof_end(ss_, pv);
                pb = Sv.prof_begin(ss_, OASIS_PROF_BICG_SPMM);
                if constexpr (DD == D && NR == D) launch_bicg_spmm(1, q, k0, c, ss_);
                else k_bicg_spmm<P, DD, NR, 1, kTileN><<<G.gs1, kBlock, G.ss, ss_>>>(q, k0, c);
                Sv.prof_end(ss_, pb);
                pv = Sv.prof_begin(ss_, OASIS_PROF_BICG_VEC);
                k_bicg_xr<P, DD, NR><<<ge_red, kBlock, 0, ss_>>>(q, k0, c);
                Sv.prof_end(ss_, pv);
                OASIS_CUDA(cudaGetLastError());
            },
            [&](cudaStream_t ss_, const Loop&) {
                k_bicg_correct<P, DD, NR><<<ge_n, kBlock, 0, ss_>>>(q, k0);
                OASIS_CUDA(cudaGetLastError());
            },
            k0, NR);
    }

    template <int NR>
    void bicg_solve(cudaStream_t s, int k0, bool graph) {
        bicg_run<D, NR>(a, s, 0, k0, graph);
    }

    // StepData of scalar `al`: its field, system, work vectors and state.
    StepData<P> scalar_data(int al) const {
        StepData<P> q = a;
        const int64_t n = Sv.m->n;
        q.u1 = Sv.c.as<S>() + (size_t)al * n;
        q.g = Sv.gc.as<S>() + (size_t)al * Sv.n_sdir;
        q.dir_index = Sv.sdir_index.p;
        q.A = Sv.Ac.as<V>();
        q.dinvA = Sv.dinvAc.as<V>();
        q.r0 = Sv.r0c.as<S>();
        q.du = Sv.dc.as<S>();
        V** w[9] = {&q.r, &q.rh, &q.p, &q.v, &q.s, &q.t, &q.ph, &q.sh, &q.dl};
        for (int k = 0; k < 9; ++k) *w[k] = Sv.sw[k].as<V>();
        q.stu = Sv.st.p + 3 + al;
        return q;
    }

    void scalars_changed() override { a.cbar = Sv.ns > 0 ? Sv.cbar.as<V>() : nullptr; }

    void scalar_solve(cudaStream_t s, bool graph) override {
        for (int al = 0; al < Sv.ns; ++al) {
            const StepData<P> q = scalar_data(al);
            Consts<V> kc = k_;
            kc.nu = (V)Sv.sc_diff[al];
            kc.hnu = (V)(0.5 * Sv.sc_diff[al]);
            kc.f[0] = (V)Sv.sc_src[al];
            k_scalar_assemble<P><<<g_sasm, kBlock, sm_v1, s>>>(q, kc);
            OASIS_CUDA(cudaGetLastError());
            bicg_run<1, 1>(q, s, 3 + al, 0, graph);
            k_scalar_finish<P><<<ge_n, kBlock, 0, s>>>(q);
            OASIS_CUDA(cudaGetLastError());
        }
    }

    void tentative_solve(cudaStream_t s, bool graph) override {
        if (Sv.prm.batch_rhs) bicg_solve<D>(s, 0, graph);
        else
            for (int k = 0; k < D; ++k) bicg_solve<1>(s, k, graph);
    }

    Ctl ctl_p(const Loop& lp) const {
        Ctl c{};
        c.rtol2 = Sv.prm.rtol_p * Sv.prm.rtol_p;
        c.inner2 = P::mixed ? Sv.prm.inner_rtol * Sv.prm.inner_rtol : 0.0;
        c.abs2 = 0.25 * c.rtol2;
        c.max_it = Sv.prm.max_it_p;
        c.sweep_cap = P::mixed ? 4000 : (1 << 30);
        c.use_cond = lp.graph;
        c.h_outer = lp.h_outer;
        c.h_inner = lp.h_inner;
        return c;
    }

    void advance_pressure(cudaStream_t s) override {
        k_pressure_advance<P><<<ge_n, kBlock, 0, s>>>(a);
        OASIS_CUDA(cudaGetLastError());
    }

    void pressure_solve(cudaStream_t s, bool graph, int inner) override {
        const int pr = Sv.prof_begin(s, OASIS_PROF_PRESSURE_RHS);
        k_tentative_velocity<P, D><<<ge_nd, kBlock, 0, s>>>(a);
        k_pressure_rhs_rows<P, D, 4, 2><<<g_rhs, kBlock, 0, s>>>(a);
        Sv.prof_end(s, pr);
        // repetitions after the first start from zero: their increment is small and
        // unrelated to the previous step's correction
        const bool learned = inner == 0 && Sv.prm.guess == OASIS_GUESS_LEARNED && Sv.net;
        int mode = (inner > 0 || Sv.prm.guess == OASIS_GUESS_ZERO) ? OASIS_GUESS_ZERO : OASIS_GUESS_PREV_PHI;
        const int pg = Sv.prof_begin(s, OASIS_PROF_GUESS);
        if (inner == 0 && (learned || Sv.record)) {
            k_guess_scales<P><<<ge_n, kBlock, 0, s>>>(a);
            k_guess_features<P><<<ge_n, kBlock, 0, s>>>(a);
            OASIS_CUDA(cudaGetLastError());
        }
        if (learned) {
            net_forward(*Sv.net, a.feat, a.gy, s);
            k_guess_judge<P><<<g_judge, kBlock, 0, s>>>(a);
            OASIS_CUDA(cudaGetLastError());
            mode = OASIS_GUESS_LEARNED;
        }
        Sv.prof_end(s, pg);
        k_phi_guess<P><<<ge_n, kBlock, 0, s>>>(a, mode);
        OASIS_CUDA(cudaGetLastError());
        if (Sv.prm.pressure_pc == OASIS_PC_AMG) {
            const AmgHierarchy& H = *Sv.m->amg;
            ProfHook hook;
            hook.ctx = &Sv;
            hook.begin = [](void* c, cudaStream_t st_, int f) { return static_cast<Solver*>(c)->prof_begin(st_, f); };
            hook.end = [](void* c, cudaStream_t st_, int h) { static_cast<Solver*>(c)->prof_end(st_, h); };
            auto vcycle = [&](cudaStream_t ss) {
                const int pa = Sv.prof_begin(ss, OASIS_PROF_AMG);
                amg_vcycle<V>(H, Sv.amgw, a.ar, a.au, a.stp, ss, &hook);
                Sv.prof_end(ss, pa);
            };
            auto update = [&](cudaStream_t ss, const Ctl& c) {
                const int pu = Sv.prof_begin(ss, OASIS_PROF_PCG_UPDATE);
                k_amg_cg_update<P><<<ge_red, kBlock, 0, ss>>>(a, c);
                Sv.prof_end(ss, pu);
                OASIS_CUDA(cudaGetLastError());
            };
            Sv.run_loops(
                s, graph, 1,
                [&](cudaStream_t ss, const Loop& lp) {
                    const Ctl c = ctl_p(lp);
                    const int po = Sv.prof_begin(ss, OASIS_PROF_OUTER);
                    k_pcg_outer_sell<P><<<g_outer_sell, kBlock, 0, ss>>>(a, c);
                    Sv.prof_end(ss, po);
                    k_amg_cg_start<P><<<ge_n, kBlock, 0, ss>>>(a);
                    vcycle(ss);
                    cg_first_fn()<<<g_cg_first, kBlock, 0, ss>>>(a, c);
                    OASIS_CUDA(cudaGetLastError());
                    update(ss, c);
                },
                // an iteration ends with the update, whose residual test sets the
                // loop's condition: a converged solve leaves the loop before another
                // V-cycle (same kernels in the same order as with the update first)
                [&](cudaStream_t ss, const Loop& lp) {
                    const Ctl c = ctl_p(lp);
                    vcycle(ss);
                    const int pq = Sv.prof_begin(ss, OASIS_PROF_PCG_SPMV);
                    amg_variant_table<P>(n_amg_v)[amg_v].pick(a)<<<amg_grid_v[amg_v], kBlock, 0, ss>>>(a, c);
                    Sv.prof_end(ss, pq);
                    OASIS_CUDA(cudaGetLastError());
                    update(ss, c);
                },
                [&](cudaStream_t ss, const Loop&) {
                    k_pcg_correct<P><<<ge_n, kBlock, 0, ss>>>(a);
                    OASIS_CUDA(cudaGetLastError());
                },
                0, 1);
            return;
        }
        Sv.run_loops(
            s, graph, 1,
            [&](cudaStream_t ss, const Loop& lp) {
                const Ctl c = ctl_p(lp);
                const int po = Sv.prof_begin(ss, OASIS_PROF_OUTER);
                k_pcg_outer_sell<P><<<g_outer_sell, kBlock, 0, ss>>>(a, c);
                Sv.prof_end(ss, po);
                const int pu = Sv.prof_begin(ss, OASIS_PROF_PCG_UPDATE);
                k_pcg_init_sell<P><<<g_sell, kBlock, 0, ss>>>(a, c);
                Sv.prof_end(ss, pu);
                OASIS_CUDA(cudaGetLastError());
            },
            [&](cudaStream_t ss, const Loop& lp) {
                const Ctl c = ctl_p(lp);
                const int pq = Sv.prof_begin(ss, OASIS_PROF_PCG_SPMV);
                iter_variants()[iter_v].fn<<<it_grid[iter_v], it_block[iter_v], it_smem[iter_v], ss>>>(a, c);
                Sv.prof_end(ss, pq);
                OASIS_CUDA(cudaGetLastError());
            },
            [&](cudaStream_t ss, const Loop&) {
                k_pcg_correct<P><<<ge_n, kBlock, 0, ss>>>(a);
                OASIS_CUDA(cudaGetLastError());
            },
            0, 1);
    }

    Ctl ctl_m(const Loop& lp) const {
        Ctl c{};
        const double tol = P::mixed ? std::max(Sv.prm.rtol_u, 1e-6) : Sv.prm.rtol_u;
        c.rtol2 = tol * tol;
        c.max_it = Sv.prm.max_it_u;
        c.use_cond = lp.graph;
        c.h_outer = lp.h_outer;
        c.h_inner = lp.h_inner;
        return c;
    }

    void update(cudaStream_t s, bool graph) override {
        if (Sv.prm.velocity_update == OASIS_UPDATE_CONSISTENT) {
            Sv.run_single(
                s, graph, 2,
                [&](cudaStream_t ss, const Loop& lp) {
                    const int pm = Sv.prof_begin(ss, OASIS_PROF_MASS);
                    k_mass_guess<P, D><<<ge_n, kBlock, 0, ss>>>(a, k_);
                    k_mass_residual<P, D><<<ge_red, kBlock, 0, ss>>>(a, ctl_m(lp));
                    Sv.prof_end(ss, pm);
                    OASIS_CUDA(cudaGetLastError());
                },
                [&](cudaStream_t ss, const Loop& lp) {
                    const Ctl c = ctl_m(lp);
                    const int pm = Sv.prof_begin(ss, OASIS_PROF_MASS);
                    k_mass_spmv<P, D><<<g_mspmv, kBlock, sm_vd, ss>>>(a, c);
                    k_mass_update<P, D><<<ge_red, kBlock, 0, ss>>>(a, c);
                    Sv.prof_end(ss, pm);
                    OASIS_CUDA(cudaGetLastError());
                });
            const int pu = Sv.prof_begin(s, OASIS_PROF_UPDATE);
            k_update<P, D, true><<<g_upd_c, kBlock, 0, s>>>(a, k_);
            Sv.prof_end(s, pu);
            OASIS_CUDA(cudaGetLastError());
            return;
        }
        const int pu = Sv.prof_begin(s, OASIS_PROF_UPDATE);
        k_update<P, D, false><<<g_upd, kBlock, sm_vd, s>>>(a, k_);
        Sv.prof_end(s, pu);
        OASIS_CUDA(cudaGetLastError());
    }

    S* state_ptr(int which) {
        switch (which) {
            case ST_U1: return a.u1;
            case ST_U2: return a.u2;
            case ST_PSTAR: return a.pstar;
            case ST_PHI: return a.phi;
            case ST_G: return const_cast<S*>(a.g);
            case ST_R0: return a.r0;
            case ST_C: return Sv.c.as<S>();
            case ST_GC: return Sv.gc.as<S>();
            default: throw Error(OASIS_EINVAL, "unknown state buffer");
        }
    }

    void to_state(cudaStream_t s, const double* src, int which, int64_t count, int comps,
                  const int32_t* perm) override {
        OASIS_CHECK(!perm || count % Sv.m->n == 0, OASIS_EINVAL, "renumbered transfer of a partial field");
        k_to_state<P><<<elem_grid(count * comps), kBlock, 0, s>>>(src, state_ptr(which), count, comps, perm,
                                                                  Sv.m->n);
        OASIS_CUDA(cudaGetLastError());
    }
    void from_state(cudaStream_t s, double* dst, int which, int64_t count, int comps,
                    const int32_t* perm) override {
        OASIS_CHECK(!perm || count % Sv.m->n == 0, OASIS_EINVAL, "renumbered transfer of a partial field");
        k_from_state<P><<<elem_grid(count * comps), kBlock, 0, s>>>(state_ptr(which), dst, count, comps, perm,
                                                                    Sv.m->n);
        OASIS_CUDA(cudaGetLastError());
    }
    const IterVariant<P>* iter_variants() const {
        int c = 0;
        return iter_variant_table<P>(c);
    }

    // Launch configuration of candidate v: one wave of 256-thread blocks over the
    // slices; the streamed shapes run as many blocks as fit (persistent), with
    // two stages of the longest slice per warp in shared memory.  False if the
    // candidate cannot run on this mesh.
    bool iter_config(const IterVariant<P>& t, int v) {
        if (!t.tma) {
            it_grid[v] = g_sell;
            it_block[v] = kBlock;
            it_smem[v] = 0;
            return true;
        }
        const size_t vb = (size_t)a.max_row * 32 * sizeof(V);
        const size_t cb = (size_t)a.max_row * 32 * (t.d16 ? 2 : 4);
        const size_t stage = (vb + cb + 127) & ~(size_t)127;
        const size_t smem = (size_t)t.wpb * 2 * stage;
        cudaFuncAttributes fa{};
        OASIS_CUDA(cudaFuncGetAttributes(&fa, t.fn));
        const size_t cap = (size_t)smem_optin() - fa.sharedSizeBytes;
        if (smem > cap) return false;
        OASIS_CUDA(cudaFuncSetAttribute(t.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cap));
        int per_sm = 0;
        OASIS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, t.fn, t.wpb * 32, smem));
        if (per_sm < 1) return false;
        const int64_t want = (a.n_slices + t.wpb - 1) / t.wpb;
        it_grid[v] = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)per_sm * num_sms()));
        it_block[v] = t.wpb * 32;
        it_smem[v] = smem;
        return true;
    }

    // Autotuner: every candidate shape of the CG iteration runs on this matrix
    // (2 untimed + 7 timed launches, CUDA events around each launch, median
    // kept) against a scratch Krylov state, so the solver's own state is not
    // touched; the iteration buffers hold no solve yet.  Every shape computes
    // the same bits, so only speed decides.
    // the multigrid CG product's shapes, timed on this matrix like the fused
    // Jacobi iteration's (forced = k >= 1 takes shape k untimed)
    void tune_amg(cudaStream_t s, int forced) {
        int count = 0;
        const AmgVariant<P>* t = amg_variant_table<P>(count);
        OASIS_CHECK(forced <= count, OASIS_EINVAL, "spmv_variant: no such candidate");
        OASIS_CHECK(forced < 1 || t[forced - 1].pick(a), OASIS_EINVAL,
                    "spmv_variant: the shape needs a layout this mesh does not have");
        for (auto& u : amg_us) u = 0.0;
        if (forced >= 1) {
            amg_v = forced - 1;
            return;
        }
        DBuf<KrylovState> scratch;
        scratch.alloc(1);
        StepData<P> d = a;
        d.stp = scratch.p;
        const Ctl c{};
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        OASIS_CUDA(cudaEventCreate(&e0));
        OASIS_CUDA(cudaEventCreate(&e1));
        // rounds over all candidates (2 untimed, then 7 timed), so that a drift of
        // the clocks or of the caches during tuning falls on every candidate alike
        constexpr int kWarm = 2, kTimed = 7;
        float ts[kAmgVariants][kTimed] = {};
        for (int r = 0; r < kWarm + kTimed; ++r)
            for (int v = 0; v < count; ++v) {
                const auto fn = t[v].pick(a);
                if (!fn) continue;                     // not timed: us stays 0
                OASIS_CUDA(cudaMemsetAsync(scratch.p, 0, sizeof(KrylovState), s));
                OASIS_CUDA(cudaEventRecord(e0, s));
                fn<<<amg_grid_v[v], kBlock, 0, s>>>(d, c);
                OASIS_CUDA(cudaGetLastError());
                OASIS_CUDA(cudaEventRecord(e1, s));
                OASIS_CUDA(cudaEventSynchronize(e1));
                if (r >= kWarm) OASIS_CUDA(cudaEventElapsedTime(&ts[v][r - kWarm], e0, e1));
            }
        int best = -1;
        for (int v = 0; v < count; ++v) {
            if (!t[v].pick(a)) continue;
            std::sort(ts[v], ts[v] + kTimed);
            amg_us[v] = 1e3 * (double)ts[v][kTimed / 2];
            if (best < 0 || amg_us[v] < amg_us[best]) best = v;
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        amg_v = best;
    }

    // the outer residual of the velocity solve's sweeps in the chosen form
    void launch_bicg_outer(const StepData<P>& q, int k0, const Ctl& c, cudaStream_t ss) const {
        const BicgVariant<P, D>& bv = bicg_variant_table<P, D>()[bicg_v];
        if (bv.outer) bv.outer<<<bicg_outer_grid[bicg_v], kBlock, 0, ss>>>(q, k0, c);
        else k_bicg_outer<P, D, D, kTileN><<<g_out_u, kBlock, sm_out_u, ss>>>(q, k0, c);
        OASIS_CUDA(cudaGetLastError());
    }

    // the d-RHS product of the velocity solve in the chosen shape
    void launch_bicg_spmm(int mode, const StepData<P>& q, int k0, const Ctl& c, cudaStream_t ss) const {
        const BicgVariant<P, D>& bv = bicg_variant_table<P, D>()[bicg_v];
        if (bv.lanes == 0) {
            if (mode == 0) bv.fn0<<<g_spmm0, kBlock, sm_spmm, ss>>>(q, k0, c);
            else bv.fn1<<<g_spmm1, kBlock, sm_spmm, ss>>>(q, k0, c);
        } else {
            (mode == 0 ? bv.fn0 : bv.fn1)<<<bicg_grid[bicg_v][mode], kBlock, 0, ss>>>(q, k0, c);
        }
        OASIS_CUDA(cudaGetLastError());
    }

    // Time both products of every shape on this solver's pattern (values zeroed,
    // scratch Krylov state, 2 untimed + 7 timed launches each, median) and keep
    // the fastest; forced = k >= 1 takes shape k untimed.
    void tune_bicg(cudaStream_t s, int forced) {
        const BicgVariant<P, D>* t = bicg_variant_table<P, D>();
        OASIS_CHECK(forced >= 0 && forced <= kBicgVariants, OASIS_EINVAL, "bicg_variant: no such candidate");
        const bool have16 = a.csr_dcol != nullptr;
        OASIS_CHECK(forced < 1 || have16 || !t[forced - 1].c16, OASIS_EINVAL,
                    "bicg_variant: 16-bit column offsets do not fit this mesh's ordering");
        const int64_t rows = Sv.m->n;
        auto wave = [&](void (*fn)(StepData<P>, int, Ctl), int lanes, int in_flight) {
            int per_sm = 0;
            OASIS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kBlock, 0));
            const int64_t per_block = (int64_t)kBlock / lanes * in_flight;
            return (int)std::max<int64_t>(
                1, std::min<int64_t>((rows + per_block - 1) / per_block, (int64_t)std::max(per_sm, 1) * num_sms()));
        };
        for (int v = 0; v < kBicgVariants; ++v) {
            if (t[v].lanes == 0) {
                bicg_grid[v][0] = g_spmm0;
                bicg_grid[v][1] = g_spmm1;
                bicg_outer_grid[v] = g_out_u;
                continue;
            }
            // each product's grid from its own occupancy (their register counts differ)
            bicg_grid[v][0] = wave(t[v].fn0, t[v].lanes, t[v].rows);
            bicg_grid[v][1] = wave(t[v].fn1, t[v].lanes, t[v].rows);
            bicg_outer_grid[v] = wave(t[v].outer, t[v].lanes, 2);
        }
        for (auto& u : bicg_us) u = 0.0;
        if (forced >= 1) {
            bicg_v = forced - 1;
            return;
        }
        OASIS_CUDA(cudaMemsetAsync(Sv.A.p, 0, Sv.A.bytes, s));
        for (auto& w : Sv.w) OASIS_CUDA(cudaMemsetAsync(w.p, 0, w.bytes, s));
        DBuf<KrylovState> scratch;
        scratch.alloc(1);
        StepData<P> d = a;
        d.stu = scratch.p;
        const Ctl c{};
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        OASIS_CUDA(cudaEventCreate(&e0));
        OASIS_CUDA(cudaEventCreate(&e1));
        // rounds over all candidates (2 untimed, then 7 timed), so that a drift of
        // the clocks or of the caches during tuning falls on every candidate alike
        constexpr int kWarm = 2, kTimed = 7;
        float ts[kBicgVariants][kTimed] = {};
        for (int r = 0; r < kWarm + kTimed; ++r)
            for (int v = 0; v < kBicgVariants; ++v) {
                if (t[v].c16 && !have16) continue;
                bicg_v = v;
                // each product from a fresh scratch state: with zeroed values the first
                // product's dots are zero, and its breakdown branch would otherwise mark
                // every column done and let the second return at once
                float t2[2];
                for (int mode = 0; mode < 2; ++mode) {
                    OASIS_CUDA(cudaMemsetAsync(scratch.p, 0, sizeof(KrylovState), s));
                    OASIS_CUDA(cudaEventRecord(e0, s));
                    launch_bicg_spmm(mode, d, 0, c, s);
                    OASIS_CUDA(cudaEventRecord(e1, s));
                    OASIS_CUDA(cudaEventSynchronize(e1));
                    OASIS_CUDA(cudaEventElapsedTime(&t2[mode], e0, e1));
                }
                if (r >= kWarm) ts[v][r - kWarm] = t2[0] + t2[1];
            }
        int best = 0;
        for (int v = 0; v < kBicgVariants; ++v) {
            if (t[v].c16 && !have16) continue;      // not timed: bicg_us stays 0
            std::sort(ts[v], ts[v] + kTimed);
            bicg_us[v] = 1e3 * (double)ts[v][kTimed / 2];
            if (bicg_us[v] < bicg_us[best]) best = v;
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        bicg_v = best;
    }

    void tune(cudaStream_t s, int forced) override {
        tune_bicg(s, Sv.prm.bicg_variant);
        if (Sv.prm.pressure_pc == OASIS_PC_AMG) {
            tune_amg(s, forced);
            return;
        }
        int count = 0;
        const IterVariant<P>* t = iter_variant_table<P>(count);
        OASIS_CHECK(forced <= count, OASIS_EINVAL, "spmv_variant: no such candidate");
        const bool have16 = a.sell_dcol != nullptr;
        OASIS_CHECK(forced < 1 || have16 || !t[forced - 1].d16, OASIS_EINVAL,
                    "spmv_variant: 16-bit column offsets do not fit this mesh's ordering");
        bool usable[OASIS_MAX_VARIANTS];
        for (int v = 0; v < count; ++v) usable[v] = iter_config(t[v], v) && (have16 || !t[v].d16);
        OASIS_CHECK(forced < 1 || usable[forced - 1], OASIS_EINVAL,
                    "spmv_variant: the streamed shape does not fit this mesh's rows in shared memory");
        for (auto& u : tune_us) u = 0.0;
        if (forced >= 1) {
            iter_v = forced - 1;
            return;
        }
        DBuf<KrylovState> scratch;
        scratch.alloc(1);
        StepData<P> d = a;
        d.stp = scratch.p;
        const Ctl c{};
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        OASIS_CUDA(cudaEventCreate(&e0));
        OASIS_CUDA(cudaEventCreate(&e1));
        constexpr int kWarm = 2, kTimed = 7;
        int best = -1;
        for (int v = 0; v < count; ++v) {
            if (!usable[v]) continue;
            float ts[kTimed];
            for (int r = 0; r < kWarm + kTimed; ++r) {
                OASIS_CUDA(cudaMemsetAsync(scratch.p, 0, sizeof(KrylovState), s));
                OASIS_CUDA(cudaEventRecord(e0, s));
                t[v].fn<<<it_grid[v], it_block[v], it_smem[v], s>>>(d, c);
                OASIS_CUDA(cudaGetLastError());
                OASIS_CUDA(cudaEventRecord(e1, s));
                OASIS_CUDA(cudaEventSynchronize(e1));
                if (r >= kWarm) OASIS_CUDA(cudaEventElapsedTime(&ts[r - kWarm], e0, e1));
            }
            std::sort(ts, ts + kTimed);
            tune_us[v] = 1e3 * (double)ts[kTimed / 2];
            if (best < 0 || tune_us[v] < tune_us[best]) best = v;
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        iter_v = best;
    }

    void tuning(oasis_tuning* out) const override {
        const BicgVariant<P, D>* bt = bicg_variant_table<P, D>();
        out->bicg_n_variants = kBicgVariants;
        out->bicg_chosen = bicg_v + 1;
        for (int v = 0; v < kBicgVariants; ++v) {
            out->bicg_lanes[v] = bt[v].lanes;
            out->bicg_rows[v] = bt[v].rows;
            out->bicg_min_blocks[v] = bt[v].minb;
            out->bicg_col16[v] = bt[v].c16;
            out->bicg_us[v] = bicg_us[v];
        }
        if (Sv.prm.pressure_pc == OASIS_PC_AMG) {
            int count = 0;
            const AmgVariant<P>* t = amg_variant_table<P>(count);
            out->n_variants = count;
            out->chosen = amg_v + 1;
            for (int v = 0; v < count; ++v) {
                out->chunk[v] = t[v].chunk;
                out->min_blocks[v] = t[v].minb;
                out->prefetch[v] = 0;
                out->col16[v] = t[v].fnp ? 2 : a.sell_dcol != nullptr;
                out->streamed[v] = 0;
                out->warps_per_block[v] = kBlock / 32;
                out->us[v] = amg_us[v];
            }
            return;
        }
        int count = 0;
        const IterVariant<P>* t = iter_variant_table<P>(count);
        out->n_variants = count;
        out->chosen = iter_v + 1;
        for (int v = 0; v < count; ++v) {
            out->chunk[v] = t[v].chunk;
            out->min_blocks[v] = t[v].minb;
            out->prefetch[v] = t[v].pf;
            out->col16[v] = t[v].d16;
            out->streamed[v] = t[v].tma;
            out->warps_per_block[v] = t[v].wpb;
            out->us[v] = tune_us[v];
        }
    }

    void amg_apply(cudaStream_t s, const void* r, void* u) override {
        DBuf<KrylovState> scratch;
        scratch.alloc(1);
        OASIS_CUDA(cudaMemsetAsync(scratch.p, 0, sizeof(KrylovState), s));
        amg_vcycle<V>(*Sv.m->amg, Sv.amgw, reinterpret_cast<const V*>(r), reinterpret_cast<V*>(u), scratch.p, s);
        OASIS_CUDA(cudaStreamSynchronize(s));
    }

    void guess_target(cudaStream_t s, float* target) override {
        k_guess_target<P><<<ge_n, kBlock, 0, s>>>(a, target);
        OASIS_CUDA(cudaGetLastError());
    }

    void a_to_double(cudaStream_t s, double* dst) override {
        k_v_to_double<V><<<elem_grid(a.nnz), kBlock, 0, s>>>(a.A, dst, a.nnz);
        OASIS_CUDA(cudaGetLastError());
    }
};

StepImpl* make_step_impl(Solver& s) {
    if (s.m->dim == 2) {
        if (s.mixed) return new StepImplT<Mixed, 2>(s);
        return new StepImplT<Fp64, 2>(s);
    }
    if (s.mixed) return new StepImplT<Mixed, 3>(s);
    return new StepImplT<Fp64, 3>(s);
}

}  // namespace oasis
