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
// equation cancels).  The systems and their solutions are those of Sec. 5;
// only the initial residual is formed without the O(1/dt) cancellation of
// b - A u^{n-1}, which keeps float32 inner solves accurate.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>

#include "device.cuh"
#include "internal.cuh"
#include "solver.cuh"

namespace oasis {

static int grid_rows(int64_t rows, int rows_per_block) {
    const int64_t want = (rows + rows_per_block - 1) / rows_per_block;
    const int64_t cap = (int64_t)num_sms() * 8;
    return (int)std::max<int64_t>(1, std::min(want, cap));
}

// Upper bound on refinement sweeps of one solve (each sweep also does at least
// one counted iteration, so max_it bounds them as well).
constexpr int kMaxSweeps = 1000;

__device__ __forceinline__ void set_cond(int use, cudaGraphConditionalHandle h, int v) {
    if (use) cudaGraphSetConditional(h, v ? 1u : 0u);
}

// =====================================================================  assembly
// beta[c][j] = w_T grad lambda_j . sum_m ubar_m, ubar = 1.5 u^{n-1} - 0.5 u^{n-2}
// (Eq. 22).  With it the P1 convection element matrix is
//   C^T_ij = w_T grad lambda_j . (sum_m ubar_m + ubar_i) = beta[T][j] + ubar_i . w_T grad lambda_j,
// w_T = |T| / ((d+1)(d+2)); the second term summed over the cells of an edge is
// ubar_i . dP_ij / (d+2) and is added in the row pass.
template <class V, int D>
__global__ void __launch_bounds__(kBlock) k_cell_beta(int64_t nc, const int32_t* __restrict__ cell_dof,
                                                      const V* __restrict__ gw, const double* __restrict__ u1,
                                                      const double* __restrict__ u2, V* __restrict__ beta) {
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nc;
         c += (int64_t)gridDim.x * blockDim.x) {
        double S[D];
#pragma unroll
        for (int k = 0; k < D; ++k) S[k] = 0.0;
#pragma unroll
        for (int m = 0; m <= D; ++m) {
            const size_t j = (size_t)__ldg(&cell_dof[c * (D + 1) + m]) * D;
#pragma unroll
            for (int k = 0; k < D; ++k) S[k] += 1.5 * __ldg(&u1[j + k]) - 0.5 * __ldg(&u2[j + k]);
        }
        V out[4];
#pragma unroll
        for (int m = 0; m <= D; ++m) {
            V acc = 0;
#pragma unroll
            for (int k = 0; k < D; ++k) acc += __ldg(&gw[((size_t)c * (D + 1) + m) * D + k]) * (V)S[k];
            out[m] = acc;
        }
        if (D == 2) out[3] = 0;
#pragma unroll
        for (int m = 0; m < 4; ++m) beta[c * 4 + m] = out[m];
    }
}

// Row pass of the convection assembly fused with Algorithm 2: for row i the
// lanes of a group own the row's pattern entries; they collect the cell terms
// beta from the incident cells (deterministic order, no atomics), add the
// dP term, and form
//   A_ij = M_ij/dt + C_ij/2 + nu K_ij/2                         (Eq. 34)
//   r0_i = f_k ML_i - sum_j (C_ij + nu K_ij) u_k,j - sum_j dP^k_ij p*_j
// which equals b_k - A u_k^{n-1} with b_k the right-hand side of Eq. 34
// (b_k = f_k ML + (2M/dt - A) u^{n-1} - dP^k p*, Algorithm 2).  Dirichlet rows
// become unit rows of A with r0 = g - u^{n-1}.
template <class V, int D, int L>
__global__ void __launch_bounds__(kBlock) k_assemble(AsmArgs<V> a) {
    constexpr int RPW = 32 / L;
    const int lane = threadIdx.x % L;
    const int sub = (threadIdx.x % 32) / L;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / 32;
    const int64_t nwarp = (int64_t)gridDim.x * blockDim.x / 32;
    double part[D];
#pragma unroll
    for (int k = 0; k < D; ++k) part[k] = 0.0;
    const V rdt = (V)(1.0 / a.dt), hnu = (V)(0.5 * a.nu), nu = (V)a.nu;
    for (int64_t w = warp; w * RPW < a.n; w += nwarp) {
        const int64_t i = w * RPW + sub;
        V racc[D];
#pragma unroll
        for (int k = 0; k < D; ++k) racc[k] = 0;
        int dir = -1;
        if (i < a.n) {
            const int32_t b = a.rp[i], len = a.rp[i + 1] - b;
            const int32_t dslot = a.diag[i] - b;
            dir = a.dir_index[i];
            V ub[D];
#pragma unroll
            for (int k = 0; k < D; ++k) ub[k] = (V)(1.5 * a.u1[i * D + k] - 0.5 * a.u2[i * D + k]);
            const int32_t q0 = a.inc_ptr[i], q1 = a.inc_ptr[i + 1];
            for (int32_t s0 = 0; s0 < len; s0 += L) {
                const int32_t s = s0 + lane;
                const bool valid = s < len;
                const uint32_t key = (uint32_t)s * 0x01010101u;
                V t1 = 0;
                for (int32_t q = q0; q < q1; ++q) {
                    const uint32_t wd = __ldg(&a.inc_slots[q]);
                    const uint32_t mt = __vcmpeq4(wd, key);
                    if (valid && mt) {
                        const int loc = (__ffs(mt) - 1) >> 3;
                        t1 += __ldg(&a.beta[(size_t)__ldg(&a.inc_cell[q]) * 4 + loc]);
                    }
                }
                if (valid) {
                    const int32_t e = b + s;
                    const int32_t j = a.col[e];
                    V gdot = 0;
                    V gv[D];
#pragma unroll
                    for (int k = 0; k < D; ++k) {
                        gv[k] = a.G[(size_t)k * a.nnz + e];
                        gdot += ub[k] * gv[k];
                    }
                    const V c = t1 + gdot * (V)(1.0 / (D + 2));
                    const V kv = a.K[e];
                    V av = a.M[e] * rdt + (V)0.5 * c + hnu * kv;
                    if (dir >= 0) av = (s == dslot) ? (V)1 : (V)0;
                    a.A[e] = av;
                    if (s == dslot) a.dinv[i] = (V)1 / av;
                    const V ck = c + nu * kv;
                    const double ps = a.pstar[j];
#pragma unroll
                    for (int k = 0; k < D; ++k) racc[k] -= ck * (V)a.u1[(size_t)j * D + k] + gv[k] * (V)ps;
                }
            }
        }
#pragma unroll
        for (int k = 0; k < D; ++k) racc[k] = group_sum<L>(racc[k]);
        if (i < a.n && lane == 0) {
#pragma unroll
            for (int k = 0; k < D; ++k) {
                double r = dir >= 0 ? a.g[(size_t)dir * D + k] - a.u1[i * D + k]
                                    : a.f[k] * a.ML[i] + (double)racc[k];
                a.r0[i * D + k] = r;
                part[k] += r * r;
            }
        }
    }
    if (grid_sum<D>(part, a.partial, &a.st->ticket) && threadIdx.x == 0) {
        KrylovState* st = a.st;
        for (int k = 0; k < 3; ++k) {
            st->bb[k] = k < D ? part[k] : 0.0;
            st->col_done[k] = k < D ? 0 : 1;
            st->in_done[k] = 1;
            st->it_total[k] = 0;
            st->rr[k] = k < D ? part[k] : 0.0;
        }
        st->sweeps = 0;
        st->it_in = 0;
        st->status = OASIS_OK;
        st->first = 1;
    }
}

// Zero Delta (the tentative correction, float64) before the solve.
template <int D>
__global__ void k_zero_du(int64_t n, double* du) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n * D; t += (int64_t)gridDim.x * blockDim.x)
        du[t] = 0.0;
}

// =====================================================================  BiCGStab
// Right-preconditioned BiCGStab (van der Vorst), Jacobi M = diag(A), run per
// column k on A Delta_k = r0_k, inside float64 refinement sweeps: every sweep
// starts from the float64 residual r = r0 - A Delta and ends with Delta += delta.
template <int NR>
__device__ __forceinline__ void load_active(const KrylovState* st, int k0, int (&act)[NR], bool& any) {
    any = false;
#pragma unroll
    for (int c = 0; c < NR; ++c) {
        act[c] = !st->col_done[k0 + c] && !st->in_done[k0 + c];
        any |= act[c] != 0;
    }
}

template <int NR>
__device__ __forceinline__ void publish_inner(KrylovState* st, int k0, const BicgCtl& ctl) {
    int any = 0;
    for (int c = 0; c < NR; ++c) any |= (!st->col_done[k0 + c] && !st->in_done[k0 + c]);
    set_cond(ctl.use_cond, ctl.h_inner, any);
}

// Outer sweep: float64 residual r = r0 - A Delta, convergence test, and start
// of a new inner solve (r, rhat = r, p = v = delta = 0).
template <class V, int D, int NR, int L>
__global__ void __launch_bounds__(kBlock) k_bicg_outer(BicgArgs<V> a, BicgCtl ctl) {
    constexpr int RPW = 32 / L;
    const int lane = threadIdx.x % L, sub = (threadIdx.x % 32) / L;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / 32;
    const int64_t nwarp = (int64_t)gridDim.x * blockDim.x / 32;
    int live[NR];
#pragma unroll
    for (int c = 0; c < NR; ++c) live[c] = !a.st->col_done[a.k0 + c];
    double part[2 * NR];
#pragma unroll
    for (int c = 0; c < 2 * NR; ++c) part[c] = 0.0;
    for (int64_t w = warp; w * RPW < a.n; w += nwarp) {
        const int64_t i = w * RPW + sub;
        double acc[NR];
#pragma unroll
        for (int c = 0; c < NR; ++c) acc[c] = 0.0;
        if (i < a.n) {
            const int32_t b = a.rp[i], e = a.rp[i + 1];
            for (int32_t q = b + lane; q < e; q += L) {
                const double av = (double)a.A[q];
                const size_t j = (size_t)a.col[q] * D + a.k0;
#pragma unroll
                for (int c = 0; c < NR; ++c) acc[c] += av * a.du[j + c];
            }
        }
#pragma unroll
        for (int c = 0; c < NR; ++c) acc[c] = group_sum<L>(acc[c]);
        if (i < a.n && lane == 0) {
#pragma unroll
            for (int c = 0; c < NR; ++c) {
                if (!live[c]) continue;
                const size_t o = (size_t)i * D + a.k0 + c;
                const double r = a.r0[o] - acc[c];
                const V rv = (V)r;
                a.r[o] = rv;
                a.rh[o] = rv;
                a.p[o] = 0;
                a.v[o] = 0;
                a.dl[o] = 0;
                part[c] += r * r;
                part[NR + c] += (double)rv * (double)rv;
            }
        }
    }
    if (grid_sum<2 * NR>(part, a.partial, &a.st->ticket) && threadIdx.x == 0) {
        KrylovState* st = a.st;
        int outer = 0;
        for (int c = 0; c < NR; ++c) {
            const int k = a.k0 + c;
            if (st->col_done[k]) continue;
            const double rr = part[c];
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
                st->rho_new[k] = part[NR + c];
                st->rr0_in[k] = part[NR + c];
                st->rr_in[k] = part[NR + c];
                outer = 1;
            }
        }
        st->sweeps += 1;
        st->it_in = 0;
        set_cond(ctl.use_cond, ctl.h_outer, outer);
        publish_inner<NR>(st, a.k0, ctl);
    }
}

// p = r + beta (p - omega v),  ph = D^{-1} p
template <class V, int D, int NR>
__global__ void __launch_bounds__(kBlock) k_bicg_dir(BicgArgs<V> a) {
    int act[NR];
    bool any;
    load_active<NR>(a.st, a.k0, act, any);
    if (!any) return;
    V beta[NR], omega[NR];
#pragma unroll
    for (int c = 0; c < NR; ++c) {
        beta[c] = (V)a.st->beta[a.k0 + c];
        omega[c] = (V)a.st->omega[a.k0 + c];
    }
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.n; i += (int64_t)gridDim.x * blockDim.x) {
        const V di = a.dinv[i];
#pragma unroll
        for (int c = 0; c < NR; ++c) {
            if (!act[c]) continue;
            const size_t o = (size_t)i * D + a.k0 + c;
            const V pv = a.r[o] + beta[c] * (a.p[o] - omega[c] * a.v[o]);
            a.p[o] = pv;
            a.ph[o] = di * pv;
        }
    }
}

// y = A x (x = ph or sh) with the dot products needed next:
//   MODE 0: v = A ph, <rhat, v>          -> alpha = rho / <rhat, v>
//   MODE 1: t = A sh, <t, s>, <t, t>     -> omega = <t, s> / <t, t>
template <class V, int D, int NR, int L, int MODE>
__global__ void __launch_bounds__(kBlock) k_bicg_spmm(BicgArgs<V> a, BicgCtl ctl) {
    int act[NR];
    bool any;
    load_active<NR>(a.st, a.k0, act, any);
    if (!any) return;
    constexpr int RPW = 32 / L;
    constexpr int NV = MODE == 0 ? NR : 2 * NR;
    const V* __restrict__ x = MODE == 0 ? a.ph : a.sh;
    V* __restrict__ y = MODE == 0 ? a.v : a.t;
    const int lane = threadIdx.x % L, sub = (threadIdx.x % 32) / L;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / 32;
    const int64_t nwarp = (int64_t)gridDim.x * blockDim.x / 32;
    double part[NV];
#pragma unroll
    for (int c = 0; c < NV; ++c) part[c] = 0.0;
    for (int64_t w = warp; w * RPW < a.n; w += nwarp) {
        const int64_t i = w * RPW + sub;
        V acc[NR];
#pragma unroll
        for (int c = 0; c < NR; ++c) acc[c] = 0;
        if (i < a.n) {
            const int32_t b = a.rp[i], e = a.rp[i + 1];
            for (int32_t q = b + lane; q < e; q += L) {
                const V av = a.A[q];
                const size_t j = (size_t)a.col[q] * D + a.k0;
#pragma unroll
                for (int c = 0; c < NR; ++c) acc[c] += av * x[j + c];
            }
        }
#pragma unroll
        for (int c = 0; c < NR; ++c) acc[c] = group_sum<L>(acc[c]);
        if (i < a.n && lane == 0) {
#pragma unroll
            for (int c = 0; c < NR; ++c) {
                if (!act[c]) continue;
                const size_t o = (size_t)i * D + a.k0 + c;
                y[o] = acc[c];
                if (MODE == 0) {
                    part[c] += (double)a.rh[o] * (double)acc[c];
                } else {
                    const double sv = (double)a.s[o];
                    part[c] += (double)acc[c] * sv;
                    part[NR + c] += (double)acc[c] * (double)acc[c];
                }
            }
        }
    }
    if (grid_sum<NV>(part, a.partial, &a.st->ticket) && threadIdx.x == 0) {
        KrylovState* st = a.st;
        for (int c = 0; c < NR; ++c) {
            if (!act[c]) continue;
            const int k = a.k0 + c;
            if (MODE == 0) {
                const double rv = part[c];
                if (rv == 0.0 || !isfinite(rv)) {
                    st->in_done[k] = 1;      // breakdown: restart from the float64 residual
                    st->it_total[k] += 1;    // counted, so that restarts end at the cap
                    st->alpha[k] = 0.0;
                } else {
                    st->alpha[k] = st->rho_new[k] / rv;
                }
            } else {
                const double ts = part[c], tt = part[NR + c];
                st->omega[k] = (tt > 0.0 && isfinite(tt)) ? ts / tt : 0.0;
            }
        }
        if (MODE == 0) publish_inner<NR>(st, a.k0, ctl);
    }
}

// s = r - alpha v,  sh = D^{-1} s
template <class V, int D, int NR>
__global__ void __launch_bounds__(kBlock) k_bicg_s(BicgArgs<V> a) {
    int act[NR];
    bool any;
    load_active<NR>(a.st, a.k0, act, any);
    if (!any) return;
    V alpha[NR];
#pragma unroll
    for (int c = 0; c < NR; ++c) alpha[c] = (V)a.st->alpha[a.k0 + c];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.n; i += (int64_t)gridDim.x * blockDim.x) {
        const V di = a.dinv[i];
#pragma unroll
        for (int c = 0; c < NR; ++c) {
            if (!act[c]) continue;
            const size_t o = (size_t)i * D + a.k0 + c;
            const V sv = a.r[o] - alpha[c] * a.v[o];
            a.s[o] = sv;
            a.sh[o] = di * sv;
        }
    }
}

// delta += alpha ph + omega sh,  r = s - omega t,  <rhat, r>, <r, r>
template <class V, int D, int NR>
__global__ void __launch_bounds__(kBlock) k_bicg_xr(BicgArgs<V> a, BicgCtl ctl) {
    int act[NR];
    bool any;
    load_active<NR>(a.st, a.k0, act, any);
    if (!any) return;
    V alpha[NR], omega[NR];
#pragma unroll
    for (int c = 0; c < NR; ++c) {
        alpha[c] = (V)a.st->alpha[a.k0 + c];
        omega[c] = (V)a.st->omega[a.k0 + c];
    }
    double part[2 * NR];
#pragma unroll
    for (int c = 0; c < 2 * NR; ++c) part[c] = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.n; i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int c = 0; c < NR; ++c) {
            if (!act[c]) continue;
            const size_t o = (size_t)i * D + a.k0 + c;
            a.dl[o] += alpha[c] * a.ph[o] + omega[c] * a.sh[o];
            const V rv = a.s[o] - omega[c] * a.t[o];
            a.r[o] = rv;
            part[c] += (double)a.rh[o] * (double)rv;
            part[NR + c] += (double)rv * (double)rv;
        }
    }
    if (grid_sum<2 * NR>(part, a.partial, &a.st->ticket) && threadIdx.x == 0) {
        KrylovState* st = a.st;
        for (int c = 0; c < NR; ++c) {
            if (!act[c]) continue;
            const int k = a.k0 + c;
            const double rho_new = part[c], rr = part[NR + c];
            st->it_total[k] += 1;
            const double om = st->omega[k];
            st->beta[k] = (st->rho_new[k] != 0.0 && om != 0.0) ? (rho_new / st->rho_new[k]) * (st->alpha[k] / om) : 0.0;
            st->rho[k] = st->rho_new[k];
            st->rho_new[k] = rho_new;
            st->rr_in[k] = rr;
            const bool stop = !isfinite(rr) || rr <= ctl.inner2 * st->rr0_in[k] ||
                              rr <= ctl.abs2 * st->bb[k] || om == 0.0 || rho_new == 0.0 ||
                              st->it_total[k] >= ctl.max_it || st->it_in + 1 >= ctl.sweep_cap;
            if (stop) st->in_done[k] = 1;
        }
        st->it_in += 1;
        publish_inner<NR>(st, a.k0, ctl);
    }
}

// Delta += delta (float64) for the columns refined in this sweep.
template <class V, int D, int NR>
__global__ void __launch_bounds__(kBlock) k_bicg_correct(BicgArgs<V> a) {
    int live[NR];
    bool any = false;
#pragma unroll
    for (int c = 0; c < NR; ++c) {
        live[c] = !a.st->col_done[a.k0 + c];
        any |= live[c] != 0;
    }
    if (!any) return;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.n; i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int c = 0; c < NR; ++c) {
            if (!live[c]) continue;
            const size_t o = (size_t)i * D + a.k0 + c;
            a.du[o] += (double)a.dl[o];
        }
    }
}

// =====================================================================  pressure
// b_phi_i = -(1/dt) sum_k sum_j dP^k_ij u_k,j^I, u^I = u^{n-1} + Delta (Sec. 5,
// algebraic pressure equation); its mean is stored for the projection on
// sum_i b_i = 0, and the pressure solve state is reset.
template <class V, int D, int L>
__global__ void __launch_bounds__(kBlock) k_pressure_rhs(PresArgs<V> a) {
    constexpr int RPW = 32 / L;
    const int lane = threadIdx.x % L, sub = (threadIdx.x % 32) / L;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / 32;
    const int64_t nwarp = (int64_t)gridDim.x * blockDim.x / 32;
    double part[1] = {0.0};
    for (int64_t w = warp; w * RPW < a.n; w += nwarp) {
        const int64_t i = w * RPW + sub;
        V acc = 0;
        if (i < a.n) {
            const int32_t b = a.rp[i], e = a.rp[i + 1];
            for (int32_t q = b + lane; q < e; q += L) {
                const size_t j = (size_t)a.col[q] * D;
#pragma unroll
                for (int k = 0; k < D; ++k) acc += a.G[(size_t)k * a.nnz + q] * (V)(a.u1[j + k] + a.du[j + k]);
            }
        }
        acc = group_sum<L>(acc);
        if (i < a.n && lane == 0) {
            const double bi = -(double)acc / a.dt;
            a.b[i] = bi;
            part[0] += bi;
        }
    }
    if (grid_sum<1>(part, a.partial, &a.st->ticket) && threadIdx.x == 0) {
        KrylovState* st = a.st;
        st->mean = part[0] / (double)a.n;
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
}

// Initial guess for phi: 0 or the previous step's correction.
__global__ void k_phi_guess(int64_t n, int mode, const double* __restrict__ prev, double* __restrict__ x) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] = mode == OASIS_GUESS_PREV_PHI ? prev[i] : 0.0;
}

// Outer sweep of the pressure CG: r = (b - mean b) - K x in float64 with the
// float64 K; starts an inner float32/float64 CG (z = D^{-1} r, p = 0, delta = 0);
// also accumulates sum_i (p*_i + x_i) for the normalisation of p.
template <class V, int L>
__global__ void __launch_bounds__(kBlock) k_pcg_outer(PcgArgs<V> a, BicgCtl ctl) {
    constexpr int RPW = 32 / L;
    const int lane = threadIdx.x % L, sub = (threadIdx.x % 32) / L;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / 32;
    const int64_t nwarp = (int64_t)gridDim.x * blockDim.x / 32;
    const bool live = !a.st->col_done[0];
    const double mean = a.st->mean;
    double part[4] = {0.0, 0.0, 0.0, 0.0};
    for (int64_t w = warp; w * RPW < a.n; w += nwarp) {
        const int64_t i = w * RPW + sub;
        double acc = 0.0;
        if (i < a.n) {
            const int32_t b = a.rp[i], e = a.rp[i + 1];
            for (int32_t q = b + lane; q < e; q += L) acc += a.K64[q] * a.x[a.col[q]];
        }
        acc = group_sum<L>(acc);
        if (i < a.n && lane == 0) {
            const double bi = a.b[i] - mean;
            const double r = bi - acc;
            const V rv = (V)r, zv = a.dinv[i] * rv;
            if (live) {
                a.r[i] = rv;
                a.z[i] = zv;
                a.p0[i] = 0;
                a.p1[i] = 0;
                a.dl[i] = 0;
            }
            part[0] += r * r;
            part[1] += (double)rv * (double)zv;
            part[2] += bi * bi;
            part[3] += a.pstar[i] + a.x[i];
        }
    }
    if (grid_sum<4>(part, a.partial, &a.st->ticket) && threadIdx.x == 0) {
        KrylovState* st = a.st;
        if (st->first) {
            st->bb[0] = part[2];
            st->first = 0;
        }
        st->psum = part[3];
        int outer = 0;
        if (!st->col_done[0]) {
            const double rr = part[0];
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
                st->rho[0] = part[1];
                st->beta[0] = 0.0;
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

// q = K p_new with p_new = z + beta p_old formed on the fly (double-buffered by
// the parity of the inner iteration), <p_new, q> -> alpha = rho / <p, q>.
template <class V, int L>
__global__ void __launch_bounds__(kBlock) k_pcg_q(PcgArgs<V> a, BicgCtl ctl) {
    if (a.st->col_done[0] || a.st->in_done[0]) return;
    constexpr int RPW = 32 / L;
    const int lane = threadIdx.x % L, sub = (threadIdx.x % 32) / L;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / 32;
    const int64_t nwarp = (int64_t)gridDim.x * blockDim.x / 32;
    const int par = a.st->it_in & 1;
    const V* __restrict__ pold = par ? a.p1 : a.p0;
    V* __restrict__ pnew = par ? a.p0 : a.p1;
    const V beta = (V)a.st->beta[0];
    double part[1] = {0.0};
    for (int64_t w = warp; w * RPW < a.n; w += nwarp) {
        const int64_t i = w * RPW + sub;
        V acc = 0;
        if (i < a.n) {
            const int32_t b = a.rp[i], e = a.rp[i + 1];
            for (int32_t q = b + lane; q < e; q += L) {
                const int32_t j = a.col[q];
                acc += a.K[q] * (a.z[j] + beta * pold[j]);
            }
        }
        acc = group_sum<L>(acc);
        if (i < a.n && lane == 0) {
            const V pv = a.z[i] + beta * pold[i];
            pnew[i] = pv;
            a.q[i] = acc;
            part[0] += (double)pv * (double)acc;
        }
    }
    if (grid_sum<1>(part, a.partial, &a.st->ticket) && threadIdx.x == 0) {
        KrylovState* st = a.st;
        const double pq = part[0];
        if (!(pq > 0.0) || !isfinite(pq)) {
            st->in_done[0] = 1;
            st->it_total[0] += 1;
            st->alpha[0] = 0.0;
            set_cond(ctl.use_cond, ctl.h_inner, 0);
        } else {
            st->alpha[0] = st->rho[0] / pq;
        }
    }
}

// delta += alpha p, r -= alpha q, z = D^{-1} r, <r, z> -> beta, <r, r> -> stop test
template <class V>
__global__ void __launch_bounds__(kBlock) k_pcg_update(PcgArgs<V> a, BicgCtl ctl) {
    if (a.st->col_done[0] || a.st->in_done[0]) return;
    const int par = a.st->it_in & 1;
    const V* __restrict__ pnew = par ? a.p0 : a.p1;
    const V alpha = (V)a.st->alpha[0];
    double part[2] = {0.0, 0.0};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.n; i += (int64_t)gridDim.x * blockDim.x) {
        a.dl[i] += alpha * pnew[i];
        const V rv = a.r[i] - alpha * a.q[i];
        const V zv = a.dinv[i] * rv;
        a.r[i] = rv;
        a.z[i] = zv;
        part[0] += (double)rv * (double)zv;
        part[1] += (double)rv * (double)rv;
    }
    if (grid_sum<2>(part, a.partial, &a.st->ticket) && threadIdx.x == 0) {
        KrylovState* st = a.st;
        const double rz = part[0], rr = part[1];
        st->it_total[0] += 1;
        st->beta[0] = st->rho[0] != 0.0 ? rz / st->rho[0] : 0.0;
        st->rho[0] = rz;
        st->rr_in[0] = rr;
        const bool stop = !isfinite(rr) || rr <= ctl.inner2 * st->rr0_in[0] || rr <= ctl.abs2 * st->bb[0] ||
                          rz == 0.0 || st->it_total[0] >= ctl.max_it || st->it_in + 1 >= ctl.sweep_cap;
        if (stop) st->in_done[0] = 1;
        st->it_in += 1;
        set_cond(ctl.use_cond, ctl.h_inner, !stop);
    }
}

template <class V>
__global__ void __launch_bounds__(kBlock) k_pcg_correct(PcgArgs<V> a) {
    if (a.st->col_done[0]) return;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.n; i += (int64_t)gridDim.x * blockDim.x)
        a.x[i] += (double)a.dl[i];
}

// =====================================================================  update
// u_k^n = u_k^I - dt (dP^k phi)_i / ML_i (Sec. 5, lumping), Dirichlet rows = g;
// p = p* + phi normalised to zero mean; rotation u^{n-2} <- u^{n-1} <- u^n,
// p* <- p, and the history of normalised corrections.
template <class V, int D, int L>
__global__ void __launch_bounds__(kBlock) k_update(UpdArgs<V> a) {
    constexpr int RPW = 32 / L;
    const int lane = threadIdx.x % L, sub = (threadIdx.x % 32) / L;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / 32;
    const int64_t nwarp = (int64_t)gridDim.x * blockDim.x / 32;
    const double mean_p = a.stp->psum / (double)a.n;
    for (int64_t w = warp; w * RPW < a.n; w += nwarp) {
        const int64_t i = w * RPW + sub;
        V acc[D];
#pragma unroll
        for (int k = 0; k < D; ++k) acc[k] = 0;
        if (i < a.n) {
            const int32_t b = a.rp[i], e = a.rp[i + 1];
            for (int32_t q = b + lane; q < e; q += L) {
                const V ph = (V)a.x[a.col[q]];
#pragma unroll
                for (int k = 0; k < D; ++k) acc[k] += a.G[(size_t)k * a.nnz + q] * ph;
            }
        }
#pragma unroll
        for (int k = 0; k < D; ++k) acc[k] = group_sum<L>(acc[k]);
        if (i < a.n && lane == 0) {
            const int dir = a.dir_index[i];
            const double iml = a.invML[i];
#pragma unroll
            for (int k = 0; k < D; ++k) {
                const size_t o = (size_t)i * D + k;
                const double u1 = a.u1[o];
                double un = u1 + a.du[o] - a.dt * (double)acc[k] * iml;
                if (dir >= 0) un = a.g[(size_t)dir * D + k];
                a.u2[o] = u1;
                a.u1[o] = un;
            }
            const double ps = a.pstar[i];
            const double pn = ps + a.x[i] - mean_p;
            const double ph = pn - ps;
            a.pstar[i] = pn;
            a.phi_out[i] = ph;
            a.phi_h2[i] = a.phi_h1[i];
            a.phi_h1[i] = ph;
        }
    }
}

// =====================================================================  driver
template <class V, int D, int L>
struct StepImplT final : StepImpl {
    Solver& S;
    explicit StepImplT(Solver& s) : S(s) {}

    AsmArgs<V> asm_args() {
        Mesh& m = *S.m;
        AsmArgs<V> a{};
        a.rp = m.row_ptr.p;
        a.col = m.col.p;
        a.diag = m.diag.p;
        a.inc_ptr = m.inc_ptr.p;
        a.inc_cell = m.inc_cell.p;
        a.inc_slots = m.inc_slots.p;
        a.beta = S.template beta<V>();
        a.M = S.template mat<V>(m.M64, m.M32);
        a.K = S.template mat<V>(m.K64, m.K32);
        a.G = S.template mat<V>(m.G64, m.G32);
        a.ML = m.ML64.p;
        a.u1 = S.u1.p;
        a.u2 = S.u2.p;
        a.pstar = S.pstar.p;
        a.dir_index = S.dir_index.p;
        a.g = S.g.p;
        for (int k = 0; k < 3; ++k) a.f[k] = S.prm.f[k];
        a.dt = S.prm.dt;
        a.nu = S.prm.nu;
        a.A = S.template A<V>();
        a.dinv = S.template dinvA<V>();
        a.r0 = S.r0u.p;
        a.st = S.st.p;
        a.partial = S.partial.p;
        a.n = m.n;
        a.nnz = m.nnz;
        return a;
    }

    void assemble(cudaStream_t s) override {
        Mesh& m = *S.m;
        k_cell_beta<V, D><<<grid_rows(m.nc, kBlock), kBlock, 0, s>>>(m.nc, m.cell_dof.p, S.template gw<V>(),
                                                                      S.u1.p, S.u2.p, S.template beta<V>());
        const int pa = S.prof_begin(s, OASIS_PROF_ASSEMBLE);
        k_assemble<V, D, L><<<grid_rows(m.n, kBlock / L), kBlock, 0, s>>>(asm_args());
        S.prof_end(s, pa);
        k_zero_du<D><<<grid_rows(m.n * D, kBlock), kBlock, 0, s>>>(m.n, S.du.p);
        OASIS_CUDA(cudaGetLastError());
    }

    BicgArgs<V> bicg_args(int k0) {
        Mesh& m = *S.m;
        BicgArgs<V> a{};
        a.rp = m.row_ptr.p;
        a.col = m.col.p;
        a.A = S.template A<V>();
        a.dinv = S.template dinvA<V>();
        a.r0 = S.r0u.p;
        a.du = S.du.p;
        V** w = S.template work<V>();
        a.r = w[0];
        a.rh = w[1];
        a.p = w[2];
        a.v = w[3];
        a.s = w[4];
        a.t = w[5];
        a.ph = w[6];
        a.sh = w[7];
        a.dl = w[8];
        a.st = S.st.p;
        a.partial = S.partial.p;
        a.n = m.n;
        a.k0 = k0;
        return a;
    }

    BicgCtl ctl_u(const Loop& lp) {
        BicgCtl c{};
        c.rtol2 = S.prm.rtol_u * S.prm.rtol_u;
        c.inner2 = S.mixed ? S.prm.inner_rtol * S.prm.inner_rtol : 0.0;
        c.abs2 = 0.25 * c.rtol2;
        c.max_it = S.prm.max_it_u;
        c.sweep_cap = S.mixed ? 400 : 1 << 30;
        c.use_cond = lp.graph;
        c.h_outer = lp.h_outer;
        c.h_inner = lp.h_inner;
        return c;
    }

    template <int NR>
    void bicg_outer(cudaStream_t s, int k0, const Loop& lp) {
        const int64_t n = S.m->n;
        k_bicg_outer<V, D, NR, L><<<grid_rows(n, kBlock / L), kBlock, 0, s>>>(bicg_args(k0), ctl_u(lp));
        OASIS_CUDA(cudaGetLastError());
    }
    template <int NR>
    void bicg_iter(cudaStream_t s, int k0, const Loop& lp) {
        const int64_t n = S.m->n;
        const int ge = grid_rows(n, kBlock), gr = grid_rows(n, kBlock / L);
        auto a = bicg_args(k0);
        auto c = ctl_u(lp);
        k_bicg_dir<V, D, NR><<<ge, kBlock, 0, s>>>(a);
        int pb = S.prof_begin(s, OASIS_PROF_BICG_SPMM);
        k_bicg_spmm<V, D, NR, L, 0><<<gr, kBlock, 0, s>>>(a, c);
        S.prof_end(s, pb);
        k_bicg_s<V, D, NR><<<ge, kBlock, 0, s>>>(a);
        pb = S.prof_begin(s, OASIS_PROF_BICG_SPMM);
        k_bicg_spmm<V, D, NR, L, 1><<<gr, kBlock, 0, s>>>(a, c);
        S.prof_end(s, pb);
        k_bicg_xr<V, D, NR><<<ge, kBlock, 0, s>>>(a, c);
        OASIS_CUDA(cudaGetLastError());
    }
    template <int NR>
    void bicg_correct(cudaStream_t s, int k0) {
        k_bicg_correct<V, D, NR><<<grid_rows(S.m->n, kBlock), kBlock, 0, s>>>(bicg_args(k0));
        OASIS_CUDA(cudaGetLastError());
    }

    template <int NR>
    void bicg_solve(cudaStream_t s, int k0, bool graph) {
        S.run_loops(
            s, graph, 0, [&](cudaStream_t ss, const Loop& lp) { bicg_outer<NR>(ss, k0, lp); },
            [&](cudaStream_t ss, const Loop& lp) { bicg_iter<NR>(ss, k0, lp); },
            [&](cudaStream_t ss, const Loop&) { bicg_correct<NR>(ss, k0); }, k0, NR);
    }

    void tentative_solve(cudaStream_t s, bool graph) override {
        if (S.prm.batch_rhs) {
            bicg_solve<D>(s, 0, graph);
        } else {
            for (int k = 0; k < D; ++k) bicg_solve<1>(s, k, graph);
        }
    }

    PresArgs<V> pres_args() {
        Mesh& m = *S.m;
        PresArgs<V> a{};
        a.rp = m.row_ptr.p;
        a.col = m.col.p;
        a.G = S.template mat<V>(m.G64, m.G32);
        a.u1 = S.u1.p;
        a.du = S.du.p;
        a.b = S.bphi.p;
        a.dt = S.prm.dt;
        a.st = S.st.p + 1;
        a.partial = S.partial.p;
        a.n = m.n;
        a.nnz = m.nnz;
        return a;
    }

    PcgArgs<V> pcg_args() {
        Mesh& m = *S.m;
        PcgArgs<V> a{};
        a.rp = m.row_ptr.p;
        a.col = m.col.p;
        a.K = S.template mat<V>(m.K64, m.K32);
        a.K64 = m.K64.p;
        a.dinv = S.mixed ? (const V*)(const void*)m.dinvK32.p : (const V*)(const void*)m.dinvK64.p;
        a.b = S.bphi.p;
        a.x = S.xp.p;
        a.pstar = S.pstar.p;
        V** w = S.template pwork<V>();
        a.r = w[0];
        a.z = w[1];
        a.p0 = w[2];
        a.p1 = w[3];
        a.q = w[4];
        a.dl = w[5];
        a.st = S.st.p + 1;
        a.partial = S.partial.p;
        a.n = m.n;
        return a;
    }

    BicgCtl ctl_p(const Loop& lp) {
        BicgCtl c{};
        c.rtol2 = S.prm.rtol_p * S.prm.rtol_p;
        c.inner2 = S.mixed ? S.prm.inner_rtol * S.prm.inner_rtol : 0.0;
        c.abs2 = 0.25 * c.rtol2;
        c.max_it = S.prm.max_it_p;
        c.sweep_cap = S.mixed ? 4000 : 1 << 30;
        c.use_cond = lp.graph;
        c.h_outer = lp.h_outer;
        c.h_inner = lp.h_inner;
        return c;
    }

    void pressure_solve(cudaStream_t s, bool graph) override {
        Mesh& m = *S.m;
        const int64_t n = m.n;
        const int ge = grid_rows(n, kBlock), gr = grid_rows(n, kBlock / L);
        const int pr = S.prof_begin(s, OASIS_PROF_PRESSURE_RHS);
        k_pressure_rhs<V, D, L><<<gr, kBlock, 0, s>>>(pres_args());
        S.prof_end(s, pr);
        const int mode = S.prm.guess == OASIS_GUESS_PREV_PHI ? OASIS_GUESS_PREV_PHI : OASIS_GUESS_ZERO;
        k_phi_guess<<<ge, kBlock, 0, s>>>(n, mode, S.phi_h1.p, S.xp.p);
        OASIS_CUDA(cudaGetLastError());
        S.run_loops(
            s, graph, 1,
            [&](cudaStream_t ss, const Loop& lp) {
                k_pcg_outer<V, L><<<gr, kBlock, 0, ss>>>(pcg_args(), ctl_p(lp));
                OASIS_CUDA(cudaGetLastError());
            },
            [&](cudaStream_t ss, const Loop& lp) {
                auto a = pcg_args();
                auto c = ctl_p(lp);
                const int pq = S.prof_begin(ss, OASIS_PROF_PCG_SPMV);
                k_pcg_q<V, L><<<gr, kBlock, 0, ss>>>(a, c);
                S.prof_end(ss, pq);
                const int pu = S.prof_begin(ss, OASIS_PROF_PCG_UPDATE);
                k_pcg_update<V><<<ge, kBlock, 0, ss>>>(a, c);
                S.prof_end(ss, pu);
                OASIS_CUDA(cudaGetLastError());
            },
            [&](cudaStream_t ss, const Loop&) {
                k_pcg_correct<V><<<ge, kBlock, 0, ss>>>(pcg_args());
                OASIS_CUDA(cudaGetLastError());
            },
            0, 1);
    }

    void update(cudaStream_t s) override {
        Mesh& m = *S.m;
        UpdArgs<V> a{};
        a.rp = m.row_ptr.p;
        a.col = m.col.p;
        a.G = S.template mat<V>(m.G64, m.G32);
        a.invML = m.invML64.p;
        a.x = S.xp.p;
        a.du = S.du.p;
        a.u1 = S.u1.p;
        a.u2 = S.u2.p;
        a.pstar = S.pstar.p;
        a.phi_out = S.phi.p;
        a.phi_h1 = S.phi_h1.p;
        a.phi_h2 = S.phi_h2.p;
        a.dir_index = S.dir_index.p;
        a.g = S.g.p;
        a.dt = S.prm.dt;
        a.stp = S.st.p + 1;
        a.n = m.n;
        a.nnz = m.nnz;
        const int pu = S.prof_begin(s, OASIS_PROF_UPDATE);
        k_update<V, D, L><<<grid_rows(m.n, kBlock / L), kBlock, 0, s>>>(a);
        S.prof_end(s, pu);
        OASIS_CUDA(cudaGetLastError());
    }
};

template <class V, int D>
static StepImpl* make_impl_l(Solver& s, int L) {
    switch (L) {
        case 8: return new StepImplT<V, D, 8>(s);
        case 16: return new StepImplT<V, D, 16>(s);
        default: throw Error(OASIS_EINVAL, "step kernels support 8 or 16 lanes per row");
    }
}

StepImpl* make_step_impl(Solver& s, int lanes) {
    const bool mixed = s.mixed;
    if (s.m->dim == 2) return mixed ? make_impl_l<float, 2>(s, lanes) : make_impl_l<double, 2>(s, lanes);
    return mixed ? make_impl_l<float, 3>(s, lanes) : make_impl_l<double, 3>(s, lanes);
}

}  // namespace oasis
