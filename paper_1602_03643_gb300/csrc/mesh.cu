// Mesh set-up: CSR sparsity pattern, dof-to-cell incidence, per-cell geometry
// and the constant matrices of Sec. 5 (M, K, dP^k, lumped mass), plus the
// stand-alone SpMV kernels.
#include <algorithm>
#include <cmath>
#include <numeric>
#include <mutex>
#include <thread>

#include "device.cuh"
#include "internal.cuh"

namespace oasis {

int num_sms() {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        OASIS_CUDA(cudaGetDevice(&dev));
        OASIS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    }
    return sms;
}

// ------------------------------------------------------------------ host build
template <class F>
static void parallel_for(int64_t n, F f) {
    int nt = (int)std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
    if (n < 20000) nt = 1;
    std::vector<std::thread> th;
    const int64_t chunk = (n + nt - 1) / nt;
    for (int t = 0; t < nt; ++t) {
        const int64_t a = t * chunk, b = std::min(n, a + chunk);
        if (a >= b) break;
        th.emplace_back([=] { f(a, b); });
    }
    for (auto& x : th) x.join();
}

Mesh* build_mesh(int dim, int64_t nv, const double* coords, int64_t nc, const int32_t* cells,
                 const int32_t* dof_of_vertex, int64_t n_dofs, const int32_t* perm) {
    OASIS_CHECK(dim == 2 || dim == 3, OASIS_EINVAL, "dim must be 2 or 3");
    OASIS_CHECK(nv > 0 && nc > 0 && coords && cells, OASIS_EINVAL, "empty mesh or null pointer");
    OASIS_CHECK(nv < INT32_MAX && nc * (dim + 1) < INT32_MAX, OASIS_EINVAL, "mesh too large for int32 indices");
    if (!dof_of_vertex) n_dofs = nv;
    OASIS_CHECK(n_dofs > 0 && n_dofs <= nv, OASIS_EINVAL, "n_dofs out of range");
    const int d1 = dim + 1;

    auto m = std::make_unique<Mesh>();
    m->dim = dim;
    m->nv = nv;
    m->nc = nc;
    m->n = n_dofs;
    if (perm) {
        // a permutation of 0 .. n_dofs-1: every value in range and seen once
        std::vector<uint8_t> seen(n_dofs, 0);
        for (int64_t d = 0; d < n_dofs; ++d) {
            OASIS_CHECK(perm[d] >= 0 && perm[d] < n_dofs, OASIS_EINVAL, "perm entry out of range");
            OASIS_CHECK(!seen[perm[d]], OASIS_EINVAL, "perm is not a permutation (repeated entry)");
            seen[perm[d]] = 1;
        }
        m->h_perm.assign(perm, perm + n_dofs);
    }
    std::vector<int32_t> cdof((size_t)nc * d1);
    for (int64_t c = 0; c < nc; ++c) {
        for (int a = 0; a < d1; ++a) {
            const int32_t v = cells[c * d1 + a];
            OASIS_CHECK(v >= 0 && v < nv, OASIS_EINVAL, "cell vertex index out of range");
            const int32_t dof = dof_of_vertex ? dof_of_vertex[v] : v;
            OASIS_CHECK(dof >= 0 && dof < n_dofs, OASIS_EINVAL, "dof_of_vertex entry out of range");
            cdof[c * d1 + a] = perm ? perm[dof] : dof;
        }
        for (int a = 0; a < d1; ++a)
            for (int b = a + 1; b < d1; ++b)
                OASIS_CHECK(cdof[c * d1 + a] != cdof[c * d1 + b], OASIS_EMESH,
                            "cell " + std::to_string(c) + " has a repeated dof");
    }
    const int64_t n = n_dofs;
    // cells stored in the order of their lowest (internal) dof, ties in the given
    // order (a counting sort): under a renumbering such as RCM, the cells a tile of
    // consecutive rows touches then sit close together, so the assembly's gathers
    // of their cell terms, and the cell pass's gathers of dof values, stay local.
    // Results depend on it only through the order of sums.
    std::vector<int32_t> cells_in((size_t)nc * d1);
    {
        std::vector<int64_t> start(n + 1, 0);
        std::vector<int32_t> low(nc);
        for (int64_t c = 0; c < nc; ++c) {
            int32_t lo = cdof[c * d1];
            for (int a = 1; a < d1; ++a) lo = std::min(lo, cdof[c * d1 + a]);
            low[c] = lo;
            start[lo + 1]++;
        }
        for (int64_t i = 0; i < n; ++i) start[i + 1] += start[i];
        std::vector<int32_t> cdof_in(cdof.size());
        for (int64_t c = 0; c < nc; ++c) {
            const int64_t o = start[low[c]]++;
            for (int a = 0; a < d1; ++a) {
                cdof_in[o * d1 + a] = cdof[c * d1 + a];
                cells_in[o * d1 + a] = cells[c * d1 + a];
            }
        }
        cdof.swap(cdof_in);
    }
    // dof -> cell incidence (counting sort keeps cells in increasing order)
    std::vector<int32_t> inc_ptr(n + 1, 0), inc_cell((size_t)nc * d1);
    for (size_t q = 0; q < cdof.size(); ++q) inc_ptr[cdof[q] + 1]++;
    for (int64_t i = 0; i < n; ++i) inc_ptr[i + 1] += inc_ptr[i];
    {
        std::vector<int32_t> fill(inc_ptr.begin(), inc_ptr.end() - 1);
        for (int64_t c = 0; c < nc; ++c)
            for (int a = 0; a < d1; ++a) inc_cell[fill[cdof[c * d1 + a]]++] = (int32_t)c;
    }
    // row pattern: union of the dofs of the incident cells
    std::vector<int32_t> row_len(n);
    parallel_for(n, [&](int64_t a, int64_t b) {
        std::vector<int32_t> buf;
        for (int64_t i = a; i < b; ++i) {
            buf.clear();
            for (int32_t q = inc_ptr[i]; q < inc_ptr[i + 1]; ++q)
                for (int k = 0; k < d1; ++k) buf.push_back(cdof[(size_t)inc_cell[q] * d1 + k]);
            std::sort(buf.begin(), buf.end());
            row_len[i] = (int32_t)(std::unique(buf.begin(), buf.end()) - buf.begin());
        }
    });
    std::vector<int32_t> row_ptr(n + 1, 0);
    for (int64_t i = 0; i < n; ++i) row_ptr[i + 1] = row_ptr[i] + row_len[i];
    const int64_t nnz = row_ptr[n];
    OASIS_CHECK(nnz < INT32_MAX, OASIS_EINVAL, "too many nonzeros for int32 indices");
    const int max_row = n ? *std::max_element(row_len.begin(), row_len.end()) : 0;
    OASIS_CHECK(max_row <= 255, OASIS_EMESH, "more than 255 pattern entries in a row");
    std::vector<int32_t> col(nnz), diag(n);
    std::vector<uint32_t> inc_slots((size_t)nc * d1);
    parallel_for(n, [&](int64_t a, int64_t b) {
        std::vector<int32_t> buf;
        for (int64_t i = a; i < b; ++i) {
            buf.clear();
            for (int32_t q = inc_ptr[i]; q < inc_ptr[i + 1]; ++q)
                for (int k = 0; k < d1; ++k) buf.push_back(cdof[(size_t)inc_cell[q] * d1 + k]);
            std::sort(buf.begin(), buf.end());
            buf.erase(std::unique(buf.begin(), buf.end()), buf.end());
            std::copy(buf.begin(), buf.end(), col.begin() + row_ptr[i]);
            diag[i] = row_ptr[i] + (int32_t)(std::lower_bound(buf.begin(), buf.end(), (int32_t)i) - buf.begin());
            for (int32_t q = inc_ptr[i]; q < inc_ptr[i + 1]; ++q) {
                uint32_t w = 0xffffffffu;
                for (int k = 0; k < d1; ++k) {
                    const int32_t dof = cdof[(size_t)inc_cell[q] * d1 + k];
                    const uint32_t slot = (uint32_t)(std::lower_bound(buf.begin(), buf.end(), dof) - buf.begin());
                    w = (w & ~(0xffu << (8 * k))) | (slot << (8 * k));
                }
                inc_slots[q] = w;
            }
        }
    });

    cudaStream_t s = 0;
    m->nnz = nnz;
    m->max_row = max_row;
    for (int64_t r0 = 0; r0 < n; r0 += kBlock) {
        const int64_t r1 = std::min<int64_t>(n, r0 + kBlock);
        m->tile_cap = std::max<int>(m->tile_cap, row_ptr[r1] - row_ptr[r0]);
    }
    for (int64_t r0 = 0; r0 < n; r0 += kTileN) {
        const int64_t r1 = std::min<int64_t>(n, r0 + kTileN);
        m->tile_cap_n = std::max<int>(m->tile_cap_n, row_ptr[r1] - row_ptr[r0]);
    }
    // row_ptr and col carry 8 padding entries so that 16-byte aligned bulk copies
    // of a tile's range never read past the allocation
    {
        std::vector<int32_t> rp_pad(row_ptr);
        rp_pad.resize(row_ptr.size() + 8, row_ptr.back());
        m->row_ptr.upload(rp_pad.data(), rp_pad.size(), s);
        std::vector<int32_t> col_pad(col);
        col_pad.resize(col.size() + 8, 0);
        m->col.upload(col_pad.data(), col_pad.size(), s);
    }
    m->diag.upload(diag.data(), diag.size(), s);
    m->cell_vert.upload(cells_in.data(), cells_in.size(), s);
    m->cell_dof.upload(cdof.data(), cdof.size(), s);
    m->coords.upload(coords, (size_t)nv * dim, s);
    m->inc_ptr.upload(inc_ptr.data(), inc_ptr.size(), s);
    m->inc_cell.upload(inc_cell.data(), inc_cell.size(), s);
    m->inc_slots.upload(inc_slots.data(), inc_slots.size(), s);
    if (!m->h_perm.empty()) m->perm.upload(m->h_perm.data(), m->h_perm.size(), s);
    m->err.alloc(1);
    OASIS_CUDA(cudaMemsetAsync(m->err.p, 0, sizeof(int32_t), s));
    OASIS_CUDA(cudaStreamSynchronize(s));
    // SELL-32 layout of the pattern
    {
        const int64_t ns = (n + 31) / 32;
        std::vector<int32_t> sptr(ns + 1, 0), slen(ns, 0);
        for (int64_t sl = 0; sl < ns; ++sl) {
            int mx = 0;
            for (int64_t i = sl * 32; i < std::min<int64_t>(n, sl * 32 + 32); ++i) mx = std::max(mx, row_len[i]);
            slen[sl] = mx;
            sptr[sl + 1] = sptr[sl] + 32 * mx;
        }
        const int64_t nsell = sptr[ns];
        OASIS_CHECK(nsell < INT32_MAX, OASIS_EINVAL, "too many padded entries for int32 indices");
        std::vector<int32_t> scol(nsell), sof(nnz);
        for (int64_t sl = 0; sl < ns; ++sl) {
            for (int l = 0; l < 32; ++l) {
                const int64_t i = sl * 32 + l;
                for (int k = 0; k < slen[sl]; ++k) {
                    const int64_t pos = sptr[sl] + 32 * k + l;
                    if (i < n && k < row_len[i]) {
                        scol[pos] = col[row_ptr[i] + k];
                        sof[row_ptr[i] + k] = (int32_t)pos;
                    } else {
                        scol[pos] = (int32_t)std::min<int64_t>(i, n - 1);
                    }
                }
            }
        }
        // modular 16-bit offsets, when they fit (the host copy lives until the
        // stream synchronisation below)
        std::vector<int16_t> dcol(nsell);
        {
            bool fits = true;
            for (int64_t sl = 0; sl < ns && fits; ++sl) {
                for (int l = 0; l < 32 && fits; ++l) {
                    const int64_t i = sl * 32 + l;
                    for (int k = 0; k < slen[sl]; ++k) {
                        const int64_t pos = sptr[sl] + 32 * k + l;
                        // the plain offset where it fits (always for the padding
                        // lanes past the last row, whose column is n - 1), else
                        // the offset modulo n, nearest to zero: the decode adds it
                        // to the row and wraps once into [0, n)
                        int64_t d = (int64_t)scol[pos] - i;
                        if (d < -32768 || d > 32767) {
                            d %= n;
                            if (d < 0) d += n;
                            if (d > n / 2) d -= n;
                        }
                        if (d < -32768 || d > 32767) {
                            fits = false;
                            break;
                        }
                        dcol[pos] = (int16_t)d;
                    }
                }
            }
            if (fits) {
                m->sell_dcol.upload(dcol.data(), dcol.size(), s);
                std::vector<int16_t> ccol((size_t)m->nnz);
                for (int64_t q = 0; q < m->nnz; ++q) ccol[q] = dcol[sof[q]];
                m->csr_dcol.upload(ccol.data(), ccol.size(), s);
                OASIS_CUDA(cudaStreamSynchronize(s));
            }
        }
        m->n_sell = nsell;
        m->sell_ptr.upload(sptr.data(), sptr.size(), s);
        m->sell_len.upload(slen.data(), slen.size(), s);
        m->sell_col.upload(scol.data(), scol.size(), s);
        m->sell_of_csr.upload(sof.data(), sof.size(), s);
        OASIS_CUDA(cudaStreamSynchronize(s));
    }
    m->h_row_ptr = std::move(row_ptr);
    m->h_col = std::move(col);
    return m.release();
}

void caller_pattern(const Mesh& m, std::vector<int32_t>& row_ptr, std::vector<int32_t>& col,
                    std::vector<int64_t>& src) {
    const int64_t n = m.n;
    row_ptr.assign(n + 1, 0);
    col.assign(m.nnz, 0);
    src.assign(m.nnz, 0);
    if (m.h_perm.empty()) {
        std::copy(m.h_row_ptr.begin(), m.h_row_ptr.begin() + n + 1, row_ptr.begin());
        std::copy(m.h_col.begin(), m.h_col.begin() + m.nnz, col.begin());
        for (int64_t e = 0; e < m.nnz; ++e) src[e] = e;
        return;
    }
    std::vector<int32_t> caller_of(n);
    for (int64_t d = 0; d < n; ++d) caller_of[m.h_perm[d]] = (int32_t)d;
    for (int64_t d = 0; d < n; ++d) {
        const int32_t r = m.h_perm[d];
        row_ptr[d + 1] = row_ptr[d] + (m.h_row_ptr[r + 1] - m.h_row_ptr[r]);
    }
    parallel_for(n, [&](int64_t a, int64_t b) {
        std::vector<std::pair<int32_t, int64_t>> buf;
        for (int64_t d = a; d < b; ++d) {
            const int32_t r = m.h_perm[d];
            buf.clear();
            for (int32_t e = m.h_row_ptr[r]; e < m.h_row_ptr[r + 1]; ++e) buf.emplace_back(caller_of[m.h_col[e]], e);
            std::sort(buf.begin(), buf.end());
            for (size_t q = 0; q < buf.size(); ++q) {
                col[row_ptr[d] + q] = buf[q].first;
                src[row_ptr[d] + q] = buf[q].second;
            }
        }
    });
}

// ------------------------------------------------------------------ geometry
// Barycentric gradients of one simplex from its Jacobian J = [x_1-x_0, ..., x_d-x_0]:
// grad lambda_k (k >= 1) is row k-1 of J^{-1}, grad lambda_0 = -sum_k grad lambda_k.
template <int D>
__global__ void k_cell_geometry(int64_t nc, const int32_t* __restrict__ cell_vert,
                                const double* __restrict__ coords, double* __restrict__ grad,
                                double* __restrict__ vol, double* __restrict__ gw64,
                                float* __restrict__ gw32, int32_t* err) {
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nc;
         c += (int64_t)gridDim.x * blockDim.x) {
        double x[D + 1][D];
        for (int a = 0; a <= D; ++a)
            for (int k = 0; k < D; ++k) x[a][k] = coords[(size_t)cell_vert[c * (D + 1) + a] * D + k];
        double J[D][D];  // J[r][col] = x_{col+1}[r] - x_0[r]
        for (int r = 0; r < D; ++r)
            for (int q = 0; q < D; ++q) J[r][q] = x[q + 1][r] - x[0][r];
        double inv[D][D], det;
        if (D == 2) {
            det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
            inv[0][0] = J[1][1];
            inv[0][1] = -J[0][1];
            inv[1][0] = -J[1][0];
            inv[1][1] = J[0][0];
        } else {
            // adjugate of a 3x3 matrix (cofactor transpose)
            const double(*a)[D] = J;
            inv[0][0] = a[1][1] * a[2][2] - a[1][2] * a[2][1];
            inv[0][1] = a[0][2] * a[2][1] - a[0][1] * a[2][2];
            inv[0][2] = a[0][1] * a[1][2] - a[0][2] * a[1][1];
            inv[1][0] = a[1][2] * a[2][0] - a[1][0] * a[2][2];
            inv[1][1] = a[0][0] * a[2][2] - a[0][2] * a[2][0];
            inv[1][2] = a[0][2] * a[1][0] - a[0][0] * a[1][2];
            inv[2][0] = a[1][0] * a[2][1] - a[1][1] * a[2][0];
            inv[2][1] = a[0][1] * a[2][0] - a[0][0] * a[2][1];
            inv[2][2] = a[0][0] * a[1][1] - a[0][1] * a[1][0];
            det = a[0][0] * inv[0][0] + a[0][1] * inv[1][0] + a[0][2] * inv[2][0];
        }
        if (!(det != 0.0) || !isfinite(det)) {
            atomicExch(err, 1);
            det = 1.0;
        }
        const double rdet = 1.0 / det;
        double g[D + 1][D];
        for (int k = 0; k < D; ++k) g[0][k] = 0.0;
        for (int a = 1; a <= D; ++a)
            for (int k = 0; k < D; ++k) {
                g[a][k] = inv[a - 1][k] * rdet;
                g[0][k] -= g[a][k];
            }
        const double v = fabs(det) / (D == 2 ? 2.0 : 6.0);
        const double w = v / ((D + 1) * (D + 2));
        vol[c] = v;
        for (int a = 0; a <= D; ++a)
            for (int k = 0; k < D; ++k) {
                const size_t o = ((size_t)c * (D + 1) + a) * D + k;
                grad[o] = g[a][k];
                gw64[o] = w * g[a][k];
                gw32[o] = (float)(w * g[a][k]);
            }
    }
}

// Row-gather assembly of the constant matrices: thread per row, summing the
// element contributions of every incident cell in increasing cell order
// (deterministic, no atomics).  Element integrals of linear Lagrange simplices:
//   M^T_ab = |T| (1 + delta_ab) / ((d+1)(d+2)),  K^T_ab = |T| grad lambda_a . grad lambda_b,
//   dP^{k,T}_ab = |T| d_k lambda_b / (d+1),        int_T lambda_a = |T| / (d+1).
template <int D>
__global__ void k_row_constant(int64_t n, const int32_t* __restrict__ row_ptr,
                               const int32_t* __restrict__ diag, const int32_t* __restrict__ inc_ptr,
                               const int32_t* __restrict__ inc_cell, const uint32_t* __restrict__ inc_slots,
                               const double* __restrict__ grad, const double* __restrict__ vol,
                               int64_t nnz, double* __restrict__ M, double* __restrict__ K,
                               double* __restrict__ G, double* __restrict__ ML) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t b = row_ptr[i], e = row_ptr[i + 1];
        for (int32_t q = b; q < e; ++q) {
            M[q] = 0.0;
            K[q] = 0.0;
            for (int k = 0; k < D; ++k) G[(size_t)k * nnz + q] = 0.0;
        }
        const uint32_t dslot = (uint32_t)(diag[i] - b);
        double ml = 0.0;
        for (int32_t q = inc_ptr[i]; q < inc_ptr[i + 1]; ++q) {
            const int32_t c = inc_cell[q];
            const uint32_t w = inc_slots[q];
            int la = 0;
            for (int a = 0; a <= D; ++a)
                if (((w >> (8 * a)) & 0xffu) == dslot) la = a;
            const double v = vol[c];
            const double* g = grad + (size_t)c * (D + 1) * D;
            ml += v / (D + 1);
            for (int a = 0; a <= D; ++a) {
                const int32_t pos = b + (int32_t)((w >> (8 * a)) & 0xffu);
                M[pos] += v * (a == la ? 2.0 : 1.0) / ((D + 1) * (D + 2));
                double kk = 0.0;
                for (int k = 0; k < D; ++k) kk += g[la * D + k] * g[a * D + k];
                K[pos] += v * kk;
                for (int k = 0; k < D; ++k) G[(size_t)k * nnz + pos] += v * g[a * D + k] / (D + 1);
            }
        }
        ML[i] = ml;
    }
}

__global__ void k_mesh_derived(int64_t n, const int32_t* __restrict__ diag, const double* __restrict__ K,
                               const double* __restrict__ ML, double* __restrict__ invML,
                               double* __restrict__ dinvK64, float* __restrict__ dinvK32,
                               float* __restrict__ ML32, float* __restrict__ invML32) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        invML[i] = 1.0 / ML[i];
        ML32[i] = (float)ML[i];
        invML32[i] = (float)(1.0 / ML[i]);
        const double kd = K[diag[i]];
        const double di = kd != 0.0 ? 1.0 / kd : 1.0;
        dinvK64[i] = di;
        dinvK32[i] = (float)di;
    }
}

// K split into float-float (hi = K rounded to float, lo = the remainder)
__global__ void k_to_ff(int64_t n, const double* __restrict__ a, float2* __restrict__ b) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float hi = (float)a[i];
        b[i] = make_float2(hi, (float)(a[i] - (double)hi));
    }
}

__global__ void k_to_f32(int64_t n, const double* __restrict__ a, float* __restrict__ b) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        b[i] = (float)a[i];
}

// K in the SELL-32 layout, in float64, float32 and float-float.
__global__ void k_csr_to_sell(int64_t nnz, const int32_t* __restrict__ sof, const double* __restrict__ v,
                              double* __restrict__ v64, float* __restrict__ v32, float2* __restrict__ vff) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t q = sof[e];
        const double x = v[e];
        const float hi = (float)x;
        v64[q] = x;
        v32[q] = hi;
        vff[q] = make_float2(hi, (float)(x - (double)hi));
    }
}

static int grid_for(int64_t items, int per_block = kBlock) {
    const int64_t want = (items + per_block - 1) / per_block;
    const int64_t cap = (int64_t)num_sms() * 8;
    return (int)std::max<int64_t>(1, std::min(want, cap));
}

void assemble_constant(Mesh& m, cudaStream_t s) {
    const int D = m.dim;
    const size_t gsz = (size_t)m.nc * (D + 1) * D;
    DBuf<double> grad, vol;
    grad.alloc(gsz);
    vol.alloc(m.nc);
    m.gw64.alloc(gsz);
    m.gw32.alloc(gsz);
    OASIS_CUDA(cudaMemsetAsync(m.err.p, 0, sizeof(int32_t), s));
    const int gc = grid_for(m.nc);
    if (D == 2)
        k_cell_geometry<2><<<gc, kBlock, 0, s>>>(m.nc, m.cell_vert.p, m.coords.p, grad.p, vol.p, m.gw64.p, m.gw32.p, m.err.p);
    else
        k_cell_geometry<3><<<gc, kBlock, 0, s>>>(m.nc, m.cell_vert.p, m.coords.p, grad.p, vol.p, m.gw64.p, m.gw32.p, m.err.p);
    OASIS_CUDA(cudaGetLastError());
    int32_t herr = 0;
    OASIS_CUDA(cudaMemcpyAsync(&herr, m.err.p, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    OASIS_CUDA(cudaStreamSynchronize(s));
    OASIS_CHECK(herr == 0, OASIS_EMESH, "degenerate (zero-volume) cell");

    m.M64.alloc(m.nnz);
    m.K64.alloc(m.nnz + 8);
    OASIS_CUDA(cudaMemsetAsync(m.K64.p, 0, (m.nnz + 8) * sizeof(double), s));
    m.G64.alloc((size_t)D * m.nnz);
    m.ML64.alloc(m.n);
    const int gr = grid_for(m.n);
    if (D == 2)
        k_row_constant<2><<<gr, kBlock, 0, s>>>(m.n, m.row_ptr.p, m.diag.p, m.inc_ptr.p, m.inc_cell.p,
                                                m.inc_slots.p, grad.p, vol.p, m.nnz, m.M64.p, m.K64.p,
                                                m.G64.p, m.ML64.p);
    else
        k_row_constant<3><<<gr, kBlock, 0, s>>>(m.n, m.row_ptr.p, m.diag.p, m.inc_ptr.p, m.inc_cell.p,
                                                m.inc_slots.p, grad.p, vol.p, m.nnz, m.M64.p, m.K64.p,
                                                m.G64.p, m.ML64.p);
    OASIS_CUDA(cudaGetLastError());
    m.invML64.alloc(m.n);
    m.dinvK64.alloc(m.n);
    m.dinvK32.alloc(m.n);
    m.ML32.alloc(m.n);
    m.invML32.alloc(m.n);
    k_mesh_derived<<<gr, kBlock, 0, s>>>(m.n, m.diag.p, m.K64.p, m.ML64.p, m.invML64.p, m.dinvK64.p, m.dinvK32.p,
                                         m.ML32.p, m.invML32.p);
    m.Kff.alloc(m.nnz);
    k_to_ff<<<grid_for(m.nnz), kBlock, 0, s>>>(m.nnz, m.K64.p, m.Kff.p);
    m.Gff.alloc((size_t)D * m.nnz);
    k_to_ff<<<grid_for((int64_t)D * m.nnz), kBlock, 0, s>>>((int64_t)D * m.nnz, m.G64.p, m.Gff.p);
    m.M32.alloc(m.nnz);
    m.K32.alloc(m.nnz + 8);
    OASIS_CUDA(cudaMemsetAsync(m.K32.p, 0, (m.nnz + 8) * sizeof(float), s));
    m.G32.alloc((size_t)D * m.nnz);
    k_to_f32<<<grid_for(m.nnz), kBlock, 0, s>>>(m.nnz, m.M64.p, m.M32.p);
    k_to_f32<<<grid_for(m.nnz), kBlock, 0, s>>>(m.nnz, m.K64.p, m.K32.p);
    k_to_f32<<<grid_for((int64_t)D * m.nnz), kBlock, 0, s>>>((int64_t)D * m.nnz, m.G64.p, m.G32.p);
    OASIS_CUDA(cudaGetLastError());
    m.K32s.alloc(m.n_sell);
    m.K64s.alloc(m.n_sell);
    m.Kffs.alloc(m.n_sell);
    OASIS_CUDA(cudaMemsetAsync(m.K32s.p, 0, m.n_sell * sizeof(float), s));
    OASIS_CUDA(cudaMemsetAsync(m.K64s.p, 0, m.n_sell * sizeof(double), s));
    OASIS_CUDA(cudaMemsetAsync(m.Kffs.p, 0, m.n_sell * sizeof(float2), s));
    k_csr_to_sell<<<grid_for(m.nnz), kBlock, 0, s>>>(m.nnz, m.sell_of_csr.p, m.K64.p, m.K64s.p, m.K32s.p, m.Kffs.p);
    m.red_partial.alloc((size_t)((m.n + kBlock - 1) / kBlock));
    m.red_ticket.alloc(1);
    OASIS_CUDA(cudaMemsetAsync(m.red_ticket.p, 0, sizeof(uint32_t), s));
    OASIS_CUDA(cudaStreamSynchronize(s));
    m.assembled = true;
}

// ------------------------------------------------------------------ SpMV
// CSR SpMV with L lanes per row (a "vector" CSR kernel): the lanes of a group
// stride over the row's entries and combine with shuffles.  The warp-level
// loop is uniform, so every shuffle has all 32 lanes present.
template <class V, int L>
__global__ void __launch_bounds__(kBlock) k_spmv(int64_t n, const int32_t* __restrict__ rp,
                                                 const int32_t* __restrict__ col,
                                                 const V* __restrict__ val, const V* __restrict__ x,
                                                 V* __restrict__ y) {
    constexpr int RPW = 32 / L;
    const int lane = threadIdx.x % L;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / 32;
    const int64_t nwarp = (int64_t)gridDim.x * blockDim.x / 32;
    const int sub = (threadIdx.x % 32) / L;
    for (int64_t w = warp; w * RPW < n; w += nwarp) {
        const int64_t i = w * RPW + sub;
        V acc = 0;
        if (i < n) {
            const int32_t b = rp[i], e = rp[i + 1];
            for (int32_t q = b + lane; q < e; q += L) acc += val[q] * __ldg(&x[col[q]]);
        }
        acc = group_sum<L>(acc);
        if (i < n && lane == 0) y[i] = acc;
    }
}

template <class V>
static void spmv_launch(const Mesh& m, const V* vals, const V* x, V* y, int lanes, cudaStream_t s) {
    const int rows_per_block = kBlock / lanes;
    const int g = grid_for(m.n, rows_per_block);
    switch (lanes) {
        case 4: k_spmv<V, 4><<<g, kBlock, 0, s>>>(m.n, m.row_ptr.p, m.col.p, vals, x, y); break;
        case 8: k_spmv<V, 8><<<g, kBlock, 0, s>>>(m.n, m.row_ptr.p, m.col.p, vals, x, y); break;
        case 16: k_spmv<V, 16><<<g, kBlock, 0, s>>>(m.n, m.row_ptr.p, m.col.p, vals, x, y); break;
        case 32: k_spmv<V, 32><<<g, kBlock, 0, s>>>(m.n, m.row_ptr.p, m.col.p, vals, x, y); break;
        default: throw Error(OASIS_EINVAL, "lanes must be 4, 8, 16 or 32");
    }
    OASIS_CUDA(cudaGetLastError());
}

// y = Mat x and x . y in float64 with 256-row tiles: an entry-parallel product
// phase into shared memory, a thread-per-row sum, one partial sum per tile in
// `tile_partial`, and a deterministic final sum (in tile order) by the block
// that takes the last ticket.  `ticket` must be zero at launch; it is left zero.
__global__ void __launch_bounds__(kBlock) k_spmv_dot_tiles(int64_t n, const int32_t* __restrict__ rp,
                                                           const int32_t* __restrict__ col,
                                                           const double* __restrict__ val,
                                                           const double* __restrict__ x, double* __restrict__ y,
                                                           double* __restrict__ tile_partial, uint32_t* ticket,
                                                           double* __restrict__ xy) {
    extern __shared__ __align__(16) unsigned char dsm[];
    double* s_prod = reinterpret_cast<double*>(dsm);
    __shared__ int32_t s_rp[kBlock + 1];
    const int64_t ntiles = (n + kBlock - 1) / kBlock;
    const int r = threadIdx.x;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t r0 = tile * kBlock;
        const int nr = (int)min((int64_t)kBlock, n - r0);
        for (int k = r; k <= nr; k += blockDim.x) s_rp[k] = rp[r0 + k];
        __syncthreads();
        const int32_t e0 = s_rp[0], e1 = s_rp[nr];
        for (int32_t e = e0 + r; e < e1; e += kBlock) s_prod[e - e0] = val[e] * x[col[e]];
        __syncthreads();
        double v[1] = {0.0};
        if (r < nr) {
            double acc = 0.0;
            for (int32_t q = s_rp[r] - e0; q < s_rp[r + 1] - e0; ++q) acc += s_prod[q];
            y[r0 + r] = acc;
            v[0] = x[r0 + r] * acc;
        }
        block_sum<1>(v);
        if (r == 0) tile_partial[tile] = v[0];
        __syncthreads();
    }
    __shared__ bool last;
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double s[1] = {0.0};
    for (int64_t t = threadIdx.x; t < ntiles; t += blockDim.x) s[0] += __ldcg(&tile_partial[t]);
    block_sum<1>(s);
    if (threadIdx.x == 0) {
        *xy = s[0];
        *ticket = 0u;
    }
}

void spmv_dot_f64(const Mesh& m, const double* vals, const double* x, double* y, double* xy, double* tile_partial,
                  uint32_t* ticket, cudaStream_t s) {
    const int64_t ntiles = (m.n + kBlock - 1) / kBlock;
    const size_t smem = (size_t)std::max(1, m.tile_cap) * sizeof(double);
    // The opt-in dynamic shared-memory size is a per-device attribute of the
    // kernel: it is set once per device (with that device current) and cached
    // under a lock, so concurrent first calls and later devices are covered.
    static std::mutex mu;
    static int rooms[256] = {0};
    int dev = 0;
    OASIS_CUDA(cudaGetDevice(&dev));
    OASIS_CHECK(dev >= 0 && dev < 256, OASIS_EINVAL, "device ordinal out of range");
    int room = 0;
    {
        std::lock_guard<std::mutex> lock(mu);
        if (!rooms[dev]) {
            int optin = 0;
            OASIS_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
            cudaFuncAttributes fa{};
            OASIS_CUDA(cudaFuncGetAttributes(&fa, k_spmv_dot_tiles));
            const int r = optin - (int)fa.sharedSizeBytes;
            OASIS_CUDA(cudaFuncSetAttribute(k_spmv_dot_tiles, cudaFuncAttributeMaxDynamicSharedMemorySize, r));
            rooms[dev] = r;
        }
        room = rooms[dev];
    }
    OASIS_CHECK(smem <= (size_t)room, OASIS_EINVAL, "a row tile needs more shared memory than the device offers");
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(ntiles, (int64_t)num_sms() * 4));
    OASIS_CUDA(cudaMemsetAsync(ticket, 0, sizeof(uint32_t), s));
    k_spmv_dot_tiles<<<grid, kBlock, smem, s>>>(m.n, m.row_ptr.p, m.col.p, vals, x, y, tile_partial, ticket, xy);
    OASIS_CUDA(cudaGetLastError());
}

// ------------------------------------------------------------------ no-alloc scratch
// Reduction scratch for oasis_spmv_dot_f64_noalloc, for callers that cannot
// allocate device memory (code running under a caller-owned memory pool or
// inside an allocator, or on a device that is already full).  Every GPU that
// loads the library holds these arrays until the process exits (516 KiB).
// One partial sum per 256-row tile: at most 65,536 tiles, i.e. 16,777,216 rows.
constexpr int64_t kNoAllocMaxTiles = 65536;
static __device__ __align__(256) double g_noalloc_partial[kNoAllocMaxTiles];
static __device__ __align__(256) uint32_t g_noalloc_ticket[64];

int64_t noalloc_max_rows() { return kNoAllocMaxTiles * kBlock; }

// Device addresses of the arrays above for the current device.  In host code
// the symbols are host-side stand-ins, not device addresses, so they are
// resolved with cudaGetSymbolAddress once per device (with that device
// current) and cached.
void noalloc_scratch(double** partial, uint32_t** ticket) {
    static std::mutex mu;
    static double* part[256] = {nullptr};
    static uint32_t* tick[256] = {nullptr};
    int dev = 0;
    OASIS_CUDA(cudaGetDevice(&dev));
    OASIS_CHECK(dev >= 0 && dev < 256, OASIS_EINVAL, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(mu);
    if (!part[dev]) {
        void* p = nullptr;
        void* t = nullptr;
        OASIS_CUDA(cudaGetSymbolAddress(&p, g_noalloc_partial));
        OASIS_CUDA(cudaGetSymbolAddress(&t, g_noalloc_ticket));
        part[dev] = static_cast<double*>(p);
        tick[dev] = static_cast<uint32_t*>(t);
    }
    *partial = part[dev];
    *ticket = tick[dev];
}

void spmv_f64(const Mesh& m, const double* vals, const double* x, double* y, int lanes, cudaStream_t s) {
    spmv_launch<double>(m, vals, x, y, lanes, s);
}
void spmv_f32(const Mesh& m, const float* vals, const float* x, float* y, int lanes, cudaStream_t s) {
    spmv_launch<float>(m, vals, x, y, lanes, s);
}

}  // namespace oasis
