// Smoothed-aggregation AMG for the pressure operator: host setup (once per
// mesh, from the assembled float64 K) and the V(1,1) cycle kernels.
#include <algorithm>
#include <map>
#include <mutex>
#include <chrono>
#include <cmath>
#include <cstring>
#include <thread>
#include <type_traits>
#include <vector>

#include <cuda_bf16.h>

#include "amg.cuh"
#include "solver.cuh"

namespace oasis {

namespace {

constexpr double kTheta = 0.08;        // strength threshold of the finest level (halved per level)
constexpr int64_t kMaxCoarse = 2048;   // dense coarsest level at or below this size
constexpr int kMaxLevels = 12;

// ------------------------------------------------------------------ host CSR
struct HCsr {
    int64_t n = 0, m = 0;              // rows, columns
    std::vector<int64_t> rp;
    std::vector<int32_t> ci;
    std::vector<double> v;
    int64_t nnz() const { return (int64_t)ci.size(); }
};

int host_threads() {
    const unsigned h = std::thread::hardware_concurrency();
    return (int)std::max(1u, std::min(h, 32u));
}

std::vector<double> diagonal(const HCsr& A) {
    std::vector<double> d(A.n, 0.0);
    for (int64_t i = 0; i < A.n; ++i)
        for (int64_t q = A.rp[i]; q < A.rp[i + 1]; ++q)
            if (A.ci[q] == i) d[i] += A.v[q];
    return d;
}

// Strong off-diagonal entries kept, weak ones added to the diagonal.  A row
// whose off-diagonals are all weak keeps its largest one (no isolated dofs).
HCsr filtered(const HCsr& A, const std::vector<double>& d, double theta) {
    HCsr F;
    F.n = A.n;
    F.m = A.m;
    F.rp.assign(A.n + 1, 0);
    F.ci.reserve(A.ci.size());
    F.v.reserve(A.v.size());
    for (int64_t i = 0; i < A.n; ++i) {
        double weak = 0.0;
        int64_t dpos = -1;
        int64_t qmax = -1;
        bool any = false;
        for (int64_t q = A.rp[i]; q < A.rp[i + 1]; ++q) {
            const int32_t j = A.ci[q];
            if (j == i) continue;
            if (qmax < 0 || std::fabs(A.v[q]) > std::fabs(A.v[qmax])) qmax = q;
            any |= std::fabs(A.v[q]) >= theta * std::sqrt(std::fabs(d[i] * d[j]));
        }
        for (int64_t q = A.rp[i]; q < A.rp[i + 1]; ++q) {
            const int32_t j = A.ci[q];
            if (j == i) {
                dpos = (int64_t)F.ci.size();
                F.ci.push_back(j);
                F.v.push_back(A.v[q]);
            } else if (std::fabs(A.v[q]) >= theta * std::sqrt(std::fabs(d[i] * d[j])) || (!any && q == qmax)) {
                F.ci.push_back(j);
                F.v.push_back(A.v[q]);
            } else {
                weak += A.v[q];
            }
        }
        if (dpos < 0) {
            dpos = (int64_t)F.ci.size();
            F.ci.push_back((int32_t)i);
            F.v.push_back(0.0);
        }
        F.v[dpos] += weak;
        F.rp[i + 1] = (int64_t)F.ci.size();
    }
    return F;
}

// rho(D^-1 A) by power iteration from a fixed start vector, with a 5 % margin.
double spectral_radius(const HCsr& A, const std::vector<double>& d) {
    std::vector<double> x(A.n), y(A.n);
    for (int64_t i = 0; i < A.n; ++i) x[i] = 1.0 + 0.5 * std::sin(0.7 * (double)i + 0.3 * (double)(i % 7));
    double lam = 1.0;
    for (int it = 0; it < 20; ++it) {
        double yy = 0.0, xx = 0.0;
        for (int64_t i = 0; i < A.n; ++i) {
            double s = 0.0;
            for (int64_t q = A.rp[i]; q < A.rp[i + 1]; ++q) s += A.v[q] * x[A.ci[q]];
            y[i] = d[i] != 0.0 ? s / d[i] : 0.0;
            yy += y[i] * y[i];
            xx += x[i] * x[i];
        }
        if (yy == 0.0) return 1.0;
        lam = std::sqrt(yy / xx);
        const double inv = 1.0 / std::sqrt(yy);
        for (int64_t i = 0; i < A.n; ++i) x[i] = y[i] * inv;
    }
    return 1.05 * lam;
}

// Greedy aggregation over the strong graph of F (every off-diagonal of F is strong).
std::vector<int32_t> aggregate(const HCsr& F, int64_t& nagg) {
    const int64_t n = F.n;
    std::vector<int32_t> agg(n, -1);
    nagg = 0;
    // 1: a root whose strong neighbours are all free takes them
    for (int64_t i = 0; i < n; ++i) {
        if (agg[i] >= 0) continue;
        bool free = true;
        for (int64_t q = F.rp[i]; q < F.rp[i + 1] && free; ++q)
            if (F.ci[q] != i && agg[F.ci[q]] >= 0) free = false;
        if (!free) continue;
        agg[i] = (int32_t)nagg;
        for (int64_t q = F.rp[i]; q < F.rp[i + 1]; ++q) agg[F.ci[q]] = (int32_t)nagg;
        ++nagg;
    }
    // 2: a free dof joins the first-phase aggregate it is most strongly tied to
    std::vector<int32_t> first = agg;
    for (int64_t i = 0; i < n; ++i) {
        if (agg[i] >= 0) continue;
        double best = -1.0;
        int32_t pick = -1;
        for (int64_t q = F.rp[i]; q < F.rp[i + 1]; ++q) {
            const int32_t j = F.ci[q];
            if (j != i && first[j] >= 0 && std::fabs(F.v[q]) > best) {
                best = std::fabs(F.v[q]);
                pick = first[j];
            }
        }
        agg[i] = pick;
    }
    // 3: what is left forms aggregates with its free strong neighbours
    for (int64_t i = 0; i < n; ++i) {
        if (agg[i] >= 0) continue;
        agg[i] = (int32_t)nagg;
        for (int64_t q = F.rp[i]; q < F.rp[i + 1]; ++q)
            if (agg[F.ci[q]] < 0) agg[F.ci[q]] = (int32_t)nagg;
        ++nagg;
    }
    return agg;
}

// P = (I - w D_F^-1 F) P_tent, P_tent[i][agg[i]] = 1.
HCsr smoothed_prolongator(const HCsr& F, const std::vector<int32_t>& agg, int64_t nagg, double w) {
    const std::vector<double> dF = diagonal(F);
    HCsr P;
    P.n = F.n;
    P.m = nagg;
    P.rp.assign(F.n + 1, 0);
    std::vector<std::pair<int32_t, double>> row;
    for (int64_t i = 0; i < F.n; ++i) {
        row.clear();
        row.emplace_back(agg[i], 1.0);
        const double s = dF[i] != 0.0 ? w / dF[i] : 0.0;
        for (int64_t q = F.rp[i]; q < F.rp[i + 1]; ++q) row.emplace_back(agg[F.ci[q]], -s * F.v[q]);
        std::sort(row.begin(), row.end(), [](const auto& a, const auto& b) { return a.first < b.first; });
        for (size_t k = 0; k < row.size();) {
            const int32_t c = row[k].first;
            double v = 0.0;
            while (k < row.size() && row[k].first == c) v += row[k++].second;
            P.ci.push_back(c);
            P.v.push_back(v);
        }
        P.rp[i + 1] = (int64_t)P.ci.size();
    }
    return P;
}

HCsr transpose(const HCsr& P) {
    HCsr R;
    R.n = P.m;
    R.m = P.n;
    R.rp.assign(P.m + 1, 0);
    for (int32_t c : P.ci) R.rp[c + 1]++;
    for (int64_t k = 0; k < P.m; ++k) R.rp[k + 1] += R.rp[k];
    R.ci.resize(P.ci.size());
    R.v.resize(P.v.size());
    std::vector<int64_t> pos(R.rp.begin(), R.rp.end() - 1);
    for (int64_t i = 0; i < P.n; ++i)
        for (int64_t q = P.rp[i]; q < P.rp[i + 1]; ++q) {
            const int64_t o = pos[P.ci[q]]++;
            R.ci[o] = (int32_t)i;
            R.v[o] = P.v[q];
        }
    return R;
}

// C = A B, row by row with a dense accumulator per thread; columns sorted.
HCsr spgemm(const HCsr& A, const HCsr& B) {
    const int64_t n = A.n;
    const int T = (int)std::min<int64_t>(host_threads(), std::max<int64_t>(1, n / 4096));
    std::vector<std::vector<int32_t>> cis(T);
    std::vector<std::vector<double>> vs(T);
    std::vector<int64_t> cnt(n, 0);
    std::vector<std::thread> th;
    auto work = [&](int t) {
        const int64_t lo = n * t / T, hi = n * (t + 1) / T;
        std::vector<double> acc(B.m, 0.0);
        std::vector<char> mark(B.m, 0);
        std::vector<int32_t> cols;
        for (int64_t i = lo; i < hi; ++i) {
            cols.clear();
            for (int64_t q = A.rp[i]; q < A.rp[i + 1]; ++q) {
                const int32_t k = A.ci[q];
                const double a = A.v[q];
                for (int64_t r = B.rp[k]; r < B.rp[k + 1]; ++r) {
                    const int32_t c = B.ci[r];
                    if (!mark[c]) {
                        mark[c] = 1;
                        cols.push_back(c);
                    }
                    acc[c] += a * B.v[r];
                }
            }
            std::sort(cols.begin(), cols.end());
            for (int32_t c : cols) {
                cis[t].push_back(c);
                vs[t].push_back(acc[c]);
                acc[c] = 0.0;
                mark[c] = 0;
            }
            cnt[i] = (int64_t)cols.size();
        }
    };
    if (T <= 1) {
        work(0);
    } else {
        for (int t = 0; t < T; ++t) th.emplace_back(work, t);
        for (auto& x : th) x.join();
    }
    HCsr C;
    C.n = n;
    C.m = B.m;
    C.rp.assign(n + 1, 0);
    for (int64_t i = 0; i < n; ++i) C.rp[i + 1] = C.rp[i] + cnt[i];
    C.ci.reserve(C.rp[n]);
    C.v.reserve(C.rp[n]);
    for (int t = 0; t < T; ++t) {
        C.ci.insert(C.ci.end(), cis[t].begin(), cis[t].end());
        C.v.insert(C.v.end(), vs[t].begin(), vs[t].end());
    }
    return C;
}

// Dense inverse of A + sigma 1 1^T (Cholesky; A symmetric positive semi-definite
// with null space 1), row-major.
std::vector<double> coarse_inverse(const HCsr& A) {
    const int64_t n = A.n;
    std::vector<double> M((size_t)n * n, 0.0);
    double tr = 0.0;
    for (int64_t i = 0; i < n; ++i)
        for (int64_t q = A.rp[i]; q < A.rp[i + 1]; ++q) {
            M[(size_t)i * n + A.ci[q]] += A.v[q];
            if (A.ci[q] == i) tr += A.v[q];
        }
    const double sigma = tr / ((double)n * (double)n);
    for (auto& x : M) x += sigma;
    // Cholesky M = L L^T in place (lower triangle)
    for (int64_t j = 0; j < n; ++j) {
        double s = M[(size_t)j * n + j];
        for (int64_t k = 0; k < j; ++k) s -= M[(size_t)j * n + k] * M[(size_t)j * n + k];
        OASIS_CHECK(s > 0.0, OASIS_EINVAL, "multigrid: coarsest operator is not positive on the complement of 1");
        const double l = std::sqrt(s);
        M[(size_t)j * n + j] = l;
        auto rows = [&](int64_t i0, int64_t i1) {
            for (int64_t i = i0; i < i1; ++i) {
                double t = M[(size_t)i * n + j];
                for (int64_t k = 0; k < j; ++k) t -= M[(size_t)i * n + k] * M[(size_t)j * n + k];
                M[(size_t)i * n + j] = t / l;
            }
        };
        const int64_t rem = n - (j + 1);
        const int T = (int)std::min<int64_t>(host_threads(), std::max<int64_t>(1, rem * j / 2000000));
        if (T <= 1) {
            rows(j + 1, n);
        } else {
            std::vector<std::thread> th;
            for (int t = 0; t < T; ++t) th.emplace_back(rows, j + 1 + rem * t / T, j + 1 + rem * (t + 1) / T);
            for (auto& x : th) x.join();
        }
    }
    // inverse column by column (columns split over the host cores): solve
    // L y = e_c, then L^T x = y
    std::vector<double> inv((size_t)n * n, 0.0);
    auto cols = [&](int64_t c0, int64_t c1) {
        std::vector<double> y(n), x(n);
        for (int64_t c = c0; c < c1; ++c) {
            for (int64_t i = 0; i < n; ++i) {
                double t = (i == c) ? 1.0 : 0.0;
                for (int64_t k = 0; k < i; ++k) t -= M[(size_t)i * n + k] * y[k];
                y[i] = t / M[(size_t)i * n + i];
            }
            for (int64_t i = n - 1; i >= 0; --i) {
                double t = y[i];
                for (int64_t k = i + 1; k < n; ++k) t -= M[(size_t)k * n + i] * x[k];
                x[i] = t / M[(size_t)i * n + i];
            }
            for (int64_t i = 0; i < n; ++i) inv[(size_t)i * n + c] = x[i];
        }
    };
    const int T = (int)std::min<int64_t>(host_threads(), std::max<int64_t>(1, n / 64));
    std::vector<std::thread> th;
    for (int t = 0; t < T; ++t) th.emplace_back(cols, n * t / T, n * (t + 1) / T);
    for (auto& x : th) x.join();
    return inv;
}

template <class T>
void upload_vec(DBuf<T>& dst, const std::vector<T>& src, cudaStream_t s) {
    dst.upload(src.data(), src.size(), s);
}

// bfloat16 bit pattern of a finite float, rounded to nearest even: add half a
// unit of the 16 dropped bits (less one when the kept part is even) and drop them
uint16_t bf16_bits(float f) {
    uint32_t u;
    std::memcpy(&u, &f, 4);
    u += 0x7FFFu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}

void upload_csr(DBuf<int32_t>& rp, DBuf<int32_t>& ci, DBuf<double>& v64, DBuf<uint16_t>& v16, const HCsr& A,
                cudaStream_t s) {
    OASIS_CHECK(A.nnz() < INT32_MAX, OASIS_EINVAL, "multigrid: level too large for int32 indices");
    std::vector<int32_t> r32(A.rp.size());
    for (size_t k = 0; k < A.rp.size(); ++k) r32[k] = (int32_t)A.rp[k];
    std::vector<uint16_t> b(A.v.size());
    for (size_t k = 0; k < A.v.size(); ++k) b[k] = bf16_bits((float)A.v[k]);
    upload_vec(rp, r32, s);
    upload_vec(ci, A.ci, s);
    upload_vec(v64, A.v, s);
    upload_vec(v16, b, s);
    OASIS_CUDA(cudaStreamSynchronize(s));
}

// Pair-packed SELL-32 copy of A for the float32 cycle (layout in amg.cuh), if A
// has at least kSellMinRows rows; otherwise `out` stays empty.  The copy is wide
// (32-bit columns) if some slice's columns span 2^16 values or more.  Entries
// keep their CSR order within a row, so a row's products are added in the same
// order as in CSR.
void build_sellp(const HCsr& A, AmgSellP& out, cudaStream_t s) {
    if (A.n < kSellMinRows) return;
    const int64_t ns = (A.n + 31) / 32;
    std::vector<int4> hdr(ns);
    int64_t words = 0;
    bool wide = false;
    for (int64_t sl = 0; sl < ns; ++sl) {
        int64_t maxlen = 0;
        int32_t lo = INT32_MAX, hi = -1;
        for (int64_t i = sl * 32; i < std::min<int64_t>(A.n, sl * 32 + 32); ++i) {
            maxlen = std::max<int64_t>(maxlen, A.rp[i + 1] - A.rp[i]);
            for (int64_t q = A.rp[i]; q < A.rp[i + 1]; ++q) {
                lo = std::min(lo, A.ci[q]);
                hi = std::max(hi, A.ci[q]);
            }
        }
        if (hi < 0) lo = hi = 0;
        wide |= (int64_t)hi - (int64_t)lo > 65535;
        const int64_t w = (maxlen + 1) / 2;
        hdr[sl] = make_int4((int)words, (int)w, lo, 0);
        words += 32 * w;
        if (words >= INT32_MAX) return;
    }
    if (wide)
        for (auto& h : hdr) h.z = 0;
    const size_t nw = (size_t)std::max<int64_t>(words, 1);
    std::vector<uint32_t> vp(nw, 0u), cp(wide ? 0 : nw, 0u);
    std::vector<uint2> cw(wide ? nw : 0, make_uint2(0u, 0u));
    double mean_w = 0.0;
    for (int64_t sl = 0; sl < ns; ++sl) {
        mean_w += hdr[sl].y;
        for (int l = 0; l < 32; ++l) {
            const int64_t i = sl * 32 + l;
            if (i >= A.n) break;
            for (int64_t k = 0; k < A.rp[i + 1] - A.rp[i]; ++k) {
                const int64_t q = A.rp[i] + k;
                const size_t o = (size_t)hdr[sl].x + 32 * (size_t)(k >> 1) + (size_t)l;
                const int sh = (int)(k & 1) * 16;
                vp[o] |= (uint32_t)bf16_bits((float)A.v[q]) << sh;
                if (wide)
                    ((k & 1) ? cw[o].y : cw[o].x) = (uint32_t)A.ci[q];
                else
                    cp[o] |= (uint32_t)(A.ci[q] - hdr[sl].z) << sh;
            }
        }
    }
    mean_w /= (double)ns;
    upload_vec(out.hdr, hdr, s);
    upload_vec(out.vp, vp, s);
    if (wide) upload_vec(out.cw, cw, s);
    else upload_vec(out.cp, cp, s);
    OASIS_CUDA(cudaStreamSynchronize(s));
    out.n = A.n;
    out.n_slices = ns;
    out.wide = wide;
    // warps per slice: enough slices x warps to fill ~2 resident waves (64 warps
    // per SM), while every warp keeps at least one full round of C2 = 4 words
    int sp = 1;
    while (sp < 4 && (double)ns * sp < 2.0 * num_sms() * 64 && mean_w >= 4.0 * 2 * sp) sp *= 2;
    out.sp = sp;
    out.c2 = sp > 1 ? 4 : (mean_w >= 12.0 ? 8 : 4);
}

// bfloat16 bit patterns of float values, round to nearest even
__global__ void k_round_bf16(int64_t n, const float* __restrict__ in, uint16_t* __restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = __bfloat16_as_ushort(__float2bfloat16_rn(in[i]));
}

// Pair-packed copy of the finest level's bfloat16 values and 16-bit column
// offsets (layout in amg.cuh).  One thread per (slice, lane); the padding entry
// of an odd-length slice takes value 0 and the lane's previous offset, so its
// gathered operand is a valid row.
__global__ void k_pack_pairs(int64_t n_slices, const int32_t* __restrict__ ptr, const int32_t* __restrict__ len,
                             const int32_t* __restrict__ ptr2, const uint16_t* __restrict__ v16,
                             const float* __restrict__ v32, const int16_t* __restrict__ dcol,
                             uint16_t* __restrict__ vp, uint16_t* __restrict__ cp, float* __restrict__ kp) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n_slices * 32;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t sl = t >> 5;
        const int l = (int)(t & 31), ln = len[sl], lp = (ln + 1) & ~1;
        uint16_t c = 0;
        for (int k = 0; k < lp; ++k) {
            uint16_t v = 0;
            float f = 0.f;
            if (k < ln) {
                const int64_t q = (int64_t)ptr[sl] + 32 * (int64_t)k + l;
                v = v16[q];
                f = v32[q];
                c = (uint16_t)dcol[q];
            }
            const int64_t o = (int64_t)ptr2[sl] + 64 * (int64_t)(k >> 1) + 2 * l + (k & 1);
            vp[o] = v;
            cp[o] = c;
            kp[o] = f;
        }
    }
}

void pack_pairs(AmgHierarchy& h, const Mesh& m, cudaStream_t s) {
    const int64_t ns = h.fine.n_slices;
    std::vector<int32_t> len(ns), ptr2(ns);
    OASIS_CUDA(cudaMemcpyAsync(len.data(), m.sell_len.p, ns * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    OASIS_CUDA(cudaStreamSynchronize(s));
    int64_t total = 0;
    for (int64_t sl = 0; sl < ns; ++sl) {
        ptr2[sl] = (int32_t)total;
        total += 32 * (int64_t)((len[sl] + 1) & ~1);
        OASIS_CHECK(total < INT32_MAX, OASIS_EINVAL, "multigrid: finest level too large for int32 positions");
    }
    upload_vec(h.fine_ptr2, ptr2, s);
    h.fine_vp.alloc((size_t)std::max<int64_t>(total / 2, 1));
    h.fine_cp.alloc((size_t)std::max<int64_t>(total / 2, 1));
    h.fine_kp.alloc((size_t)std::max<int64_t>(total / 2, 1));
    k_pack_pairs<<<(int)std::max<int64_t>(1, std::min<int64_t>((ns * 32 + kBlock - 1) / kBlock, 4096)), kBlock, 0, s>>>(
        ns, m.sell_ptr.p, m.sell_len.p, h.fine_ptr2.p, h.fine16.p, m.K32s.p, m.sell_dcol.p,
        reinterpret_cast<uint16_t*>(h.fine_vp.p), reinterpret_cast<uint16_t*>(h.fine_cp.p),
        reinterpret_cast<float*>(h.fine_kp.p));
    OASIS_CUDA(cudaGetLastError());
    OASIS_CUDA(cudaStreamSynchronize(s));
    h.fine.ptr2 = h.fine_ptr2.p;
    h.fine.vp = h.fine_vp.p;
    h.fine.cp = h.fine_cp.p;
    h.fine.kp = h.fine_kp.p;
}

}  // namespace

void amg_build(Mesh& m, cudaStream_t s) {
    if (m.amg) return;
    OASIS_CHECK(m.assembled, OASIS_EINVAL, "mesh not assembled");
    OASIS_CHECK(m.sell_ptr.p && m.K32s.p, OASIS_EINVAL, "multigrid: the mesh has no SELL-32 copy of K");
    const auto t0 = std::chrono::steady_clock::now();
    auto h = std::make_shared<AmgHierarchy>();
    HCsr A;
    A.n = A.m = m.n;
    A.rp.assign(m.h_row_ptr.begin(), m.h_row_ptr.end());
    A.ci = m.h_col;
    A.ci.resize(m.nnz);
    A.v.resize(m.nnz);
    OASIS_CUDA(cudaMemcpyAsync(A.v.data(), m.K64.p, m.nnz * sizeof(double), cudaMemcpyDeviceToHost, s));
    OASIS_CUDA(cudaStreamSynchronize(s));
    while (true) {
        auto L = std::make_unique<AmgLevelDev>();
        L->n = A.n;
        L->nnz = A.nnz();
        const std::vector<double> d = diagonal(A);
        std::vector<double> dinv(A.n);
        for (int64_t i = 0; i < A.n; ++i) dinv[i] = d[i] != 0.0 ? 1.0 / d[i] : 0.0;
        std::vector<float> dinv32(dinv.begin(), dinv.end());
        upload_vec(L->d64, dinv, s);
        upload_vec(L->d32, dinv32, s);
        L->omega = 4.0 / (3.0 * spectral_radius(A, d));
        if (h->lv.empty()) {
            h->fine.n = m.n;
            h->fine.n_slices = (m.n + 31) / 32;
            h->fine.ptr = m.sell_ptr.p;
            h->fine.len = m.sell_len.p;
            h->fine.col = m.sell_col.p;
            h->fine.dcol = m.sell_dcol.p;
            h->fine.v64 = m.K64s.p;
            h->fine16.alloc(m.n_sell);
            k_round_bf16<<<(int)std::max<int64_t>(1, std::min<int64_t>((m.n_sell + kBlock - 1) / kBlock, 4096)), kBlock, 0, s>>>(
                m.n_sell, m.K32s.p, h->fine16.p);
            OASIS_CUDA(cudaGetLastError());
            h->fine.v16 = h->fine16.p;
            if (m.sell_dcol.p) pack_pairs(*h, m, s);
            L->rp = m.row_ptr.p;
            L->ci = m.col.p;
            L->a64 = m.K64.p;
        } else {
            upload_csr(L->own_rp, L->own_ci, L->own_a64, L->own_a16, A, s);
            L->rp = L->own_rp.p;
            L->ci = L->own_ci.p;
            L->a64 = L->own_a64.p;
            L->a16 = L->own_a16.p;
            build_sellp(A, L->sa, s);
        }
        h->sizes.push_back(A.n);
        h->nnzs.push_back(A.nnz());
        // coarsen; a level that barely shrinks is aggregated again with every
        // connection strong
        const double theta = kTheta * std::pow(0.5, (double)h->lv.size());
        HCsr F = filtered(A, d, theta);
        int64_t nagg = 0;
        std::vector<int32_t> agg = aggregate(F, nagg);
        if ((double)nagg > 0.6 * (double)A.n) {
            F = filtered(A, d, 0.0);
            agg = aggregate(F, nagg);
        }
        const double wP = 4.0 / (3.0 * spectral_radius(F, diagonal(F)));
        const HCsr P = smoothed_prolongator(F, agg, nagg, wP);
        const HCsr R = transpose(P);
        h->pnnzs.push_back(P.nnz());
        upload_csr(L->p_rp, L->p_ci, L->p64, L->p16, P, s);
        upload_csr(L->r_rp, L->r_ci, L->r64, L->r16, R, s);
        build_sellp(R, L->sr, s);
        build_sellp(P, L->sp, s);
        auto lanes = [](int64_t nnz, int64_t rows) {
            const double mean = rows ? (double)nnz / (double)rows : 1.0;
            int g = 4;
            while (g < 32 && g * 4 < mean) g *= 2;
            return g;
        };
        L->g_a = lanes(A.nnz(), A.n);
        L->g_r = lanes(R.nnz(), R.n);
        L->g_p = lanes(P.nnz(), P.n);
        h->lv.push_back(std::move(L));
        HCsr Ac = spgemm(R, spgemm(A, P));
        A = std::move(Ac);
        const bool small = A.n <= kMaxCoarse;
        const bool stalled = (double)A.n > 0.8 * (double)h->sizes.back();
        if (small || stalled || (int)h->lv.size() >= kMaxLevels) break;
    }
    OASIS_CHECK(A.n <= 2 * kMaxCoarse, OASIS_EINVAL, "multigrid: coarsening stalled above the dense size");
    h->nc = A.n;
    h->sizes.push_back(A.n);
    h->nnzs.push_back(A.nnz());
    const std::vector<double> inv = coarse_inverse(A);
    // rows padded to a multiple of 4 entries (16-byte vector loads)
    h->ld = (A.n + 3) / 4 * 4;
    std::vector<double> inv_ld((size_t)A.n * h->ld, 0.0);
    for (int64_t i = 0; i < A.n; ++i)
        for (int64_t c = 0; c < A.n; ++c) inv_ld[(size_t)i * h->ld + c] = inv[(size_t)i * A.n + c];
    std::vector<float> inv32(inv_ld.begin(), inv_ld.end());
    upload_vec(h->inv64, inv_ld, s);
    upload_vec(h->inv32, inv32, s);
    OASIS_CUDA(cudaStreamSynchronize(s));
    h->setup_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    m.amg = std::move(h);
}

void AmgWork::alloc(const AmgHierarchy& h, size_t vbytes) {
    const size_t L = h.lv.size();
    x.resize(L + 1);
    xo.resize(L + 1);
    res.resize(L + 1);
    rin.resize(L + 1);
    for (size_t l = 0; l <= L; ++l) {
        // the dense level's input is read with vector loads up to ld: zero padding
        const int64_t n = l < L ? h.lv[l]->n : h.ld;
        const size_t cnt = ((size_t)n * vbytes + 7) / 8;
        x[l].alloc(cnt);
        xo[l].alloc(cnt);
        res[l].alloc(cnt);
        rin[l].alloc(cnt);
        if (l == L) OASIS_CUDA(cudaMemset(rin[l].p, 0, rin[l].bytes()));
    }
}

// ------------------------------------------------------------------ kernels
namespace {

__device__ __forceinline__ bool amg_done(const KrylovState* st) { return st->col_done[0] || st->in_done[0]; }

template <int G, class V>
__device__ __forceinline__ V group_sum(V v) {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// CSR row kernels of the coarser levels and the transfers.  Rows are served by
// groups of G lanes (G divides 32); every group keeps U rows in flight: the row
// pointers of its U rows are loaded together, then per round one entry of each
// unfinished row (value, column, then the gathered operand), so that a warp has
// U independent load chains where one row at a time would wait on each chain in
// turn.  Lane lg of a group adds the entries lg, lg + G, ... of its row in that
// order and the group sums the lanes with a fixed shuffle tree, whatever U is.
// The batch loop is uniform across the warp (all shuffles have the full warp).
enum AmgRowMode { kRowPre = 0, kRowPost = 1, kRowProlong = 2, kRowRestrict = 3 };

// Values as stored for the cycle of value type V: float64 for the float64
// cycle; bfloat16 bit patterns (uint16_t) for the float32 one, widened by a
// shift on load (measured at 128^3: 100.6 steps/s against 98.1 with float32
// values, the same CG iterations).
template <class V>
using StoredT = typename std::conditional<sizeof(V) == 8, double, uint16_t>::type;
__device__ __forceinline__ float stored_value(uint16_t b) { return __uint_as_float((uint32_t)b << 16); }
__device__ __forceinline__ double stored_value(double v) { return v; }
template <class V>
const StoredT<V>* stored(const uint16_t* b, const double* d) {
    if constexpr (sizeof(V) == 8) return d;
    else return b;
}

template <class V, class AV>
struct AmgRowArgs {
    int64_t n;
    const int32_t* __restrict__ rp;
    const int32_t* __restrict__ ci;
    const AV* __restrict__ a;
    const V* __restrict__ d;     // 1 / a_ii (smoothing)
    V w;                         // Jacobi weight (smoothing)
    const V* __restrict__ r;     // right-hand side of the level (smoothing)
    const V* __restrict__ x;     // post: the iterate
    const V* __restrict__ v;     // transfers: the vector multiplied
    V* __restrict__ out;         // pre: x; post: the smoothed iterate; transfers: y
    V* __restrict__ res;         // pre: the residual
    const KrylovState* st;
};

// MODE kRowPre:      x = w D^-1 r, res = r - A x (smoothing from zero; the gathered
//                    operand is w d_j r_j);
//      kRowPost:     out = x + w D^-1 (r - A x);
//      kRowProlong:  out += P v;
//      kRowRestrict: out = R v.
template <class V, class AV, int G, int U, int MODE>
__device__ __forceinline__ void amg_rows(const AmgRowArgs<V, AV>& p) {
    if (amg_done(p.st)) return;
    constexpr int RPW = 32 / G;
    const int lane = threadIdx.x & 31, lg = lane & (G - 1), grp = lane / G;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t base = w0 * RPW * U; base < p.n; base += nw * RPW * U) {
        int64_t i[U];
        int32_t q[U], e[U];
        V sum[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            i[u] = base + u * RPW + grp;
            const bool ok = i[u] < p.n;
            q[u] = ok ? p.rp[i[u]] + lg : 0;
            e[u] = ok ? p.rp[i[u] + 1] : 0;
            sum[u] = 0;
        }
        bool more = false;
#pragma unroll
        for (int u = 0; u < U; ++u) more |= q[u] < e[u];
        while (more) {
            int32_t j[U];
            V av[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const bool has = q[u] < e[u];
                j[u] = has ? p.ci[q[u]] : 0;
                av[u] = has ? (V)stored_value(p.a[q[u]]) : V(0);
            }
            V g[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if constexpr (MODE == kRowPre) g[u] = p.w * p.d[j[u]] * p.r[j[u]];
                else if constexpr (MODE == kRowPost) g[u] = p.x[j[u]];
                else g[u] = p.v[j[u]];
            }
            more = false;
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (q[u] < e[u]) {
                    sum[u] += av[u] * g[u];
                    q[u] += G;
                }
                more |= q[u] < e[u];
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const V t = group_sum<G>(sum[u]);
            if (i[u] < p.n && lg == 0) {
                const int64_t ii = i[u];
                if constexpr (MODE == kRowPre) {
                    p.res[ii] = p.r[ii] - t;
                    p.out[ii] = p.w * p.d[ii] * p.r[ii];
                } else if constexpr (MODE == kRowPost) {
                    p.out[ii] = p.x[ii] + p.w * p.d[ii] * (p.r[ii] - t);
                } else if constexpr (MODE == kRowProlong) {
                    p.out[ii] = p.out[ii] + t;
                } else {
                    p.out[ii] = t;
                }
            }
        }
    }
}

// rows in flight per lane group: more for short rows (few entries per lane)
template <int G>
constexpr int amg_rows_u() {
    return G <= 8 ? 4 : 2;
}

template <class V, class AV, int G>
__global__ void __launch_bounds__(kBlock) k_amg_pre(AmgRowArgs<V, AV> p) {
    amg_rows<V, AV, G, amg_rows_u<G>(), kRowPre>(p);
}
template <class V, class AV, int G>
__global__ void __launch_bounds__(kBlock) k_amg_post(AmgRowArgs<V, AV> p) {
    amg_rows<V, AV, G, amg_rows_u<G>(), kRowPost>(p);
}
template <class V, class AV, int G>
__global__ void __launch_bounds__(kBlock) k_amg_restrict(AmgRowArgs<V, AV> p) {
    amg_rows<V, AV, G, amg_rows_u<G>(), kRowRestrict>(p);
}
template <class V, class AV, int G>
__global__ void __launch_bounds__(kBlock) k_amg_prolong(AmgRowArgs<V, AV> p) {
    amg_rows<V, AV, G, amg_rows_u<G>(), kRowProlong>(p);
}

// Finest level on SELL-32: one warp per slice of 32 rows, lane l owns row
// 32 s + l; entry k of the row sits at ptr[s] + 32 k + l (padding: a valid
// column and a zero value).  Four entries per lane have their column and value
// loads issued together, then their gathers; products are added in entry order.
template <bool D16>
__device__ __forceinline__ int32_t fine_col(const AmgSellView& F, int64_t q, int32_t row) {
    if constexpr (D16) {
        int32_t j = row + (int32_t)F.dcol[q];
        const int32_t n = (int32_t)F.n;
        j = j < 0 ? j + n : j;
        return j >= n ? j - n : j;
    } else {
        return F.col[q];
    }
}

// PRE: x = w D^-1 r and res = r - A x (smoothing from zero); else
// out = x + w D^-1 (r - A x).  The gathered operand is w d_j r_j (PRE) or x_j.
// (Two slices per warp in flight were measured slower at 128^3: 61 against
// 47 us per sweep, the extra registers costing more resident warps than the
// second chain gains.)
// AV is the stored value type (StoredT).

template <class V, class AV, bool D16, bool PRE>
__global__ void __launch_bounds__(kBlock) k_amg_fine(AmgSellView F, const AV* __restrict__ av,
                                                     const V* __restrict__ d, V w, const V* __restrict__ r,
                                                     const V* __restrict__ x, V* __restrict__ out,
                                                     V* __restrict__ res, const KrylovState* st) {
    if (amg_done(st)) return;
    constexpr int C = 4;
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t sl = w0; sl < F.n_slices; sl += nw) {
        const int64_t i = sl * 32 + lane;
        const int32_t row = (int32_t)i;
        const int len = F.len[sl];
        const int64_t base = (int64_t)F.ptr[sl] + lane;
        V s = 0;
        for (int k = 0; k < len; k += C) {
            int32_t j[C];
            V kv[C];
#pragma unroll
            for (int u = 0; u < C; ++u) {
                const int64_t q = base + 32 * (int64_t)(k + u);
                const bool ok = k + u < len;
                j[u] = ok ? fine_col<D16>(F, q, row) : 0;
                kv[u] = ok ? (V)stored_value(av[q]) : V(0);
            }
            V g[C];
#pragma unroll
            for (int u = 0; u < C; ++u) g[u] = PRE ? w * d[j[u]] * r[j[u]] : x[j[u]];
#pragma unroll
            for (int u = 0; u < C; ++u)
                if (k + u < len) s += kv[u] * g[u];
        }
        if (i < F.n) {
            if constexpr (PRE) {
                res[i] = r[i] - s;
                out[i] = w * d[i] * r[i];
            } else {
                out[i] = x[i] + w * d[i] * (r[i] - s);
            }
        }
    }
}

// The float32 sweep on the pair-packed copy: per round C2 words of values and
// C2 of offsets (2 C2 entries) are loaded, then their 2 C2 gathers; products
// are added in entry order, as in k_amg_fine (same bits: the padding entry
// adds 0 times a valid operand).
constexpr int kFinePairWords = 4;
template <bool PRE, int C2>
__global__ void __launch_bounds__(kBlock) k_amg_fine_pairs(AmgSellView F, const float* __restrict__ d, float w,
                                                           const float* __restrict__ r, const float* __restrict__ x,
                                                           float* __restrict__ out, float* __restrict__ res,
                                                           const KrylovState* st) {
    if (amg_done(st)) return;
    const uint32_t* __restrict__ vp = F.vp;
    const uint32_t* __restrict__ cp = F.cp;
    const int32_t n32 = (int32_t)F.n;
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t sl = w0; sl < F.n_slices; sl += nw) {
        const int64_t i = sl * 32 + lane;
        const int32_t row = (int32_t)i;
        const int words = (F.len[sl] + 1) >> 1;
        // 32-bit word offsets (the copy holds fewer than 2^31 entries)
        const uint32_t base = (uint32_t)(F.ptr2[sl] >> 1) + (uint32_t)lane;
        float sum = 0.f;
        for (int k = 0; k < words; k += C2) {
            uint32_t vw[C2], cw[C2];
#pragma unroll
            for (int u = 0; u < C2; ++u) {
                const uint32_t q = base + 32u * (uint32_t)(k + u);
                const bool ok = k + u < words;
                vw[u] = ok ? vp[q] : 0u;
                cw[u] = ok ? cp[q] : 0u;
            }
            float g[2 * C2];
#pragma unroll
            for (int e = 0; e < 2 * C2; ++e) {
                const uint32_t half = (e & 1) ? (cw[e >> 1] >> 16) : (cw[e >> 1] & 0xFFFFu);
                int32_t j = row + (int32_t)(int16_t)half;
                j = j < 0 ? j + n32 : j;
                j = j >= n32 ? j - n32 : j;
                g[e] = PRE ? w * d[j] * r[j] : x[j];
            }
#pragma unroll
            for (int u = 0; u < C2; ++u)
                if (k + u < words) {
                    sum += __uint_as_float(vw[u] << 16) * g[2 * u];
                    sum += __uint_as_float(vw[u] & 0xFFFF0000u) * g[2 * u + 1];
                }
        }
        if (i < F.n) {
            if constexpr (PRE) {
                res[i] = r[i] - sum;
                out[i] = w * d[i] * r[i];
            } else {
                out[i] = x[i] + w * d[i] * (r[i] - sum);
            }
        }
    }
}

// A pair-packed SELL-32 operator of the float32 cycle (AmgSellP) as the kernels
// see it.
struct SellPView {
    int64_t n, n_slices;
    const int4* __restrict__ hdr;
    const uint32_t* __restrict__ vp;
    const uint32_t* __restrict__ cp;
    const uint2* __restrict__ cw;
};

// Row kernels of the float32 cycle on a pair-packed SELL-32 operator, the modes
// of amg_rows (pre: x = w D^-1 r, res = r - A x; post: out = src + w D^-1 (r - A src);
// prolong: out += P src; restrict: out = R src).  SP warps serve one slice: warp
// p of the slice takes the rounds p, p + SP, ... of C2 words each; per round it
// loads C2 words of values and C2 of offsets (W: C2 pairs of whole columns) per
// lane (2 C2 entries), then their 2 C2 gathers, and adds the products in entry
// order.  With SP > 1 the partial sums meet in shared memory and the slice's
// first warp adds them in warp order.  (A level of 250k rows is only ~7,800
// slices: one warp per slice leaves half the SM's warp slots empty and every
// warp a long chain of dependent loads.)
template <int MODE, int C2, bool W, int SP>
__global__ void __launch_bounds__(kBlock) k_amg_sellp(SellPView S, const float* __restrict__ d, float w,
                                                      const float* __restrict__ r, const float* __restrict__ src,
                                                      float* __restrict__ out, float* __restrict__ res,
                                                      const KrylovState* st) {
    if (amg_done(st)) return;
    constexpr int kWarps = kBlock / 32, kSlices = kWarps / SP;
    static_assert(kWarps % SP == 0, "warps per slice must divide the block's warps");
    __shared__ float part[SP > 1 ? kWarps : 1][32];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int sub = wib % SP, ls = wib / SP;
    const int64_t groups = (S.n_slices + kSlices - 1) / kSlices;
    for (int64_t gi = blockIdx.x; gi < groups; gi += gridDim.x) {     // uniform over the block
        const int64_t sl = gi * kSlices + ls;
        float sum = 0.f;
        if (sl < S.n_slices) {
            const int4 h = S.hdr[sl];
            const uint32_t base = (uint32_t)h.x + (uint32_t)lane;
            for (int k = sub * C2; k < h.y; k += SP * C2) {
                uint32_t vw[C2];
                uint2 cw[C2];
#pragma unroll
                for (int u = 0; u < C2; ++u) {
                    const uint32_t q = base + 32u * (uint32_t)(k + u);
                    const bool ok = k + u < h.y;
                    vw[u] = ok ? S.vp[q] : 0u;
                    if constexpr (W) {
                        cw[u] = ok ? S.cw[q] : make_uint2(0u, 0u);
                    } else {
                        const uint32_t c = ok ? S.cp[q] : 0u;
                        cw[u] = make_uint2(c & 0xFFFFu, c >> 16);
                    }
                }
                float g[2 * C2];
#pragma unroll
                for (int e = 0; e < 2 * C2; ++e) {
                    const int32_t j = h.z + (int32_t)((e & 1) ? cw[e >> 1].y : cw[e >> 1].x);
                    if constexpr (MODE == kRowPre) g[e] = w * d[j] * r[j];
                    else g[e] = src[j];
                }
#pragma unroll
                for (int u = 0; u < C2; ++u)
                    if (k + u < h.y) {
                        sum += __uint_as_float(vw[u] << 16) * g[2 * u];
                        sum += __uint_as_float(vw[u] & 0xFFFF0000u) * g[2 * u + 1];
                    }
            }
        }
        if constexpr (SP > 1) {
            part[wib][lane] = sum;
            __syncthreads();
            if (sub == 0) {
                sum = part[wib][lane];
#pragma unroll
                for (int p = 1; p < SP; ++p) sum += part[wib + p][lane];
            }
            __syncthreads();
        }
        const int64_t i = sl * 32 + lane;
        if (sub == 0 && sl < S.n_slices && i < S.n) {
            if constexpr (MODE == kRowPre) {
                res[i] = r[i] - sum;
                out[i] = w * d[i] * r[i];
            } else if constexpr (MODE == kRowPost) {
                out[i] = src[i] + w * d[i] * (r[i] - sum);
            } else if constexpr (MODE == kRowProlong) {
                out[i] = out[i] + sum;
            } else {
                out[i] = sum;
            }
        }
    }
}

// coarsest level: x = inv r with inv dense and row-major, leading dimension ld
// (a multiple of 4, zero-padded) and r zero-padded to ld; one block of 128
// threads per row, 16-byte loads (float4 / double2), the block's sum in a fixed
// order.
__device__ __forceinline__ float dot_vec(const float4& a, const float4& b) {
    return a.x * b.x + a.y * b.y + a.z * b.z + a.w * b.w;
}
__device__ __forceinline__ double dot_vec(const double2& a, const double2& b) { return a.x * b.x + a.y * b.y; }

constexpr int kDenseBlock = 128;

template <class V>
__global__ void __launch_bounds__(kDenseBlock) k_amg_dense(int64_t n, int64_t ld, const V* __restrict__ inv,
                                                           const V* __restrict__ r, V* __restrict__ x,
                                                           const KrylovState* st) {
    if (amg_done(st)) return;
    using V2 = typename std::conditional<sizeof(V) == 4, float4, double2>::type;
    constexpr int E = (int)(sizeof(V2) / sizeof(V));
    __shared__ V sh[kDenseBlock / 32];
    const int64_t nv = ld / E;
    const V2* rv = reinterpret_cast<const V2*>(r);
    for (int64_t i = blockIdx.x; i < n; i += gridDim.x) {
        const V2* row = reinterpret_cast<const V2*>(inv + (size_t)i * ld);
        V acc = 0;
#pragma unroll 4
        for (int64_t c = threadIdx.x; c < nv; c += kDenseBlock) acc += dot_vec(row[c], rv[c]);
        acc = group_sum<32>(acc);
        if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
        __syncthreads();
        if (threadIdx.x == 0) x[i] = (sh[0] + sh[1]) + (sh[2] + sh[3]);
        __syncthreads();
    }
}

// Blocks of `fn` (kBlock threads, no dynamic shared memory) resident on one SM
// of the current device, from the occupancy calculator, cached per device and
// kernel: grids of grid-stride kernels stay within one wave.
int resident_blocks(const void* fn) {
    static std::mutex mu;
    static std::map<std::pair<int, const void*>, int> cache;
    int dev = 0;
    OASIS_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(mu);
    auto it = cache.find({dev, fn});
    if (it != cache.end()) return it->second;
    int per_sm = 0;
    OASIS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kBlock, 0));
    per_sm = std::max(1, per_sm);
    cache[{dev, fn}] = per_sm;
    return per_sm;
}

// finest-level sweeps: one warp per slice pair at a time, one resident wave
int fine_grid(const AmgSellView& F, const void* fn) {
    const int64_t want = (F.n_slices + kBlock / 32 - 1) / (kBlock / 32);
    return (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)num_sms() * resident_blocks(fn)));
}

int amg_grid(int64_t rows, int G, int U, const void* fn) {
    const int64_t per_block = (int64_t)kBlock / G * U;
    const int64_t want = (rows + per_block - 1) / per_block;
    return (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)num_sms() * resident_blocks(fn)));
}

template <class V>
const V* pick(const float* f, const double* d) {
    if constexpr (sizeof(V) == 4) return reinterpret_cast<const V*>(f);
    else return reinterpret_cast<const V*>(d);
}

// one finest-level sweep (PRE: from zero, with the residual), values and
// column form as the view holds them
template <class V, bool PRE>
void launch_fine(const AmgSellView& F, const V* d, V w, const V* r, const V* x, V* out, V* res,
                 const KrylovState* st, cudaStream_t s) {
    using AV = StoredT<V>;
    const AV* av = stored<V>(F.v16, F.v64);
    if constexpr (sizeof(V) == 4) {
        if (F.vp) {
            constexpr int C2 = kFinePairWords;
            k_amg_fine_pairs<PRE, C2><<<fine_grid(F, (const void*)k_amg_fine_pairs<PRE, C2>), kBlock, 0, s>>>(
                F, d, w, r, x, out, res, st);
            return;
        }
    }
    if (F.dcol)
        k_amg_fine<V, AV, true, PRE><<<fine_grid(F, (const void*)k_amg_fine<V, AV, true, PRE>), kBlock, 0, s>>>(
            F, av, d, w, r, x, out, res, st);
    else
        k_amg_fine<V, AV, false, PRE><<<fine_grid(F, (const void*)k_amg_fine<V, AV, false, PRE>), kBlock, 0, s>>>(
            F, av, d, w, r, x, out, res, st);
}

// one float32-cycle row kernel on a pair-packed SELL-32 operator: one warp per
// slice at a time, one resident wave
template <int MODE, int C2, bool W, int SP>
void launch_sellp_c(const SellPView& v, const float* d, float w, const float* r, const float* src, float* out,
                    float* res, const KrylovState* st, cudaStream_t s) {
    constexpr int kSlices = kBlock / 32 / SP;
    const int64_t want = (v.n_slices + kSlices - 1) / kSlices;
    const int per_sm = resident_blocks((const void*)k_amg_sellp<MODE, C2, W, SP>);
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)num_sms() * per_sm));
    k_amg_sellp<MODE, C2, W, SP><<<grid, kBlock, 0, s>>>(v, d, w, r, src, out, res, st);
}

template <int MODE, bool W>
void launch_sellp_w(const AmgSellP& A, const SellPView& v, const float* d, float w, const float* r, const float* src,
                    float* out, float* res, const KrylovState* st, cudaStream_t s) {
    switch (A.sp * 16 + A.c2) {
        case 4 * 16 + 4: launch_sellp_c<MODE, 4, W, 4>(v, d, w, r, src, out, res, st, s); break;
        case 2 * 16 + 4: launch_sellp_c<MODE, 4, W, 2>(v, d, w, r, src, out, res, st, s); break;
        case 1 * 16 + 8: launch_sellp_c<MODE, 8, W, 1>(v, d, w, r, src, out, res, st, s); break;
        default: launch_sellp_c<MODE, 4, W, 1>(v, d, w, r, src, out, res, st, s); break;
    }
}

template <int MODE>
void launch_sellp(const AmgSellP& A, const float* d, float w, const float* r, const float* src, float* out,
                  float* res, const KrylovState* st, cudaStream_t s) {
    const SellPView v{A.n, A.n_slices, A.hdr.p, A.vp.p, A.cp.p, A.cw.p};
    if (A.wide) launch_sellp_w<MODE, true>(A, v, d, w, r, src, out, res, st, s);
    else launch_sellp_w<MODE, false>(A, v, d, w, r, src, out, res, st, s);
}

}  // namespace

// Launch a row kernel with G lanes per row, G chosen at run time.
#define AMG_LAUNCH(GG, KERNEL, ROWS, ARGS)                                                                  \
    KERNEL<V, AV, GG><<<amg_grid(ROWS, GG, amg_rows_u<GG>(), (const void*)KERNEL<V, AV, GG>), kBlock, 0, s>>>(ARGS)
#define AMG_DISPATCH(G, KERNEL, ROWS, ARGS)                                                                   \
    switch (G) {                                                                                              \
        case 4: AMG_LAUNCH(4, KERNEL, ROWS, ARGS); break;                                                     \
        case 8: AMG_LAUNCH(8, KERNEL, ROWS, ARGS); break;                                                     \
        case 16: AMG_LAUNCH(16, KERNEL, ROWS, ARGS); break;                                                   \
        default: AMG_LAUNCH(32, KERNEL, ROWS, ARGS); break;                                                   \
    }

template <class V>
void amg_vcycle(const AmgHierarchy& h, AmgWork& wk, const V* r, V* u, const KrylovState* st, cudaStream_t s,
                const ProfHook* prof) {
    const int L = (int)h.lv.size();
    // the pair-packed copies serve the float32 cycle only
    auto sellp_ok = [](const AmgSellP& A) { return sizeof(V) == 4 && A.n > 0; };
    int ph = -1;
    auto pbeg = [&](int family) {
        if (prof && prof->begin) ph = prof->begin(prof->ctx, s, family);
    };
    auto pend = [&]() {
        if (prof && prof->end) prof->end(prof->ctx, s, ph);
    };
    using AV = StoredT<V>;
    auto vec = [](DBuf<double>& b) { return reinterpret_cast<V*>(b.p); };
    // level inputs: rin[0] = r; outputs: xo[0] = u
    auto rin = [&](int l) -> const V* { return l == 0 ? r : vec(wk.rin[l]); };
    auto xo = [&](int l) -> V* { return l == 0 ? u : vec(wk.xo[l]); };
    for (int l = 0; l < L; ++l) {
        const AmgLevelDev& lv = *h.lv[l];
        const AV* a = stored<V>(lv.a16, lv.a64);
        const V* d = pick<V>(lv.d32.p, lv.d64.p);
        const V w = (V)lv.omega;
        if (l == 0) {
            pbeg(OASIS_PROF_AMG_FINE);
            launch_fine<V, true>(h.fine, d, w, rin(0), nullptr, vec(wk.x[0]), vec(wk.res[0]), st, s);
            pend();
        } else {
            pbeg(OASIS_PROF_AMG_COARSE);
            if (sellp_ok(lv.sa)) {
                if constexpr (sizeof(V) == 4)
                    launch_sellp<kRowPre>(lv.sa, d, w, rin(l), nullptr, vec(wk.x[l]), vec(wk.res[l]), st, s);
            } else {
                AmgRowArgs<V, AV> ra{lv.n, lv.rp, lv.ci, a, d, w, rin(l), nullptr, nullptr, vec(wk.x[l]),
                                     vec(wk.res[l]), st};
                AMG_DISPATCH(lv.g_a, k_amg_pre, lv.n, ra);
            }
            pend();
        }
        const int64_t nc = l + 1 < L ? h.lv[l + 1]->n : h.nc;
        const AV* rv = stored<V>(lv.r16.p, lv.r64.p);
        pbeg(OASIS_PROF_AMG_TRANSFER);
        if (sellp_ok(lv.sr)) {
            if constexpr (sizeof(V) == 4)
                launch_sellp<kRowRestrict>(lv.sr, nullptr, 0.f, nullptr, vec(wk.res[l]), vec(wk.rin[l + 1]), nullptr,
                                           st, s);
        } else {
            AmgRowArgs<V, AV> rr{nc, lv.r_rp.p, lv.r_ci.p, rv, nullptr, V(0), nullptr, nullptr, vec(wk.res[l]),
                                 vec(wk.rin[l + 1]), nullptr, st};
            AMG_DISPATCH(lv.g_r, k_amg_restrict, nc, rr);
        }
        pend();
    }
    pbeg(OASIS_PROF_AMG_COARSE);
    k_amg_dense<V><<<(int)std::max<int64_t>(1, h.nc), kDenseBlock, 0, s>>>(h.nc, h.ld, pick<V>(h.inv32.p, h.inv64.p),
                                                                     vec(wk.rin[L]),
                                                         vec(wk.xo[L]), st);
    pend();
    for (int l = L - 1; l >= 0; --l) {
        const AmgLevelDev& lv = *h.lv[l];
        const AV* a = stored<V>(lv.a16, lv.a64);
        const V* d = pick<V>(lv.d32.p, lv.d64.p);
        const V w = (V)lv.omega;
        const AV* pv = stored<V>(lv.p16.p, lv.p64.p);
        pbeg(OASIS_PROF_AMG_TRANSFER);
        if (sellp_ok(lv.sp)) {
            if constexpr (sizeof(V) == 4)
                launch_sellp<kRowProlong>(lv.sp, nullptr, 0.f, nullptr, xo(l + 1), vec(wk.x[l]), nullptr, st, s);
        } else {
            AmgRowArgs<V, AV> pr{lv.n, lv.p_rp.p, lv.p_ci.p, pv, nullptr, V(0), nullptr, nullptr, xo(l + 1),
                                 vec(wk.x[l]), nullptr, st};
            AMG_DISPATCH(lv.g_p, k_amg_prolong, lv.n, pr);
        }
        pend();
        if (l == 0) {
            pbeg(OASIS_PROF_AMG_FINE);
            launch_fine<V, false>(h.fine, d, w, rin(0), vec(wk.x[0]), xo(0), nullptr, st, s);
            pend();
        } else {
            pbeg(OASIS_PROF_AMG_COARSE);
            if (sellp_ok(lv.sa)) {
                if constexpr (sizeof(V) == 4)
                    launch_sellp<kRowPost>(lv.sa, d, w, rin(l), vec(wk.x[l]), xo(l), nullptr, st, s);
            } else {
                AmgRowArgs<V, AV> po{lv.n, lv.rp, lv.ci, a, d, w, rin(l), vec(wk.x[l]), nullptr, xo(l), nullptr, st};
                AMG_DISPATCH(lv.g_a, k_amg_post, lv.n, po);
            }
            pend();
        }
    }
    OASIS_CUDA(cudaGetLastError());
}
#undef AMG_DISPATCH
#undef AMG_LAUNCH

template void amg_vcycle<float>(const AmgHierarchy&, AmgWork&, const float*, float*, const KrylovState*, cudaStream_t,
                                const ProfHook*);
template void amg_vcycle<double>(const AmgHierarchy&, AmgWork&, const double*, double*, const KrylovState*,
                                 cudaStream_t, const ProfHook*);

}  // namespace oasis
