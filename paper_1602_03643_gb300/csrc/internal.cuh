// Internal declarations shared by the translation units of liboasis.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <memory>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/oasis.h"

namespace oasis {

// Error carried from deep inside the library to the C ABI boundary.
struct Error : std::runtime_error {
    int code;
    Error(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};

#define OASIS_CUDA(call)                                                                   \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            throw ::oasis::Error(e_ == cudaErrorMemoryAllocation ? OASIS_ENOMEM : OASIS_ECUDA, \
                                 std::string(#call) + ": " + cudaGetErrorString(e_));      \
    } while (0)

#define OASIS_CHECK(cond, code, msg)                                                       \
    do {                                                                                   \
        if (!(cond)) throw ::oasis::Error((code), (msg));                                  \
    } while (0)

constexpr int kBlock = 256;          // threads per block for every kernel here
constexpr int kTile = kBlock;        // rows of a row tile (kern.cuh)
// Narrow tiles (half the rows, same block size) for kernels whose per-entry
// shared-memory staging would otherwise limit residency: the entry phase still
// runs on every thread, the row phase on the first kTileN.
constexpr int kTileN = kBlock / 2;

// Owning device buffer (cudaMalloc at creation, cudaFree at destruction).
template <class T>
struct DBuf {
    T* p = nullptr;
    size_t n = 0;
    DBuf() = default;
    DBuf(const DBuf&) = delete;
    DBuf& operator=(const DBuf&) = delete;
    DBuf(DBuf&& o) noexcept : p(o.p), n(o.n) {
        o.p = nullptr;
        o.n = 0;
    }
    DBuf& operator=(DBuf&& o) noexcept {
        if (this != &o) {
            release();
            p = o.p;
            n = o.n;
            o.p = nullptr;
            o.n = 0;
        }
        return *this;
    }
    ~DBuf() { release(); }
    void alloc(size_t count) {
        release();
        n = count;
        if (count) OASIS_CUDA(cudaMalloc(&p, count * sizeof(T)));
    }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
    }
    void upload(const T* host, size_t count, cudaStream_t s) {
        alloc(count);
        if (count) OASIS_CUDA(cudaMemcpyAsync(p, host, count * sizeof(T), cudaMemcpyHostToDevice, s));
    }
    size_t bytes() const { return n * sizeof(T); }
};

struct AmgHierarchy;

// The mesh: sparsity pattern, incidence and constant matrices (all on device).
struct Mesh {
    int dim = 0;
    int64_t nv = 0, nc = 0, n = 0, nnz = 0;
    int max_row = 0;
    // host copies needed later
    std::vector<int32_t> h_row_ptr, h_col;
    // Dof renumbering given at creation: internal dof = h_perm[caller dof]
    // (empty: the caller's order is the internal one).  `perm` is its device
    // copy, used by the field transfers.
    std::vector<int32_t> h_perm;
    DBuf<int32_t> perm;
    int32_t internal_dof(int32_t caller) const { return h_perm.empty() ? caller : h_perm[caller]; }
    // device: pattern
    DBuf<int32_t> row_ptr, col, diag;          // diag[i] = position of (i, i)
    // device: cells
    DBuf<int32_t> cell_vert;                   // [nc][dim+1] vertex indices
    DBuf<int32_t> cell_dof;                    // [nc][dim+1] dofs
    DBuf<double> coords;                       // [nv][dim]
    // device: dof -> cell incidence, sorted by cell; slots packs, per incidence,
    // the position (within the row) of each of the cell's dofs, 8 bits each.
    DBuf<int32_t> inc_ptr, inc_cell;
    DBuf<uint32_t> inc_slots;
    // device: geometry and constant matrices
    DBuf<double> gw64;                         // [nc][dim+1][dim]  |T|/((d+1)(d+2)) grad lambda_j
    DBuf<float> gw32;
    DBuf<double> M64, K64, G64;                // G64: [dim][nnz]
    DBuf<float> M32, K32, G32;
    DBuf<double> ML64, invML64, dinvK64;       // [n]
    DBuf<float> ML32, invML32, dinvK32;
    DBuf<float2> Kff;                          // K as float-float (hi, lo)
    DBuf<float2> Gff;                          // dP^k as float-float, [dim][nnz]
    int tile_cap = 0;                          // max entries of a 256-row tile
    int tile_cap_n = 0;                        // max entries of a 128-row tile
    // SELL-32 (sliced ELLPACK, slices of 32 rows, column-major inside a slice):
    // entry k of row 32 s + l sits at sell_ptr[s] + 32 k + l; short rows are
    // padded with their own index and a zero value.  sell_of_csr maps a CSR
    // entry to its SELL position.
    int64_t n_sell = 0;
    DBuf<int32_t> sell_ptr, sell_len, sell_col, sell_of_csr;
    // The same columns as 16-bit offsets from the row, taken modulo n (so that
    // periodic wrap-around neighbours stay short): j = row + d, then + n if
    // negative, - n if >= n.  Built only when every offset fits (empty else).
    DBuf<int16_t> sell_dcol;
    DBuf<int16_t> csr_dcol;                    // the same offsets in CSR order (built with sell_dcol)
    DBuf<float> K32s;
    DBuf<double> K64s;
    DBuf<float2> Kffs;
    DBuf<double> red_partial;                  // one partial sum per 256-row tile
    DBuf<uint32_t> red_ticket;
    DBuf<int32_t> err;                         // device error flag for setup kernels
    bool assembled = false;
    std::shared_ptr<AmgHierarchy> amg;         // pressure multigrid, built on first use
};

// Device-resident scalars of one Krylov solve (up to 3 right-hand sides).
// Float copies of the coefficients are kept so that float32 kernels never
// convert from float64 (a float64 instruction is ~64x a float32 one on GB300).
struct KrylovState {
    double rho[3], rho_new[3], alpha[3], omega[3], beta[3];
    double bb[3];          // ||reference||^2 for the relative criterion
    double rr[3];          // last float64-quality residual^2 of the outer sweep
    double rr0_in[3];      // start of the current inner solve
    double rr_in[3];       // recurrence residual^2 of the inner solve
    double mean;           // pressure: mean of the right-hand side
    double psum;           // pressure: sum of p* + phi (normalisation)
    float alpha_f[3], omega_f[3], beta_f[3];
    float mean_hi, mean_lo, meanp_hi, meanp_lo;
    double gscale[2];      // learned guess: rms of the right-hand side and of phi^{n-1}
    float gscale_f[2];
    double guess_rr[2];    // residual^2 of the learned guess and of the fallback
    int32_t col_done[3];   // converged (float64-quality residual)
    int32_t in_done[3];    // inner solve finished for this sweep
    int32_t it_total[3];
    int32_t it_in;         // inner iteration counter (parity of double buffers)
    int32_t sweeps;
    int32_t status;        // OASIS_OK / ENOTCONV / EBREAKDOWN / ENAN
    int32_t guess_used;
    int32_t first;         // 1 before the first residual of a solve
    uint32_t ticket;       // last-block reduction ticket
};

struct Solver;

// Kernels and launchers (step.cu)
void spmv_f64(const Mesh& m, const double* vals, const double* x, double* y, int lanes, cudaStream_t s);
void spmv_f32(const Mesh& m, const float* vals, const float* x, float* y, int lanes, cudaStream_t s);
void spmv_dot_f64(const Mesh& m, const double* vals, const double* x, double* y, double* xy, double* tile_partial,
                  uint32_t* ticket, cudaStream_t s);
void noalloc_scratch(double** partial, uint32_t** ticket);
int64_t noalloc_max_rows();

int num_sms();

}  // namespace oasis
