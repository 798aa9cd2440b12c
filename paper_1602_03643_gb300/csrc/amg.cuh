// Smoothed-aggregation algebraic multigrid for the pressure operator K.
//
// The paper preconditions the pressure solve with algebraic multigrid (hypre
// BoomerAMG, Sec. 6); this is a smoothed-aggregation hierarchy built for the
// pure-Neumann P1 Laplacian:
//   * strength: |a_ij| >= theta sqrt(a_ii a_jj); the filtered operator A_F drops
//     weak off-diagonal entries into the diagonal (row sums kept);
//   * greedy aggregation over the strong graph (root + strong neighbours, then
//     attach leftovers to the aggregate they connect to most strongly, then
//     aggregate what remains), in dof order, so the hierarchy is deterministic;
//   * prolongator P = (I - w_P D_F^-1 A_F) P_tent with P_tent = aggregate
//     indicators (entries 1) and w_P = 4 / (3 rho(D_F^-1 A_F)); because A_F 1 = 0,
//     P maps coarse constants to fine constants and every coarse operator
//     A_c = P^T A P keeps the constant null space exactly;
//   * coarsest level (<= 2048 dofs): the dense inverse of A_c + sigma 1 1^T, which
//     acts as the pseudo-inverse of A_c on right-hand sides orthogonal to 1.
// The V(1,1) cycle uses one damped-Jacobi sweep (w_s = 4 / (3 rho(D^-1 A)))
// before and after the coarse correction, with restriction P^T: a symmetric
// positive semi-definite preconditioner, as CG requires.  The finest level's
// sweeps read K in the mesh's SELL-32 layout; coarser levels and the transfers
// are CSR, and the float32 cycle reads a pair-packed SELL-32 copy of each of
// them that is large enough (AmgSellP; 16-bit column offsets where they fit).
#pragma once

#include <memory>

#include "internal.cuh"

namespace oasis {

// Pair-packed SELL-32 copy of a CSR operator of the float32 cycle (a coarser
// level's matrix, a restriction or a prolongation): rows in slices of 32, lane l
// of slice s owns row 32 s + l; hdr[s] = {word offset, words per lane, base
// column, 0}; entries 2k and 2k + 1 of lane l sit in the 32-bit word at
// hdr[s].x + 32 k + l, as two bfloat16 values in vp (low half: entry 2k) and two
// 16-bit offsets from the slice's base column in cp.  Padding entries carry value
// 0 and offset 0 (column = base, a valid row of the operand).  Where some
// slice's columns spread over 2^16 or more values, the copy is wide: the two
// columns of word w are stored whole in cw[w] (base 0), cp is empty.
struct AmgSellP {
    int64_t n = 0, n_slices = 0;
    int c2 = 4;                        // words per lane loaded per round
    int sp = 1;                        // warps serving one slice (1, 2 or 4)
    bool wide = false;
    DBuf<int4> hdr;
    DBuf<uint32_t> vp, cp;
    DBuf<uint2> cw;
};

struct AmgLevelDev {
    int64_t n = 0, nnz = 0;
    // operator of this level (level 0 points at the mesh's K)
    const int32_t *rp = nullptr, *ci = nullptr;
    const double* a64 = nullptr;
    const uint16_t* a16 = nullptr;     // bfloat16 bit patterns (the float32 cycle; null on level 0,
                                       // whose sweeps read the SELL-32 view)
    DBuf<int32_t> own_rp, own_ci;
    DBuf<double> own_a64;
    DBuf<uint16_t> own_a16;
    DBuf<float> d32;                   // 1 / a_ii
    DBuf<double> d64;
    double omega = 0.0;                // Jacobi weight of the smoother
    int g_a = 4, g_r = 8, g_p = 4;     // lanes per row for A, R = P^T and P (from mean row lengths)
    // prolongation to this level from the next coarser one, and its transpose
    DBuf<int32_t> p_rp, p_ci, r_rp, r_ci;
    DBuf<double> p64, r64;
    DBuf<uint16_t> p16, r16;
    // pair-packed SELL-32 copies for the float32 cycle of this level's operator
    // (levels >= 1), of R and of P, where the operator has at least
    // kSellMinRows rows (n = 0: the CSR kernels serve)
    AmgSellP sa, sr, sp;
};

constexpr int64_t kSellMinRows = 65536;

// SELL-32 view of the finest operator (the mesh's K): the fine-level smoothers
// read it with one lane per row, coalesced column/value loads, and 16-bit column
// offsets where the mesh has them.  The float32 cycle reads its values rounded
// to bfloat16 (v16, the bit patterns), as it does every level's operator and
// transfer: a preconditioner needs no more than a few digits of them, the
// rounded operators are still symmetric (equal entries round alike) and the
// rounded restriction is still the transpose of the rounded prolongation, so
// the cycle stays a symmetric preconditioner.
//
// Where the 16-bit offsets exist, the float32 cycle reads a pair-packed copy:
// a slice's rows padded to an even length, entries k and k+1 of lane l in one
// 32-bit word at word ptr2[s] / 2 + 32 (k / 2) + l (vp: two bfloat16 values,
// low half entry k; cp: two column offsets), so one load brings two entries.
// kp holds the float32 values in the same layout, two per 8-byte word, for the
// float32 CG product w = K u (which needs K exactly as the inner system has it).
struct AmgSellView {
    int64_t n = 0, n_slices = 0;
    const int32_t *ptr = nullptr, *len = nullptr, *col = nullptr;
    const int16_t* dcol = nullptr;
    const double* v64 = nullptr;
    const uint16_t* v16 = nullptr;
    const int32_t* ptr2 = nullptr;
    const uint32_t *vp = nullptr, *cp = nullptr;
    const float2* kp = nullptr;
};

struct AmgHierarchy {
    AmgSellView fine;
    DBuf<uint16_t> fine16;                           // storage of fine.v16
    DBuf<int32_t> fine_ptr2;                         // storage of the pair-packed copy
    DBuf<uint32_t> fine_vp, fine_cp;
    DBuf<float2> fine_kp;
    std::vector<std::unique_ptr<AmgLevelDev>> lv;   // lv[0] fine ... lv[L-1] coarsest
    int64_t nc = 0;                                  // size of the dense coarsest level
    int64_t ld = 0;                                  // its row stride: nc rounded up to 4
    DBuf<float> inv32;                               // [nc][ld], zero-padded
    DBuf<double> inv64;
    double setup_s = 0.0;
    std::vector<int64_t> sizes;                      // rows per level (incl. coarsest)
    std::vector<int64_t> nnzs;
    std::vector<int64_t> pnnzs;                      // prolongator nnz per level (level k+1 -> k)
};

// Build (once per mesh) from the assembled float64 K; no-op if present.
void amg_build(Mesh& m, cudaStream_t s);

// Per-solver work vectors of the V-cycle.
struct AmgWork {
    std::vector<DBuf<double>> x, xo, res, rin;   // raw storage; viewed as V
    void alloc(const AmgHierarchy& h, size_t vbytes);
};

// Optional timing of the V-cycle's kernels by family (eager profiling): begin
// returns a handle that end closes; both are no-ops when the hook is absent.
struct ProfHook {
    void* ctx = nullptr;
    int (*begin)(void* ctx, cudaStream_t s, int family) = nullptr;
    void (*end)(void* ctx, cudaStream_t s, int handle) = nullptr;
};

// u = M r with one V(1,1) cycle (device arrays of n_0 values of type V).  The
// kernels return at once when `done` (the CG's col_done / in_done flags) is set.
template <class V>
void amg_vcycle(const AmgHierarchy& h, AmgWork& w, const V* r, V* u, const KrylovState* st, cudaStream_t s,
                const ProfHook* prof = nullptr);

}  // namespace oasis
