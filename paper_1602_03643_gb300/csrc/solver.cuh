// Solver object, kernel argument blocks and the Krylov loop driver.
#pragma once

#include <functional>
#include <memory>
#include <utility>
#include <vector>

#include "amg.cuh"
#include "internal.cuh"

namespace oasis {

// Raw device buffer whose element type depends on the precision policy
// (8-byte state entries are double in float64 mode and float2 float-float in
// mixed mode; V entries are double or float).
struct RBuf {
    void* p = nullptr;
    size_t bytes = 0;
    RBuf() = default;
    RBuf(const RBuf&) = delete;
    RBuf& operator=(const RBuf&) = delete;
    ~RBuf() {
        if (p) cudaFree(p);
    }
    void alloc(size_t b, cudaStream_t s) {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = b;
        if (b) {
            OASIS_CUDA(cudaMalloc(&p, b));
            OASIS_CUDA(cudaMemsetAsync(p, 0, b, s));
        }
    }
    template <class T> T* as() const { return reinterpret_cast<T*>(p); }
};

// Per-row state of the pressure CG that neighbours gather: the residual r,
// w = K M^-1 r, s = K p and M^-1 = 1 / K_ii, as one aligned 4-vector so that a
// neighbour costs one 16-byte (float) or 32-byte (double) load.
template <class V>
struct alignas(4 * sizeof(V)) CgQuad {
    V r, w, s, d;
};

template <class P>
struct StepData {
    using V = typename P::V;
    using S = typename P::S;
    // pattern / mesh
    const int32_t *rp, *col, *diag, *inc_ptr, *inc_cell, *cell_dof;
    const uint32_t* inc_slots;
    const V *M, *K, *G, *gw, *ML;     // G: [D][nnz]; gw: [nc][D+1][D]
    const S* Kout;                    // float64-quality K for the pressure residual
    const S* Gout;                    // float64-quality dP^k for the pressure right-hand side
    const V *dinvK, *invML;
    // state (S)
    S *u1, *u2, *du, *r0, *pstar, *x, *b, *phi, *phi_h1, *phi_h2;
    const S* g;                       // [n_dir][D]
    const int32_t* dir_index;
    // tentative system (V)
    V *A, *dinvA, *beta, *beta2;     // beta2: cell terms of u^{n-2} (explicit convection only)
    V* ubar;                          // [n][D] convecting velocity 1.5 u^{n-1} - 0.5 u^{n-2} (Eq. 22)
    S* uI;                            // [n][D] tentative velocity u^{n-1} + Delta (pressure right-hand side)
    // BiCGStab work [n][D] (V)
    V *r, *rh, *p, *v, *s, *t, *ph, *sh, *dl;
    // CG work: gathered quads double-buffered by iteration parity; p; delta; x rounded
    CgQuad<V> *pq0, *pq1;
    V *pp, *pdl, *xv;
    V *ar, *as, *aw, *au;             // multigrid-preconditioned CG: r, s, w = K u, u = M r
    float* feat;                      // learned guess: features [n][3]
    float* gy;                        // learned guess: network output [n]
    V *mx, *mr, *mz, *mp, *mq;        // consistent-mass update [n][D]: increment, r, z, p, q = M p
    V* cbar;                          // passive scalars: C(ubar) per pattern entry, written by the
                                      // velocity assembly when non-null
    KrylovState *stu, *stp, *stm;
    void* partial;
    double f[3];
    double dt, nu;
    int64_t n, nnz, nc;
    int max_row;
    int tile_cap;
    // SELL-32 copy of K
    int64_t n_slices;
    const int32_t *sell_ptr, *sell_len, *sell_col;
    const int16_t* sell_dcol;         // modular 16-bit column offsets, or null
    const int16_t* csr_dcol;          // the same offsets in CSR order, or null
    // the finest multigrid level's pair-packed copy of K (float32 values two per
    // word, offsets two per word, word offset of each slice x 2), or null
    const float2* kpair;
    const uint32_t* cpair;
    const int32_t* ptr2;
    const V* Ks;
    const S* Kouts;
};

struct Ctl {
    double rtol2;       // float64 stopping test: ||r||^2 <= rtol2 * bb
    double inner2;      // inner solve: relative reduction^2 of its own start residual
    double abs2;        // inner solve also ends at ||r_in||^2 <= abs2 * bb
    int max_it;         // total iterations over all sweeps
    int sweep_cap;      // iterations per sweep
    int use_cond;       // 1 inside a captured graph
    cudaGraphConditionalHandle h_outer, h_inner;
};

struct Loop {
    int graph = 0;
    cudaGraphConditionalHandle h_outer = 0, h_inner = 0;
};

struct StepImpl {
    virtual ~StepImpl() = default;
    virtual void assemble(cudaStream_t s) = 0;
    virtual void tentative_solve(cudaStream_t s, bool graph) = 0;
    // inner = index of the repetition within the step (Algorithm 1)
    virtual void pressure_solve(cudaStream_t s, bool graph, int inner) = 0;
    // p* <- p (normalised) between repetitions, velocities untouched
    virtual void advance_pressure(cudaStream_t s) = 0;
    // velocity update (lumped, or the consistent-mass solve then the update)
    virtual void update(cudaStream_t s, bool graph) = 0;
    // passive scalars: assembly, BiCGStab and update of every scalar
    virtual void scalar_solve(cudaStream_t s, bool graph) = 0;
    // the solver's scalar buffers were (re)allocated or removed
    virtual void scalars_changed() = 0;
    // Component-major float64 arrays [comps][count] <-> the state (dof-major,
    // storage type).  With `perm` (the mesh's device renumbering, period n_dofs)
    // entry i of the array is caller index i: it lands at internal index
    // (i / n) n + perm[i mod n]; without it the indices are equal.
    virtual void to_state(cudaStream_t s, const double* src_soa, int which, int64_t count, int comps,
                          const int32_t* perm) = 0;
    virtual void from_state(cudaStream_t s, double* dst_soa, int which, int64_t count, int comps,
                            const int32_t* perm) = 0;
    virtual void a_to_double(cudaStream_t s, double* dst) = 0;
    virtual void guess_target(cudaStream_t s, float* target) = 0;
    // time the candidate shapes of the CG iteration kernel on this matrix and keep
    // the fastest (forced = k >= 1 takes shape k untimed)
    virtual void tune(cudaStream_t s, int forced) = 0;
    virtual void tuning(oasis_tuning* out) const = 0;
    virtual void amg_apply(cudaStream_t s, const void* r, void* u) = 0;
};

// state buffers addressable by to_state / from_state
enum StateId { ST_U1 = 0, ST_U2, ST_PSTAR, ST_PHI, ST_G, ST_R0, ST_C, ST_GC, ST_COUNT };

using LoopFn = std::function<void(cudaStream_t, const Loop&)>;

struct Solver {
    Mesh* m = nullptr;
    oasis_params prm{};
    bool mixed = false;
    int64_t n_dir = 0;
    double t = 0.0;
    DBuf<int32_t> dir_index;
    RBuf g, u1, u2, du, r0, pstar, x, b, phi, phi_h1, phi_h2;          // S
    RBuf A, dinvA, beta, beta2;                                        // V
    RBuf ubar;                                                         // V [n][D]
    RBuf uI;                                                           // S [n][D]
    RBuf w[9];                                                         // V [n][D]
    RBuf pw[3];                                                        // V [n]
    RBuf pq[2];                                                        // CgQuad<V> [n]
    RBuf amg_vec[4];                                                   // V [n]: r, s, w, u (multigrid CG)
    RBuf mw[5];                                                        // V [n][D]: consistent-mass CG
    // passive scalars (oasis_solver_set_scalars)
    int ns = 0;
    int64_t n_sdir = 0;
    double sc_diff[OASIS_MAX_SCALARS] = {0}, sc_src[OASIS_MAX_SCALARS] = {0};
    DBuf<int32_t> sdir_index;                                          // [n]: index in the set, or -1
    RBuf c, gc;                                                        // S [ns][n], S [ns][n_sdir]
    RBuf cbar, Ac;                                                     // V [nnz]
    RBuf dinvAc;                                                       // V [n]
    RBuf r0c, dc;                                                      // S [n]
    RBuf sw[9];                                                        // V [n]: BiCGStab work
    DBuf<double> cstage;                                               // [ns][max(n, n_sdir)] host copies
    AmgWork amgw;                                                      // V-cycle work vectors
    DBuf<float> feat, gy;                                              // learned-guess features / output
    struct Net* net = nullptr;                                         // attached network (not owned)
    bool record = false;                                               // compute features every step
    RBuf Kout;                                                         // S [nnz]
    DBuf<double> stage;                                                // [max(n, n_dir) * D]
    static constexpr int kStates = 3 + OASIS_MAX_SCALARS;
    DBuf<KrylovState> st;                                              // [0] velocity, [1] pressure, [2] mass,
                                                                       // [3 + a] scalar a
    int n_states() const { return 3 + ns; }                            // mirrored to the host each step
    RBuf partial;
    KrylovState* h_st = nullptr;                                       // pinned mirror [kStates]
    std::unique_ptr<StepImpl> impl;
    cudaStream_t cap[3] = {nullptr, nullptr, nullptr};
    cudaGraphExec_t gexec = nullptr;
    cudaGraph_t graph = nullptr;
    // eager-mode kernel timing (CUDA events around selected launches)
    static constexpr int kProfFamilies = 14;
    bool prof_on = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_pool;
    std::vector<std::pair<int, int>> ev_used;
    double prof_ms[kProfFamilies] = {0};
    int64_t prof_n[kProfFamilies] = {0};
    int prof_begin(cudaStream_t s, int family);
    void prof_end(cudaStream_t s, int idx);
    void prof_collect();

    void run_loops(cudaStream_t s, bool graph_mode, int which, const LoopFn& outer, const LoopFn& inner,
                   const LoopFn& correct, int k0 = 0, int nr = 3);
    // start; while (inner cond) { iter }: a single Krylov sweep whose kernels
    // set h_inner (graph) or in_done[0] of state `which` (eager polls)
    void run_single(cudaStream_t s, bool graph_mode, int which, const LoopFn& start, const LoopFn& iter);
    void poll(cudaStream_t s, int which);
    void step(cudaStream_t s);
    void enqueue_step(cudaStream_t s, bool graph);
    void capture();
    ~Solver();
};

StepImpl* make_step_impl(Solver& s);
Mesh* build_mesh(int dim, int64_t nv, const double* coords, int64_t nc, const int32_t* cells,
                 const int32_t* dof_of_vertex, int64_t n_dofs, const int32_t* perm);
// Pattern of the mesh in the caller's dof order (see Mesh::h_perm): row_ptr,
// col, and for each caller entry the index of the same entry in the internal
// pattern.
void caller_pattern(const Mesh& m, std::vector<int32_t>& row_ptr, std::vector<int32_t>& col,
                    std::vector<int64_t>& src);
void assemble_constant(Mesh& m, cudaStream_t s);

}  // namespace oasis
