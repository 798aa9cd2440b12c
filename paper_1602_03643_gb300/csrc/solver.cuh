// Solver object, kernel argument blocks and the Krylov loop driver.
#pragma once

#include <functional>
#include <memory>
#include <utility>
#include <vector>

#include "internal.cuh"

namespace oasis {

template <class V>
struct AsmArgs {
    const int32_t *rp, *col, *diag, *inc_ptr, *inc_cell;
    const uint32_t* inc_slots;
    const V* beta;
    const V *M, *K, *G;
    const double* ML;
    const double *u1, *u2, *pstar;
    const int32_t* dir_index;
    const double* g;
    double f[3];
    double dt, nu;
    V* A;
    V* dinv;
    double* r0;
    KrylovState* st;
    double* partial;
    int64_t n, nnz;
};

template <class V>
struct BicgArgs {
    const int32_t *rp, *col;
    const V* A;
    const V* dinv;
    const double* r0;
    double* du;
    V *r, *rh, *p, *v, *s, *t, *ph, *sh, *dl;
    KrylovState* st;
    double* partial;
    int64_t n;
    int k0;
};

struct BicgCtl {
    double rtol2;       // float64 stopping test: ||r||^2 <= rtol2 * bb
    double inner2;      // inner solve: relative reduction^2 of its own start residual
    double abs2;        // inner solve: ||r_in||^2 <= abs2 * bb also ends the sweep
    int max_it;         // total iterations over all sweeps
    int sweep_cap;      // iterations per sweep
    int use_cond;       // 1 inside a captured graph
    cudaGraphConditionalHandle h_outer, h_inner;
};

template <class V>
struct PresArgs {
    const int32_t *rp, *col;
    const V* G;
    const double *u1, *du;
    double* b;
    double dt;
    KrylovState* st;
    double* partial;
    int64_t n, nnz;
};

template <class V>
struct PcgArgs {
    const int32_t *rp, *col;
    const V* K;
    const double* K64;
    const V* dinv;
    const double* b;
    double* x;
    const double* pstar;
    V *r, *z, *p0, *p1, *q, *dl;
    KrylovState* st;
    double* partial;
    int64_t n;
};

template <class V>
struct UpdArgs {
    const int32_t *rp, *col;
    const V* G;
    const double* invML;
    const double *x, *du;
    double *u1, *u2, *pstar, *phi_out, *phi_h1, *phi_h2;
    const int32_t* dir_index;
    const double* g;
    double dt;
    const KrylovState* stp;
    int64_t n, nnz;
};

struct Loop {
    int graph = 0;
    cudaGraphConditionalHandle h_outer = 0, h_inner = 0;
};

struct StepImpl {
    virtual ~StepImpl() = default;
    virtual void assemble(cudaStream_t s) = 0;
    virtual void tentative_solve(cudaStream_t s, bool graph) = 0;
    virtual void pressure_solve(cudaStream_t s, bool graph) = 0;
    virtual void update(cudaStream_t s) = 0;
};

using LoopFn = std::function<void(cudaStream_t, const Loop&)>;

struct Solver {
    Mesh* m = nullptr;
    oasis_params prm{};
    bool mixed = false;
    int lanes = 16;
    int64_t n_dir = 0;
    double t = 0.0;
    DBuf<int32_t> dir_index;
    DBuf<double> g;                            // [n_dir][D]
    DBuf<double> u1, u2, du, r0u;              // [n][D]
    DBuf<double> pstar, phi, phi_h1, phi_h2, bphi, xp;   // [n]
    DBuf<double> A64, dA64, beta64;
    DBuf<float> A32, dA32, beta32;
    DBuf<double> w64[9];
    DBuf<float> w32[9];
    DBuf<double> q64[6];
    DBuf<float> q32[6];
    double* w64p[9];
    float* w32p[9];
    double* q64p[6];
    float* q32p[6];
    DBuf<KrylovState> st;                      // [0] velocity, [1] pressure
    DBuf<double> partial;
    KrylovState* h_st = nullptr;               // pinned mirror [2]
    std::unique_ptr<StepImpl> impl;
    cudaStream_t cap[3] = {nullptr, nullptr, nullptr};
    cudaGraphExec_t gexec = nullptr;
    cudaGraph_t graph = nullptr;
    bool stepped = false;
    DBuf<double> stage;                        // [n][D] staging for host transfers
    DBuf<float> stage32;                       // [nnz] float32 -> float64 staging
    // eager-mode kernel timing (CUDA events around selected launches)
    static constexpr int kProfFamilies = 6;
    bool prof_on = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_pool;
    std::vector<std::pair<int, int>> ev_used;  // (family, pool index)
    double prof_ms[kProfFamilies] = {0};
    int64_t prof_n[kProfFamilies] = {0};
    int prof_begin(cudaStream_t s, int family);
    void prof_end(cudaStream_t s, int idx);
    void prof_collect();

    template <class V> V* beta();
    template <class V> const V* gw();
    template <class V> V* A();
    template <class V> V* dinvA();
    template <class V> V** work();
    template <class V> V** pwork();
    template <class V> const V* mat(const DBuf<double>& d, const DBuf<float>& f) {
        if constexpr (sizeof(V) == 8) return (const V*)(const void*)d.p;
        else return (const V*)(const void*)f.p;
    }

    // Runs a refinement loop: outer(); while(inner active) inner(); correct(); ...
    // `which` selects the KrylovState (0 velocity, 1 pressure); [k0, k0+nr) the columns.
    void run_loops(cudaStream_t s, bool graph_mode, int which, const LoopFn& outer, const LoopFn& inner,
                   const LoopFn& correct, int k0 = 0, int nr = 3);
    void poll(cudaStream_t s, int which);
    void step(cudaStream_t s);
    void capture();
    ~Solver();
};

template <> inline double* Solver::beta<double>() { return beta64.p; }
template <> inline float* Solver::beta<float>() { return beta32.p; }
template <> inline const double* Solver::gw<double>() { return m->gw64.p; }
template <> inline const float* Solver::gw<float>() { return m->gw32.p; }
template <> inline double* Solver::A<double>() { return A64.p; }
template <> inline float* Solver::A<float>() { return A32.p; }
template <> inline double* Solver::dinvA<double>() { return dA64.p; }
template <> inline float* Solver::dinvA<float>() { return dA32.p; }
template <> inline double** Solver::work<double>() { return w64p; }
template <> inline float** Solver::work<float>() { return w32p; }
template <> inline double** Solver::pwork<double>() { return q64p; }
template <> inline float** Solver::pwork<float>() { return q32p; }

StepImpl* make_step_impl(Solver& s, int lanes);
Mesh* build_mesh(int dim, int64_t nv, const double* coords, int64_t nc, const int32_t* cells,
                 const int32_t* dof_of_vertex, int64_t n_dofs);
void assemble_constant(Mesh& m, cudaStream_t s);

}  // namespace oasis
