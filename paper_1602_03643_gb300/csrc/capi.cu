// C ABI of liboasis (declared in include/oasis.h) and the host side of the
// solver: buffer allocation, field transfer, the eager and graph step drivers.
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "device.cuh"
#include "internal.cuh"
#include "solver.cuh"
#include "kern.cuh"
#include "amg.cuh"
#include "net.cuh"

namespace oasis {

static thread_local std::string g_last_error;

// ------------------------------------------------------------------ loops
void Solver::poll(cudaStream_t s, int which) {
    OASIS_CUDA(cudaMemcpyAsync(h_st + which, st.p + which, sizeof(KrylovState), cudaMemcpyDeviceToHost, s));
    OASIS_CUDA(cudaStreamSynchronize(s));
}

static cudaGraph_t capture_graph_of(cudaStream_t s) {
    cudaStreamCaptureStatus cs;
    cudaGraph_t g = nullptr;
    OASIS_CUDA(cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, nullptr, nullptr, nullptr));
    OASIS_CHECK(cs == cudaStreamCaptureStatusActive, OASIS_ECUDA, "stream is not capturing");
    return g;
}

// Append a WHILE conditional node to the graph being captured on `s`; returns
// its body graph.  The stream's capture continues after the node.
static cudaGraph_t add_while(cudaStream_t s, cudaGraphConditionalHandle h) {
    cudaStreamCaptureStatus cs;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    size_t ndeps = 0;
    OASIS_CUDA(cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, nullptr, &ndeps));
    cudaGraphNodeParams np{};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    OASIS_CUDA(cudaGraphAddNode(&node, g, deps, nullptr, ndeps, &np));
    cudaGraph_t body = np.conditional.phGraph_out[0];
    OASIS_CUDA(cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    return body;
}

void Solver::run_loops(cudaStream_t s, bool graph_mode, int which, const LoopFn& outer, const LoopFn& inner,
                       const LoopFn& correct, int k0, int nr) {
    if (!graph_mode) {
        Loop lp;
        const int chunk = 4;
        for (int guard = 0; guard < 1000000; ++guard) {
            outer(s, lp);
            poll(s, which);
            bool live = false;
            for (int k = k0; k < k0 + nr && k < 3; ++k) live |= !h_st[which].col_done[k];
            if (!live) return;
            for (;;) {
                for (int c = 0; c < chunk; ++c) inner(s, lp);
                poll(s, which);
                bool act = false;
                for (int k = k0; k < k0 + nr && k < 3; ++k)
                    act |= !h_st[which].col_done[k] && !h_st[which].in_done[k];
                if (!act) break;
            }
            correct(s, lp);
        }
        throw Error(OASIS_ENOTCONV, "refinement loop did not terminate");
    }
    // graph: while (outer cond) { outer; while (inner cond) { inner }; correct }
    cudaGraph_t g = capture_graph_of(s);
    Loop lp;
    lp.graph = 1;
    OASIS_CUDA(cudaGraphConditionalHandleCreate(&lp.h_outer, g, 1, cudaGraphCondAssignDefault));
    cudaGraph_t outer_body = add_while(s, lp.h_outer);
    cudaStream_t s1 = cap[1], s2 = cap[2];
    OASIS_CUDA(cudaStreamBeginCaptureToGraph(s1, outer_body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    OASIS_CUDA(cudaGraphConditionalHandleCreate(&lp.h_inner, outer_body, 0, 0));
    outer(s1, lp);
    cudaGraph_t inner_body = add_while(s1, lp.h_inner);
    OASIS_CUDA(cudaStreamBeginCaptureToGraph(s2, inner_body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    inner(s2, lp);
    cudaGraph_t tmp;
    OASIS_CUDA(cudaStreamEndCapture(s2, &tmp));
    correct(s1, lp);
    OASIS_CUDA(cudaStreamEndCapture(s1, &tmp));
}

void Solver::run_single(cudaStream_t s, bool graph_mode, int which, const LoopFn& start, const LoopFn& iter) {
    if (!graph_mode) {
        Loop lp;
        const int chunk = 4;
        start(s, lp);
        for (int guard = 0; guard < 1000000; ++guard) {
            poll(s, which);
            if (h_st[which].in_done[0]) return;
            for (int c = 0; c < chunk; ++c) iter(s, lp);
        }
        throw Error(OASIS_ENOTCONV, "Krylov loop did not terminate");
    }
    cudaGraph_t g = capture_graph_of(s);
    Loop lp;
    lp.graph = 1;
    OASIS_CUDA(cudaGraphConditionalHandleCreate(&lp.h_inner, g, 0, 0));
    start(s, lp);
    cudaGraph_t body = add_while(s, lp.h_inner);
    cudaStream_t s1 = cap[1];
    OASIS_CUDA(cudaStreamBeginCaptureToGraph(s1, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    iter(s1, lp);
    cudaGraph_t tmp;
    OASIS_CUDA(cudaStreamEndCapture(s1, &tmp));
}

int Solver::prof_begin(cudaStream_t s, int family) {
    if (!prof_on || prm.use_graph) return -1;
    const size_t idx = ev_used.size();
    if (idx >= ev_pool.size()) {
        cudaEvent_t a, b;
        OASIS_CUDA(cudaEventCreate(&a));
        OASIS_CUDA(cudaEventCreate(&b));
        ev_pool.emplace_back(a, b);
    }
    ev_used.emplace_back(family, (int)idx);
    OASIS_CUDA(cudaEventRecord(ev_pool[idx].first, s));
    return (int)idx;
}

void Solver::prof_end(cudaStream_t s, int idx) {
    if (idx < 0) return;
    OASIS_CUDA(cudaEventRecord(ev_pool[idx].second, s));
}

void Solver::prof_collect() {
    for (auto& fu : ev_used) {
        float ms = 0.f;
        OASIS_CUDA(cudaEventSynchronize(ev_pool[fu.second].second));
        OASIS_CUDA(cudaEventElapsedTime(&ms, ev_pool[fu.second].first, ev_pool[fu.second].second));
        prof_ms[fu.first] += ms;
        prof_n[fu.first] += 1;
    }
    ev_used.clear();
}

void Solver::step(cudaStream_t s) {
    const bool graph_mode = prm.use_graph != 0;
    if (graph_mode) {
        if (!gexec) capture();
        OASIS_CUDA(cudaGraphLaunch(gexec, s));
    } else {
        enqueue_step(s, false);
        OASIS_CUDA(cudaMemcpyAsync(h_st, st.p, n_states() * sizeof(KrylovState), cudaMemcpyDeviceToHost, s));
        if (prof_on) prof_collect();
    }
    t += prm.dt;
}

// One time step (Algorithm 1): assembly, then per inner repetition the
// tentative and pressure solves (p* advanced and the tentative residual
// re-formed between repetitions), the passive scalars (they use only the old
// velocities), then the velocity update (lumped, or the consistent-mass solve).
void Solver::enqueue_step(cudaStream_t s, bool graph_mode) {
    const int ni = std::max(1, prm.inner_iters);
    impl->assemble(s);
    for (int it = 0; it < ni; ++it) {
        if (it > 0) {
            impl->advance_pressure(s);
            impl->assemble(s);
        }
        impl->tentative_solve(s, graph_mode);
        impl->pressure_solve(s, graph_mode, it);
    }
    if (ns > 0) impl->scalar_solve(s, graph_mode);
    impl->update(s, graph_mode);
}

void Solver::capture() {
    cudaStream_t s = cap[0];
    OASIS_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    try {
        enqueue_step(s, true);
        OASIS_CUDA(cudaMemcpyAsync(h_st, st.p, n_states() * sizeof(KrylovState), cudaMemcpyDeviceToHost, s));
    } catch (...) {
        cudaGraph_t g;
        cudaStreamEndCapture(s, &g);
        if (g) cudaGraphDestroy(g);
        throw;
    }
    OASIS_CUDA(cudaStreamEndCapture(s, &graph));
    OASIS_CUDA(cudaGraphInstantiate(&gexec, graph, 0));
}

Solver::~Solver() {
    for (auto& e : ev_pool) {
        cudaEventDestroy(e.first);
        cudaEventDestroy(e.second);
    }
    if (gexec) cudaGraphExecDestroy(gexec);
    if (graph) cudaGraphDestroy(graph);
    for (auto& c : cap)
        if (c) cudaStreamDestroy(c);
    if (h_st) cudaFreeHost(h_st);
}

static Solver* create_solver(Mesh* m, const oasis_params* prm, int64_t n_dir, const int32_t* dir,
                             cudaStream_t s) {
    OASIS_CHECK(m && prm, OASIS_EINVAL, "null mesh or params");
    OASIS_CHECK(m->assembled, OASIS_EINVAL, "call oasis_assemble_constant first");
    OASIS_CHECK(prm->dt > 0 && prm->nu >= 0, OASIS_EINVAL, "dt must be > 0 and nu >= 0");
    OASIS_CHECK(prm->rtol_u > 0 && prm->rtol_p > 0, OASIS_EINVAL, "tolerances must be > 0");
    OASIS_CHECK(prm->max_it_u > 0 && prm->max_it_p > 0, OASIS_EINVAL, "iteration caps must be > 0");
    OASIS_CHECK(prm->precision == OASIS_FP64 || prm->precision == OASIS_MIXED, OASIS_EINVAL, "precision");
    OASIS_CHECK(prm->guess >= 0 && prm->guess <= 2, OASIS_EINVAL, "guess");
    OASIS_CHECK(prm->spmv_variant >= 0 && prm->spmv_variant <= OASIS_MAX_VARIANTS, OASIS_EINVAL, "spmv_variant");
    OASIS_CHECK(prm->bicg_variant >= 0 && prm->bicg_variant <= 8, OASIS_EINVAL, "bicg_variant");
    OASIS_CHECK(prm->pressure_pc == OASIS_PC_JACOBI || prm->pressure_pc == OASIS_PC_AMG, OASIS_EINVAL,
                "pressure_pc");
    OASIS_CHECK(prm->inner_iters >= 0 && prm->inner_iters <= 16, OASIS_EINVAL, "inner_iters must be in [0, 16]");
    OASIS_CHECK(prm->convection == OASIS_CONV_ABCN || prm->convection == OASIS_CONV_ABE, OASIS_EINVAL, "convection");
    OASIS_CHECK(prm->velocity_update == OASIS_UPDATE_LUMPED || prm->velocity_update == OASIS_UPDATE_CONSISTENT,
                OASIS_EINVAL, "velocity_update");
    OASIS_CHECK(n_dir >= 0 && (n_dir == 0 || dir), OASIS_EINVAL, "dirichlet dofs");
    OASIS_CHECK(m->max_row <= 64, OASIS_EMESH, "rows with more than 64 pattern entries are not supported");
    auto S = std::make_unique<Solver>();
    S->m = m;
    S->prm = *prm;
    S->mixed = prm->precision == OASIS_MIXED;
    if (S->mixed && !(S->prm.inner_rtol > 0 && S->prm.inner_rtol < 1)) S->prm.inner_rtol = 1e-4;
    const int D = m->dim;
    const int64_t n = m->n;
    const size_t vb = S->mixed ? sizeof(float) : sizeof(double);   // value bytes
    const size_t sb = 8;                                             // state bytes (double or float2)
    S->n_dir = n_dir;
    std::vector<int32_t> di(n, -1);
    for (int64_t q = 0; q < n_dir; ++q) {
        OASIS_CHECK(dir[q] >= 0 && dir[q] < n, OASIS_EINVAL, "dirichlet dof out of range");
        const int32_t i = m->internal_dof(dir[q]);
        OASIS_CHECK(di[i] < 0, OASIS_EINVAL, "repeated dirichlet dof");
        di[i] = (int32_t)q;
    }
    S->dir_index.upload(di.data(), n, s);
    S->g.alloc(sb * std::max<int64_t>(1, n_dir * D), s);
    for (RBuf* b : {&S->u1, &S->u2, &S->du, &S->r0, &S->uI}) b->alloc(sb * n * D, s);
    for (RBuf* b : {&S->pstar, &S->x, &S->b, &S->phi, &S->phi_h1, &S->phi_h2}) b->alloc(sb * n, s);
    S->A.alloc(vb * m->nnz, s);
    S->dinvA.alloc(vb * n, s);
    S->beta.alloc(vb * m->nc * 4, s);
    if (prm->convection == OASIS_CONV_ABE) S->beta2.alloc(vb * m->nc * 4, s);
    else S->ubar.alloc(vb * n * D, s);
    for (auto& w : S->w) w.alloc(vb * n * D, s);
    for (auto& w : S->pw) w.alloc(vb * n, s);
    for (auto& q : S->pq) q.alloc(4 * vb * n, s);
    if (prm->velocity_update == OASIS_UPDATE_CONSISTENT)
        for (auto& w : S->mw) w.alloc(vb * n * D, s);
    if (prm->pressure_pc == OASIS_PC_AMG) {
        amg_build(*m, s);
        S->amgw.alloc(*m->amg, vb);
        for (auto& v : S->amg_vec) v.alloc(vb * n, s);
    }
    S->feat.alloc((size_t)n * 3);
    S->gy.alloc((size_t)n);
    OASIS_CUDA(cudaMemsetAsync(S->feat.p, 0, S->feat.bytes(), s));
    OASIS_CUDA(cudaMemsetAsync(S->gy.p, 0, S->gy.bytes(), s));
    // host transfers stage through here: the fields u, p, phi side by side, or the
    // Dirichlet values
    S->stage.alloc(std::max<int64_t>(n * (D + 2), n_dir * D));
    S->st.alloc(Solver::kStates);
    OASIS_CUDA(cudaMemsetAsync(S->st.p, 0, S->st.bytes(), s));
    // per-block partial sums: up to 8 values of 16 bytes per block, for grids of
    // at most max(8 blocks per SM, one block per 256 rows)
    const int64_t max_blocks = std::max<int64_t>((int64_t)num_sms() * 8, (n + kBlock - 1) / kBlock + 1);
    S->partial.alloc((size_t)max_blocks * 8 * 16, s);
    OASIS_CUDA(cudaHostAlloc(&S->h_st, Solver::kStates * sizeof(KrylovState), cudaHostAllocDefault));
    std::memset(S->h_st, 0, Solver::kStates * sizeof(KrylovState));
    for (auto& c : S->cap) OASIS_CUDA(cudaStreamCreateWithFlags(&c, cudaStreamNonBlocking));
    S->impl.reset(make_step_impl(*S));
    S->impl->tune(s, prm->spmv_variant);
    OASIS_CUDA(cudaStreamSynchronize(s));
    return S.release();
}

static void fill_stats(const Solver& S, oasis_step_stats* o) {
    std::memset(o, 0, sizeof(*o));
    const KrylovState& u = S.h_st[0];
    const KrylovState& p = S.h_st[1];
    for (int al = 0; al < S.ns; ++al) {
        const KrylovState& cs = S.h_st[3 + al];
        o->it_c = std::max(o->it_c, cs.it_total[0]);
        o->res_c = std::max(o->res_c, cs.bb[0] > 0 ? std::sqrt(cs.rr[0] / cs.bb[0]) : 0.0);
    }
    const KrylovState& mm = S.h_st[2];
    const bool cons = S.prm.velocity_update == OASIS_UPDATE_CONSISTENT;
    o->status = u.status != OASIS_OK ? u.status : p.status != OASIS_OK ? p.status : cons ? mm.status : OASIS_OK;
    for (int al = 0; al < S.ns && o->status == OASIS_OK; ++al) o->status = S.h_st[3 + al].status;
    if (cons) {
        o->it_m = mm.it_total[0];
        for (int k = 0; k < S.m->dim && k < 3; ++k) o->res_m[k] = mm.bb[k] > 0 ? std::sqrt(mm.rr[k] / mm.bb[k]) : 0.0;
    }
    for (int k = 0; k < 3; ++k) {
        o->it_u[k] = k < S.m->dim ? u.it_total[k] : 0;
        o->res_u[k] = (k < S.m->dim && u.bb[k] > 0) ? std::sqrt(u.rr[k] / u.bb[k]) : 0.0;
    }
    o->sweeps_u = u.sweeps;
    o->it_p = p.it_total[0];
    o->sweeps_p = p.sweeps;
    o->res_p = p.bb[0] > 0 ? std::sqrt(p.rr[0] / p.bb[0]) : 0.0;
    if (S.prm.guess == OASIS_GUESS_LEARNED && S.net) {
        o->guess_used = p.guess_used;
        for (int k = 0; k < 2; ++k) o->guess_res[k] = p.bb[0] > 0 ? std::sqrt(p.guess_rr[k] / p.bb[0]) : 0.0;
    } else o->guess_used = S.prm.guess == OASIS_GUESS_ZERO ? OASIS_GUESS_ZERO : OASIS_GUESS_PREV_PHI;
    o->t = S.t;
}

}  // namespace oasis

using namespace oasis;

template <class F>
static int guarded(F&& f) {
    try {
        g_last_error.clear();
        f();
        return OASIS_OK;
    } catch (const Error& e) {
        g_last_error = e.what();
        return e.code;
    } catch (const std::bad_alloc&) {
        g_last_error = "host allocation failed";
        return OASIS_ENOMEM;
    } catch (const std::exception& e) {
        g_last_error = e.what();
        return OASIS_EINVAL;
    }
}

static cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// Host copy of a per-entry (pattern order) or per-dof array in the internal
// order, written out in the caller's order.
static void to_caller_order(const Mesh& m, bool per_dof, const std::vector<double>& internal, double* out) {
    if (m.h_perm.empty()) {
        std::memcpy(out, internal.data(), internal.size() * sizeof(double));
        return;
    }
    if (per_dof) {
        for (int64_t d = 0; d < m.n; ++d) out[d] = internal[m.h_perm[d]];
        return;
    }
    std::vector<int32_t> rp, ci;
    std::vector<int64_t> src;
    caller_pattern(m, rp, ci, src);
    for (int64_t e = 0; e < m.nnz; ++e) out[e] = internal[src[e]];
}

extern "C" {

int oasis_version(void) { return 100; }

const char* oasis_last_error(void) { return g_last_error.c_str(); }

int oasis_mesh_create(int32_t dim, int64_t n_vertices, const double* coords, int64_t n_cells,
                      const int32_t* cells, const int32_t* dof_of_vertex, int64_t n_dofs, const int32_t* perm,
                      oasis_mesh** out) {
    return guarded([&] {
        OASIS_CHECK(out, OASIS_EINVAL, "null output pointer");
        *out = reinterpret_cast<oasis_mesh*>(
            build_mesh(dim, n_vertices, coords, n_cells, cells, dof_of_vertex, n_dofs, perm));
    });
}

int oasis_mesh_info(const oasis_mesh* mesh, int64_t* n_dofs, int64_t* n_cells, int64_t* nnz) {
    return guarded([&] {
        const Mesh* m = reinterpret_cast<const Mesh*>(mesh);
        OASIS_CHECK(m, OASIS_EINVAL, "null mesh");
        if (n_dofs) *n_dofs = m->n;
        if (n_cells) *n_cells = m->nc;
        if (nnz) *nnz = m->nnz;
    });
}

int oasis_assemble_constant(oasis_mesh* mesh, void* stream) {
    return guarded([&] {
        Mesh* m = reinterpret_cast<Mesh*>(mesh);
        OASIS_CHECK(m, OASIS_EINVAL, "null mesh");
        assemble_constant(*m, as_stream(stream));
    });
}

int oasis_mesh_get_pattern(const oasis_mesh* mesh, int32_t* row_ptr, int32_t* col) {
    return guarded([&] {
        const Mesh* m = reinterpret_cast<const Mesh*>(mesh);
        OASIS_CHECK(m && row_ptr && col, OASIS_EINVAL, "null pointer");
        std::vector<int32_t> rp, ci;
        std::vector<int64_t> src;
        caller_pattern(*m, rp, ci, src);
        std::memcpy(row_ptr, rp.data(), rp.size() * sizeof(int32_t));
        std::memcpy(col, ci.data(), ci.size() * sizeof(int32_t));
    });
}

int oasis_mesh_get_matrix(const oasis_mesh* mesh, int32_t which, double* values) {
    return guarded([&] {
        const Mesh* m = reinterpret_cast<const Mesh*>(mesh);
        OASIS_CHECK(m && values, OASIS_EINVAL, "null pointer");
        OASIS_CHECK(m->assembled, OASIS_EINVAL, "mesh not assembled");
        const double* src = nullptr;
        size_t cnt = m->nnz;
        if (which == OASIS_MAT_M) src = m->M64.p;
        else if (which == OASIS_MAT_K) src = m->K64.p;
        else if (which >= OASIS_MAT_G0 && which < OASIS_MAT_G0 + m->dim) src = m->G64.p + (size_t)(which - OASIS_MAT_G0) * m->nnz;
        else if (which == -1) {
            src = m->ML64.p;
            cnt = m->n;
        } else
            throw Error(OASIS_EINVAL, "unknown matrix");
        OASIS_CUDA(cudaDeviceSynchronize());
        std::vector<double> internal(cnt);
        OASIS_CUDA(cudaMemcpy(internal.data(), src, cnt * sizeof(double), cudaMemcpyDeviceToHost));
        to_caller_order(*m, which == -1, internal, values);
    });
}

static const void* const_matrix(const Mesh* m, int which, bool f32) {
    if (which == OASIS_MAT_M) return f32 ? (const void*)m->M32.p : (const void*)m->M64.p;
    if (which == OASIS_MAT_K) return f32 ? (const void*)m->K32.p : (const void*)m->K64.p;
    if (which >= OASIS_MAT_G0 && which < OASIS_MAT_G0 + m->dim) {
        const size_t o = (size_t)(which - OASIS_MAT_G0) * m->nnz;
        return f32 ? (const void*)(m->G32.p + o) : (const void*)(m->G64.p + o);
    }
    throw Error(OASIS_EINVAL, "unknown matrix");
}

int oasis_spmv_f64(const oasis_mesh* mesh, int32_t which, const double* x, double* y, int32_t lanes, void* stream) {
    return guarded([&] {
        const Mesh* m = reinterpret_cast<const Mesh*>(mesh);
        OASIS_CHECK(m && x && y, OASIS_EINVAL, "null pointer");
        OASIS_CHECK(m->assembled, OASIS_EINVAL, "mesh not assembled");
        spmv_f64(*m, (const double*)const_matrix(m, which, false), x, y, lanes ? lanes : 16, as_stream(stream));
    });
}

int oasis_spmv_f32(const oasis_mesh* mesh, int32_t which, const float* x, float* y, int32_t lanes, void* stream) {
    return guarded([&] {
        const Mesh* m = reinterpret_cast<const Mesh*>(mesh);
        OASIS_CHECK(m && x && y, OASIS_EINVAL, "null pointer");
        OASIS_CHECK(m->assembled, OASIS_EINVAL, "mesh not assembled");
        spmv_f32(*m, (const float*)const_matrix(m, which, true), x, y, lanes ? lanes : 16, as_stream(stream));
    });
}

int oasis_spmv_dot_f64(const oasis_mesh* mesh, int32_t which, const double* x, double* y, double* xy,
                       void* stream) {
    return guarded([&] {
        const Mesh* m = reinterpret_cast<const Mesh*>(mesh);
        OASIS_CHECK(m && x && y && xy, OASIS_EINVAL, "null pointer");
        OASIS_CHECK(m->assembled, OASIS_EINVAL, "mesh not assembled");
        spmv_dot_f64(*m, (const double*)const_matrix(m, which, false), x, y, xy, m->red_partial.p, m->red_ticket.p,
                     as_stream(stream));
    });
}

int oasis_spmv_dot_f64_noalloc(const oasis_mesh* mesh, int32_t which, const double* x, double* y, double* xy,
                               void* stream) {
    return guarded([&] {
        const Mesh* m = reinterpret_cast<const Mesh*>(mesh);
        OASIS_CHECK(m && x && y && xy, OASIS_EINVAL, "null pointer");
        // the size bound depends on the mesh alone, so it is checked first
        OASIS_CHECK(m->n <= noalloc_max_rows(), OASIS_EINVAL,
                    "n_dofs = " + std::to_string(m->n) + " exceeds the static scratch of the no-alloc entry point (at "
                    "most " + std::to_string(noalloc_max_rows()) + " rows); use oasis_spmv_dot_f64");
        OASIS_CHECK(m->assembled, OASIS_EINVAL, "mesh not assembled");
        double* partial = nullptr;
        uint32_t* ticket = nullptr;
        noalloc_scratch(&partial, &ticket);
        spmv_dot_f64(*m, (const double*)const_matrix(m, which, false), x, y, xy, partial, ticket, as_stream(stream));
    });
}

int oasis_solver_create(oasis_mesh* mesh, const oasis_params* params, int64_t n_dirichlet,
                        const int32_t* dirichlet_dofs, void* stream, oasis_solver** out) {
    return guarded([&] {
        OASIS_CHECK(out, OASIS_EINVAL, "null output pointer");
        *out = reinterpret_cast<oasis_solver*>(
            create_solver(reinterpret_cast<Mesh*>(mesh), params, n_dirichlet, dirichlet_dofs, as_stream(stream)));
    });
}

int oasis_set_fields(oasis_solver* solver, const double* u_nm1, const double* u_nm2, const double* p, double t,
                     int32_t on_device, void* stream) {
    return guarded([&] {
        Solver* S = reinterpret_cast<Solver*>(solver);
        OASIS_CHECK(S && u_nm1 && u_nm2 && p, OASIS_EINVAL, "null pointer");
        cudaStream_t s = as_stream(stream);
        const int D = S->m->dim;
        const int64_t n = S->m->n;
        const double* srcs[3] = {u_nm1, u_nm2, p};
        const int ids[3] = {ST_U1, ST_U2, ST_PSTAR};
        const int comps[3] = {D, D, 1};
        for (int q = 0; q < 3; ++q) {
            const double* src = srcs[q];
            if (!on_device) {
                OASIS_CUDA(cudaMemcpyAsync(S->stage.p, src, n * comps[q] * sizeof(double), cudaMemcpyHostToDevice, s));
                src = S->stage.p;
            }
            S->impl->to_state(s, src, ids[q], n, comps[q], S->m->perm.p);
            OASIS_CUDA(cudaStreamSynchronize(s));
        }
        for (RBuf* b : {&S->phi, &S->phi_h1, &S->phi_h2}) OASIS_CUDA(cudaMemsetAsync(b->p, 0, b->bytes, s));
        OASIS_CUDA(cudaStreamSynchronize(s));
        S->t = t;
    });
}

int oasis_set_dirichlet(oasis_solver* solver, const double* g, int32_t on_device, void* stream) {
    return guarded([&] {
        Solver* S = reinterpret_cast<Solver*>(solver);
        OASIS_CHECK(S, OASIS_EINVAL, "null solver");
        if (S->n_dir == 0) return;
        OASIS_CHECK(g, OASIS_EINVAL, "null values");
        cudaStream_t s = as_stream(stream);
        const int D = S->m->dim;
        const int64_t nd = S->n_dir;
        const double* src = g;
        if (!on_device) {
            OASIS_CUDA(cudaMemcpyAsync(S->stage.p, g, nd * D * sizeof(double), cudaMemcpyHostToDevice, s));
            src = S->stage.p;
        }
        S->impl->to_state(s, src, ST_G, nd, D, nullptr);
        if (!on_device) OASIS_CUDA(cudaStreamSynchronize(s));
    });
}

static void drop_graph(Solver* S);

int oasis_solver_set_scalars(oasis_solver* solver, int32_t n_scalars, const double* diffusivity,
                             const double* source, int64_t n_dirichlet, const int32_t* dirichlet_dofs) {
    return guarded([&] {
        Solver* S = reinterpret_cast<Solver*>(solver);
        OASIS_CHECK(S, OASIS_EINVAL, "null solver");
        OASIS_CHECK(n_scalars >= 0 && n_scalars <= OASIS_MAX_SCALARS, OASIS_EINVAL, "n_scalars out of range");
        OASIS_CHECK(n_scalars == 0 || (diffusivity && source), OASIS_EINVAL, "null diffusivity or source");
        OASIS_CHECK(n_dirichlet >= 0 && (n_dirichlet == 0 || dirichlet_dofs), OASIS_EINVAL, "scalar dirichlet dofs");
        const int64_t n = S->m->n;
        for (int al = 0; al < n_scalars; ++al)
            OASIS_CHECK(diffusivity[al] >= 0 && std::isfinite(diffusivity[al]) && std::isfinite(source[al]),
                        OASIS_EINVAL, "diffusivity must be finite and >= 0, source finite");
        std::vector<int32_t> di(n, -1);
        for (int64_t q = 0; q < n_dirichlet; ++q) {
            OASIS_CHECK(dirichlet_dofs[q] >= 0 && dirichlet_dofs[q] < n, OASIS_EINVAL, "scalar dirichlet dof out of range");
            const int32_t i = S->m->internal_dof(dirichlet_dofs[q]);
            OASIS_CHECK(di[i] < 0, OASIS_EINVAL, "repeated scalar dirichlet dof");
            di[i] = (int32_t)q;
        }
        drop_graph(S);
        cudaStream_t s = nullptr;
        OASIS_CUDA(cudaDeviceSynchronize());
        const size_t vb = S->mixed ? sizeof(float) : sizeof(double), sb = 8;
        const int64_t nnz = S->m->nnz;
        const bool on = n_scalars > 0;
        S->ns = n_scalars;
        S->n_sdir = on ? n_dirichlet : 0;
        for (int al = 0; al < OASIS_MAX_SCALARS; ++al) {
            S->sc_diff[al] = al < n_scalars ? diffusivity[al] : 0.0;
            S->sc_src[al] = al < n_scalars ? source[al] : 0.0;
        }
        if (on) S->sdir_index.upload(di.data(), n, s);
        else S->sdir_index.alloc(0);
        S->c.alloc(on ? sb * n * n_scalars : 0, s);
        S->gc.alloc(on ? sb * std::max<int64_t>(1, n_dirichlet * n_scalars) : 0, s);
        S->cbar.alloc(on ? vb * nnz : 0, s);
        S->Ac.alloc(on ? vb * nnz : 0, s);
        S->dinvAc.alloc(on ? vb * n : 0, s);
        S->r0c.alloc(on ? sb * n : 0, s);
        S->dc.alloc(on ? sb * n : 0, s);
        for (auto& w : S->sw) w.alloc(on ? vb * n : 0, s);
        S->cstage.alloc(on ? (size_t)n_scalars * std::max<int64_t>(n, n_dirichlet) : 0);
        OASIS_CUDA(cudaMemsetAsync(S->st.p + 3, 0, OASIS_MAX_SCALARS * sizeof(KrylovState), s));
        OASIS_CUDA(cudaStreamSynchronize(s));
        S->impl->scalars_changed();
    });
}

int oasis_set_scalar_fields(oasis_solver* solver, const double* c, int32_t on_device, void* stream) {
    return guarded([&] {
        Solver* S = reinterpret_cast<Solver*>(solver);
        OASIS_CHECK(S && c, OASIS_EINVAL, "null pointer");
        OASIS_CHECK(S->ns > 0, OASIS_EINVAL, "no scalars (oasis_solver_set_scalars)");
        cudaStream_t s = as_stream(stream);
        const int64_t count = S->m->n * S->ns;
        const double* src = c;
        if (!on_device) {
            OASIS_CUDA(cudaMemcpyAsync(S->cstage.p, c, count * sizeof(double), cudaMemcpyHostToDevice, s));
            src = S->cstage.p;
        }
        S->impl->to_state(s, src, ST_C, count, 1, S->m->perm.p);
        OASIS_CUDA(cudaStreamSynchronize(s));
    });
}

int oasis_get_scalar_fields(oasis_solver* solver, double* c, int32_t on_device, void* stream) {
    return guarded([&] {
        Solver* S = reinterpret_cast<Solver*>(solver);
        OASIS_CHECK(S && c, OASIS_EINVAL, "null pointer");
        OASIS_CHECK(S->ns > 0, OASIS_EINVAL, "no scalars (oasis_solver_set_scalars)");
        cudaStream_t s = as_stream(stream);
        const int64_t count = S->m->n * S->ns;
        if (on_device) {
            S->impl->from_state(s, c, ST_C, count, 1, S->m->perm.p);
            return;
        }
        S->impl->from_state(s, S->cstage.p, ST_C, count, 1, S->m->perm.p);
        OASIS_CUDA(cudaMemcpyAsync(c, S->cstage.p, count * sizeof(double), cudaMemcpyDeviceToHost, s));
        OASIS_CUDA(cudaStreamSynchronize(s));
    });
}

int oasis_set_scalar_dirichlet(oasis_solver* solver, const double* g, int32_t on_device, void* stream) {
    return guarded([&] {
        Solver* S = reinterpret_cast<Solver*>(solver);
        OASIS_CHECK(S, OASIS_EINVAL, "null solver");
        OASIS_CHECK(S->ns > 0, OASIS_EINVAL, "no scalars (oasis_solver_set_scalars)");
        if (S->n_sdir == 0) return;
        OASIS_CHECK(g, OASIS_EINVAL, "null values");
        cudaStream_t s = as_stream(stream);
        const int64_t count = S->n_sdir * S->ns;
        const double* src = g;
        if (!on_device) {
            OASIS_CUDA(cudaMemcpyAsync(S->cstage.p, g, count * sizeof(double), cudaMemcpyHostToDevice, s));
            src = S->cstage.p;
        }
        S->impl->to_state(s, src, ST_GC, count, 1, nullptr);
        OASIS_CUDA(cudaStreamSynchronize(s));
    });
}

int oasis_step(oasis_solver* solver, void* stream, oasis_step_stats* stats) {
    int rc = guarded([&] {
        Solver* S = reinterpret_cast<Solver*>(solver);
        OASIS_CHECK(S, OASIS_EINVAL, "null solver");
        S->step(as_stream(stream));
        if (stats) {
            OASIS_CUDA(cudaStreamSynchronize(as_stream(stream)));
            fill_stats(*S, stats);
            if (stats->status != OASIS_OK)
                throw Error(stats->status, "step failed: status " + std::to_string(stats->status));
        }
    });
    return rc;
}

int oasis_last_stats(oasis_solver* solver, oasis_step_stats* stats) {
    return guarded([&] {
        Solver* S = reinterpret_cast<Solver*>(solver);
        OASIS_CHECK(S && stats, OASIS_EINVAL, "null pointer");
        OASIS_CUDA(cudaDeviceSynchronize());
        fill_stats(*S, stats);
        if (stats->status != OASIS_OK) throw Error(stats->status, "step failed: status " + std::to_string(stats->status));
    });
}

int oasis_get_fields(oasis_solver* solver, double* u, double* p, double* phi, int32_t on_device, void* stream) {
    return guarded([&] {
        Solver* S = reinterpret_cast<Solver*>(solver);
        OASIS_CHECK(S, OASIS_EINVAL, "null solver");
        cudaStream_t s = as_stream(stream);
        const int D = S->m->dim;
        const int64_t n = S->m->n;
        double* outs[3] = {u, p, phi};
        const int ids[3] = {ST_U1, ST_PSTAR, ST_PHI};
        const int comps[3] = {D, 1, 1};
        const int64_t at[3] = {0, (int64_t)D * n, (int64_t)(D + 1) * n};   // places in the stage
        // every field converted first, then the copies to the host, then one
        // synchronisation (a copy overlaps the next field's conversion)
        bool any = false;
        for (int q = 0; q < 3; ++q) {
            if (!outs[q]) continue;
            double* dst = on_device ? outs[q] : S->stage.p + at[q];
            S->impl->from_state(s, dst, ids[q], n, comps[q], S->m->perm.p);
            if (!on_device)
                OASIS_CUDA(cudaMemcpyAsync(outs[q], S->stage.p + at[q], n * comps[q] * sizeof(double),
                                           cudaMemcpyDeviceToHost, s));
            any = true;
        }
        if (any && !on_device) OASIS_CUDA(cudaStreamSynchronize(s));
    });
}

int oasis_get_tentative_system(oasis_solver* solver, double* A_values, double* r0, void* stream) {
    return guarded([&] {
        Solver* S = reinterpret_cast<Solver*>(solver);
        OASIS_CHECK(S, OASIS_EINVAL, "null solver");
        cudaStream_t s = as_stream(stream);
        const int D = S->m->dim;
        const int64_t n = S->m->n, nnz = S->m->nnz;
        S->impl->assemble(s);
        if (A_values) {
            DBuf<double> tmp;
            tmp.alloc(nnz);
            S->impl->a_to_double(s, tmp.p);
            std::vector<double> internal(nnz);
            OASIS_CUDA(cudaMemcpyAsync(internal.data(), tmp.p, nnz * sizeof(double), cudaMemcpyDeviceToHost, s));
            OASIS_CUDA(cudaStreamSynchronize(s));
            to_caller_order(*S->m, false, internal, A_values);
        }
        if (r0) {
            S->impl->from_state(s, S->stage.p, ST_R0, n, D, S->m->perm.p);
            OASIS_CUDA(cudaMemcpyAsync(r0, S->stage.p, n * D * sizeof(double), cudaMemcpyDeviceToHost, s));
        }
        OASIS_CUDA(cudaStreamSynchronize(s));
    });
}

int oasis_profile(oasis_solver* solver, int32_t enable) {
    return guarded([&] {
        Solver* S = reinterpret_cast<Solver*>(solver);
        OASIS_CHECK(S, OASIS_EINVAL, "null solver");
        S->prof_on = enable != 0;
        for (int f = 0; f < Solver::kProfFamilies; ++f) {
            S->prof_ms[f] = 0.0;
            S->prof_n[f] = 0;
        }
    });
}

int oasis_profile_read(oasis_solver* solver, int32_t family, int64_t* launches, double* total_ms) {
    return guarded([&] {
        Solver* S = reinterpret_cast<Solver*>(solver);
        OASIS_CHECK(S && launches && total_ms, OASIS_EINVAL, "null pointer");
        OASIS_CHECK(family >= 0 && family < Solver::kProfFamilies, OASIS_EINVAL, "unknown kernel family");
        *launches = S->prof_n[family];
        *total_ms = S->prof_ms[family];
    });
}

// ------------------------------------------------------------------ learned guess
static void drop_graph(Solver* S) {
    if (S->gexec) cudaGraphExecDestroy(S->gexec);
    if (S->graph) cudaGraphDestroy(S->graph);
    S->gexec = nullptr;
    S->graph = nullptr;
}

int oasis_net_create(const oasis_mesh* mesh, oasis_net** out) {
    return guarded([&] {
        const Mesh* m = reinterpret_cast<const Mesh*>(mesh);
        OASIS_CHECK(m && out, OASIS_EINVAL, "null pointer");
        *out = reinterpret_cast<oasis_net*>(net_create(*m));
    });
}

int oasis_net_set_params(oasis_net* net, const float* params) {
    return guarded([&] {
        Net* N = reinterpret_cast<Net*>(net);
        OASIS_CHECK(N && params, OASIS_EINVAL, "null pointer");
        net_set_params(*N, params);
    });
}

int oasis_net_get_params(const oasis_net* net, float* params) {
    return guarded([&] {
        const Net* N = reinterpret_cast<const Net*>(net);
        OASIS_CHECK(N && params, OASIS_EINVAL, "null pointer");
        OASIS_CUDA(cudaDeviceSynchronize());
        OASIS_CUDA(cudaMemcpy(params, N->p32.p, kNetParams * sizeof(float), cudaMemcpyDeviceToHost));
    });
}

int oasis_net_forward(oasis_net* net, const float* features, float* y, void* stream) {
    return guarded([&] {
        Net* N = reinterpret_cast<Net*>(net);
        OASIS_CHECK(N && features && y, OASIS_EINVAL, "null pointer");
        net_forward(*N, features, y, as_stream(stream));
        net_check(*N, as_stream(stream));
    });
}

int oasis_net_backward(oasis_net* net, const float* features, const float* target, float* grad, float* loss,
                       void* stream) {
    return guarded([&] {
        Net* N = reinterpret_cast<Net*>(net);
        OASIS_CHECK(N && features && target, OASIS_EINVAL, "null pointer");
        net_backward(*N, features, target, grad, loss, as_stream(stream));
    });
}

int oasis_net_adam(oasis_net* net, const float* grad, float lr, float beta1, float beta2, float eps, int32_t step,
                   void* stream) {
    return guarded([&] {
        Net* N = reinterpret_cast<Net*>(net);
        OASIS_CHECK(N && step >= 1 && lr > 0, OASIS_EINVAL, "bad arguments");
        net_adam(*N, grad, lr, beta1, beta2, eps, step, as_stream(stream));
    });
}

void oasis_net_destroy(oasis_net* net) {
    Net* N = reinterpret_cast<Net*>(net);
    if (N) {
        cudaDeviceSynchronize();
        delete N;
    }
}

int oasis_solver_set_guess_net(oasis_solver* solver, oasis_net* net) {
    return guarded([&] {
        Solver* S = reinterpret_cast<Solver*>(solver);
        OASIS_CHECK(S, OASIS_EINVAL, "null solver");
        Net* N = reinterpret_cast<Net*>(net);
        OASIS_CHECK(!N || N->m == S->m, OASIS_EINVAL, "the network was created on another mesh");
        S->net = N;
        drop_graph(S);
    });
}

int oasis_solver_record_guess(oasis_solver* solver, int32_t on) {
    return guarded([&] {
        Solver* S = reinterpret_cast<Solver*>(solver);
        OASIS_CHECK(S, OASIS_EINVAL, "null solver");
        S->record = on != 0;
        drop_graph(S);
    });
}

int oasis_get_guess_sample(oasis_solver* solver, float* features, float* target, void* stream) {
    return guarded([&] {
        Solver* S = reinterpret_cast<Solver*>(solver);
        OASIS_CHECK(S && features && target, OASIS_EINVAL, "null pointer");
        OASIS_CHECK(S->record || (S->prm.guess == OASIS_GUESS_LEARNED && S->net), OASIS_EINVAL,
                    "enable oasis_solver_record_guess (or a learned guess) before the step");
        cudaStream_t s = as_stream(stream);
        OASIS_CUDA(cudaMemcpyAsync(features, S->feat.p, S->feat.bytes(), cudaMemcpyDeviceToDevice, s));
        S->impl->guess_target(s, target);
    });
}

int oasis_get_amg_info(const oasis_solver* solver, oasis_amg_info* out) {
    return guarded([&] {
        const Solver* S = reinterpret_cast<const Solver*>(solver);
        OASIS_CHECK(S && out, OASIS_EINVAL, "null pointer");
        OASIS_CHECK(S->prm.pressure_pc == OASIS_PC_AMG && S->m->amg, OASIS_EINVAL,
                    "the solver was not created with OASIS_PC_AMG");
        std::memset(out, 0, sizeof(*out));
        const AmgHierarchy& h = *S->m->amg;
        out->levels = (int32_t)std::min<size_t>(16, h.sizes.size());
        for (int k = 0; k < out->levels; ++k) {
            out->rows[k] = h.sizes[k];
            out->nnz[k] = h.nnzs[k];
            out->p_nnz[k] = k < (int)h.pnnzs.size() ? h.pnnzs[k] : 0;
            if (k < (int)h.lv.size()) {
                const AmgLevelDev& lv = *h.lv[k];
                out->packed[k] = (lv.sa.n > 0 ? 1 : 0) | (lv.sr.n > 0 ? 2 : 0) | (lv.sp.n > 0 ? 4 : 0) |
                                 (lv.sa.wide ? 8 : 0) | (lv.sr.wide ? 16 : 0) | (lv.sp.wide ? 32 : 0);
            }
        }
        out->setup_s = h.setup_s;
    });
}

int oasis_amg_apply(oasis_solver* solver, const void* r, void* u, void* stream) {
    return guarded([&] {
        Solver* S = reinterpret_cast<Solver*>(solver);
        OASIS_CHECK(S && r && u, OASIS_EINVAL, "null pointer");
        OASIS_CHECK(S->prm.pressure_pc == OASIS_PC_AMG && S->m->amg, OASIS_EINVAL,
                    "the solver was not created with OASIS_PC_AMG");
        cudaStream_t s = as_stream(stream);
        S->impl->amg_apply(s, r, u);
        OASIS_CUDA(cudaStreamSynchronize(s));
    });
}

int oasis_get_tuning(const oasis_solver* solver, oasis_tuning* out) {
    return guarded([&] {
        const Solver* S = reinterpret_cast<const Solver*>(solver);
        OASIS_CHECK(S && out, OASIS_EINVAL, "null pointer");
        std::memset(out, 0, sizeof(*out));
        S->impl->tuning(out);
    });
}

void oasis_solver_destroy(oasis_solver* solver) {
    Solver* S = reinterpret_cast<Solver*>(solver);
    if (S) {
        cudaDeviceSynchronize();
        delete S;
    }
}

void oasis_mesh_destroy(oasis_mesh* mesh) {
    Mesh* m = reinterpret_cast<Mesh*>(mesh);
    if (m) {
        cudaDeviceSynchronize();
        delete m;
    }
}

}  // extern "C"
