/*
 * oasis.h -- C ABI of the GB300 (sm_103a) P1-P1 incremental pressure-correction
 * (IPCS, "ABCN" convection) Navier-Stokes time step on simplex meshes.
 *
 * The scheme is the fractional-step method of Sec. 2 (Eqs. 17-19, convection
 * Eq. 22 or Eq. 21, Algorithm 1 with one or more inner iterations), discretised
 * with P1 elements for velocity and pressure as in Sec. 3, and organised as the
 * high-performance solver of Sec. 5: constant matrices M, K, dP^k preassembled
 * once, the convection matrix reassembled every step into the fixed sparsity
 * pattern and combined with M and K by Algorithm 2, a Krylov solve per velocity
 * component with one shared coefficient matrix (Eq. 35), a pressure-correction
 * Poisson solve (Sec. 5, the algebraic form of Eq. 18), the velocity update
 * with the lumped or the consistent mass matrix (Sec. 5), and optional passive
 * scalars (the scalar equation of Sec. 3).
 *
 * Conventions shared by every entry point
 *   - Return value: 0 on success, a negative OASIS_E* code on failure.  No C++
 *     exception crosses the ABI.  oasis_last_error() returns a thread-local
 *     message describing the last failure of the calling thread.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     All device work of a call is ordered on that stream.
 *   - Host arrays are read during the call only and never retained.  Device
 *     memory behind oasis_mesh / oasis_solver is allocated by the library at
 *     creation time (and by the configuration call oasis_solver_set_scalars)
 *     and released by the matching destroy call.  The field copies and the
 *     kernels of oasis_step allocate no device memory; the first oasis_step of
 *     a graph-mode solver captures and instantiates the step's CUDA graph, and
 *     the test hooks oasis_get_tentative_system and oasis_amg_apply use
 *     temporary buffers.
 *   - Fields are float64, component-major: u[k * n_dofs + i] is component k of
 *     dof i.  Indices are int32, zero based.
 *   - Dof order.  Every per-dof array and dof index that crosses a field call
 *     (oasis_set_fields, oasis_get_fields, oasis_set_scalar_fields,
 *     oasis_get_scalar_fields, oasis_get_tentative_system, the Dirichlet dof
 *     lists of oasis_solver_create and oasis_solver_set_scalars) and the pattern
 *     and matrices of oasis_mesh_get_pattern / oasis_mesh_get_matrix are in the
 *     CALLER's dof order.  The library stores and computes in its internal order,
 *     the caller's renumbered by the `perm` of oasis_mesh_create (identical when
 *     perm is NULL).  The kernel-level vector entry points (oasis_spmv_*,
 *     oasis_net_forward / _backward, oasis_get_guess_sample, oasis_amg_apply)
 *     exchange device vectors in the internal order: entry perm[d] belongs to
 *     caller dof d.
 *   - Handles are not reentrant: calls on one solver must not overlap.
 *     Different solvers (and meshes) are independent.
 */
#ifndef OASIS_H
#define OASIS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define OASIS_OK 0
#define OASIS_EINVAL (-1)      /* bad argument (null pointer, size, index out of range) */
#define OASIS_ECUDA (-2)       /* a CUDA runtime call failed */
#define OASIS_EMESH (-3)       /* degenerate cell or a cell with repeated dofs */
#define OASIS_ENOTCONV (-4)    /* a Krylov solve hit its iteration cap */
#define OASIS_EBREAKDOWN (-5)  /* BiCGStab/CG breakdown (a zero inner product) */
#define OASIS_ENAN (-6)        /* a non-finite value appeared in a solve */
#define OASIS_ENOMEM (-7)      /* device allocation failed at creation time */
#define OASIS_EWAIT (-8)       /* a bounded device-side wait exceeded its time limit (~2 s);
                                  the kernel returned without hanging */

#define OASIS_FP64 0           /* every value and every operation in float64 */
#define OASIS_MIXED 1          /* float32 matrices and inner Krylov iterations inside
                                  float64 iterative refinement (float64 residual,
                                  float64 dot-product accumulation, float64 geometry) */

#define OASIS_GUESS_ZERO 0     /* pressure solve starts from phi = 0, i.e. p = p* */
#define OASIS_GUESS_PREV_PHI 1 /* starts from the previous step's correction phi */
#define OASIS_GUESS_LEARNED 2  /* starts from the network's guess (oasis_solver_set_guess_net)
                                  when its residual ||b - K phi0|| is smaller than that of
                                  the fallback phi^{n-1} (the residual is the judge) */

#define OASIS_MAT_M 0          /* M_ij = int phi_j phi_i            (Sec. 5) */
#define OASIS_MAT_K 1          /* K_ij = int grad phi_j . grad phi_i (Sec. 5) */
#define OASIS_MAT_G0 2         /* dP^k_ij = int d_k phi_j phi_i, k = 0, 1, 2 (Eq. 31) */
#define OASIS_MAT_G1 3
#define OASIS_MAT_G2 4
#define OASIS_MAT_A 5          /* coefficient matrix of Eq. 35 after the last assembly */

typedef struct oasis_mesh oasis_mesh;
typedef struct oasis_solver oasis_solver;

/* Parameters of the scheme and of its solvers. */
typedef struct oasis_params {
    double nu;             /* kinematic viscosity */
    double dt;             /* time step (constant, Sec. 2) */
    double f[3];           /* constant body force; int f_k phi_i = f_k * ML_i */
    double rtol_u;         /* tentative velocity: stop when ||r|| <= rtol_u ||r_0||,
                              r_0 = b - A u^{n-1}; the iteration starts from the
                              extrapolation 2 u^{n-1} - u^{n-2} */
    double rtol_p;         /* pressure correction: stop when ||r|| <= rtol_p ||b_phi||,
                              b_phi the right-hand side (the residual of phi = 0) */
    int32_t max_it_u;      /* cap on BiCGStab iterations per solve (all sweeps) */
    int32_t max_it_p;      /* cap on CG iterations per solve (all sweeps) */
    int32_t precision;     /* OASIS_FP64 or OASIS_MIXED */
    double inner_rtol;     /* OASIS_MIXED: relative reduction asked of each float32 inner
                              solve before the float64 residual is recomputed */
    int32_t batch_rhs;     /* 1: the d velocity components in one d-RHS BiCGStab
                              (one matrix read per product); 0: one solve per component */
    int32_t use_graph;     /* 1: the whole step runs as one CUDA graph, Krylov loops as
                              conditional WHILE nodes; 0: eager launches with host polls */
    int32_t guess;         /* OASIS_GUESS_* */
    int32_t spmv_variant;  /* shape of the pressure-CG product kernel (the fused Jacobi
                              iteration, or the multigrid CG product with OASIS_PC_AMG):
                              0 = autotune at solver creation (every candidate timed on
                              this matrix, the fastest kept); k >= 1 = candidate k of
                              oasis_get_tuning */
    int32_t pressure_pc;   /* OASIS_PC_JACOBI or OASIS_PC_AMG (preconditioner of the
                              pressure CG) */
    int32_t inner_iters;   /* inner velocity/pressure iterations of Algorithm 1 (0 or 1 =
                              one): the tentative and pressure solves are repeated with
                              p* = the newest pressure (A unchanged), the last pressure
                              increment drives the velocity update.  Repetitions after the
                              first start the pressure solve from zero.  The statistics of
                              a step describe its last repetition.  At most 16. */
    int32_t convection;    /* OASIS_CONV_ABCN (Eq. 22, default) or OASIS_CONV_ABE (Eq. 21) */
    int32_t velocity_update; /* OASIS_UPDATE_LUMPED (default) or OASIS_UPDATE_CONSISTENT */
    int32_t bicg_variant;  /* shape of the d-RHS product of the batched tentative BiCGStab:
                              0 = autotune at solver creation (every candidate timed on this
                              mesh's pattern, the fastest kept); k >= 1 = candidate k of
                              oasis_get_tuning's bicg_* fields.  The shapes add a row's
                              products in different orders: they agree to rounding, and a
                              solver keeps its shape for its life. */
} oasis_params;

/* Velocity update of the projection (Sec. 5).  LUMPED: u_k^n = u_k^I - dt
 * (dP^k phi) / ML, one pass.  CONSISTENT: M u_k^n = M u_k^I - dt dP^k phi with
 * Dirichlet rows u^n = g, solved for the increment u^n - u^I by a d-RHS CG on the
 * interior block of M with the lumped mass as preconditioner (a multiple of
 * diag M for P1 elements), started from the lumped increment and stopped at
 * ||r|| <= tol ||dt dP^k phi|| per component (interior rows), tol = rtol_u for
 * OASIS_FP64 and max(rtol_u, 1e-6) for OASIS_MIXED, whose solve runs in float32
 * (the increment is O(dt), so its float32 error stays far below that of u^n).
 * The solve's iterations count against max_it_u; hitting the cap sets the
 * step's status to OASIS_ENOTCONV. */
#define OASIS_UPDATE_LUMPED 0
#define OASIS_UPDATE_CONSISTENT 1

/* Convection forms (Sec. 3).  ABCN: B = ubar . grad u~ with ubar = 1.5 u^{n-1} -
 * 0.5 u^{n-2} and the Crank-Nicolson u~, implicit: A = M/dt + C(ubar)/2 + nu K/2.
 * ABE: explicit Adams-Bashforth B = 1.5 u^{n-1}.grad u^{n-1} - 0.5 u^{n-2}.grad u^{n-2}
 * on the right-hand side: A = M/dt + nu K/2 (the same matrix every step). */
#define OASIS_CONV_ABCN 0
#define OASIS_CONV_ABE 1

/* Preconditioners of the pressure CG.  The paper preconditions its pressure solve
 * with algebraic multigrid (Sec. 6); OASIS_PC_AMG is a smoothed-aggregation
 * hierarchy of K built once per mesh on the host (strength threshold 0.08,
 * greedy aggregation, Jacobi-smoothed prolongator, Galerkin coarse operators,
 * dense coarsest level <= 2048 dofs) applied as one V(1,1) cycle with damped
 * Jacobi smoothing: a symmetric positive semi-definite preconditioner. */
#define OASIS_PC_JACOBI 0
#define OASIS_PC_AMG 1

/* Candidate shapes of the pressure-CG product kernel (SELL-32, one warp per
 * 32 rows; with OASIS_PC_AMG the multigrid CG product, whose candidates vary
 * the entries per lane and the blocks per SM only) and what the autotuner
 * measured.  A shape is the number of entries
 * per lane whose column/value loads are issued before their gathers, the
 * resident blocks per SM that the register budget is sized for, whether the
 * next chunk's loads are issued before the current products (prefetch), and
 * whether columns are read as 16-bit offsets from the row taken modulo the dof
 * count (col16 = 1; only where every offset fits, else the candidate is not
 * timed; col16 = 2: the float32 multigrid CG product on the pair-packed copy of
 * K, two entries' values and offsets per load, where the multigrid hierarchy
 * has one; chunk is then entries per round),
 * and whether the slice's values and columns are streamed into shared memory
 * by the bulk-copy engine, two slices ahead per warp (streamed). */
#define OASIS_MAX_VARIANTS 16
typedef struct oasis_tuning {
    int32_t n_variants;
    int32_t chosen;                        /* 1-based candidate in use */
    int32_t chunk[OASIS_MAX_VARIANTS];
    int32_t min_blocks[OASIS_MAX_VARIANTS];
    int32_t prefetch[OASIS_MAX_VARIANTS];
    int32_t col16[OASIS_MAX_VARIANTS];
    int32_t streamed[OASIS_MAX_VARIANTS];  /* 1: values and columns streamed into shared
                                              memory by bulk copies (persistent grid) */
    int32_t warps_per_block[OASIS_MAX_VARIANTS];
    double us[OASIS_MAX_VARIANTS];         /* median time per launch; 0 if not timed */
    /* The d-RHS product of the batched tentative BiCGStab (both products of one
     * iteration timed together): lanes = 0 is the row-tile form (rows per tile in
     * bicg_rows, the entries of a tile read coalesced and summed per row through
     * shared memory); lanes = G > 0 is the row-split form, G lanes per row and
     * bicg_rows rows in flight per lane group, its registers capped for
     * bicg_min_blocks resident blocks per SM (1: no cap); bicg_col16 = 1: the
     * columns are read as 16-bit offsets from the row, modulo n (only where every
     * neighbour of the mesh's ordering fits; not timed, us = 0, elsewhere). */
    int32_t bicg_n_variants;
    int32_t bicg_chosen;                   /* 1-based */
    int32_t bicg_lanes[8];
    int32_t bicg_rows[8];
    int32_t bicg_min_blocks[8];
    double bicg_us[8];                     /* median time of the two products; 0 if not timed */
    int32_t bicg_col16[8];
} oasis_tuning;

/* Per-step solver statistics. */
typedef struct oasis_step_stats {
    int32_t status;        /* OASIS_OK or the failing OASIS_E* code of the step */
    int32_t it_u[3];       /* BiCGStab iterations per velocity component */
    int32_t sweeps_u;      /* refinement sweeps (float64 residual evaluations) */
    int32_t it_p;          /* CG iterations of the pressure solve */
    int32_t sweeps_p;
    int32_t guess_used;    /* OASIS_GUESS_* actually used this step */
    double res_u[3];       /* final ||r|| / ||r_0|| per component (float64 residual) */
    double res_p;          /* final ||r|| / ||b_phi|| */
    double t;              /* time t^n reached by the step */
    double guess_res[2];   /* OASIS_GUESS_LEARNED: ||b - K phi0|| / ||b|| of the network's
                              guess [0] and of the fallback phi^{n-1} [1]; else 0 */
    double res_m[3];       /* OASIS_UPDATE_CONSISTENT: final recurrence ||r|| / ||dt dP^k phi||
                              of the mass solve per component; else 0 */
    int32_t it_m;          /* OASIS_UPDATE_CONSISTENT: CG iterations of the mass solve */
    int32_t it_c;          /* passive scalars: most BiCGStab iterations over the scalars */
    double res_c;          /* passive scalars: largest final ||r|| / ||r_0|| over the scalars */
} oasis_step_stats;

/* Library version (major * 10000 + minor * 100 + patch). */
int oasis_version(void);

/* Message of the last failure on this thread ("" if none).  Owned by the library. */
const char* oasis_last_error(void);

/* Create a P1 mesh.
 *   dim           2 (triangles) or 3 (tetrahedra)
 *   coords        host, [n_vertices][dim] vertex coordinates
 *   cells         host, [n_cells][dim+1] vertex indices, any orientation
 *   dof_of_vertex host, [n_vertices] dof of each vertex, or NULL for the identity
 *                 (periodic meshes identify image vertices through this map)
 *   n_dofs        number of dofs (max(dof_of_vertex) + 1; n_vertices if the map is NULL)
 *   perm          host, [n_dofs] or NULL: a renumbering of the dofs (for example
 *                 reverse Cuthill-McKee, for locality of the sparse products),
 *                 perm[d] = the library's internal index of the caller's dof d.
 *                 It must be a permutation of 0 .. n_dofs-1.  The library stores
 *                 the pattern, the matrices and the state in that internal order;
 *                 the field calls still take and return the caller's order (see
 *                 "Dof order" above), so results do not depend on perm beyond
 *                 the solvers' tolerances (the order of floating-point sums and
 *                 the multigrid aggregation follow the internal numbering).
 * Builds the shared CSR sparsity pattern of all matrices (Sec. 5: "computed on
 * the first assemble"; the assembled system's dof numbering is free, Sec. 5) and
 * the dof-to-cell incidence used by the assembly kernels; copies everything to
 * the current device.  The cells are stored in the order of their lowest
 * internal dof (ties in the given order), so the given cell order matters only
 * through the order of floating-point sums.
 * Errors: OASIS_EINVAL (sizes, out-of-range index, perm not a permutation),
 * OASIS_EMESH (a cell whose dofs repeat, or more than 255 pattern entries in one
 * row), OASIS_ENOMEM. */
int oasis_mesh_create(int32_t dim, int64_t n_vertices, const double* coords, int64_t n_cells,
                      const int32_t* cells, const int32_t* dof_of_vertex, int64_t n_dofs,
                      const int32_t* perm, oasis_mesh** out);

/* Sizes of the mesh and of its sparsity pattern (any pointer may be NULL). */
int oasis_mesh_info(const oasis_mesh* mesh, int64_t* n_dofs, int64_t* n_cells, int64_t* nnz);

/* Preassemble the constant matrices of Sec. 5 on the device: M, K, dP^k
 * (k < dim) and the lumped mass ML_i = sum_j M_ij (Sec. 5, velocity update),
 * plus the per-cell float64 geometry (Jacobian inverse, volume) reused by the
 * per-step convection assembly.  Deterministic (no atomics).
 * Errors: OASIS_EMESH if a cell has zero volume; OASIS_ECUDA. */
int oasis_assemble_constant(oasis_mesh* mesh, void* stream);

/* Copy the sparsity pattern to host in the caller's dof order: row_ptr [n_dofs+1],
 * col [nnz] (sorted per row). */
int oasis_mesh_get_pattern(const oasis_mesh* mesh, int32_t* row_ptr, int32_t* col);

/* Copy the float64 values of a constant matrix (OASIS_MAT_M, _K, _G0.._G2) to a
 * host array [nnz] in the order of oasis_mesh_get_pattern (caller's dof order), or
 * with which = -1 the lumped mass [n_dofs].  Synchronises the device. */
int oasis_mesh_get_matrix(const oasis_mesh* mesh, int32_t which, double* values);

/* y = Mat x on device vectors of length n_dofs (float64, internal dof order), Mat
 * one of the constant matrices, with `lanes` lanes per row (0 = 16).  For
 * kernel-level tests and bandwidth measurements. */
int oasis_spmv_f64(const oasis_mesh* mesh, int32_t which, const double* x, double* y,
                   int32_t lanes, void* stream);
/* Same in float32 values and vectors (the values are the float32 copy of the matrix). */
int oasis_spmv_f32(const oasis_mesh* mesh, int32_t which, const float* x, float* y,
                   int32_t lanes, void* stream);

/* y = Mat x and *xy = x . y in float64 (for K this is the energy product p . K p
 * of the CG iteration, Sec. 6 solvers), on device vectors of length n_dofs; xy
 * is one double in device memory.  Row tiles of 256 rows, one partial sum per
 * tile in scratch owned by the mesh (allocated by oasis_assemble_constant), and
 * a deterministic final sum in tile order.  Calls on one mesh must not overlap
 * on the GPU (they share that scratch). */
int oasis_spmv_dot_f64(const oasis_mesh* mesh, int32_t which, const double* x, double* y, double* xy,
                       void* stream);

/* The same product and dot as oasis_spmv_dot_f64, for callers that cannot
 * allocate device memory (code that runs under a caller-owned memory pool, inside
 * an allocator, or on a device whose memory is already committed): this call
 * allocates nothing.  The paper has no counterpart; it is a deployment variant.
 *   - Its reduction scratch is a file-scope __device__ array of 516 KiB that
 *     every GPU loading the library holds until process exit; it limits n_dofs
 *     to 16,777,216 (65,536 tiles of 256 rows).  Larger meshes: OASIS_EINVAL.
 *   - The first call on a device resolves the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture.
 *   - Every call on every mesh shares the one array, and it keeps the last
 *     call's contents (the ticket word that must start at zero is cleared by
 *     each call, on `stream`).  Calls that overlap on the GPU race: order them
 *     on one stream or synchronise between them. */
int oasis_spmv_dot_f64_noalloc(const oasis_mesh* mesh, int32_t which, const double* x, double* y, double* xy,
                               void* stream);

/* Create a solver on an assembled mesh.
 *   dirichlet_dofs host, [n_dirichlet] distinct dofs carrying velocity Dirichlet
 *                  values (the same set for every component, Sec. 5 after Eq. 35)
 * The pressure has no Dirichlet condition: its right-hand side is projected on
 * sum_i b_i = 0 and p is normalised to zero mean after each solve.
 * Allocates every device buffer the step needs (no allocation afterwards).
 * With spmv_variant = 0 the CG iteration kernel is autotuned here (timed on
 * `stream`; every candidate computes the same sums in the same order, so the
 * choice changes the speed, not the result). */
int oasis_solver_create(oasis_mesh* mesh, const oasis_params* params, int64_t n_dirichlet,
                        const int32_t* dirichlet_dofs, void* stream, oasis_solver** out);

/* Set the state before a step: u^{n-1}, u^{n-2} ([dim][n_dofs]), the tentative
 * pressure p* = p^{n-3/2} ([n_dofs]) and the time t^{n-1}.  on_device = 1: the
 * pointers are device pointers; 0: host pointers (copied synchronously).
 * Resets the pressure-correction history used by the guesses. */
int oasis_set_fields(oasis_solver* s, const double* u_nm1, const double* u_nm2, const double* p,
                     double t, int32_t on_device, void* stream);

/* Set the velocity Dirichlet values g[k * n_dirichlet + m] for dof dirichlet_dofs[m]
 * at the time t^n of the next step.  Values persist until the next call. */
int oasis_set_dirichlet(oasis_solver* s, const double* g, int32_t on_device, void* stream);

/* Advance one time step (Algorithm 1; params.inner_iters repetitions):
 *   assemble C into A and form the tentative right-hand side (Algorithm 2),
 *   solve A u_k^I = b_k for the dim components, solve the pressure correction,
 *   solve the passive scalars if any (oasis_solver_set_scalars), normalise p,
 *   update u (params.velocity_update), rotate u^{n-2} <- u^{n-1} <- u^n and
 *   p* <- p.
 * If stats is NULL the call only enqueues work on `stream` and returns OASIS_OK;
 * a failure of the step is reported by the next oasis_last_stats().  If stats is
 * non-NULL the call waits for the step and returns its status. */
int oasis_step(oasis_solver* s, void* stream, oasis_step_stats* stats);

/* Wait for the last step and return its statistics and status. */
int oasis_last_stats(oasis_solver* s, oasis_step_stats* stats);

/* ---- Passive scalars (the scalar equation of Sec. 3) -------------------------
 * Scalar alpha with diffusivity D_a and constant source f_a is advanced after the
 * tentative and pressure solves of every step (Algorithm 1 solves it after the
 * velocity correction; it uses only the old velocities, so the order is free):
 *   A_a = M/dt + C(ubar)/2 + D_a K/2,  ubar = 1.5 u^{n-1} - 0.5 u^{n-2} (whichever
 *   convection form the velocity uses), b_a = (M/dt - C/2 - D_a K/2) c^{n-1} + f_a ML,
 *   rows of the scalars' Dirichlet set: unit rows, c^n = g_a(t^n) (values re-imposed
 *   after the solve).
 * Solved in delta form A_a (c^n - c^{n-1}) = b_a - A_a c^{n-1} by the tentative
 * solver's BiCGStab (Jacobi, refinement in OASIS_MIXED) with rtol_u and max_it_u.
 * C(ubar) is kept from the velocity assembly (one extra nnz array).
 *
 * oasis_solver_set_scalars: n_scalars in [0, OASIS_MAX_SCALARS] (0 removes them);
 * diffusivity and source host arrays [n_scalars] (D_a >= 0); dirichlet_dofs host
 * [n_dirichlet], distinct, in range (may differ from the velocity's set).  The
 * fields start at 0 and the Dirichlet values at 0.  Drops a captured graph.
 * Errors: OASIS_EINVAL (sizes, index, negative diffusivity), OASIS_ENOMEM. */
#define OASIS_MAX_SCALARS 8
int oasis_solver_set_scalars(oasis_solver* s, int32_t n_scalars, const double* diffusivity,
                             const double* source, int64_t n_dirichlet, const int32_t* dirichlet_dofs);
/* c[a * n_dofs + i] = c_a at dof i (float64; on_device as for oasis_set_fields). */
int oasis_set_scalar_fields(oasis_solver* s, const double* c, int32_t on_device, void* stream);
int oasis_get_scalar_fields(oasis_solver* s, double* c, int32_t on_device, void* stream);
/* g[a * n_dirichlet + m]: value of scalar a at dirichlet_dofs[m] at the time t^n of
 * the next step.  Values persist until the next call. */
int oasis_set_scalar_dirichlet(oasis_solver* s, const double* g, int32_t on_device, void* stream);

/* Copy out the current state: u = u^n ([dim][n_dofs]), p = p^{n-1/2} ([n_dofs]),
 * phi = p^{n-1/2} - p* ([n_dofs]); any of them may be NULL.  on_device as above.
 * Synchronises `stream` when copying to host. */
int oasis_get_fields(oasis_solver* s, double* u, double* p, double* phi, int32_t on_device,
                     void* stream);

/* Run only the assembly of the next step (Algorithm 2) on the current state and
 * copy to host the coefficient matrix A [nnz] (in the order of
 * oasis_mesh_get_pattern; Dirichlet rows already unit rows) and the initial
 * tentative residual r0 = b - A u^{n-1} ([dim][n_dofs], caller's dof order).  The
 * state is not advanced.  For parity tests. */
int oasis_get_tentative_system(oasis_solver* s, double* A_values, double* r0, void* stream);

/* ---- Learned initial guess for the pressure-correction solve -------------------
 * The paper has no learned component: this is a project addition.  A two-layer
 * message-passing network on the sparsity graph of the mesh (width 32, bfloat16
 * weights, float32 accumulation) maps per-dof inputs
 *   x_i = (b_i / s_b, phi^{n-1}_i / s_phi, phi^{n-2}_i / s_phi),
 * b the projected right-hand side, s_b = rms(b), s_phi = rms(phi^{n-1}), to y_i;
 * the guess is phi0 = s_phi y.  Training minimises mean (y_i - phi_i / s_phi)^2.
 * Parameters: 2339 floats in the order W1a[32][3], W1b[32][3], c1[32],
 * W2a[32][32], W2b[32][32], c2[32], w3[32], c3, a[2]. */
#define OASIS_NET_PARAMS 2339
typedef struct oasis_net oasis_net;

/* Network with work buffers for the mesh's dofs; parameters start at zero. */
int oasis_net_create(const oasis_mesh* mesh, oasis_net** out);
/* Set / get the float32 master parameters (host arrays of OASIS_NET_PARAMS);
 * setting also refreshes the bfloat16 copy used by the kernels and resets Adam. */
int oasis_net_set_params(oasis_net* net, const float* params);
int oasis_net_get_params(const oasis_net* net, float* params);
/* y = net(features); device arrays [n_dofs][3] and [n_dofs].  Layer 2's dense
 * product runs on the tensor cores (tcgen05, bfloat16 weights, float32
 * accumulation, float32 activations split into three bfloat16 terms).  Waits for
 * `stream`; OASIS_EWAIT if the kernel's bounded wait for the tensor core ran out
 * (y is then incomplete). */
int oasis_net_forward(oasis_net* net, const float* features, float* y, void* stream);
/* Gradient of the loss with respect to the parameters (device [OASIS_NET_PARAMS],
 * or NULL for the network's own buffer) and the loss (device [1] or NULL) for one
 * sample (features, target: device). */
int oasis_net_backward(oasis_net* net, const float* features, const float* target, float* grad, float* loss,
                       void* stream);
/* One Adam step (Kingma & Ba) with the given gradient (device, NULL = own buffer). */
int oasis_net_adam(oasis_net* net, const float* grad, float lr, float beta1, float beta2, float eps,
                   int32_t step, void* stream);
void oasis_net_destroy(oasis_net* net);
/* Attach a network (or NULL) to a solver created on the same mesh; used when
 * params.guess == OASIS_GUESS_LEARNED.  Drops a captured graph (recaptured at the
 * next step). */
int oasis_solver_set_guess_net(oasis_solver* s, oasis_net* net);
/* on = 1: compute the network inputs every step, so that oasis_get_guess_sample
 * can return training samples. */
int oasis_solver_record_guess(oasis_solver* s, int32_t on);
/* Training sample of the last step: the inputs [n_dofs][3] and the target
 * phi / s_phi [n_dofs] (device arrays). */
int oasis_get_guess_sample(oasis_solver* s, float* features, float* target, void* stream);

/* Multigrid hierarchy of a solver created with OASIS_PC_AMG. */
typedef struct oasis_amg_info {
    int32_t levels;                /* operator levels, the dense coarsest one included */
    int64_t rows[16];
    int64_t nnz[16];
    double setup_s;                /* host setup time (once per mesh) */
    int64_t p_nnz[16];             /* entries of the prolongation from level k+1 to level k
                                      (k < levels - 1); its transpose, the restriction, has
                                      as many */
    int32_t packed[16];            /* operators of level k that the float32 cycle reads in
                                      pair-packed SELL-32 form (bfloat16 values, 16-bit
                                      column offsets) instead of CSR: bit 0 the level's
                                      matrix, bit 1 the restriction to level k+1, bit 2 the
                                      prolongation from it; bits 3, 4, 5: that copy keeps
                                      32-bit columns (its columns spread too far) */
} oasis_amg_info;
int oasis_get_amg_info(const oasis_solver* s, oasis_amg_info* out);

/* u = M r with one V-cycle of the solver's hierarchy, in the solver's inner
 * precision (float64 for OASIS_FP64, float32 for OASIS_MIXED); r, u device
 * arrays of n_dofs values.  Synchronises `stream`.  Test hook. */
int oasis_amg_apply(oasis_solver* s, const void* r, void* u, void* stream);

/* What the autotuner of oasis_solver_create chose for this solver. */
int oasis_get_tuning(const oasis_solver* s, oasis_tuning* out);

/* Kernel families timed by oasis_profile (eager mode only; graph steps are not
 * instrumented). */
#define OASIS_PROF_PCG_SPMV 0      /* fused pressure-CG iteration: w = K M^-1 r on SELL-32
                                      with the vector updates and the three dot products */
#define OASIS_PROF_BICG_SPMM 1     /* the d-RHS products of the tentative BiCGStab */
#define OASIS_PROF_ASSEMBLE 2      /* fused convection assembly + Algorithm 2 row pass */
#define OASIS_PROF_PCG_UPDATE 3    /* Jacobi CG: start of each refinement sweep (w0 = K M^-1 r0,
                                      dots); multigrid CG: the vector update of every iteration
                                      (p, s, the increment, r and ||r||^2) */
#define OASIS_PROF_UPDATE 4        /* velocity update (lumped, or the final pass of the
                                      consistent one) + rotation */
#define OASIS_PROF_PRESSURE_RHS 5  /* pressure right-hand side */
#define OASIS_PROF_GUESS 6         /* learned guess: input scaling, network forward, judge */
#define OASIS_PROF_AMG 7           /* multigrid V-cycles of the pressure CG */
#define OASIS_PROF_MASS 8          /* consistent-mass update: the mass CG's start and iterations */
/* Parts of OASIS_PROF_AMG (each V-cycle kernel is counted in one of them): */
#define OASIS_PROF_AMG_FINE 9      /* smoothing sweeps of the finest level (the mesh's K) */
#define OASIS_PROF_AMG_TRANSFER 10 /* restriction P^T and prolongation P, every level */
#define OASIS_PROF_AMG_COARSE 11   /* smoothing sweeps of the coarser levels and the dense
                                      coarsest solve */
#define OASIS_PROF_BICG_VEC 12     /* vector kernels of the tentative BiCGStab iteration (search
                                      direction, s update, solution/residual update + dots) */
#define OASIS_PROF_OUTER 13        /* float64-quality residuals of the refinement sweeps (the
                                      tentative solve's r = r0 - A Delta and the pressure's
                                      r = b - K x) */

/* enable = 1: from now on, eager steps record CUDA events around the launches
 * of the kernel families above; the counters are reset by every call. */
int oasis_profile(oasis_solver* s, int32_t enable);

/* Launch count and summed device time (ms) of one kernel family since the last
 * oasis_profile call. */
int oasis_profile_read(oasis_solver* s, int32_t family, int64_t* launches, double* total_ms);

void oasis_solver_destroy(oasis_solver* s);
void oasis_mesh_destroy(oasis_mesh* mesh);

#ifdef __cplusplus
}
#endif
#endif /* OASIS_H */
