/*
 * fvgb.h -- C ABI of libfvgb, a GB300 (sm_103a) finite-volume PISO / SIMPLE
 * solver core for incompressible flow on unstructured, face-addressed meshes.
 *
 * Method: T. Tomczak, K. Zadarnowska, Z. Koza, M. Matyka, L. Miroslaw,
 * "Complete PISO and SIMPLE solvers on Graphics Processing Units".
 *   Sec. 3    PISO (momentum solve, then pressure solves with explicit
 *             velocity corrections) and SIMPLE (the steady-state variant),
 *             finite-volume discretisation; Jacobi-preconditioned CG for the
 *             pressure equation, Jacobi-preconditioned BiCGStab for momentum.
 *   Sec. 3.1  mesh model: N cells, every face shared by two cells or on the
 *             boundary; A_ij != 0 iff cells i, j share a face or i == j; the
 *             matrix is accessed by rows (SMVP) and by columns.
 *   Sec. 4.2  double precision.
 *
 * Conventions for every call:
 *  - Every function returns an fv_status; no exception or abort crosses the
 *    ABI.  On error, fv_last_error() returns a thread-local message.
 *  - "host" pointers are CPU memory, read or written before the call returns;
 *    "device" pointers are CUDA global memory on the current device, borrowed
 *    for the duration of the call only.  The library owns all mesh, case and
 *    solver memory, allocated at create time; no step allocates.
 *  - Arrays of 3-vectors are component-major (SoA): x[c * n + i].
 *  - Indices are int32; floating point is IEEE double unless stated.
 *  - Work is enqueued on the CUDA stream given at create time (NULL = legacy
 *    default stream).  Calls that return statistics synchronise that stream.
 */
#ifndef FVGB_H
#define FVGB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    FV_OK = 0,
    FV_E_INVALID = 1,        /* bad argument or malformed mesh */
    FV_E_CUDA = 2,           /* a CUDA runtime call failed */
    FV_E_NOMEM = 3,          /* device or host allocation failed */
    FV_E_NOT_CONVERGED = 4,  /* a solver reached its iteration limit (stats filled) */
    FV_E_DIVERGED = 5,       /* NaN/Inf or breakdown in a solver (stats filled) */
    FV_E_TIMEOUT = 6,        /* a bounded device-side wait gave up */
    FV_E_UNSUPPORTED = 7
} fv_status;

/* Boundary patch kinds (the paper's cases: no-slip / moving walls, inlets
 * with time-dependent velocity, zero-pressure outlets, Sec. 4.1). */
typedef enum {
    FV_PATCH_WALL = 0,    /* fixed velocity (may move / vary in time), zero-gradient p */
    FV_PATCH_INLET = 1,   /* fixed velocity, zero-gradient p */
    FV_PATCH_OUTLET = 2,  /* zero-gradient velocity, fixed p */
    FV_PATCH_EMPTY = 3    /* front/back of a one-cell-thick 2-D mesh: ignored */
} fv_patch_type;

typedef enum { FV_PREC_FP64 = 0, FV_PREC_MIXED = 1 } fv_precision;

typedef struct {
    int32_t type;   /* fv_patch_type */
    int32_t start;  /* first boundary face of the patch, 0 .. B-1 */
    int32_t size;   /* number of faces */
    int32_t pad_;
    double u[3];    /* initial uniform velocity (fixed-velocity patches) */
    double p;       /* initial uniform pressure (outlets) */
} fv_patch;

/* Mesh description (Sec. 3.1).  All pointers are host arrays, copied.
 * Faces 0..F-1 are internal, F..F+B-1 boundary, boundary faces grouped by
 * patch.  Sf points out of the owner (towards the neighbour). */
typedef struct {
    int32_t n_cells;            /* N  > 0 */
    int32_t n_internal_faces;   /* F >= 0 */
    int32_t n_boundary_faces;   /* B >= 0 */
    int32_t n_patches;
    const int32_t *owner;       /* [F+B] */
    const int32_t *neighbour;   /* [F]   */
    const double *Sf;           /* [3][F+B] face area vectors */
    const double *Cf;           /* [3][F+B] face centres */
    const double *C;            /* [3][N]   cell centroids */
    const double *V;            /* [N]      cell volumes, > 0 */
    const fv_patch *patches;    /* [n_patches], tiling 0..B-1 */
    int32_t renumber;           /* 0 keep cell order, 1 reverse Cuthill-McKee */
    int32_t pad_;
} fv_mesh_desc;

typedef struct fv_mesh fv_mesh;
typedef struct fv_case fv_case;

/* Per linear solve. */
typedef struct {
    int32_t iters;     /* Krylov iterations (SMVPs for CG; FP32 inner ones for mixed) */
    int32_t status;    /* fv_status of this solve */
    double res0;       /* initial ||b - A x0||_2 / ||b||_2 */
    double res;        /* final ||r||_2 / ||b||_2: recursively updated r (FP64 CG,
                          BiCGStab) or the true FP64 residual (mixed precision) */
    int32_t outer;     /* FP64 residual passes (mixed precision), else 1 */
    int32_t pad_;
} fv_solve_stats;

#define FV_MAX_CORR 8

typedef struct {
    fv_solve_stats u[3];              /* momentum components */
    fv_solve_stats p[FV_MAX_CORR];    /* pressure solves in order: corrector k, non-orthogonal
                                         loop j at k (1 + n_nonorth) + j (PISO); loop j (SIMPLE) */
    int32_t n_p;
    int32_t status;                   /* worst status of the step */
    double init_res_max;              /* SIMPLE outer residual (see fv_simple_iter) */
} fv_step_stats;

typedef struct {
    double dt;             /* time step */
    int32_t n_corr;        /* pressure correctors per step, 1..FV_MAX_CORR */
    int32_t p_maxit;       /* CG iteration limit */
    double p_tol;          /* CG: ||r|| <= p_tol ||b|| */
    double u_tol;          /* BiCGStab: ||r|| <= u_tol ||b|| */
    int32_t u_maxit;       /* BiCGStab iteration limit */
    int32_t p_ref_cell;    /* reference cell (caller's numbering) pinned to
                              p_ref_value when no outlet patch exists; -1 none */
    double p_ref_value;
    int32_t n_nonorth;     /* non-orthogonal correctors: each pressure corrector
                              solves 1 + n_nonorth times, the explicit
                              non-orthogonal term re-evaluated from the newest
                              pressure before each re-solve; the flux is
                              corrected after the last.  0 = one solve.
                              n_corr * (1 + n_nonorth) <= FV_MAX_CORR. */
    int32_t pad_;
} fv_piso_params;

typedef struct {
    double alpha_u, alpha_p;   /* momentum (implicit) and pressure (explicit) relaxation */
    double p_tol, p_reltol;    /* CG: ||r|| <= max(p_tol ||b||, p_reltol ||r0||) */
    double u_tol, u_reltol;    /* BiCGStab, same rule */
    int32_t p_maxit, u_maxit;
    int32_t p_ref_cell;        /* as in fv_piso_params */
    int32_t n_nonorth;         /* as in fv_piso_params; 1 + n_nonorth <= FV_MAX_CORR */
    double p_ref_value;
} fv_simple_params;

typedef struct {
    double tol;      /* ||r|| <= max(tol ||b||, reltol ||r0||) */
    double reltol;
    int32_t maxit;
    int32_t pad_;
} fv_pcg_params;

/* ---------------------------------------------------------------- mesh -- */

/* Validate and set up a mesh (Sec. 3.1): optional reverse Cuthill-McKee cell
 * renumbering, faces re-oriented so that owner < neighbour and sorted by
 * (owner, neighbour), boundary faces sorted by (patch, owner, original
 * index); face geometry (interpolation weights, delta coefficients,
 * non-orthogonal correction vectors) computed on the device; row-access
 * structures built once and shared by all matrices.
 * desc: host, copied.  stream: cudaStream_t or NULL, used for all later work
 * on this mesh and its cases.  Errors: FV_E_INVALID for owner/neighbour out
 * of range, owner == neighbour, a cell pair with two faces, V <= 0, patches
 * not tiling the boundary; FV_E_NOMEM / FV_E_CUDA. */
fv_status fv_mesh_create(const fv_mesh_desc *desc, void *stream, fv_mesh **out);
fv_status fv_mesh_destroy(fv_mesh *mesh);

/* Host-only variant of the addressing step (no GPU touched): the renumbering
 * of fv_mesh_create.  new_of_old_cell [N], new_of_old_face [F+B],
 * flipped [F+B] (1 where the face orientation was reversed): host outputs. */
fv_status fv_mesh_plan(const fv_mesh_desc *desc, int32_t *new_of_old_cell,
                       int32_t *new_of_old_face, int8_t *flipped);

fv_status fv_mesh_cell_order(const fv_mesh *mesh, int32_t *new_of_old /* host [N] */);
fv_status fv_mesh_face_order(const fv_mesh *mesh, int32_t *new_of_old /* host [F+B] */,
                             int8_t *flipped /* host [F+B] or NULL */);
/* sizes: n_cells, n_internal_faces, n_boundary_faces, nonorthogonal (0/1) */
fv_status fv_mesh_info(const fv_mesh *mesh, int32_t *info /* host [4] */);
/* internal-order addressing: owner [F+B], neighbour [F] (device outputs) */
fv_status fv_mesh_addressing(const fv_mesh *mesh, int32_t *owner, int32_t *neighbour);

/* ---------------------------------------------------------------- case -- */

/* A flow case on a mesh: kinematic viscosity nu, fields u, p, phi (zero),
 * boundary values from the patch descriptions.  precision FV_PREC_MIXED runs
 * the pressure CG as an FP32 inner solve inside an FP64 defect-correction
 * loop; everything else stays FP64. */
fv_status fv_case_create(const fv_mesh *mesh, double nu, int32_t precision, fv_case **out);
fv_status fv_case_destroy(fv_case *cs);

/* Fields: u [3][N], p [N], phi [F+B] (face flux, positive along Sf).
 * Device pointers; original_order = 1 means the caller's cell and face
 * numbering and face orientation, 0 the internal one.  Any pointer may be
 * NULL to skip that field. */
fv_status fv_case_set_fields(fv_case *cs, const double *u, const double *p, const double *phi,
                             int32_t original_order);
fv_status fv_case_get_fields(const fv_case *cs, double *u, double *p, double *phi,
                             int32_t original_order);
/* Same with host buffers; synchronous (the caller's buffers may be reused or
 * read on return).  Where the device reaches pageable host memory through the
 * host's page tables (NVLink-C2C systems such as GB300), the copy and
 * permutation kernels read and write the caller's buffers directly; elsewhere,
 * or with the environment variable FVGB_HOST_STAGING=1 at mesh creation, each
 * field goes through a pinned staging buffer.  Same values either way. */
fv_status fv_case_set_fields_host(fv_case *cs, const double *u, const double *p,
                                  const double *phi, int32_t original_order);
fv_status fv_case_get_fields_host(const fv_case *cs, double *u, double *p, double *phi,
                                  int32_t original_order);

/* Time-dependent boundary conditions (Sec. 1 and 6 of the paper): a uniform
 * value for patch q (u for fixed-velocity patches, p for outlets); u NULL
 * keeps the velocity values.  Stream-ordered and asynchronous (one small
 * kernel on the mesh's stream, values passed by value): a value set between
 * two enqueued steps applies from the second one, and the call may be
 * captured in a CUDA graph.  Errors: FV_E_INVALID for a bad patch index. */
fv_status fv_patch_set_value(fv_case *cs, int32_t q, const double u[3], double p);
/* Per-face values for patch q in the caller's face order within the patch:
 * u host [3][size] (NULL keeps), p host [size] (NULL keeps). */
fv_status fv_patch_set_face_values(fv_case *cs, int32_t q, const double *u, const double *p);

/* One PISO time step (Sec. 3): assemble the momentum matrix, solve the three
 * velocity components by Jacobi-BiCGStab, then n_corr times: H/A, predicted
 * face flux, pressure matrix, Jacobi-PCG pressure solve, flux correction,
 * velocity correction.  stats: host, may be NULL (then the call does not
 * synchronise).  Returns the worst solver status (FV_E_NOT_CONVERGED,
 * FV_E_DIVERGED, FV_E_TIMEOUT) when stats are requested. */
fv_status fv_piso_step(fv_case *cs, const fv_piso_params *prm, fv_step_stats *stats);

/* One SIMPLE iteration (Sec. 3): as PISO without the time derivative, with
 * implicit momentum relaxation alpha_u, one pressure solve, the flux
 * corrected with the solved pressure, then p relaxed explicitly by alpha_p
 * and u corrected with the relaxed pressure.  stats->init_res_max = max of
 * max_c ||b_c - M u_c|| / max_c ||b_c|| and ||b_p - A p|| / ||phi*||_2
 * (initial residuals). */
fv_status fv_simple_iter(fv_case *cs, const fv_simple_params *prm, fv_step_stats *stats);

/* Statistics of the last fv_piso_step / fv_simple_iter / graph replay of
 * this case (useful when the step was enqueued with stats = NULL).
 * Synchronises the stream.  stats: host. */
fv_status fv_case_last_stats(fv_case *cs, fv_step_stats *stats);

/* Capture one PISO step of this case into a CUDA graph (once per parameter
 * set) and replay it n_steps times on the mesh's stream, which must not be
 * the legacy default stream.  stats (host, may be NULL) receive the last
 * replay's statistics. */
fv_status fv_piso_run_graph(fv_case *cs, const fv_piso_params *prm, int32_t n_steps,
                            fv_step_stats *stats);

/* ------------------------------------------------------------ batches -- */

/* Many independent cases advanced together (not in the paper, which runs one
 * case per GPU).  The n meshes (host descriptions, copied; every mesh must be
 * connected) are joined into one block-diagonal mesh renumbered by reverse
 * Cuthill-McKee; case c has kinematic viscosity nu[c] and, when
 * p_ref_cells[c] >= 0 (caller's numbering of that case), that reference
 * pressure cell (p_ref_cells may be NULL for cases with outlets).  Every PISO
 * stage is one launch over all cases: assembly and corrections over all
 * cells, the Krylov solves one block per case from a queue of cases ordered
 * by size.  precision: FV_PREC_FP64 or FV_PREC_MIXED (pressure solve as in
 * fv_pcg_solve_mixed, per case).  stream as in fv_mesh_create.  Errors:
 * FV_E_INVALID for NULL arrays, n < 1, an unknown precision, a negative
 * viscosity, a mesh description that fails fv_mesh_create's validation or a
 * batch whose joined mesh exceeds int32 indexing; FV_E_NOMEM / FV_E_CUDA when
 * memory runs out.  fv_batch_destroy releases everything (NULL is a no-op). */
typedef struct fv_batch fv_batch;
fv_status fv_batch_create(const fv_mesh_desc *descs, int32_t n, const double *nu,
                          const int32_t *p_ref_cells, int32_t precision, void *stream,
                          fv_batch **out);
fv_status fv_batch_destroy(fv_batch *bt);
/* One PISO step of every case; prm->p_ref_cell is ignored (per-case pins
 * come from fv_batch_create).  per_case: host [n] or NULL (no sync). */
fv_status fv_batch_piso_step(fv_batch *bt, const fv_piso_params *prm, fv_step_stats *per_case);
/* Capture one batched step into a CUDA graph (once per parameter set and
 * schedule) and replay it n_steps times. */
fv_status fv_batch_run_graph(fv_batch *bt, const fv_piso_params *prm, int32_t n_steps,
                             fv_step_stats *per_case);
/* Fields of case c in its own original numbering: u [3][N_c], p [N_c],
 * phi [F_c + B_c] (host, any may be NULL).  Synchronous. */
fv_status fv_batch_get_fields(const fv_batch *bt, int32_t c, double *u, double *p, double *phi);
/* Schedules of the per-case Krylov kernels: info = {threads per block, rows
 * per thread per loop trip, block reduction (0 shuffle tree, 1 shared-memory
 * staging), number of schedules, blocks per case in the pressure solve (a
 * thread-block cluster sharing the case through distributed shared
 * memory)}. */
fv_status fv_batch_schedule_info(int32_t schedule, int32_t *info /* host [5] */);
fv_status fv_batch_set_schedule(fv_batch *bt, int32_t schedule);
/* Autotuner: time one PISO step with every schedule from the current state
 * (restored after each trial), keep the fastest; best (host, may be NULL)
 * receives its index, ms (host [number of schedules] or NULL) the times. */
fv_status fv_batch_autotune(fv_batch *bt, const fv_piso_params *prm, int32_t *best, double *ms);

/* ------------------------------------------------------------ solvers -- */

/* Jacobi-preconditioned CG on the symmetric matrix (diag, upper) in LDU form
 * (Sec. 3, Sec. 4.3.2: SMVP, daxpy, dot product, reduction, diagonal
 * preconditioner), in the mesh's internal face order: row owner[f] holds
 * upper[f] in column neighbour[f] and vice versa.  diag [N], upper [F],
 * b [N]: device, read; x [N]: device, initial guess in, solution out.
 * Stops at ||b - A x||_2 <= max(tol ||b||_2, reltol ||r0||_2) with the
 * recursively updated residual; ||b|| = 0 gives x = 0.  stats: host, may be
 * NULL.  Returns FV_E_NOT_CONVERGED / FV_E_DIVERGED / FV_E_TIMEOUT as
 * described above; synchronises the mesh's stream. */
fv_status fv_pcg_solve(const fv_mesh *mesh, const double *diag, const double *upper,
                       const double *b, double *x, const fv_pcg_params *prm,
                       fv_solve_stats *stats);

/* Allocation-free variant of fv_pcg_solve (no counterpart in the paper; it
 * serves callers of this library).  Same arguments, same kernel and the same
 * result; the difference is where the solver's work vectors live.
 * fv_pcg_solve uses memory that fv_mesh_create allocated; this call uses a
 * fixed array of device memory declared statically in the library (about
 * 14 MiB, present on every GPU that loads the library until it is
 * unloaded) and calls no cudaMalloc, cudaFree or other allocating routine.
 * It is meant for callers that cannot allow device allocation when they
 * solve: applications whose device memory is all handed out by their own
 * allocator or pool, and code that runs while a stream capture in global
 * mode is active in the process, where allocation calls are refused.
 * Limits: at most 131072 cells and 1048576 row-structure entries of the
 * mesh; larger meshes return FV_E_INVALID with a message.  The first call
 * on a device looks up the array's device address (make that first call
 * before any stream capture).  Every call uses the same array and leaves
 * its contents behind; the call clears what must start at zero.  Calls that
 * overlap on the GPU (different streams, other threads) race on the array:
 * issue them one after another. */
fv_status fv_pcg_solve_noalloc(const fv_mesh *mesh, const double *diag, const double *upper,
                               const double *b, double *x, const fv_pcg_params *prm,
                               fv_solve_stats *stats);

/* The same solve with the mixed-precision method of FV_PREC_MIXED cases (not
 * in the paper): defect correction in FP64 -- true residual b - A x with the
 * FP64 matrix, its norm and the stopping test, x += correction -- around an
 * FP32 Jacobi-CG on an FP32 copy of the symmetrically scaled matrix (inner
 * dot products summed in FP64 across threads).  Stops on the true FP64
 * residual: ||b - A x||_2 <= max(tol ||b||_2, reltol ||r0||_2); maxit bounds
 * the FP32 inner iterations.  Arguments as fv_pcg_solve; diag and upper are
 * not modified. */
fv_status fv_pcg_solve_mixed(const fv_mesh *mesh, const double *diag, const double *upper,
                             const double *b, double *x, const fv_pcg_params *prm,
                             fv_solve_stats *stats);

/* Jacobi (right) preconditioned BiCGStab on the non-symmetric LDU matrix
 * (diag, upper, lower) (Sec. 3, momentum systems), same conventions as
 * fv_pcg_solve: lower[f] is the entry in row neighbour[f], column owner[f]. */
fv_status fv_bicgstab_solve(const fv_mesh *mesh, const double *diag, const double *upper,
                            const double *lower, const double *b, double *x,
                            const fv_pcg_params *prm, fv_solve_stats *stats);

/* ---------------------------------------------- multigrid pressure CG -- */
/* CG preconditioned by one aggregation-multigrid V-cycle: the stronger
 * pressure solver the paper's discussion (Sec. 5 and 6) calls for, where
 * its GPU code uses Jacobi-CG and its CPU comparison uses OpenFOAM's GAMG.
 * Hierarchy (once per mesh, host, from the geometry): level 0 is the cell
 * graph weighted by |S_f| Delta_f; each level comes from two pairwise-
 * matching passes; coarsening stops at <= 32 nodes.  Per solve (device):
 * Galerkin coarse matrices P^T A P with piecewise-constant P, the coarsest
 * factored by Cholesky; the V-cycle smooths with two weighted-Jacobi sweeps
 * (omega 2/3) before and after the coarse correction, which is added with
 * the over-correction factor 1.8 (keeps the cycle SPD).  The CG's stopping
 * rule, warm start and statistics are those of fv_pcg_solve. */
typedef enum { FV_PSOLVER_JACOBI = 0, FV_PSOLVER_AMG = 1 } fv_pressure_solver;

/* Symmetric A (diag [N], upper [F], device, the mesh's internal order).
 * The first call on a mesh builds the hierarchy (synchronous; later calls
 * reuse it).  Errors: FV_E_INVALID (arguments), FV_E_UNSUPPORTED (the
 * coarsening stalls above 64 nodes, e.g. a graph of isolated cells),
 * FV_E_NOT_CONVERGED / FV_E_DIVERGED as fv_pcg_solve (DIVERGED also when a
 * coarse matrix is not positive definite). */
fv_status fv_pcg_solve_amg(const fv_mesh *mesh, const double *diag, const double *upper,
                           const double *b, double *x, const fv_pcg_params *prm,
                           fv_solve_stats *stats);
/* The same solve with the V-cycle in FP32 (level matrices, vectors and
 * smoothing sweeps; the coarsest factor, the CG recurrences, its residual,
 * reductions, stopping test and solution stay FP64).  The preconditioner
 * changes by about 1e-7 relative, so iterates differ from fv_pcg_solve_amg
 * at that level while the final FP64 residual meets the same tolerance. */
fv_status fv_pcg_solve_amg_mixed(const fv_mesh *mesh, const double *diag, const double *upper,
                                 const double *b, double *x, const fv_pcg_params *prm,
                                 fv_solve_stats *stats);
/* Build the hierarchy if needed; *n_levels and, if sizes is not NULL, the
 * node count of every level (sizes [n_levels], at most 24). */
fv_status fv_amg_info(const fv_mesh *mesh, int32_t *n_levels, int32_t *sizes);
/* Pressure solver of a case's PISO steps and SIMPLE iterations (default
 * FV_PSOLVER_JACOBI).  Selecting FV_PSOLVER_AMG builds the mesh's
 * hierarchy now (synchronous), so later steps may be captured in graphs;
 * in a mixed-precision case the V-cycle runs in FP32
 * (fv_pcg_solve_amg_mixed). */
fv_status fv_case_set_pressure_solver(fv_case *cs, int32_t solver);
/* Host only (no GPU): one coarsening level of a graph of n nodes and ne
 * edges (ea < eb, ordered by (ea, eb), weights ew > 0): agg [n] (node ->
 * aggregate), emap [ne] (edge -> coarse edge, -1 inside an aggregate), the
 * coarse graph in cea, ceb, cew (capacity ne) with *n_coarse nodes and
 * *ne_coarse edges.  FV_E_INVALID for malformed graphs. */
fv_status fv_amg_coarsen_host(int32_t n, int32_t ne, const int32_t *ea, const int32_t *eb,
                              const double *ew, int32_t *agg, int32_t *emap, int32_t *n_coarse,
                              int32_t *ne_coarse, int32_t *cea, int32_t *ceb, double *cew);

/* ------------------------------------------------------------ kernels -- */

/* Gauss gradient of a cell field (Sec. 4.3.3): grad x_P = (1/V_P) sum_f S_f
 * x_f with linearly interpolated x_f and boundary values xb [B] (internal
 * boundary-face order); x [N], xb [B], g [3][N]: device. */
fv_status fv_gauss_grad(const fv_mesh *mesh, const double *x, const double *xb, double *g);

/* LDU matrix-vector product y = A x (the paper's SMVP); device arrays in the
 * mesh's internal order. */
fv_status fv_ldu_matvec(const fv_mesh *mesh, const double *diag, const double *upper,
                        const double *lower, const double *x, double *y);

/* ------------------------------------------- hybrid ELL + J storage -- */
/* The paper's matrix storage (Sec. 3.1, its ELL / J / CRS example): the
 * first K entries of each row (diagonal included, columns ascending) in ELL
 * arrays V (values) and I (columns); the transpose-index array J, where
 * J[i][k] is the ELL slot of the transposed entry A_ji in row j = I[i][k],
 * so the same arrays can be read by columns (STMVP); the entries beyond the
 * K-th of a row in CRS arrays.  The solver path does not use this storage
 * (its SELL-32 rows are assembled from both sides of each face and never
 * read by columns); it is provided for comparison.
 * Encodings: empty ELL slot I = J = -1; a transposed entry in the CRS part
 * at position p is named by -2 - p (in J and in crs_tr).  Without a CRS
 * part, I and J are also packed as Q = K I + J (the paper's remark on
 * combining them; its other formula, K J + I, is not decodable when I >= K,
 * so K I + J is used). */
typedef struct fv_ellj fv_ellj;

/* Host only (no GPU): build the arrays for a structurally symmetric
 * pattern given as row_ptr [n+1], col [row_ptr[n]] (columns strictly
 * ascending per row).  Outputs are row-major n x K as in the paper: I, J
 * [n*K]; crs_ptr [n+1]; crs_col, crs_tr [*n_crs].  With I == NULL only
 * crs_ptr and *n_crs are produced (size query).  FV_E_INVALID: bad
 * arguments, unsorted or out-of-range columns, an entry without transpose. */
fv_status fv_ellj_build_host(int32_t n, const int32_t *row_ptr, const int32_t *col, int32_t K,
                             int32_t *I, int32_t *J, int32_t *crs_ptr, int32_t *crs_col,
                             int32_t *crs_tr, int32_t *n_crs);
/* The storage of the mesh's LDU pattern (internal order) with width K
 * (0 = the most frequent row length).  Index arrays are built on the host
 * and copied to the device (synchronous); the library owns them. */
fv_status fv_ellj_create(const fv_mesh *mesh, int32_t K, fv_ellj **out);
fv_status fv_ellj_destroy(fv_ellj *ellj);
/* K and the number of CRS entries (either pointer may be NULL). */
fv_status fv_ellj_info(const fv_ellj *ellj, int32_t *K, int32_t *n_crs);
/* Scatter an LDU matrix (diag [N], upper/lower [F], device, internal order)
 * into V [K*N] (device, slot k of row i at k*N + i; empty slots set to 0)
 * and C [n_crs] (device; may be NULL when n_crs == 0).  Asynchronous on the
 * mesh's stream. */
fv_status fv_ellj_from_ldu(const fv_ellj *ellj, const double *diag, const double *upper,
                           const double *lower, double *V, double *C);
/* y = A x (mode 0, by rows), y = A^T x (mode 1, by columns through I and
 * J), or y = A^T x through the packed Q (mode 2; FV_E_UNSUPPORTED when the
 * storage has a CRS part).  V, C, x, y: device; asynchronous. */
fv_status fv_ellj_spmv(const fv_ellj *ellj, const double *V, const double *C, const double *x,
                       double *y, int32_t mode);

/* ---------------------------------------------------------- profiling -- */

/* Per-stage device time, measured with CUDA events recorded on the mesh's
 * stream around each stage of fv_piso_step / fv_simple_iter (the paper
 * profiles its solver per component, Sec. 4.3.2-4.3.3).  Stages: */
enum {
    FV_PROF_MOMENTUM = 0,   /* momentum assembly + grad p (+ grad u) */
    FV_PROF_BICGSTAB = 1,   /* momentum solve */
    FV_PROF_HBYA = 2,       /* H/A, rAU */
    FV_PROF_PRESSURE = 3,   /* pressure assembly */
    FV_PROF_PCG = 4,        /* pressure solve */
    FV_PROF_CORRECT = 5,    /* flux and velocity correction */
    FV_PROF_OTHER = 6,      /* residual reductions, copies */
    FV_PROF_NSTAGE = 7
};
/* on = 1 starts recording (direct launches only; graph replays are not
 * instrumented), 0 stops.  Kernel launches are counted either way. */
fv_status fv_profile_enable(int32_t on);
/* ms [FV_PROF_NSTAGE]: accumulated device milliseconds per stage;
 * launches [FV_PROF_NSTAGE]: kernel launches per stage (host arrays, either
 * may be NULL).  Waits for pending events; reset = 1 clears the totals. */
fv_status fv_profile_read(double *ms, int64_t *launches, int32_t reset);

/* ---------------------------------------------------------- utilities -- */

const char *fv_last_error(void);
/* Spin limit of device-side grid barriers (iterations); 0 restores the
 * default.  A barrier that exceeds it makes the solve return FV_E_TIMEOUT. */
fv_status fv_set_barrier_spin_limit(int64_t limit);
/* Device memory held by a case (bytes), including its mesh. */
fv_status fv_case_memory(const fv_case *cs, int64_t *bytes);

#ifdef __cplusplus
}
#endif
#endif /* FVGB_H */
