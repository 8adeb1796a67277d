// fvgb_internal.h -- internal data structures of libfvgb (not part of the ABI).
//
// Device layout (all in HBM, internal = renumbered order):
//  * faces 0..F-1 internal (owner < neighbour, sorted by (owner, neighbour)),
//    F..F+B-1 boundary (sorted by patch, owner, original index);
//  * face geometry SoA: Sf[3][M], magSf[M], w[F], delta[M], kv[3][F] (M = F+B);
//  * row access for every matrix (the paper's "access by rows", Sec. 3.1):
//    SELL-32 -- rows in slices of 32 (one warp), slice s holds K_s columns,
//    entry k of row 32 s + l at slice_ptr[s] + 32 k + l; per entry the
//    neighbour cell (col) and the face (sface); padding entries have
//    sface = -1 and col = the row itself.  Matrix off-diagonals are stored
//    in the same slots, so a face's coefficient appears once per side;
//  * boundary faces of each cell: bptr[N+1] into bface[] (0..B-1, empty
//    patches left out).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/fvgb.h"

namespace fvgb {

constexpr int kSlice = 32;

void set_error(const char *fmt, ...);
fv_status cuda_status(cudaError_t e, const char *what);

#define FV_CUDA(call)                                                   \
    do {                                                                \
        cudaError_t e__ = (call);                                       \
        if (e__ != cudaSuccess) return ::fvgb::cuda_status(e__, #call); \
    } while (0)

#define FV_CHECK(cond, code, ...)                \
    do {                                         \
        if (!(cond)) {                           \
            ::fvgb::set_error(__VA_ARGS__);      \
            return code;                         \
        }                                        \
    } while (0)

// device allocation registry (freed by the owner's destructor)
struct DeviceArena {
    std::vector<void *> ptrs;
    size_t bytes = 0;
    fv_status alloc(void **p, size_t n);
    template <class T>
    fv_status alloc_n(T **p, size_t n) { return alloc(reinterpret_cast<void **>(p), n * sizeof(T)); }
    void release();
};

// Host-side addressing plan (RCM order, face order) -- pure host code.
struct MeshPlan {
    int N = 0, F = 0, B = 0;
    std::vector<int32_t> cell_new_of_old, face_new_of_old;
    std::vector<int8_t> flipped;
    std::vector<int32_t> own, nei;          // internal order [M], [F]
    std::vector<int32_t> bpatch;            // internal boundary order [B]
    // SELL-32 rows over internal neighbours
    int nslice = 0;
    std::vector<int32_t> slice_ptr, col, sface;
    // boundary faces per cell (non-empty patches)
    std::vector<int32_t> bptr, bface;
};
fv_status build_plan(const fv_mesh_desc *d, MeshPlan *plan);

// Solve statistics as kept on the device.
struct DevSolveStats {
    int32_t iters;
    int32_t status;
    double res0;
    double res;
    int32_t outer;
    int32_t pad;
};

// Grid barrier state (bounded spin, coop.cuh); zeroed before each launch.
struct GridBar {
    unsigned int count;     // arrivals so far in this launch
    unsigned int spare;
    int err;                // first error recorded by a waiter (FV_E_TIMEOUT)
    int pad;
};

// Persistent Krylov workspace, sized for one mesh.
struct KrylovWork {
    int G = 0;               // cooperative grid size of the BiCGStab kernel
    int Gcg = 0;             // cooperative grid size of the CG kernel (one block per SM)
    int block = 0;
    int cg_res_max = 0;      // dynamic shared memory the resident CG form may use (bytes)
    int mix_res_max = 0;     // the same for the resident mixed-precision CG form
    int cgcg_res_max = 0;    // the same for the Chronopoulos-Gear mixed-precision form
    int mixed_form = 2;      // mixed CG inner order: 0 textbook, 1 Chronopoulos-Gear, 2 by regime
    double *val = nullptr;   // SELL values (scaled copy for CG)
    double *val2 = nullptr;  // second SELL value buffer (BiCGStab input copy)
    double *dinv = nullptr;  // [N] (BiCGStab) / scaling s (CG)
    double *r = nullptr, *p = nullptr, *q = nullptr, *y = nullptr;   // CG [N]
    double *bv[9] = {};      // BiCGStab: r, rh, p, v, y(s), z, t ... per component [3N] each
    float *val32 = nullptr;      // FP32 scaled SELL values (mixed precision, lazily)
    float *f32[6] = {};          // FP32 inner vectors r, p, q, e, w, v [N]
    float *f32p[2] = {};         // Chronopoulos-Gear form: s = A^ p, w = A^ r [N]
    double *partials = nullptr;  // [2][G][8]
    GridBar *bar = nullptr;
    DevSolveStats *stats = nullptr;  // [4] scratch for stand-alone calls
};

// aggregation-multigrid preconditioned CG (amg.cu)
struct AmgData;
void amg_release(AmgData *a);
struct AmgProblem {
    const double *diag;      // [N]
    const double *off;       // [F] symmetric off-diagonal per internal face, times off_sign
    double off_sign;
    const double *b;         // [N]
    double *x;               // [N] in/out
    double tol, reltol;
    int maxit;
    DevSolveStats *stats;    // device
    int fp32 = 0;            // V-cycle in FP32 (mixed precision)
};

}  // namespace fvgb

struct fv_mesh {
    int N = 0, F = 0, B = 0, M = 0, np = 0;
    int nonorth = 0;
    cudaStream_t stream = nullptr;
    int device = 0;                   // CUDA device current at fv_mesh_create
    int sm_count = 0;
    int host_direct = 0;              // kernels may read/write pageable host memory (see case.cu)
    std::vector<fv_patch> patches;
    fvgb::MeshPlan plan;              // host copy of the addressing
    fvgb::DeviceArena arena;
    // device addressing
    int32_t *own = nullptr, *nei = nullptr;
    int32_t *slice_ptr = nullptr, *col = nullptr, *sface = nullptr;
    int nslice = 0, nnz = 0;
    int32_t *bptr = nullptr, *bface = nullptr;
    int8_t *btype = nullptr;          // patch type of each boundary face [B]
    int32_t *cell_new_of_old = nullptr, *face_new_of_old = nullptr;
    int8_t *flipped = nullptr;
    // device geometry
    double *Sf = nullptr, *magSf = nullptr, *w = nullptr, *delta = nullptr, *kv = nullptr;
    double *V = nullptr, *Vinv = nullptr;
    fvgb::KrylovWork kw;
    fvgb::AmgData *amg = nullptr;     // multigrid hierarchy, built on first use
};

namespace fvgb {
fv_status amg_prepare(fv_mesh *m);
fv_status launch_pcg_amg(const fv_mesh *m, const AmgProblem &pb);
}

struct fv_case {
    const fv_mesh *mesh = nullptr;
    double nu = 0.0;
    int precision = FV_PREC_FP64;
    int psolver = FV_PSOLVER_JACOBI;
    fvgb::DeviceArena arena;
    // state
    double *u = nullptr, *p = nullptr, *phi = nullptr;   // [3N], [N], [M]
    double *ub = nullptr, *pb = nullptr;                 // boundary values [3B], [B]
    // momentum system
    double *Md = nullptr, *Mo = nullptr, *src = nullptr, *gradp = nullptr, *gradU = nullptr;
    // pressure step
    double *HbyA = nullptr, *rAU = nullptr, *Pd = nullptr, *Po = nullptr, *pbv = nullptr;
    double *phis = nullptr, *af = nullptr, *nof = nullptr, *pold = nullptr;
    // mixed-precision pressure solve
    float *Po32 = nullptr;
    double *resid = nullptr;
    double *tmp = nullptr;                   // field exchange temporary [max(3N, M)]
    double *nu_cell = nullptr;               // per-cell viscosity (batched cases) or nullptr
    int8_t *pin = nullptr;                   // per-cell reference-pressure flags or nullptr
    // per-step statistics
    fvgb::DevSolveStats *dstats = nullptr;   // [3 + FV_MAX_CORR + 2]
    double *dsimple = nullptr;               // SIMPLE residual partials/finals
    fvgb::DevSolveStats *hstats = nullptr;   // pinned mirror
    double *hsimple = nullptr;
    // host staging (pinned)
    double *hstage = nullptr;
    size_t hstage_bytes = 0;
    cudaGraphExec_t graph = nullptr;
    int last_np = 0;                         // pressure solves of the last step
    bool last_simple = false;
    fv_piso_params graph_prm{};
};

namespace fvgb {

// mesh.cu
fv_status upload_mesh(fv_mesh *m, const fv_mesh_desc *d);

// assembly.cu -- kernels launched on the mesh's stream
struct StepArgs {
    double dt_inv;      // 1/dt (PISO) or 0 (SIMPLE)
    double alpha_u;     // 1 (PISO) or relaxation factor
    int ref_cell;       // internal index or -1
    double p_ref;
};
fv_status launch_grad_u(const fv_case *c);
fv_status launch_momentum(const fv_case *c, const StepArgs &a);
fv_status launch_hbya(const fv_case *c);
fv_status launch_pressure(const fv_case *c, const StepArgs &a);
fv_status launch_grad_p(const fv_case *c);
fv_status launch_correct_piso(const fv_case *c);
fv_status launch_correct_simple(const fv_case *c, double alpha_p);
fv_status launch_simple_residuals_mom(const fv_case *c);
fv_status launch_simple_residuals_p(const fv_case *c);
fv_status launch_gauss_grad(const fv_mesh *m, const double *x, const double *xb, double *g);
fv_status launch_ldu_matvec(const fv_mesh *m, const double *diag, const double *upper,
                            const double *lower, const double *x, double *y);
fv_status launch_ldu_to_sell(const fv_mesh *m, const double *upper, const double *lower,
                             double *val);
fv_status launch_permute_cells(const fv_mesh *m, int ncomp, const double *src, double *dst,
                               int to_internal);
fv_status launch_permute_faces(const fv_mesh *m, const double *src, double *dst, int to_internal);
fv_status launch_patch_fill(const fv_case *c, int start, int n, const double *u, double p);

// krylov.cu
struct CgProblem {
    const double *diag;      // [N]
    double *val;             // SELL off-diagonals, unscaled on entry, scaled on exit
    const double *b;         // [N]
    double *x;               // [N] in/out
    double tol, reltol;
    int maxit;
    DevSolveStats *stats;    // device
};
fv_status launch_pcg(const fv_mesh *m, const CgProblem &pb);

// FP32-inside-FP64 defect-correction CG (the FP64 values are not modified)
struct MixedProblem {
    const double *diag;
    const double *val;       // SELL off-diagonals, unscaled FP64
    const double *b;
    double *x;
    double tol, reltol;
    int maxit;               // budget of inner iterations
    DevSolveStats *stats;
};
fv_status launch_pcg_mixed(const fv_mesh *m, const MixedProblem &pb);

// work vectors of one CG solve supplied by the caller
struct CgScratch {
    double *s, *r, *p, *q, *y;   // [N] each
    double *partials;            // [2][max_blocks][8]
    int max_blocks;
    GridBar *bar;
};
fv_status launch_pcg_scratch(const fv_mesh *m, const CgProblem &pb, const CgScratch &ws);

struct BicgProblem {
    const double *diag;      // [N]
    const double *val;       // SELL off-diagonals (non-symmetric)
    const double *b;         // [3][N] right-hand sides, or nullptr with src/gradp below
    const double *src;       // [3][N]   b_c = src_c - V gradp_c when b == nullptr
    const double *gradp;     // [3][N]
    double *x;               // [3][N] in/out
    int ncomp;
    double tol, reltol;
    int maxit;
    DevSolveStats *stats;    // device [ncomp]
};
fv_status launch_bicgstab(const fv_mesh *m, const BicgProblem &pb);
fv_status krylov_setup(fv_mesh *m);
extern long long g_spin_limit;

// profile.cu
int prof_begin(int stage, cudaStream_t s);
void prof_end(int id, cudaStream_t s);
void prof_count(int stage, int n);

}  // namespace fvgb
