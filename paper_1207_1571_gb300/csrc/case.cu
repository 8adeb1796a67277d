// case.cu -- flow cases, the PISO time step and the SIMPLE iteration (paper
// Sec. 3), stand-alone solver entry points and CUDA-graph replay.
//
// A PISO step is a fixed sequence of launches on the mesh's stream:
//   [grad u (non-orthogonal meshes)] -> momentum assembly + grad p ->
//   BiCGStab (three components, one cooperative launch) ->
//   n_corr x { H/A and rAU -> (1 + n_nonorth) x { [grad p] -> pressure
//   assembly -> CG (one cooperative launch) } -> flux + velocity
//   correction }.
// Nothing leaves the device inside a step; statistics are copied back only
// when the caller asks for them.  Because the sequence is fixed, it can be
// captured once into a CUDA graph and replayed.
#include <cstring>
#include <new>

#include "fvgb_internal.h"

using namespace fvgb;

namespace {

fv_status stage(fv_case *c, size_t bytes)
{
    if (c->hstage_bytes >= bytes) return FV_OK;
    if (c->hstage) cudaFreeHost(c->hstage);
    c->hstage = nullptr;
    c->hstage_bytes = 0;
    FV_CUDA(cudaMallocHost(&c->hstage, bytes));
    c->hstage_bytes = bytes;
    return FV_OK;
}

bool has_outlet(const fv_mesh *m)
{
    for (const fv_patch &p : m->patches)
        if (p.type == FV_PATCH_OUTLET && p.size > 0) return true;
    return false;
}

fv_status check_ref(const fv_case *c, int ref_cell, int *ref_internal)
{
    const fv_mesh *m = c->mesh;
    if (ref_cell >= 0) {
        FV_CHECK(ref_cell < m->N, FV_E_INVALID, "p_ref_cell %d out of range", ref_cell);
        *ref_internal = m->plan.cell_new_of_old[ref_cell];
    } else {
        FV_CHECK(has_outlet(m), FV_E_INVALID,
                 "a closed domain (no outlet patch) needs a pressure reference cell");
        *ref_internal = -1;
    }
    return FV_OK;
}

void fill_solve(fv_solve_stats *o, const DevSolveStats &d)
{
    o->iters = d.iters;
    o->status = d.status;
    o->res0 = d.res0;
    o->res = d.res;
    o->outer = d.outer;
    o->pad_ = 0;
}

// pressure solve of a step: FP64 CG, or the mixed-precision method
fv_status launch_pressure_solve(const fv_case *c, double tol, double reltol, int maxit,
                                DevSolveStats *st)
{
    if (c->psolver == FV_PSOLVER_AMG) {
        // the face coefficients a_f of the pressure assembly are -upper; a
        // mixed-precision case smooths in FP32
        AmgProblem ap{c->Pd, c->af, -1.0, c->pbv, c->p, tol, reltol, maxit, st,
                      c->precision == FV_PREC_MIXED ? 1 : 0};
        return launch_pcg_amg(c->mesh, ap);
    }
    if (c->precision == FV_PREC_MIXED) {
        MixedProblem mp{c->Pd, c->Po, c->pbv, c->p, tol, reltol, maxit, st};
        return launch_pcg_mixed(c->mesh, mp);
    }
    CgProblem cp{c->Pd, c->Po, c->pbv, c->p, tol, reltol, maxit, st};
    return launch_pcg(c->mesh, cp);
}

int worse(int a, int b)
{
    // timeout > diverged > not converged > ok
    auto rank = [](int s) {
        return s == FV_E_TIMEOUT ? 3 : s == FV_E_DIVERGED ? 2 : s == FV_E_NOT_CONVERGED ? 1 : 0;
    };
    return rank(b) > rank(a) ? b : a;
}

fv_status read_stats(fv_case *c, int n_p, fv_step_stats *out, bool simple)
{
    const fv_mesh *m = c->mesh;
    const int n = 3 + FV_MAX_CORR;
    FV_CUDA(cudaMemcpyAsync(c->hstats, c->dstats, sizeof(DevSolveStats) * n,
                            cudaMemcpyDeviceToHost, m->stream));
    if (simple)
        FV_CUDA(cudaMemcpyAsync(c->hsimple, c->dsimple, sizeof(double) * 4, cudaMemcpyDeviceToHost,
                                m->stream));
    FV_CUDA(cudaStreamSynchronize(m->stream));
    std::memset(out, 0, sizeof(*out));
    int st = FV_OK;
    for (int k = 0; k < 3; ++k) {
        fill_solve(&out->u[k], c->hstats[k]);
        st = worse(st, c->hstats[k].status);
    }
    for (int k = 0; k < n_p; ++k) {
        fill_solve(&out->p[k], c->hstats[3 + k]);
        st = worse(st, c->hstats[3 + k].status);
    }
    out->n_p = n_p;
    out->status = st;
    out->init_res_max = simple ? c->hsimple[2] : 0.0;
    return (fv_status)st;
}

// Run one stage: CUDA events around it when profiling is on, launch count.
#define STAGE(stg, nlaunch, call)                          \
    do {                                                   \
        const int id__ = prof_begin((stg), m->stream);     \
        const fv_status s__ = (call);                      \
        prof_end(id__, m->stream);                         \
        prof_count((stg), (nlaunch));                      \
        if (s__ != FV_OK) return s__;                      \
    } while (0)

fv_status piso_enqueue(fv_case *c, const fv_piso_params *prm, int ref)
{
    const fv_mesh *m = c->mesh;
    StepArgs sa{1.0 / prm->dt, 1.0, ref, prm->p_ref_value};
    if (m->nonorth) STAGE(FV_PROF_MOMENTUM, 1, launch_grad_u(c));
    STAGE(FV_PROF_MOMENTUM, 1, launch_momentum(c, sa));
    BicgProblem bp{c->Md, c->Mo, nullptr, c->src, c->gradp, c->u, 3, prm->u_tol, 0.0,
                   prm->u_maxit, c->dstats};
    STAGE(FV_PROF_BICGSTAB, 1, launch_bicgstab(m, bp));
    const int nl = 1 + prm->n_nonorth;
    for (int k = 0; k < prm->n_corr; ++k) {
        STAGE(FV_PROF_HBYA, 1, launch_hbya(c));
        for (int j = 0; j < nl; ++j) {
            // non-orthogonal corrector: explicit term from the newest pressure
            if (j > 0) STAGE(FV_PROF_PRESSURE, 1, launch_grad_p(c));
            STAGE(FV_PROF_PRESSURE, 1, launch_pressure(c, sa));
            STAGE(FV_PROF_PCG, 1, launch_pressure_solve(c, prm->p_tol, 0.0, prm->p_maxit,
                                                        c->dstats + 3 + k * nl + j));
        }
        STAGE(FV_PROF_CORRECT, 1, launch_correct_piso(c));
    }
    return FV_OK;
}

fv_status check_piso(const fv_piso_params *prm)
{
    FV_CHECK(prm != nullptr, FV_E_INVALID, "params are NULL");
    FV_CHECK(prm->dt > 0.0, FV_E_INVALID, "dt must be positive");
    FV_CHECK(prm->n_corr >= 1 && prm->n_corr <= FV_MAX_CORR, FV_E_INVALID,
             "n_corr must be in 1..%d", FV_MAX_CORR);
    FV_CHECK(prm->n_nonorth >= 0 && prm->n_corr * (1 + prm->n_nonorth) <= FV_MAX_CORR,
             FV_E_INVALID, "n_corr * (1 + n_nonorth) must be at most %d", FV_MAX_CORR);
    FV_CHECK(prm->p_maxit >= 0 && prm->u_maxit >= 0, FV_E_INVALID, "negative iteration limit");
    FV_CHECK(prm->p_tol >= 0.0 && prm->u_tol >= 0.0, FV_E_INVALID, "negative tolerance");
    return FV_OK;
}

}  // namespace

extern "C" fv_status fv_case_create(const fv_mesh *m, double nu, int32_t precision, fv_case **out)
{
    FV_CHECK(m && out, FV_E_INVALID, "NULL argument");
    FV_CHECK(nu >= 0.0, FV_E_INVALID, "negative viscosity");
    FV_CHECK(precision == FV_PREC_FP64 || precision == FV_PREC_MIXED, FV_E_INVALID,
             "unknown precision %d", precision);
    *out = nullptr;
    fv_case *c = new (std::nothrow) fv_case();
    FV_CHECK(c != nullptr, FV_E_NOMEM, "host allocation failed");
    c->mesh = m;
    c->nu = nu;
    c->precision = precision;
    const size_t N = m->N, M = m->M, B = m->B, F = m->F;
    const size_t nb = (N + 255) / 256;
    DeviceArena &a = c->arena;
    fv_status st = FV_OK;
    auto A = [&](double **p, size_t n) {
        if (st == FV_OK) st = a.alloc_n(p, n);
        if (st == FV_OK) st = cudaMemsetAsync(*p, 0, sizeof(double) * (n ? n : 1), m->stream) == cudaSuccess
                                  ? FV_OK : FV_E_CUDA;
    };
    A(&c->u, 3 * N); A(&c->p, N); A(&c->phi, M); A(&c->ub, 3 * B); A(&c->pb, B);
    A(&c->Md, N); A(&c->Mo, (size_t)m->nnz); A(&c->src, 3 * N); A(&c->gradp, 3 * N);
    A(&c->gradU, m->nonorth ? 9 * N : 1);
    A(&c->HbyA, 3 * N); A(&c->rAU, N); A(&c->Pd, N); A(&c->Po, (size_t)m->nnz); A(&c->pbv, N);
    A(&c->phis, M); A(&c->af, M); A(&c->nof, F ? F : 1); A(&c->pold, N);
    A(&c->resid, nb * 8); A(&c->dsimple, 4);
    double *tmp = nullptr;
    A(&tmp, 3 * N > M ? 3 * N : M);
    if (st == FV_OK) st = a.alloc_n(&c->dstats, 3 + FV_MAX_CORR);
    if (st == FV_OK && cudaMemsetAsync(c->dstats, 0, sizeof(DevSolveStats) * (3 + FV_MAX_CORR), m->stream) != cudaSuccess)
        st = FV_E_CUDA;
    if (st == FV_OK && cudaMallocHost(&c->hstats, sizeof(DevSolveStats) * (3 + FV_MAX_CORR)) != cudaSuccess)
        st = FV_E_NOMEM;
    if (st == FV_OK && cudaMallocHost(&c->hsimple, sizeof(double) * 4) != cudaSuccess) st = FV_E_NOMEM;
    if (st != FV_OK) {
        fv_case_destroy(c);
        return st;
    }
    c->tmp = tmp;
    c->hsimple[0] = c->hsimple[1] = c->hsimple[2] = 0.0;
    // boundary values from the patch descriptions
    for (int q = 0; q < m->np; ++q) {
        const fv_patch &pt = m->patches[q];
        if (pt.type == FV_PATCH_EMPTY) continue;
        st = fv_patch_set_value(c, q, pt.u, pt.p);
        if (st != FV_OK) { fv_case_destroy(c); return st; }
    }
    cudaError_t e = cudaStreamSynchronize(m->stream);
    if (e != cudaSuccess) { fv_case_destroy(c); return cuda_status(e, "case init"); }
    *out = c;
    return FV_OK;
}

extern "C" fv_status fv_case_destroy(fv_case *c)
{
    if (!c) return FV_OK;
    cudaStreamSynchronize(c->mesh->stream);
    if (c->graph) cudaGraphExecDestroy(c->graph);
    if (c->hstats) cudaFreeHost(c->hstats);
    if (c->hsimple) cudaFreeHost(c->hsimple);
    if (c->hstage) cudaFreeHost(c->hstage);
    c->arena.release();
    delete c;
    return FV_OK;
}

extern "C" fv_status fv_case_memory(const fv_case *c, int64_t *bytes)
{
    FV_CHECK(c && bytes, FV_E_INVALID, "NULL argument");
    *bytes = (int64_t)(c->arena.bytes + c->mesh->arena.bytes);
    return FV_OK;
}

extern "C" fv_status fv_case_set_fields(fv_case *c, const double *u, const double *p,
                                        const double *phi, int32_t original_order)
{
    FV_CHECK(c, FV_E_INVALID, "NULL case");
    const fv_mesh *m = c->mesh;
    fv_status st;
    if (u) {
        if (original_order) { if ((st = launch_permute_cells(m, 3, u, c->u, 1)) != FV_OK) return st; }
        else FV_CUDA(cudaMemcpyAsync(c->u, u, sizeof(double) * 3 * m->N, cudaMemcpyDefault, m->stream));
    }
    if (p) {
        if (original_order) { if ((st = launch_permute_cells(m, 1, p, c->p, 1)) != FV_OK) return st; }
        else FV_CUDA(cudaMemcpyAsync(c->p, p, sizeof(double) * m->N, cudaMemcpyDefault, m->stream));
    }
    if (phi) {
        if (original_order) { if ((st = launch_permute_faces(m, phi, c->phi, 1)) != FV_OK) return st; }
        else FV_CUDA(cudaMemcpyAsync(c->phi, phi, sizeof(double) * m->M, cudaMemcpyDefault, m->stream));
    }
    return FV_OK;
}

extern "C" fv_status fv_case_get_fields(const fv_case *c, double *u, double *p, double *phi,
                                        int32_t original_order)
{
    FV_CHECK(c, FV_E_INVALID, "NULL case");
    const fv_mesh *m = c->mesh;
    fv_status st;
    if (u) {
        if (original_order) { if ((st = launch_permute_cells(m, 3, c->u, u, 0)) != FV_OK) return st; }
        else FV_CUDA(cudaMemcpyAsync(u, c->u, sizeof(double) * 3 * m->N, cudaMemcpyDefault, m->stream));
    }
    if (p) {
        if (original_order) { if ((st = launch_permute_cells(m, 1, c->p, p, 0)) != FV_OK) return st; }
        else FV_CUDA(cudaMemcpyAsync(p, c->p, sizeof(double) * m->N, cudaMemcpyDefault, m->stream));
    }
    if (phi) {
        if (original_order) { if ((st = launch_permute_faces(m, c->phi, phi, 0)) != FV_OK) return st; }
        else FV_CUDA(cudaMemcpyAsync(phi, c->phi, sizeof(double) * m->M, cudaMemcpyDefault, m->stream));
    }
    return FV_OK;
}

// Host variants.  Where the device reaches pageable host memory through the
// host's page tables (GB300 with NVLink-C2C), the copy and permutation
// kernels read or write the caller's buffers directly (m->host_direct);
// otherwise each field goes through one pinned staging buffer and one device
// temporary.  Both return once the caller's buffers may be reused or read.
extern "C" fv_status fv_case_set_fields_host(fv_case *c, const double *u, const double *p,
                                             const double *phi, int32_t original_order)
{
    FV_CHECK(c, FV_E_INVALID, "NULL case");
    const fv_mesh *m = c->mesh;
    if (m->host_direct) {
        const fv_status sd = fv_case_set_fields(c, u, p, phi, original_order);
        if (sd != FV_OK) return sd;
        FV_CUDA(cudaStreamSynchronize(m->stream));
        return FV_OK;
    }
    const size_t n3 = 3 * (size_t)m->N, n1 = m->N, nm = m->M;
    fv_status st = stage(c, sizeof(double) * (n3 > nm ? n3 : nm));
    if (st != FV_OK) return st;
    struct Item { const double *h; size_t n; int kind; } items[3] = {{u, n3, 0}, {p, n1, 1}, {phi, nm, 2}};
    for (const Item &it : items) {
        if (!it.h) continue;
        std::memcpy(c->hstage, it.h, sizeof(double) * it.n);
        FV_CUDA(cudaMemcpyAsync(c->tmp, c->hstage, sizeof(double) * it.n, cudaMemcpyHostToDevice, m->stream));
        st = fv_case_set_fields(c, it.kind == 0 ? c->tmp : nullptr, it.kind == 1 ? c->tmp : nullptr,
                                it.kind == 2 ? c->tmp : nullptr, original_order);
        if (st != FV_OK) return st;
        FV_CUDA(cudaStreamSynchronize(m->stream));
    }
    return FV_OK;
}

extern "C" fv_status fv_case_get_fields_host(const fv_case *cc, double *u, double *p, double *phi,
                                             int32_t original_order)
{
    FV_CHECK(cc, FV_E_INVALID, "NULL case");
    fv_case *c = const_cast<fv_case *>(cc);
    const fv_mesh *m = c->mesh;
    if (m->host_direct) {
        const fv_status sd = fv_case_get_fields(c, u, p, phi, original_order);
        if (sd != FV_OK) return sd;
        FV_CUDA(cudaStreamSynchronize(m->stream));
        return FV_OK;
    }
    const size_t n3 = 3 * (size_t)m->N, n1 = m->N, nm = m->M;
    fv_status st = stage(c, sizeof(double) * (n3 > nm ? n3 : nm));
    if (st != FV_OK) return st;
    struct Item { double *h; size_t n; int kind; } items[3] = {{u, n3, 0}, {p, n1, 1}, {phi, nm, 2}};
    for (const Item &it : items) {
        if (!it.h) continue;
        st = fv_case_get_fields(c, it.kind == 0 ? c->tmp : nullptr, it.kind == 1 ? c->tmp : nullptr,
                                it.kind == 2 ? c->tmp : nullptr, original_order);
        if (st != FV_OK) return st;
        FV_CUDA(cudaMemcpyAsync(c->hstage, c->tmp, sizeof(double) * it.n, cudaMemcpyDeviceToHost, m->stream));
        FV_CUDA(cudaStreamSynchronize(m->stream));
        std::memcpy(it.h, c->hstage, sizeof(double) * it.n);
    }
    return FV_OK;
}

// Boundary values live in device arrays in internal boundary-face order;
// patch q occupies boundary faces [start, start + size) in that order too.
static fv_status put_patch(fv_case *c, int q, const double *u_int /*[3][size] or NULL*/,
                           const double *p_int /*[size] or NULL*/)
{
    const fv_mesh *m = c->mesh;
    const fv_patch &pt = m->patches[q];
    const size_t n = pt.size;
    if (n == 0) return FV_OK;
    fv_status st = stage(c, sizeof(double) * 4 * n);
    if (st != FV_OK) return st;
    FV_CUDA(cudaStreamSynchronize(m->stream));   // staging buffer may still be in use
    if (u_int) std::memcpy(c->hstage, u_int, sizeof(double) * 3 * n);
    if (p_int) std::memcpy(c->hstage + 3 * n, p_int, sizeof(double) * n);
    if (u_int)
        for (int cc = 0; cc < 3; ++cc)
            FV_CUDA(cudaMemcpyAsync(c->ub + (size_t)cc * m->B + pt.start, c->hstage + cc * n,
                                    sizeof(double) * n, cudaMemcpyHostToDevice, m->stream));
    if (p_int)
        FV_CUDA(cudaMemcpyAsync(c->pb + pt.start, c->hstage + 3 * n, sizeof(double) * n,
                                cudaMemcpyHostToDevice, m->stream));
    FV_CUDA(cudaStreamSynchronize(m->stream));
    return FV_OK;
}

extern "C" fv_status fv_patch_set_value(fv_case *c, int32_t q, const double u[3], double p)
{
    FV_CHECK(c && q >= 0 && q < c->mesh->np, FV_E_INVALID, "bad patch index %d", q);
    const fv_patch &pt = c->mesh->patches[q];
    return launch_patch_fill(c, pt.start, pt.size, u, p);
}

extern "C" fv_status fv_patch_set_face_values(fv_case *c, int32_t q, const double *u, const double *p)
{
    FV_CHECK(c && q >= 0 && q < c->mesh->np, FV_E_INVALID, "bad patch index %d", q);
    const fv_mesh *m = c->mesh;
    const fv_patch &pt = m->patches[q];
    const size_t n = pt.size;
    std::vector<double> uu(u ? 3 * n : 0), pp(p ? n : 0);
    for (size_t j = 0; j < n; ++j) {
        const int b = m->plan.face_new_of_old[m->F + pt.start + j] - m->F - pt.start;
        if (u)
            for (int cc = 0; cc < 3; ++cc) uu[cc * n + b] = u[cc * n + j];
        if (p) pp[b] = p[j];
    }
    return put_patch(c, q, u ? uu.data() : nullptr, p ? pp.data() : nullptr);
}

extern "C" fv_status fv_piso_step(fv_case *c, const fv_piso_params *prm, fv_step_stats *stats)
{
    FV_CHECK(c, FV_E_INVALID, "NULL case");
    fv_status st = check_piso(prm);
    if (st != FV_OK) return st;
    int ref = -1;
    if ((st = check_ref(c, prm->p_ref_cell, &ref)) != FV_OK) return st;
    if ((st = piso_enqueue(c, prm, ref)) != FV_OK) return st;
    c->last_np = prm->n_corr * (1 + prm->n_nonorth);
    c->last_simple = false;
    if (!stats) return FV_OK;
    return read_stats(c, c->last_np, stats, false);
}

extern "C" fv_status fv_case_last_stats(fv_case *c, fv_step_stats *stats)
{
    FV_CHECK(c && stats, FV_E_INVALID, "NULL argument");
    return read_stats(c, c->last_np, stats, c->last_simple);
}

extern "C" fv_status fv_simple_iter(fv_case *c, const fv_simple_params *prm, fv_step_stats *stats)
{
    FV_CHECK(c && prm, FV_E_INVALID, "NULL argument");
    FV_CHECK(prm->alpha_u > 0.0 && prm->alpha_u <= 1.0 && prm->alpha_p > 0.0 && prm->alpha_p <= 1.0,
             FV_E_INVALID, "relaxation factors must be in (0, 1]");
    FV_CHECK(prm->p_maxit >= 0 && prm->u_maxit >= 0, FV_E_INVALID, "negative iteration limit");
    FV_CHECK(prm->n_nonorth >= 0 && 1 + prm->n_nonorth <= FV_MAX_CORR, FV_E_INVALID,
             "1 + n_nonorth must be at most %d", FV_MAX_CORR);
    const fv_mesh *m = c->mesh;
    int ref = -1;
    fv_status st = check_ref(c, prm->p_ref_cell, &ref);
    if (st != FV_OK) return st;
    StepArgs sa{0.0, prm->alpha_u, ref, prm->p_ref_value};
    if (m->nonorth) STAGE(FV_PROF_MOMENTUM, 1, launch_grad_u(c));
    STAGE(FV_PROF_MOMENTUM, 1, launch_momentum(c, sa));
    STAGE(FV_PROF_OTHER, 1, launch_simple_residuals_mom(c));
    BicgProblem bp{c->Md, c->Mo, nullptr, c->src, c->gradp, c->u, 3, prm->u_tol, prm->u_reltol,
                   prm->u_maxit, c->dstats};
    STAGE(FV_PROF_BICGSTAB, 1, launch_bicgstab(m, bp));
    STAGE(FV_PROF_HBYA, 1, launch_hbya(c));
    STAGE(FV_PROF_PRESSURE, 1, launch_pressure(c, sa));
    STAGE(FV_PROF_OTHER, 2, launch_simple_residuals_p(c));
    FV_CUDA(cudaMemcpyAsync(c->pold, c->p, sizeof(double) * m->N, cudaMemcpyDeviceToDevice, m->stream));
    const int nl = 1 + prm->n_nonorth;
    for (int j = 0; j < nl; ++j) {
        if (j > 0) {
            STAGE(FV_PROF_PRESSURE, 1, launch_grad_p(c));
            STAGE(FV_PROF_PRESSURE, 1, launch_pressure(c, sa));
        }
        STAGE(FV_PROF_PCG, 1, launch_pressure_solve(c, prm->p_tol, prm->p_reltol, prm->p_maxit,
                                                    c->dstats + 3 + j));
    }
    STAGE(FV_PROF_CORRECT, 2, launch_correct_simple(c, prm->alpha_p));
    c->last_np = nl;
    c->last_simple = true;
    if (!stats) return FV_OK;
    return read_stats(c, nl, stats, true);
}

extern "C" fv_status fv_piso_run_graph(fv_case *c, const fv_piso_params *prm, int32_t n_steps,
                                       fv_step_stats *stats)
{
    FV_CHECK(c, FV_E_INVALID, "NULL case");
    fv_status st = check_piso(prm);
    if (st != FV_OK) return st;
    FV_CHECK(n_steps >= 0, FV_E_INVALID, "negative step count");
    const fv_mesh *m = c->mesh;
    FV_CHECK(m->stream != nullptr, FV_E_UNSUPPORTED, "graph replay needs a non-default stream");
    int ref = -1;
    if ((st = check_ref(c, prm->p_ref_cell, &ref)) != FV_OK) return st;
    if (c->graph && std::memcmp(&c->graph_prm, prm, sizeof(*prm)) != 0) {
        cudaGraphExecDestroy(c->graph);
        c->graph = nullptr;
    }
    if (!c->graph) {
        cudaGraph_t g = nullptr;
        FV_CUDA(cudaStreamBeginCapture(m->stream, cudaStreamCaptureModeThreadLocal));
        st = piso_enqueue(c, prm, ref);
        cudaError_t e = cudaStreamEndCapture(m->stream, &g);
        if (st != FV_OK) { if (g) cudaGraphDestroy(g); return st; }
        if (e != cudaSuccess) return cuda_status(e, "cudaStreamEndCapture");
        e = cudaGraphInstantiate(&c->graph, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) { c->graph = nullptr; return cuda_status(e, "cudaGraphInstantiate"); }
        c->graph_prm = *prm;
    }
    for (int s = 0; s < n_steps; ++s) FV_CUDA(cudaGraphLaunch(c->graph, m->stream));
    c->last_np = prm->n_corr * (1 + prm->n_nonorth);
    c->last_simple = false;
    if (!stats) return FV_OK;
    return read_stats(c, c->last_np, stats, false);
}

// ------------------------------------------------ stand-alone operators --

extern "C" fv_status fv_pcg_solve(const fv_mesh *mc, const double *diag, const double *upper,
                                  const double *b, double *x, const fv_pcg_params *prm,
                                  fv_solve_stats *stats)
{
    FV_CHECK(mc && diag && b && x && prm, FV_E_INVALID, "NULL argument");
    FV_CHECK(mc->F == 0 || upper, FV_E_INVALID, "upper is NULL");
    FV_CHECK(prm->maxit >= 0 && prm->tol >= 0.0 && prm->reltol >= 0.0, FV_E_INVALID, "bad params");
    fv_mesh *m = const_cast<fv_mesh *>(mc);
    fv_status st = launch_ldu_to_sell(m, upper, upper, m->kw.val);
    if (st != FV_OK) return st;
    CgProblem cp{diag, m->kw.val, b, x, prm->tol, prm->reltol, prm->maxit, m->kw.stats};
    if ((st = launch_pcg(m, cp)) != FV_OK) return st;
    DevSolveStats h;
    FV_CUDA(cudaMemcpyAsync(&h, m->kw.stats, sizeof(h), cudaMemcpyDeviceToHost, m->stream));
    FV_CUDA(cudaStreamSynchronize(m->stream));
    if (stats) fill_solve(stats, h);
    return (fv_status)h.status;
}

static fv_status pcg_solve_amg(const fv_mesh *mc, const double *diag, const double *upper,
                               const double *b, double *x, const fv_pcg_params *prm,
                               fv_solve_stats *stats, int fp32)
{
    FV_CHECK(mc && diag && b && x && prm, FV_E_INVALID, "NULL argument");
    FV_CHECK(mc->F == 0 || upper, FV_E_INVALID, "upper is NULL");
    FV_CHECK(prm->maxit >= 0 && prm->tol >= 0.0 && prm->reltol >= 0.0, FV_E_INVALID, "bad params");
    fv_mesh *m = const_cast<fv_mesh *>(mc);
    fv_status st = amg_prepare(m);
    if (st != FV_OK) return st;
    AmgProblem ap{diag, upper, 1.0, b, x, prm->tol, prm->reltol, prm->maxit, m->kw.stats, fp32};
    if ((st = launch_pcg_amg(m, ap)) != FV_OK) return st;
    DevSolveStats h;
    FV_CUDA(cudaMemcpyAsync(&h, m->kw.stats, sizeof(h), cudaMemcpyDeviceToHost, m->stream));
    FV_CUDA(cudaStreamSynchronize(m->stream));
    if (stats) fill_solve(stats, h);
    return (fv_status)h.status;
}

extern "C" fv_status fv_pcg_solve_amg(const fv_mesh *mc, const double *diag, const double *upper,
                                      const double *b, double *x, const fv_pcg_params *prm,
                                      fv_solve_stats *stats)
{
    return pcg_solve_amg(mc, diag, upper, b, x, prm, stats, 0);
}

extern "C" fv_status fv_pcg_solve_amg_mixed(const fv_mesh *mc, const double *diag,
                                            const double *upper, const double *b, double *x,
                                            const fv_pcg_params *prm, fv_solve_stats *stats)
{
    return pcg_solve_amg(mc, diag, upper, b, x, prm, stats, 1);
}

extern "C" fv_status fv_case_set_pressure_solver(fv_case *c, int32_t solver)
{
    FV_CHECK(c, FV_E_INVALID, "NULL case");
    FV_CHECK(solver == FV_PSOLVER_JACOBI || solver == FV_PSOLVER_AMG, FV_E_INVALID,
             "unknown pressure solver %d", solver);
    if (solver == FV_PSOLVER_AMG) {
        fv_status st = amg_prepare(const_cast<fv_mesh *>(c->mesh));
        if (st != FV_OK) return st;
    }
    if (c->psolver != solver && c->graph) {
        cudaGraphExecDestroy(c->graph);
        c->graph = nullptr;
    }
    c->psolver = solver;
    return FV_OK;
}

extern "C" fv_status fv_pcg_solve_mixed(const fv_mesh *mc, const double *diag, const double *upper,
                                        const double *b, double *x, const fv_pcg_params *prm,
                                        fv_solve_stats *stats)
{
    FV_CHECK(mc && diag && b && x && prm, FV_E_INVALID, "NULL argument");
    FV_CHECK(mc->F == 0 || upper, FV_E_INVALID, "upper is NULL");
    FV_CHECK(prm->maxit >= 0 && prm->tol >= 0.0 && prm->reltol >= 0.0, FV_E_INVALID, "bad params");
    fv_mesh *m = const_cast<fv_mesh *>(mc);
    fv_status st = launch_ldu_to_sell(m, upper, upper, m->kw.val);
    if (st != FV_OK) return st;
    MixedProblem mp{diag, m->kw.val, b, x, prm->tol, prm->reltol, prm->maxit, m->kw.stats};
    if ((st = launch_pcg_mixed(m, mp)) != FV_OK) return st;
    DevSolveStats h;
    FV_CUDA(cudaMemcpyAsync(&h, m->kw.stats, sizeof(h), cudaMemcpyDeviceToHost, m->stream));
    FV_CUDA(cudaStreamSynchronize(m->stream));
    if (stats) fill_solve(stats, h);
    return (fv_status)h.status;
}

extern "C" fv_status fv_bicgstab_solve(const fv_mesh *mc, const double *diag, const double *upper,
                                       const double *lower, const double *b, double *x,
                                       const fv_pcg_params *prm, fv_solve_stats *stats)
{
    FV_CHECK(mc && diag && b && x && prm, FV_E_INVALID, "NULL argument");
    FV_CHECK(mc->F == 0 || (upper && lower), FV_E_INVALID, "upper/lower is NULL");
    FV_CHECK(prm->maxit >= 0 && prm->tol >= 0.0 && prm->reltol >= 0.0, FV_E_INVALID, "bad params");
    fv_mesh *m = const_cast<fv_mesh *>(mc);
    fv_status st = launch_ldu_to_sell(m, upper, lower, m->kw.val2);
    if (st != FV_OK) return st;
    BicgProblem bp{diag, m->kw.val2, b, nullptr, nullptr, x, 1, prm->tol, prm->reltol, prm->maxit,
                   m->kw.stats};
    if ((st = launch_bicgstab(m, bp)) != FV_OK) return st;
    DevSolveStats h;
    FV_CUDA(cudaMemcpyAsync(&h, m->kw.stats, sizeof(h), cudaMemcpyDeviceToHost, m->stream));
    FV_CUDA(cudaStreamSynchronize(m->stream));
    if (stats) fill_solve(stats, h);
    return (fv_status)h.status;
}

extern "C" fv_status fv_gauss_grad(const fv_mesh *m, const double *x, const double *xb, double *g)
{
    FV_CHECK(m && x && g && (m->B == 0 || xb), FV_E_INVALID, "NULL argument");
    fv_status st = launch_gauss_grad(m, x, xb, g);
    if (st != FV_OK) return st;
    FV_CUDA(cudaStreamSynchronize(m->stream));
    return FV_OK;
}

extern "C" fv_status fv_ldu_matvec(const fv_mesh *m, const double *diag, const double *upper,
                                   const double *lower, const double *x, double *y)
{
    FV_CHECK(m && diag && x && y, FV_E_INVALID, "NULL argument");
    FV_CHECK(m->F == 0 || (upper && lower), FV_E_INVALID, "upper/lower is NULL");
    fv_status st = launch_ldu_matvec(m, diag, upper, lower, x, y);
    if (st != FV_OK) return st;
    FV_CUDA(cudaStreamSynchronize(m->stream));
    return FV_OK;
}
