// mesh.cu -- fv_mesh_create / destroy and the one-time geometry kernel.
//
// Geometry (the paper defers the discretisation to the textbook finite-volume
// method, Sec. 3): for an internal face with owner P, neighbour N, area
// vector S (P -> N), n = S/|S|, d = C_N - C_P:
//   w     = n.(C_N - Cf) / (n.(C_N - Cf) + n.(Cf - C_P))   face value
//           x_f = w x_P + (1 - w) x_N;
//   delta = 1 / max(n.d, 0.05 |d|);   k = n - delta d  (over-relaxed split of
//           S into |S| delta d + |S| k, the non-orthogonal correction);
// boundary faces use d = Cf - C_P and carry no k.
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>

#include "fvgb_internal.h"

namespace fvgb {

static thread_local char g_err[512] = "";

void set_error(const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

fv_status cuda_status(cudaError_t e, const char *what)
{
    set_error("%s: %s", what, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? FV_E_NOMEM : FV_E_CUDA;
}

// Fault injection for tests: FVGB_FAIL_ALLOC_AFTER=k makes the (k+1)-th
// device allocation of the process fail with FV_E_NOMEM (host-side only).
static long long alloc_budget()
{
    static long long left = [] {
        const char *e = getenv("FVGB_FAIL_ALLOC_AFTER");
        return e ? atoll(e) : -1LL;
    }();
    return left < 0 ? 1 : left--;
}

fv_status DeviceArena::alloc(void **p, size_t n)
{
    *p = nullptr;
    if (alloc_budget() == 0) {
        set_error("device allocation refused (FVGB_FAIL_ALLOC_AFTER)");
        return FV_E_NOMEM;
    }
    if (n == 0) n = 16;
    n = (n + 255) & ~size_t(255);
    cudaError_t e = cudaMalloc(p, n);
    if (e != cudaSuccess) {
        *p = nullptr;
        return cuda_status(e, "cudaMalloc");
    }
    ptrs.push_back(*p);
    bytes += n;
    return FV_OK;
}

void DeviceArena::release()
{
    for (void *p : ptrs) cudaFree(p);
    ptrs.clear();
    bytes = 0;
}

// Face geometry, one thread per face.  Uses explicit products (no fused
// multiply-add in the dot products) so that the values follow the formulas
// above term by term.
__global__ void k_face_geometry(int F, int M, int N, const int32_t *__restrict__ own,
                                const int32_t *__restrict__ nei, const double *__restrict__ Sf,
                                const double *__restrict__ Cf, const double *__restrict__ C,
                                double *__restrict__ magSf, double *__restrict__ w,
                                double *__restrict__ delta, double *__restrict__ kv,
                                int *__restrict__ nonorth)
{
    int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= M) return;
    double S[3], n[3], d[3], cf[3], cp[3];
    const int P = own[f];
    for (int c = 0; c < 3; ++c) {
        S[c] = Sf[(size_t)c * M + f];
        cf[c] = Cf[(size_t)c * M + f];
        cp[c] = C[(size_t)c * N + P];
    }
    double mag = sqrt(__dadd_rn(__dadd_rn(__dmul_rn(S[0], S[0]), __dmul_rn(S[1], S[1])),
                                __dmul_rn(S[2], S[2])));
    magSf[f] = mag;
    for (int c = 0; c < 3; ++c) n[c] = S[c] / mag;
    if (f < F) {
        const int Q = nei[f];
        double cn[3];
        for (int c = 0; c < 3; ++c) cn[c] = C[(size_t)c * N + Q];
        double a1 = 0.0, a2 = 0.0;
        for (int c = 0; c < 3; ++c) {
            a1 = __dadd_rn(a1, __dmul_rn(n[c], cn[c] - cf[c]));
            a2 = __dadd_rn(a2, __dmul_rn(n[c], cf[c] - cp[c]));
        }
        w[f] = a1 / (a1 + a2);
        for (int c = 0; c < 3; ++c) d[c] = cn[c] - cp[c];
    } else {
        for (int c = 0; c < 3; ++c) d[c] = cf[c] - cp[c];
    }
    double nd = __dadd_rn(__dadd_rn(__dmul_rn(n[0], d[0]), __dmul_rn(n[1], d[1])), __dmul_rn(n[2], d[2]));
    double dm = sqrt(__dadd_rn(__dadd_rn(__dmul_rn(d[0], d[0]), __dmul_rn(d[1], d[1])),
                               __dmul_rn(d[2], d[2])));
    double lim = 0.05 * dm;
    double de = 1.0 / (nd > lim ? nd : lim);
    delta[f] = de;
    if (f < F) {
        double kk = 0.0;
        for (int c = 0; c < 3; ++c) {
            double k = n[c] - __dmul_rn(de, d[c]);
            kv[(size_t)c * F + f] = k;
            kk = __dadd_rn(kk, __dmul_rn(k, k));
        }
        // the explicit non-orthogonal terms are active for the whole mesh
        // when any internal face has |k| > 1e-8 (|k| is dimensionless)
        if (sqrt(kk) > 1e-8) atomicOr(nonorth, 1);
    }
}

__global__ void k_recip(int n, const double *__restrict__ x, double *__restrict__ y)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = 1.0 / x[i];
}

template <class T>
static fv_status upload(DeviceArena &a, T **dst, const T *src, size_t n, cudaStream_t s)
{
    fv_status st = a.alloc_n(dst, n);
    if (st != FV_OK) return st;
    if (n) FV_CUDA(cudaMemcpyAsync(*dst, src, n * sizeof(T), cudaMemcpyHostToDevice, s));
    return FV_OK;
}

fv_status upload_mesh(fv_mesh *m, const fv_mesh_desc *d)
{
    const MeshPlan &pl = m->plan;
    const int N = m->N, F = m->F, B = m->B, M = m->M;
    cudaStream_t s = m->stream;
    DeviceArena &a = m->arena;
    fv_status st;
#define UP(dst, src, n) if ((st = upload(a, &(dst), (src), (n), s)) != FV_OK) return st
    UP(m->own, pl.own.data(), (size_t)M);
    UP(m->nei, pl.nei.data(), (size_t)F);
    UP(m->slice_ptr, pl.slice_ptr.data(), pl.slice_ptr.size());
    UP(m->col, pl.col.data(), pl.col.size());
    UP(m->sface, pl.sface.data(), pl.sface.size());
    UP(m->bptr, pl.bptr.data(), pl.bptr.size());
    UP(m->bface, pl.bface.data(), pl.bface.size());
    UP(m->cell_new_of_old, pl.cell_new_of_old.data(), (size_t)N);
    UP(m->face_new_of_old, pl.face_new_of_old.data(), (size_t)M);
    UP(m->flipped, pl.flipped.data(), (size_t)M);
    m->nslice = pl.nslice;
    m->nnz = (int)pl.col.size();
    std::vector<int8_t> bt(B);
    for (int k = 0; k < B; ++k) bt[k] = (int8_t)m->patches[pl.bpatch[k]].type;
    UP(m->btype, bt.data(), (size_t)B);

    // geometry inputs in internal order (host permutation, then upload)
    std::vector<double> Sf((size_t)3 * M), Cf((size_t)3 * M), C((size_t)3 * N), V(N);
    for (int f = 0; f < M; ++f) {
        const int g = pl.face_new_of_old[f];
        const double sg = pl.flipped[f] ? -1.0 : 1.0;
        for (int c = 0; c < 3; ++c) {
            Sf[(size_t)c * M + g] = sg * d->Sf[(size_t)c * M + f];
            Cf[(size_t)c * M + g] = d->Cf[(size_t)c * M + f];
        }
    }
    for (int i = 0; i < N; ++i) {
        const int j = pl.cell_new_of_old[i];
        for (int c = 0; c < 3; ++c) C[(size_t)c * N + j] = d->C[(size_t)c * N + i];
        V[j] = d->V[i];
    }
    UP(m->Sf, Sf.data(), Sf.size());
    UP(m->V, V.data(), V.size());
    // temporaries of the geometry kernel, freed when this function returns
    struct Tmp {
        DeviceArena a;
        ~Tmp() { a.release(); }
    } tmp;
    double *dCf = nullptr, *dC = nullptr;
    int *dflag = nullptr;
    if ((st = tmp.a.alloc_n(&dCf, Cf.size())) != FV_OK) return st;
    if ((st = tmp.a.alloc_n(&dC, C.size())) != FV_OK) return st;
    if ((st = tmp.a.alloc_n(&dflag, 1)) != FV_OK) return st;
    FV_CUDA(cudaMemcpyAsync(dCf, Cf.data(), sizeof(double) * Cf.size(), cudaMemcpyHostToDevice, s));
    FV_CUDA(cudaMemcpyAsync(dC, C.data(), sizeof(double) * C.size(), cudaMemcpyHostToDevice, s));
    FV_CUDA(cudaMemsetAsync(dflag, 0, sizeof(int), s));
    if ((st = a.alloc_n(&m->magSf, M)) != FV_OK) return st;
    if ((st = a.alloc_n(&m->w, F)) != FV_OK) return st;
    if ((st = a.alloc_n(&m->delta, M)) != FV_OK) return st;
    if ((st = a.alloc_n(&m->kv, (size_t)3 * F)) != FV_OK) return st;
    if ((st = a.alloc_n(&m->Vinv, N)) != FV_OK) return st;
#undef UP
    if (M > 0)
        k_face_geometry<<<(M + 255) / 256, 256, 0, s>>>(F, M, N, m->own, m->nei, m->Sf, dCf, dC,
                                                        m->magSf, m->w, m->delta, m->kv, dflag);
    k_recip<<<(N + 255) / 256, 256, 0, s>>>(N, m->V, m->Vinv);
    FV_CUDA(cudaGetLastError());
    int flag = 0;
    FV_CUDA(cudaMemcpyAsync(&flag, dflag, sizeof(int), cudaMemcpyDeviceToHost, s));
    FV_CUDA(cudaStreamSynchronize(s));
    m->nonorth = flag;
    return FV_OK;
}

}  // namespace fvgb

using namespace fvgb;

extern "C" const char *fv_last_error(void) { return g_err; }

extern "C" fv_status fv_mesh_create(const fv_mesh_desc *desc, void *stream, fv_mesh **out)
{
    FV_CHECK(out != nullptr, FV_E_INVALID, "out is NULL");
    *out = nullptr;
    fv_mesh *m = new (std::nothrow) fv_mesh();
    FV_CHECK(m != nullptr, FV_E_NOMEM, "host allocation failed");
    fv_status st;
    try {
        st = build_plan(desc, &m->plan);
        if (st != FV_OK) { delete m; return st; }
        m->N = desc->n_cells;
        m->F = desc->n_internal_faces;
        m->B = desc->n_boundary_faces;
        m->M = m->F + m->B;
        m->np = desc->n_patches;
        m->patches.assign(desc->patches, desc->patches + desc->n_patches);
        m->stream = static_cast<cudaStream_t>(stream);
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        m->device = dev;
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&m->sm_count, cudaDevAttrMultiProcessorCount, dev);
        int pageable = 0, host_tables = 0;
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&pageable, cudaDevAttrPageableMemoryAccess, dev);
        if (e == cudaSuccess)
            e = cudaDeviceGetAttribute(&host_tables, cudaDevAttrPageableMemoryAccessUsesHostPageTables, dev);
        if (e != cudaSuccess) { delete m; return cuda_status(e, "device query"); }
        // host-buffer field exchange straight from and to the caller's memory
        // where the device reaches pageable memory through the host's page
        // tables; FVGB_HOST_STAGING=1 keeps the pinned staging copy
        const char *staging = std::getenv("FVGB_HOST_STAGING");
        m->host_direct = pageable && host_tables && !(staging && std::atoi(staging) != 0);
        st = upload_mesh(m, desc);
        if (st == FV_OK) st = krylov_setup(m);
    } catch (const std::bad_alloc &) {
        set_error("host allocation failed in fv_mesh_create");
        st = FV_E_NOMEM;
    }
    if (st != FV_OK) {
        m->arena.release();
        delete m;
        return st;
    }
    *out = m;
    return FV_OK;
}

extern "C" fv_status fv_mesh_destroy(fv_mesh *m)
{
    if (!m) return FV_OK;
    cudaStreamSynchronize(m->stream);
    fvgb::amg_release(m->amg);
    m->amg = nullptr;
    m->arena.release();
    delete m;
    return FV_OK;
}

extern "C" fv_status fv_mesh_cell_order(const fv_mesh *m, int32_t *new_of_old)
{
    FV_CHECK(m && new_of_old, FV_E_INVALID, "NULL argument");
    std::memcpy(new_of_old, m->plan.cell_new_of_old.data(), sizeof(int32_t) * m->N);
    return FV_OK;
}

extern "C" fv_status fv_mesh_face_order(const fv_mesh *m, int32_t *new_of_old, int8_t *flipped)
{
    FV_CHECK(m && new_of_old, FV_E_INVALID, "NULL argument");
    std::memcpy(new_of_old, m->plan.face_new_of_old.data(), sizeof(int32_t) * m->M);
    if (flipped) std::memcpy(flipped, m->plan.flipped.data(), m->M);
    return FV_OK;
}

extern "C" fv_status fv_mesh_info(const fv_mesh *m, int32_t *info)
{
    FV_CHECK(m && info, FV_E_INVALID, "NULL argument");
    info[0] = m->N;
    info[1] = m->F;
    info[2] = m->B;
    info[3] = m->nonorth;
    return FV_OK;
}

extern "C" fv_status fv_mesh_addressing(const fv_mesh *m, int32_t *owner, int32_t *neighbour)
{
    FV_CHECK(m, FV_E_INVALID, "NULL mesh");
    if (owner)
        FV_CUDA(cudaMemcpyAsync(owner, m->own, sizeof(int32_t) * m->M, cudaMemcpyDeviceToDevice,
                                m->stream));
    if (neighbour && m->F)
        FV_CUDA(cudaMemcpyAsync(neighbour, m->nei, sizeof(int32_t) * m->F,
                                cudaMemcpyDeviceToDevice, m->stream));
    FV_CUDA(cudaStreamSynchronize(m->stream));
    return FV_OK;
}
