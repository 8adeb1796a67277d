// ellj.cu -- the paper's hybrid matrix storage (Sec. 3.1): ELL for the first
// K entries of every row, the transpose-index array J that lets the same
// arrays be read by columns, and CRS for the entries that do not fit.
//
// The solver path keeps its matrices in SELL-32 slots filled row by row
// (both cells of a face evaluate the face's coefficient), so it never reads
// a matrix by columns.  This storage is the paper's alternative; it is
// provided with its own assembly from LDU coefficients and the row (SMVP)
// and column (STMVP) products so the two layouts can be compared.
//
// Device layout: slot k of row i at k * N + i (coalesced across a warp).
// Locations of matrix entries are encoded as k * N + i (ELL) or -1 - p (CRS
// position p).
#include <algorithm>
#include <new>
#include <vector>

#include "fvgb_internal.h"

using namespace fvgb;

struct fv_ellj {
    int N = 0, F = 0, K = 0, ncrs = 0;
    cudaStream_t stream = nullptr;
    DeviceArena arena;
    int32_t *I = nullptr, *J = nullptr, *Q = nullptr;          // [K][N]
    int32_t *crs_ptr = nullptr, *crs_col = nullptr, *crs_tr = nullptr;
    int32_t *loc_diag = nullptr, *loc_up = nullptr, *loc_lo = nullptr;
};

namespace {

constexpr int kEllBlock = 256;

// Where entry (row, c) lives: its ELL slot, or -2 - p for CRS position p.
// Columns of a row are ascending, so the entry is found by bisection.
int find_entry(const int32_t *row_ptr, const int32_t *col, int K, const int32_t *crs_ptr,
               int row, int c)
{
    const int32_t *b = col + row_ptr[row], *e = col + row_ptr[row + 1];
    const int32_t *it = std::lower_bound(b, e, c);
    if (it == e || *it != c) return -1;
    const int t = (int)(it - b);
    return t < K ? t : -2 - (crs_ptr[row] + (t - K));
}

__global__ void k_ellj_from_ldu(int N, int F, const int32_t *__restrict__ loc_diag,
                                const int32_t *__restrict__ loc_up,
                                const int32_t *__restrict__ loc_lo,
                                const double *__restrict__ diag, const double *__restrict__ upper,
                                const double *__restrict__ lower, double *__restrict__ V,
                                double *__restrict__ C)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < N) {
        const int l = loc_diag[t];
        if (l >= 0) V[l] = diag[t];
        else C[-1 - l] = diag[t];
    }
    if (t < F) {
        const int lu = loc_up[t], ll = loc_lo[t];
        if (lu >= 0) V[lu] = upper[t];
        else C[-1 - lu] = upper[t];
        if (ll >= 0) V[ll] = lower[t];
        else C[-1 - ll] = lower[t];
    }
}

__global__ void k_ellj_zero_pad(int N, int K, const int32_t *__restrict__ I, double *__restrict__ V)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    for (int k = 0; k < K; ++k)
        if (I[(size_t)k * N + i] < 0) V[(size_t)k * N + i] = 0.0;
}

// y = A x: ELL slots, then the row's CRS tail (column order).
__global__ void k_ellj_spmv(int N, int K, const int32_t *__restrict__ I,
                            const int32_t *__restrict__ crs_ptr, const int32_t *__restrict__ crs_col,
                            const double *__restrict__ V, const double *__restrict__ C,
                            const double *__restrict__ x, double *__restrict__ y)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    double acc = 0.0;
    for (int k = 0; k < K; ++k) {
        const int c = I[(size_t)k * N + i];
        if (c >= 0) acc += V[(size_t)k * N + i] * x[c];
    }
    if (crs_ptr)
        for (int p = crs_ptr[i]; p < crs_ptr[i + 1]; ++p) acc += C[p] * x[crs_col[p]];
    y[i] = acc;
}

// y = A^T x by columns: entry (i, j) of the pattern names the transposed
// entry A_ji through J (ELL slot in row j, or -2 - p in the CRS part).
__global__ void k_ellj_stmvp(int N, int K, const int32_t *__restrict__ I,
                             const int32_t *__restrict__ J, const int32_t *__restrict__ crs_ptr,
                             const int32_t *__restrict__ crs_col, const int32_t *__restrict__ crs_tr,
                             const double *__restrict__ V, const double *__restrict__ C,
                             const double *__restrict__ x, double *__restrict__ y)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    double acc = 0.0;
    for (int k = 0; k < K; ++k) {
        const int j = I[(size_t)k * N + i];
        if (j < 0) continue;
        const int l = J[(size_t)k * N + i];
        const double a = l >= 0 ? V[(size_t)l * N + j] : C[-2 - l];
        acc += a * x[j];
    }
    if (crs_ptr)
        for (int p = crs_ptr[i]; p < crs_ptr[i + 1]; ++p) {
            const int j = crs_col[p], l = crs_tr[p];
            const double a = l >= 0 ? V[(size_t)l * N + j] : C[-2 - l];
            acc += a * x[j];
        }
    y[i] = acc;
}

// Same product through the packed index Q = K I + J (matrices without a CRS
// part): one integer load per slot instead of two.
__global__ void k_ellj_stmvp_q(int N, int K, const int32_t *__restrict__ Q,
                               const double *__restrict__ V, const double *__restrict__ x,
                               double *__restrict__ y)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    double acc = 0.0;
    for (int k = 0; k < K; ++k) {
        const int q = Q[(size_t)k * N + i];
        if (q < 0) continue;
        const int j = q / K, l = q - j * K;
        acc += V[(size_t)l * N + j] * x[j];
    }
    y[i] = acc;
}

int blocks(int n) { return (n + kEllBlock - 1) / kEllBlock; }

}  // namespace

extern "C" fv_status fv_ellj_build_host(int32_t n, const int32_t *row_ptr, const int32_t *col,
                                        int32_t K, int32_t *I, int32_t *J, int32_t *crs_ptr,
                                        int32_t *crs_col, int32_t *crs_tr, int32_t *n_crs)
{
    FV_CHECK(n >= 0 && row_ptr && (n == 0 || col) && crs_ptr && n_crs, FV_E_INVALID,
             "bad arguments");
    FV_CHECK(K >= 1, FV_E_INVALID, "K must be at least 1");
    crs_ptr[0] = 0;
    for (int i = 0; i < n; ++i) {
        const int len = row_ptr[i + 1] - row_ptr[i];
        FV_CHECK(len >= 0, FV_E_INVALID, "row_ptr not monotone at row %d", i);
        for (int t = 1; t < len; ++t)
            FV_CHECK(col[row_ptr[i] + t - 1] < col[row_ptr[i] + t], FV_E_INVALID,
                     "columns of row %d not strictly ascending", i);
        crs_ptr[i + 1] = crs_ptr[i] + std::max(0, len - K);
    }
    *n_crs = crs_ptr[n];
    if (!I) return FV_OK;
    FV_CHECK(J && (crs_ptr[n] == 0 || (crs_col && crs_tr)), FV_E_INVALID, "output arrays missing");
    for (int i = 0; i < n; ++i) {
        const int r0 = row_ptr[i], len = row_ptr[i + 1] - r0;
        for (int t = 0; t < std::max(len, (int)K); ++t) {
            if (t >= len) {   // empty ELL slot
                I[(size_t)i * K + t] = -1;
                J[(size_t)i * K + t] = -1;
                continue;
            }
            const int c = col[r0 + t];
            FV_CHECK(c >= 0 && c < n, FV_E_INVALID, "column %d out of range in row %d", c, i);
            const int tr = find_entry(row_ptr, col, K, crs_ptr, c, i);
            FV_CHECK(tr != -1, FV_E_INVALID, "entry (%d,%d) has no transpose", i, c);
            if (t < K) {
                I[(size_t)i * K + t] = c;
                J[(size_t)i * K + t] = tr;
            } else {
                const int p = crs_ptr[i] + (t - K);
                crs_col[p] = c;
                crs_tr[p] = tr;
            }
        }
    }
    return FV_OK;
}

extern "C" fv_status fv_ellj_create(const fv_mesh *m, int32_t K, fv_ellj **out)
{
    FV_CHECK(m && out, FV_E_INVALID, "NULL argument");
    FV_CHECK(K >= 0, FV_E_INVALID, "negative K");
    *out = nullptr;
    const int N = m->N, F = m->F;
    const MeshPlan &pl = m->plan;
    // row structure: diagonal and both sides of every internal face, ascending
    std::vector<int32_t> row_ptr(N + 1, 0), col;
    for (int f = 0; f < F; ++f) { ++row_ptr[pl.own[f] + 1]; ++row_ptr[pl.nei[f] + 1]; }
    for (int i = 0; i < N; ++i) row_ptr[i + 1] += row_ptr[i] + 1;
    col.resize(row_ptr[N]);
    {
        std::vector<int32_t> fill(row_ptr.begin(), row_ptr.end() - 1);
        for (int i = 0; i < N; ++i) col[fill[i]++] = i;
        for (int f = 0; f < F; ++f) {
            col[fill[pl.own[f]]++] = pl.nei[f];
            col[fill[pl.nei[f]]++] = pl.own[f];
        }
        for (int i = 0; i < N; ++i) std::sort(col.begin() + row_ptr[i], col.begin() + row_ptr[i + 1]);
    }
    if (K == 0) {   // the most frequent row length (the larger one on a tie)
        std::vector<int> hist;
        for (int i = 0; i < N; ++i) {
            const int len = row_ptr[i + 1] - row_ptr[i];
            if (len >= (int)hist.size()) hist.resize(len + 1, 0);
            ++hist[len];
        }
        K = 1;
        for (int l = 1; l < (int)hist.size(); ++l)
            if (hist[l] >= hist[K]) K = l;
    }
    FV_CHECK((int64_t)K * N < (int64_t)1 << 31, FV_E_INVALID, "K x N exceeds the int32 range");
    std::vector<int32_t> I((size_t)N * K), J((size_t)N * K), crs_ptr(N + 1);
    int32_t ncrs = 0;
    fv_status st = fv_ellj_build_host(N, row_ptr.data(), col.data(), K, nullptr, nullptr,
                                      crs_ptr.data(), nullptr, nullptr, &ncrs);
    if (st != FV_OK) return st;
    std::vector<int32_t> crs_col(std::max(ncrs, 1)), crs_tr(std::max(ncrs, 1));
    st = fv_ellj_build_host(N, row_ptr.data(), col.data(), K, I.data(), J.data(), crs_ptr.data(),
                            crs_col.data(), crs_tr.data(), &ncrs);
    if (st != FV_OK) return st;
    // device layout [K][N] and entry locations for the LDU assembly
    std::vector<int32_t> Ic((size_t)N * K), Jc((size_t)N * K), Qc;
    for (int i = 0; i < N; ++i)
        for (int k = 0; k < K; ++k) {
            Ic[(size_t)k * N + i] = I[(size_t)i * K + k];
            Jc[(size_t)k * N + i] = J[(size_t)i * K + k];
        }
    if (ncrs == 0) {
        Qc.resize((size_t)N * K);
        for (size_t e = 0; e < Qc.size(); ++e) Qc[e] = Ic[e] < 0 ? -1 : K * Ic[e] + Jc[e];
    }
    auto loc = [&](int row, int c) {
        const int t = find_entry(row_ptr.data(), col.data(), K, crs_ptr.data(), row, c);
        return t >= 0 ? t * N + row : -1 - (-2 - t);
    };
    std::vector<int32_t> ld(N), lu(std::max(F, 1)), ll(std::max(F, 1));
    for (int i = 0; i < N; ++i) ld[i] = loc(i, i);
    for (int f = 0; f < F; ++f) {
        lu[f] = loc(pl.own[f], pl.nei[f]);
        ll[f] = loc(pl.nei[f], pl.own[f]);
    }
    fv_ellj *e = new (std::nothrow) fv_ellj();
    FV_CHECK(e != nullptr, FV_E_NOMEM, "host allocation failed");
    e->N = N; e->F = F; e->K = K; e->ncrs = ncrs; e->stream = m->stream;
    auto up = [&](int32_t **d, const std::vector<int32_t> &h) -> fv_status {
        fv_status s = e->arena.alloc_n(d, h.size());
        if (s != FV_OK) return s;
        if (cudaMemcpy(*d, h.data(), sizeof(int32_t) * h.size(), cudaMemcpyHostToDevice) != cudaSuccess)
            return FV_E_CUDA;
        return FV_OK;
    };
    if ((st = up(&e->I, Ic)) == FV_OK && (st = up(&e->J, Jc)) == FV_OK &&
        (st = up(&e->loc_diag, ld)) == FV_OK && (st = up(&e->loc_up, lu)) == FV_OK &&
        (st = up(&e->loc_lo, ll)) == FV_OK) {
        if (ncrs > 0) {
            if ((st = up(&e->crs_ptr, crs_ptr)) == FV_OK && (st = up(&e->crs_col, crs_col)) == FV_OK)
                st = up(&e->crs_tr, crs_tr);
        } else {
            st = up(&e->Q, Qc);
        }
    }
    if (st != FV_OK) {
        e->arena.release();
        delete e;
        return st;
    }
    *out = e;
    return FV_OK;
}

extern "C" fv_status fv_ellj_destroy(fv_ellj *e)
{
    if (!e) return FV_OK;
    cudaStreamSynchronize(e->stream);
    e->arena.release();
    delete e;
    return FV_OK;
}

extern "C" fv_status fv_ellj_info(const fv_ellj *e, int32_t *K, int32_t *n_crs)
{
    FV_CHECK(e, FV_E_INVALID, "NULL storage");
    if (K) *K = e->K;
    if (n_crs) *n_crs = e->ncrs;
    return FV_OK;
}

extern "C" fv_status fv_ellj_from_ldu(const fv_ellj *e, const double *diag, const double *upper,
                                      const double *lower, double *V, double *C)
{
    FV_CHECK(e && diag && V && (e->F == 0 || (upper && lower)), FV_E_INVALID, "NULL argument");
    FV_CHECK(e->ncrs == 0 || C, FV_E_INVALID, "C is NULL but the storage has a CRS part");
    const int n = std::max(e->N, e->F);
    if (e->N > 0) {
        k_ellj_zero_pad<<<blocks(e->N), kEllBlock, 0, e->stream>>>(e->N, e->K, e->I, V);
        FV_CUDA(cudaGetLastError());
    }
    if (n > 0) {
        k_ellj_from_ldu<<<blocks(n), kEllBlock, 0, e->stream>>>(e->N, e->F, e->loc_diag, e->loc_up,
                                                                e->loc_lo, diag, upper, lower, V, C);
        FV_CUDA(cudaGetLastError());
    }
    return FV_OK;
}

extern "C" fv_status fv_ellj_spmv(const fv_ellj *e, const double *V, const double *C,
                                  const double *x, double *y, int32_t mode)
{
    FV_CHECK(e && V && x && y, FV_E_INVALID, "NULL argument");
    FV_CHECK(e->ncrs == 0 || C, FV_E_INVALID, "C is NULL but the storage has a CRS part");
    FV_CHECK(mode >= 0 && mode <= 2, FV_E_INVALID, "unknown mode %d", mode);
    FV_CHECK(mode != 2 || e->Q, FV_E_UNSUPPORTED, "the packed index needs a storage without CRS part");
    if (e->N == 0) return FV_OK;
    if (mode == 0)
        k_ellj_spmv<<<blocks(e->N), kEllBlock, 0, e->stream>>>(e->N, e->K, e->I, e->crs_ptr,
                                                               e->crs_col, V, C, x, y);
    else if (mode == 1)
        k_ellj_stmvp<<<blocks(e->N), kEllBlock, 0, e->stream>>>(e->N, e->K, e->I, e->J, e->crs_ptr,
                                                                e->crs_col, e->crs_tr, V, C, x, y);
    else
        k_ellj_stmvp_q<<<blocks(e->N), kEllBlock, 0, e->stream>>>(e->N, e->K, e->Q, V, x, y);
    FV_CUDA(cudaGetLastError());
    return FV_OK;
}
