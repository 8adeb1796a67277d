// mesh_plan.cpp -- host-side, one-time mesh addressing (no GPU involved).
//
// The paper's mesh model (Sec. 3.1): N cells, every face shared by two cells
// or a boundary face; the matrix pattern is the cell adjacency plus the
// diagonal.  Its index arrays are built once and shared by every matrix and
// face field (Sec. 3.1).  This file validates the description, renumbers the
// cells by reverse Cuthill-McKee (so neighbouring cells sit close in memory
// and row gathers stay in cache), orients and sorts the faces, and builds the
// SELL-32 row structure plus the per-cell boundary-face lists.
//
// Renumbering rule (fixed so that the result is reproducible bit for bit):
// start from the unvisited cell of smallest degree (lowest index on ties),
// breadth-first search appending each dequeued cell's unvisited neighbours
// in ascending (degree, index) order, restart the same way for further
// components, then reverse the whole sequence.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstring>
#include <numeric>

#include "fvgb_internal.h"

namespace fvgb {

static fv_status validate(const fv_mesh_desc *d)
{
    FV_CHECK(d != nullptr, FV_E_INVALID, "mesh description is NULL");
    const int N = d->n_cells, F = d->n_internal_faces, B = d->n_boundary_faces;
    FV_CHECK(N > 0 && F >= 0 && B >= 0, FV_E_INVALID, "bad sizes N=%d F=%d B=%d", N, F, B);
    FV_CHECK((long long)F + B < (1LL << 31) - 1, FV_E_INVALID, "too many faces");
    FV_CHECK(d->owner && d->Sf && d->Cf && d->C && d->V, FV_E_INVALID, "NULL mesh array");
    FV_CHECK(F == 0 || d->neighbour, FV_E_INVALID, "neighbour array is NULL");
    FV_CHECK(d->n_patches >= 0 && (d->n_patches == 0 || d->patches), FV_E_INVALID,
             "bad patch list");
    const int M = F + B;
    for (int f = 0; f < M; ++f)
        FV_CHECK(d->owner[f] >= 0 && d->owner[f] < N, FV_E_INVALID,
                 "owner[%d] = %d out of range", f, d->owner[f]);
    for (int f = 0; f < F; ++f) {
        FV_CHECK(d->neighbour[f] >= 0 && d->neighbour[f] < N, FV_E_INVALID,
                 "neighbour[%d] = %d out of range", f, d->neighbour[f]);
        FV_CHECK(d->neighbour[f] != d->owner[f], FV_E_INVALID,
                 "face %d has owner == neighbour", f);
    }
    for (int i = 0; i < N; ++i)
        FV_CHECK(d->V[i] > 0.0 && std::isfinite(d->V[i]), FV_E_INVALID,
                 "cell %d has volume %g", i, d->V[i]);
    for (int f = 0; f < M; ++f) {
        double s2 = 0.0;
        for (int c = 0; c < 3; ++c) s2 += d->Sf[(size_t)c * M + f] * d->Sf[(size_t)c * M + f];
        FV_CHECK(s2 > 0.0 && std::isfinite(s2), FV_E_INVALID, "face %d has zero area", f);
    }
    int next = 0;
    for (int q = 0; q < d->n_patches; ++q) {
        const fv_patch &p = d->patches[q];
        FV_CHECK(p.type >= FV_PATCH_WALL && p.type <= FV_PATCH_EMPTY, FV_E_INVALID,
                 "patch %d has type %d", q, p.type);
        FV_CHECK(p.start == next && p.size >= 0, FV_E_INVALID,
                 "patches must tile the boundary in order (patch %d)", q);
        next += p.size;
    }
    FV_CHECK(next == B, FV_E_INVALID, "patches cover %d of %d boundary faces", next, B);
    return FV_OK;
}

// Reverse Cuthill-McKee with the tie rules stated at the top of the file.
static void rcm(int N, int F, const int32_t *own, const int32_t *nei,
                std::vector<int32_t> &new_of_old)
{
    std::vector<int32_t> deg(N, 0);
    for (int f = 0; f < F; ++f) { ++deg[own[f]]; ++deg[nei[f]]; }
    std::vector<int64_t> ptr(N + 1, 0);
    for (int i = 0; i < N; ++i) ptr[i + 1] = ptr[i] + deg[i];
    std::vector<int32_t> adj(ptr[N]);
    std::vector<int64_t> pos(ptr.begin(), ptr.end() - 1);
    for (int f = 0; f < F; ++f) {
        adj[pos[own[f]]++] = nei[f];
        adj[pos[nei[f]]++] = own[f];
    }
    auto by_deg_idx = [&](int32_t a, int32_t b) {
        return deg[a] != deg[b] ? deg[a] < deg[b] : a < b;
    };
    for (int i = 0; i < N; ++i) std::sort(adj.begin() + ptr[i], adj.begin() + ptr[i + 1], by_deg_idx);
    // candidates for component starts, in (degree, index) order
    std::vector<int32_t> starts(N);
    std::iota(starts.begin(), starts.end(), 0);
    std::stable_sort(starts.begin(), starts.end(),
                     [&](int32_t a, int32_t b) { return deg[a] < deg[b]; });
    std::vector<char> seen(N, 0);
    std::vector<int32_t> order;
    order.reserve(N);
    size_t head = 0, cursor = 0;
    while ((int)order.size() < N) {
        while (seen[starts[cursor]]) ++cursor;
        int32_t s = starts[cursor];
        seen[s] = 1;
        order.push_back(s);
        while (head < order.size()) {
            int32_t v = order[head++];
            for (int64_t k = ptr[v]; k < ptr[v + 1]; ++k) {
                int32_t u = adj[k];
                if (!seen[u]) { seen[u] = 1; order.push_back(u); }
            }
        }
    }
    new_of_old.assign(N, 0);
    for (int i = 0; i < N; ++i) new_of_old[order[N - 1 - i]] = i;
}

fv_status build_plan(const fv_mesh_desc *d, MeshPlan *pl)
{
    fv_status st = validate(d);
    if (st != FV_OK) return st;
    const int N = d->n_cells, F = d->n_internal_faces, B = d->n_boundary_faces, M = F + B;
    pl->N = N; pl->F = F; pl->B = B;
    if (d->renumber) {
        rcm(N, F, d->owner, d->neighbour, pl->cell_new_of_old);
    } else {
        pl->cell_new_of_old.resize(N);
        std::iota(pl->cell_new_of_old.begin(), pl->cell_new_of_old.end(), 0);
    }
    const std::vector<int32_t> &no = pl->cell_new_of_old;

    // internal faces: (lo, hi) after renumbering, sorted
    std::vector<int32_t> lo(F), hi(F), idx(F);
    pl->flipped.assign(M, 0);
    for (int f = 0; f < F; ++f) {
        int32_t a = no[d->owner[f]], b = no[d->neighbour[f]];
        lo[f] = std::min(a, b);
        hi[f] = std::max(a, b);
        pl->flipped[f] = a > b ? 1 : 0;
        idx[f] = f;
    }
    std::sort(idx.begin(), idx.end(), [&](int32_t x, int32_t y) {
        return lo[x] != lo[y] ? lo[x] < lo[y] : (hi[x] != hi[y] ? hi[x] < hi[y] : x < y);
    });
    for (int k = 1; k < F; ++k)
        FV_CHECK(!(lo[idx[k]] == lo[idx[k - 1]] && hi[idx[k]] == hi[idx[k - 1]]), FV_E_INVALID,
                 "faces %d and %d join the same two cells", idx[k - 1], idx[k]);
    pl->face_new_of_old.assign(M, 0);
    pl->own.assign(M, 0);
    pl->nei.assign(F, 0);
    for (int k = 0; k < F; ++k) {
        pl->face_new_of_old[idx[k]] = k;
        pl->own[k] = lo[idx[k]];
        pl->nei[k] = hi[idx[k]];
    }
    // boundary faces: (patch, new owner, original index)
    std::vector<int32_t> patch_of(B, 0), bidx(B);
    for (int q = 0; q < d->n_patches; ++q)
        for (int j = 0; j < d->patches[q].size; ++j) patch_of[d->patches[q].start + j] = q;
    std::iota(bidx.begin(), bidx.end(), 0);
    std::sort(bidx.begin(), bidx.end(), [&](int32_t x, int32_t y) {
        if (patch_of[x] != patch_of[y]) return patch_of[x] < patch_of[y];
        int32_t ox = no[d->owner[F + x]], oy = no[d->owner[F + y]];
        return ox != oy ? ox < oy : x < y;
    });
    pl->bpatch.assign(B, 0);
    for (int k = 0; k < B; ++k) {
        pl->face_new_of_old[F + bidx[k]] = F + k;
        pl->own[F + k] = no[d->owner[F + bidx[k]]];
        pl->bpatch[k] = patch_of[bidx[k]];
    }

    // SELL-32 rows: internal neighbours of each cell, ascending column
    std::vector<int32_t> rdeg(N, 0);
    for (int f = 0; f < F; ++f) { ++rdeg[pl->own[f]]; ++rdeg[pl->nei[f]]; }
    std::vector<int64_t> rptr(N + 1, 0);
    for (int i = 0; i < N; ++i) rptr[i + 1] = rptr[i] + rdeg[i];
    std::vector<int32_t> rcol(rptr[N]), rface(rptr[N]);
    {
        std::vector<int64_t> fill(rptr.begin(), rptr.end() - 1);
        // faces are sorted by owner, so visiting them in order fills lower
        // entries (col < row) by ascending owner and upper entries by
        // ascending neighbour: every row ends up sorted without a sort
        for (int f = 0; f < F; ++f) {
            int32_t a = pl->own[f], b = pl->nei[f];
            rcol[fill[b]] = a; rface[fill[b]++] = f;
        }
        for (int f = 0; f < F; ++f) {
            int32_t a = pl->own[f], b = pl->nei[f];
            rcol[fill[a]] = b; rface[fill[a]++] = f;
        }
    }
    pl->nslice = (N + kSlice - 1) / kSlice;
    pl->slice_ptr.assign(pl->nslice + 1, 0);
    for (int s = 0; s < pl->nslice; ++s) {
        int K = 0;
        for (int l = 0; l < kSlice; ++l) {
            int i = s * kSlice + l;
            if (i < N) K = std::max(K, rdeg[i]);
        }
        pl->slice_ptr[s + 1] = pl->slice_ptr[s] + K * kSlice;
    }
    FV_CHECK((long long)pl->slice_ptr[pl->nslice] < (1LL << 31), FV_E_INVALID,
             "row structure too large");
    pl->col.assign(pl->slice_ptr[pl->nslice], 0);
    pl->sface.assign(pl->slice_ptr[pl->nslice], -1);
    for (int s = 0; s < pl->nslice; ++s) {
        int K = (pl->slice_ptr[s + 1] - pl->slice_ptr[s]) / kSlice;
        for (int l = 0; l < kSlice; ++l) {
            int i = s * kSlice + l;
            for (int k = 0; k < K; ++k) {
                int64_t e = pl->slice_ptr[s] + (int64_t)k * kSlice + l;
                if (i < N && k < rdeg[i]) {
                    pl->col[e] = rcol[rptr[i] + k];
                    pl->sface[e] = rface[rptr[i] + k];
                } else {
                    pl->col[e] = i < N ? i : 0;
                    pl->sface[e] = -1;
                }
            }
        }
    }
    // boundary faces per cell (empty patches are ignored everywhere)
    pl->bptr.assign(N + 1, 0);
    for (int k = 0; k < B; ++k)
        if (d->patches[pl->bpatch[k]].type != FV_PATCH_EMPTY) ++pl->bptr[pl->own[F + k] + 1];
    for (int i = 0; i < N; ++i) pl->bptr[i + 1] += pl->bptr[i];
    pl->bface.assign(pl->bptr[N], 0);
    {
        std::vector<int32_t> fill(pl->bptr.begin(), pl->bptr.end() - 1);
        for (int k = 0; k < B; ++k)
            if (d->patches[pl->bpatch[k]].type != FV_PATCH_EMPTY)
                pl->bface[fill[pl->own[F + k]]++] = k;
    }
    return FV_OK;
}

}  // namespace fvgb

extern "C" fv_status fv_mesh_plan(const fv_mesh_desc *desc, int32_t *new_of_old_cell,
                                  int32_t *new_of_old_face, int8_t *flipped)
{
    try {
        fvgb::MeshPlan pl;
        fv_status st = fvgb::build_plan(desc, &pl);
        if (st != FV_OK) return st;
        if (new_of_old_cell)
            std::memcpy(new_of_old_cell, pl.cell_new_of_old.data(), sizeof(int32_t) * pl.N);
        if (new_of_old_face)
            std::memcpy(new_of_old_face, pl.face_new_of_old.data(),
                        sizeof(int32_t) * (pl.F + pl.B));
        if (flipped) std::memcpy(flipped, pl.flipped.data(), pl.F + pl.B);
        return FV_OK;
    } catch (...) {
        fvgb::set_error("host allocation failed in fv_mesh_plan");
        return FV_E_NOMEM;
    }
}
