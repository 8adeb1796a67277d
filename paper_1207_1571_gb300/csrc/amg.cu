// amg.cu -- aggregation-multigrid preconditioned CG for the pressure
// equation: the stronger pressure solver the paper's discussion (Sec. 5,
// Sec. 6) names as the way past Jacobi-CG, built for one GB300.
//
// Setup, once per mesh (host): a hierarchy of aggregates from the geometry
// alone.  Level 0 is the cell graph with edge weights |S_f| Delta_f; each
// level's aggregates come from two pairwise-matching passes (a node is
// paired with its unassigned neighbour of largest weight, or joins its
// strongest neighbour's aggregate when all are taken; weights within a
// relative 1e-9 tie and the lower index wins); the coarse graph joins two
// aggregates that share an edge, with summed weight, edges ordered by
// (lower, higher) aggregate.  Coarsening stops at <= 32 nodes or when a
// level shrinks by less than 10 %.
//
// Per solve (device, one cooperative launch): Galerkin coarse matrices
// A_c = P^T A P for piecewise-constant P (coarse diagonal = members'
// diagonals + twice the coefficients of the edges inside the aggregate;
// coarse edge = sum of its fine edges; every sum in ascending fine index),
// the coarsest matrix factored by Cholesky, then CG preconditioned by one
// V-cycle: per level two weighted-Jacobi sweeps (omega = 2/3) from zero,
// the residual summed over each aggregate, the coarse correction added with
// the over-correction factor 1.8, two sweeps again.
//
// GB300 mapping: levels with many rows run over the whole grid with the
// bounded grid barrier between dependent phases; the small levels (and the
// coarsest solve) run inside block 0 with block barriers only, while the
// other blocks wait at the next grid barrier.  Pre-smoothing's first sweep
// is fused into the phase that produces the level's right-hand side, the
// residual into the restriction, and the prolongation into the first
// post-smoothing sweep, so a grid level costs four grid barriers per cycle.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "fvgb_internal.h"
#include "coop.cuh"

namespace fvgb {

constexpr int kAmgMaxLev = 24;
constexpr int kAmgNmin = 32;           // coarsest level size target
constexpr int kAmgCoarseMax = 64;      // largest coarsest level handled on the device
constexpr int kAmgBlock = 512;
constexpr int kAmgBlockRows = 256;     // levels up to this size run inside block 0
constexpr int kAmgShadowMax = 64 << 10; // largest shared-memory copy of those levels
constexpr double kAmgTie = 1e-9;
constexpr double kAmgOmega = 2.0 / 3.0;
constexpr double kAmgAlpha = 1.8;

// ------------------------------------------------------ host: hierarchy --

namespace {

struct Graph {
    int n = 0;
    std::vector<int32_t> a, b;     // edges, a < b, ordered by (a, b)
    std::vector<double> w;
};

bool prefer(double wc, int jc, double wb, int jb)
{
    if (jb < 0) return true;
    if (wc > wb * (1.0 + kAmgTie)) return true;
    return wc >= wb * (1.0 - kAmgTie) && jc < jb;
}

// One pairwise-matching pass; returns the number of aggregates.
int match(const Graph &g, std::vector<int32_t> &assign)
{
    const size_t ne = g.a.size();
    std::vector<int32_t> off(g.n + 1, 0);
    for (size_t e = 0; e < ne; ++e) { ++off[g.a[e] + 1]; ++off[g.b[e] + 1]; }
    for (int i = 0; i < g.n; ++i) off[i + 1] += off[i];
    std::vector<int32_t> nb(2 * ne), cur(off.begin(), off.end() - 1);
    std::vector<double> nw(2 * ne);
    for (size_t e = 0; e < ne; ++e) {
        nb[cur[g.a[e]]] = g.b[e]; nw[cur[g.a[e]]++] = g.w[e];
        nb[cur[g.b[e]]] = g.a[e]; nw[cur[g.b[e]]++] = g.w[e];
    }
    assign.assign(g.n, -1);
    int na = 0;
    for (int i = 0; i < g.n; ++i) {
        if (assign[i] >= 0) continue;
        int best = -1, any = -1;
        double wbest = 0.0, wany = 0.0;
        for (int t = off[i]; t < off[i + 1]; ++t) {
            const int j = nb[t];
            if (assign[j] < 0 && prefer(nw[t], j, wbest, best)) { best = j; wbest = nw[t]; }
            if (prefer(nw[t], j, wany, any)) { any = j; wany = nw[t]; }
        }
        if (best >= 0) assign[i] = assign[best] = na++;
        else assign[i] = any >= 0 ? assign[any] : na++;
    }
    return na;
}

// Coarse graph of an assignment; emap: fine edge -> coarse edge or -1.
Graph contract(const Graph &g, const std::vector<int32_t> &assign, int na,
               std::vector<int32_t> &emap)
{
    const size_t ne = g.a.size();
    emap.assign(ne, -1);
    std::vector<std::pair<uint64_t, int32_t>> key;
    key.reserve(ne);
    for (size_t e = 0; e < ne; ++e) {
        const uint32_t p = assign[g.a[e]], q = assign[g.b[e]];
        if (p == q) continue;
        const uint64_t lo = std::min(p, q), hi = std::max(p, q);
        key.emplace_back((lo << 32) | hi, (int32_t)e);
    }
    std::sort(key.begin(), key.end());
    Graph c;
    c.n = na;
    for (size_t t = 0; t < key.size(); ++t) {
        if (t == 0 || key[t].first != key[t - 1].first) {
            c.a.push_back((int32_t)(key[t].first >> 32));
            c.b.push_back((int32_t)(key[t].first & 0xffffffffu));
            c.w.push_back(0.0);
        }
        emap[key[t].second] = (int32_t)c.a.size() - 1;
    }
    for (size_t e = 0; e < ne; ++e)
        if (emap[e] >= 0) c.w[emap[e]] += g.w[e];
    return c;
}

// One level: two matching passes composed.
Graph coarsen(const Graph &g, std::vector<int32_t> &agg, std::vector<int32_t> &emap)
{
    std::vector<int32_t> a1, a2, m1, m2;
    const int n1 = match(g, a1);
    const Graph g1 = contract(g, a1, n1, m1);
    const int n2 = match(g1, a2);
    Graph g2 = contract(g1, a2, n2, m2);
    agg.resize(g.n);
    for (int i = 0; i < g.n; ++i) agg[i] = a2[a1[i]];
    emap.resize(g.a.size());
    for (size_t e = 0; e < g.a.size(); ++e) emap[e] = m1[e] < 0 ? -1 : m2[m1[e]];
    return g2;
}

}  // namespace

// ---------------------------------------------------- device hierarchy --

struct AmgLevelDev {
    int n, ne;
    // rows in SELL-32 slices: entry k of row i at sptr[i / 32] + 32 k + i % 32,
    // columns ascending; padding has column i, edge -1, value 0
    const int32_t *sptr, *scol, *sedge;
    double *sval;                            // coefficient of every slot (set per solve)
    const int32_t *agg;                      // -> next level (nullptr at the coarsest)
    const int32_t *mptr, *memb;              // members in the finer level (l > 0)
    const int32_t *iptr, *inner;             // finer-level edges inside the aggregate (l > 0)
    const int32_t *eptr, *elist;             // finer-level edges of each edge (l > 0)
    double *d, *o, *dinv;                    // matrix (level 0: d copied per solve, o unused)
    double *b, *x, *xa;                      // right-hand side, iterates
    // FP32 copies the cycle smooths with in mixed precision
    float *sval32, *d32, *dinv32, *b32, *x32, *xa32;
};

struct AmgData {
    int L = 0;                // index of the coarsest level
    int G = 1;                // levels 0..G-1 run over the whole grid
    int grid = 0;             // cooperative grid size
    int dyn_bytes = 0;        // dynamic shared memory of the solve kernel
    int shadow = 0;           // block 0 keeps levels G..L in shared memory
    int lev_table_bytes = 0;
    int n[kAmgMaxLev] = {}, ne[kAmgMaxLev] = {};
    AmgLevelDev *lev = nullptr;      // device copy of the level table
    int *coarse_ok = nullptr;
    double *z = nullptr, *p = nullptr, *q = nullptr, *r = nullptr;
    DeviceArena arena;
};

void amg_release(AmgData *a)
{
    if (!a) return;
    a->arena.release();
    delete a;
}

namespace {

struct AmgArgs {
    int L, G, nc;
    const AmgLevelDev *lev;
    const double *d0, *o0;     // level-0 matrix: diagonal [N] and edge coefficients [F]
    double o0_sign;            // o = o0_sign * o0[f] (-1 when o0 holds the positive a_f)
    int fp32;                  // the V-cycle in FP32 (mixed precision)
    int shadow;                // block 0 keeps levels G..L in shared memory
    int lev_table_bytes;       // room of the shared-memory level table (16-byte multiple)
    const double *b;
    double *x, *r, *z, *p, *q;
    double *partA, *partB;
    int *coarse_ok;            // written by block 0 during setup, read after a barrier
    GridBar *bar;
    long long spin;
    double tol, reltol;
    int maxit;
    DevSolveStats *stats;
};

struct AmgScal {
    double alpha, beta, rho, thresh, nb, nr0, nr;
    int phase;    // 0 iterate, 1 converged, 2 not converged, 3 breakdown, 4 zero rhs, 5 bad coarse
};

// Rows [lo, hi) of level l owned by this block (whole grid) or all rows
// (block 0 alone).
struct Span {
    int lo, hi;
};

__device__ __forceinline__ Span grid_rows(int n)
{
    // whole 32-row slices per block, so a warp's rows share a slice
    const int nsl = (n + 31) >> 5;
    const int chunk = ((nsl + gridDim.x - 1) / gridDim.x) * 32;
    const int lo = min(n, (int)blockIdx.x * chunk);
    return {lo, min(n, lo + chunk)};
}

struct SRow {
    int e0, K;
};

__device__ __forceinline__ SRow srow(const AmgLevelDev &L, int i)
{
    const int s = i >> 5;
    const int p0 = L.sptr[s], p1 = L.sptr[s + 1];
    return {p0 + (i & 31), (p1 - p0) >> 5};
}

__device__ __forceinline__ double coef(const AmgArgs &a, const AmgLevelDev &L, int l, int e)
{
    return l == 0 ? a.o0_sign * a.o0[e] : L.o[e];
}

__device__ __forceinline__ double diagv(const AmgArgs &a, const AmgLevelDev &L, int l, int i)
{
    return l == 0 ? a.d0[i] : L.d[i];
}

// (A x)_i on level l (coefficients from the per-entry copy: no edge indirection)
__device__ __forceinline__ double row_ax(const AmgArgs &a, const AmgLevelDev &L, int l, int i,
                                         const double *x)
{
    double t = diagv(a, L, l, i) * x[i];
    const SRow r = srow(L, i);
    for (int k = 0; k < r.K; ++k) {
        const int e = r.e0 + 32 * k;
        t += L.sval[e] * x[L.scol[e]];
    }
    return t;
}

// The arrays a V-cycle in value type V works on (FP64, or the FP32 copies).
template <class V> struct VL;
template <> struct VL<double> {
    __device__ static const double *sval(const AmgLevelDev &L) { return L.sval; }
    __device__ static const double *d(const AmgLevelDev &L) { return L.d; }
    __device__ static const double *dinv(const AmgLevelDev &L) { return L.dinv; }
    __device__ static double *b(const AmgLevelDev &L) { return L.b; }
    __device__ static double *x(const AmgLevelDev &L) { return L.x; }
    __device__ static double *xa(const AmgLevelDev &L) { return L.xa; }
};
template <> struct VL<float> {
    __device__ static const float *sval(const AmgLevelDev &L) { return L.sval32; }
    __device__ static const float *d(const AmgLevelDev &L) { return L.d32; }
    __device__ static const float *dinv(const AmgLevelDev &L) { return L.dinv32; }
    __device__ static float *b(const AmgLevelDev &L) { return L.b32; }
    __device__ static float *x(const AmgLevelDev &L) { return L.x32; }
    __device__ static float *xa(const AmgLevelDev &L) { return L.xa32; }
};

// (A x)_i on a level in the cycle's value type
template <class V>
__device__ __forceinline__ V row_axv(const AmgLevelDev &L, int i, const V *x)
{
    const V *sv = VL<V>::sval(L);
    V t = VL<V>::d(L)[i] * x[i];
    const SRow r = srow(L, i);
    for (int k = 0; k < r.K; ++k) {
        const int e = r.e0 + 32 * k;
        t += sv[e] * x[L.scol[e]];
    }
    return t;
}

// Level 0 per solve: per-entry coefficients from the caller's edge array,
// the diagonal and its reciprocal (and their FP32 copies in mixed precision).
__device__ void phase_rows0(const AmgArgs &a, Span s, int t0, int step)
{
    const AmgLevelDev &L = a.lev[0];
    for (int i = s.lo + t0; i < s.hi; i += step) {
        const double d = a.d0[i];
        L.d[i] = d;
        L.dinv[i] = 1.0 / d;
        if (a.fp32) {
            L.d32[i] = (float)d;
            L.dinv32[i] = (float)(1.0 / d);
        }
        const SRow r = srow(L, i);
        for (int k = 0; k < r.K; ++k) {
            const int e = r.e0 + 32 * k;
            const int E = L.sedge[e];
            const double v = E < 0 ? 0.0 : coef(a, L, 0, E);
            L.sval[e] = v;
            if (a.fp32) L.sval32[e] = (float)v;
        }
    }
}

// ---- level phases over the rows [s.lo, s.hi) with thread stride `step` --

// Galerkin coarse matrix of level l (>= 1) from level l - 1.
__device__ void phase_galerkin(const AmgArgs &a, int l, Span s, int t0, int step)
{
    const AmgLevelDev &C = a.lev[l], &F = a.lev[l - 1];
    for (int I = s.lo + t0; I < s.hi; I += step) {
        double v = 0.0;
        for (int k = C.mptr[I]; k < C.mptr[I + 1]; ++k) v += diagv(a, F, l - 1, C.memb[k]);
        for (int k = C.iptr[I]; k < C.iptr[I + 1]; ++k) v += 2.0 * coef(a, F, l - 1, C.inner[k]);
        C.d[I] = v;
        C.dinv[I] = 1.0 / v;
        if (a.fp32) {
            C.d32[I] = (float)v;
            C.dinv32[I] = (float)(1.0 / v);
        }
        // the row's coefficients: the same sums as the edge phase below
        const SRow r = srow(C, I);
        for (int q = 0; q < r.K; ++q) {
            const int e = r.e0 + 32 * q;
            const int E = C.sedge[e];
            double w = 0.0;
            if (E >= 0)
                for (int k = C.eptr[E]; k < C.eptr[E + 1]; ++k) w += coef(a, F, l - 1, C.elist[k]);
            C.sval[e] = w;
            if (a.fp32) C.sval32[e] = (float)w;
        }
    }
}

__device__ void phase_galerkin_edges(const AmgArgs &a, int l, Span s, int t0, int step)
{
    const AmgLevelDev &C = a.lev[l], &F = a.lev[l - 1];
    for (int E = s.lo + t0; E < s.hi; E += step) {
        double v = 0.0;
        for (int k = C.eptr[E]; k < C.eptr[E + 1]; ++k) v += coef(a, F, l - 1, C.elist[k]);
        C.o[E] = v;
    }
}

// x = x + omega (b - A x) / d, from xin to xout
template <class V>
__device__ void phase_sweep(const AmgLevelDev *lv, int l, const V *xin, V *xout, Span s, int t0,
                            int step)
{
    const AmgLevelDev &L = lv[l];
    const V *b = VL<V>::b(L), *dinv = VL<V>::dinv(L);
    const V w = (V)kAmgOmega;
    for (int i = s.lo + t0; i < s.hi; i += step)
        xout[i] = xin[i] + w * (b[i] - row_axv<V>(L, i, xin)) * dinv[i];
}

// b_{l+1} = P^T (b - A xa) over each aggregate, and the next level's first
// sweep from zero: x_{l+1} = omega b_{l+1} / d_{l+1}.
template <class V>
__device__ void phase_restrict(const AmgLevelDev *lv, int l, Span s, int t0, int step)
{
    const AmgLevelDev &F = lv[l], &C = lv[l + 1];
    const V *fb = VL<V>::b(F), *fxa = VL<V>::xa(F), *cdinv = VL<V>::dinv(C);
    V *cb = VL<V>::b(C), *cx = VL<V>::x(C);
    for (int I = s.lo + t0; I < s.hi; I += step) {
        V v = 0;
        for (int k = C.mptr[I]; k < C.mptr[I + 1]; ++k) {
            const int i = C.memb[k];
            v += fb[i] - row_axv<V>(F, i, fxa);
        }
        cb[I] = v;
        cx[I] = (V)kAmgOmega * v * cdinv[I];
    }
}

// x = xa + alpha P e_c, then one sweep; neighbours' prolonged values are
// formed on the fly.
template <class V>
__device__ void phase_prolong_sweep(const AmgLevelDev *lv, int l, Span s, int t0, int step)
{
    const AmgLevelDev &L = lv[l];
    const V *ec = VL<V>::xa(lv[l + 1]);
    const V *xa = VL<V>::xa(L), *sv = VL<V>::sval(L), *d = VL<V>::d(L);
    const V *b = VL<V>::b(L), *dinv = VL<V>::dinv(L);
    V *x = VL<V>::x(L);
    const V al = (V)kAmgAlpha;
    for (int i = s.lo + t0; i < s.hi; i += step) {
        const V xi = xa[i] + al * ec[L.agg[i]];
        V t = d[i] * xi;
        const SRow r = srow(L, i);
        for (int k = 0; k < r.K; ++k) {
            const int e = r.e0 + 32 * k;
            const int j = L.scol[e];
            t += sv[e] * (xa[j] + al * ec[L.agg[j]]);
        }
        x[i] = xi + (V)kAmgOmega * (b[i] - t) * dinv[i];
    }
}

// Coarsest level: dense Cholesky factor (once per solve) by warp 0 of
// block 0, kept in block 0's shared memory `c` for the whole solve (every
// step of the triangular solves then costs a shared-memory access, not an
// L2 round trip); returns false if the matrix is not positive definite.
__device__ bool coarse_factor(const AmgArgs &a, double *c)
{
    const AmgLevelDev &C = a.lev[a.L];
    const int n = a.nc, lane = threadIdx.x & 31;
    for (int t = lane; t < n * n; t += 32) c[t] = 0.0;
    __syncwarp();
    for (int i = lane; i < n; i += 32) c[i * n + i] = diagv(a, C, a.L, i);
    for (int i = lane; i < n; i += 32) {
        const SRow r = srow(C, i);
        for (int k = 0; k < r.K; ++k) {
            const int e = r.e0 + 32 * k;
            if (C.sedge[e] >= 0) c[i * n + C.scol[e]] = C.sval[e];
        }
    }
    __syncwarp();
    bool ok = true;
    for (int j = 0; j < n; ++j) {
        // left-looking column j: lanes own the rows i >= j
        double s = c[j * n + j];
        for (int k = 0; k < j; ++k) s -= c[j * n + k] * c[j * n + k];
        if (!(s > 0.0)) ok = false;
        const double ljj = sqrt(s > 0.0 ? s : 1.0);
        for (int i = j + 1 + lane; i < n; i += 32) {
            double t = c[i * n + j];
            for (int k = 0; k < j; ++k) t -= c[i * n + k] * c[j * n + k];
            c[i * n + j] = t / ljj;
        }
        __syncwarp();
        if (lane == 0) c[j * n + j] = ljj;
        __syncwarp();
    }
    return ok;
}

// xa_L = A_L^-1 b_L with the FP64 factor c (shared memory; warp 0 of block
// 0), working vector y in shared memory
template <class V>
__device__ void coarse_solve(const AmgArgs &a, const AmgLevelDev *lv, const double *c, double *y)
{
    const AmgLevelDev &C = lv[a.L];
    const int n = a.nc, lane = threadIdx.x & 31;
    const V *cb = VL<V>::b(C);
    V *cxa = VL<V>::xa(C);
    for (int i = lane; i < n; i += 32) y[i] = (double)cb[i];
    __syncwarp();
    for (int k = 0; k < n; ++k) {            // forward: L y = b
        const double yk = y[k] / c[k * n + k];
        __syncwarp();
        for (int i = k + 1 + lane; i < n; i += 32) y[i] -= c[i * n + k] * yk;
        if (lane == 0) y[k] = yk;
        __syncwarp();
    }
    for (int k = n - 1; k >= 0; --k) {       // backward: L^T x = y
        const double xk = y[k] / c[k * n + k];
        __syncwarp();
        for (int i = lane; i < k; i += 32) y[i] -= c[k * n + i] * xk;
        if (lane == 0) y[k] = xk;
        __syncwarp();
    }
    for (int i = lane; i < n; i += 32) cxa[i] = (V)y[i];
    __syncwarp();
}

// The levels from G down to the coarsest and back, inside block 0, on the
// level table lv (the shared-memory copy of those levels when it exists).
template <class V>
__device__ void block_levels_down_up(const AmgArgs &a, const AmgLevelDev *lv, const double *chol,
                                     double *cy)
{
    const int t0 = threadIdx.x, step = blockDim.x;
    for (int l = a.G; l < a.L; ++l) {
        const Span s{0, lv[l].n};
        phase_sweep<V>(lv, l, VL<V>::x(lv[l]), VL<V>::xa(lv[l]), s, t0, step);
        __syncthreads();
        phase_restrict<V>(lv, l, Span{0, lv[l + 1].n}, t0, step);
        __syncthreads();
    }
    if (threadIdx.x < 32) coarse_solve<V>(a, lv, chol, cy);
    __syncthreads();
    for (int l = a.L - 1; l >= a.G; --l) {
        const Span s{0, lv[l].n};
        phase_prolong_sweep<V>(lv, l, s, t0, step);
        __syncthreads();
        phase_sweep<V>(lv, l, VL<V>::x(lv[l]), VL<V>::xa(lv[l]), s, t0, step);
        __syncthreads();
    }
}

// Shared-memory copy of the levels G..L for block 0 (their matrices are
// fixed for the solve once the Galerkin products are formed): the row
// structure, coefficients, diagonal and its reciprocal, the vectors of the
// cycle in value type V, the aggregate maps and the member lists the
// restriction sums over.  Thread 0 lays the arrays out in `dyn` and fills
// the level table `sl`; the block copies the arrays.  Level G's right-hand
// side and first iterate come from the grid phase of every cycle and its
// result goes back to it (shadow_in / shadow_out).
template <class V>
__device__ void shadow_setup(const AmgArgs &a, AmgLevelDev *sl, unsigned char *dyn)
{
    if (threadIdx.x == 0) {
        size_t off = 0;
        auto take = [&](size_t bytes) {
            unsigned char *p = dyn + off;
            off += (bytes + 15) & ~(size_t)15;
            return p;
        };
        for (int l = a.G; l <= a.L; ++l) {
            const AmgLevelDev &g = a.lev[l];
            AmgLevelDev &d = sl[l];
            d = g;
            const int n = g.n, nsl = (n + 31) >> 5;
            const int slots = g.sptr[nsl];
            V *sv = (V *)take(sizeof(V) * slots);
            V *dd = (V *)take(sizeof(V) * n);
            V *di = (V *)take(sizeof(V) * n);
            V *bb = (V *)take(sizeof(V) * n);
            V *xx = (V *)take(sizeof(V) * n);
            V *xa = (V *)take(sizeof(V) * n);
            if (sizeof(V) == 8) {
                d.sval = (double *)sv; d.d = (double *)dd; d.dinv = (double *)di;
                d.b = (double *)bb; d.x = (double *)xx; d.xa = (double *)xa;
            } else {
                d.sval32 = (float *)sv; d.d32 = (float *)dd; d.dinv32 = (float *)di;
                d.b32 = (float *)bb; d.x32 = (float *)xx; d.xa32 = (float *)xa;
            }
            d.sptr = (const int32_t *)take(sizeof(int32_t) * (nsl + 1));
            d.scol = (const int32_t *)take(sizeof(int32_t) * slots);
            d.agg = l < a.L ? (const int32_t *)take(sizeof(int32_t) * n) : nullptr;
            if (l > a.G) {
                d.mptr = (const int32_t *)take(sizeof(int32_t) * (n + 1));
                d.memb = (const int32_t *)take(sizeof(int32_t) * g.mptr[n]);
            }
        }
    }
    __syncthreads();
    for (int l = a.G; l <= a.L; ++l) {
        const AmgLevelDev &g = a.lev[l], &d = sl[l];
        const int n = g.n, nsl = (n + 31) >> 5;
        const int slots = g.sptr[nsl];
        V *sv = (V *)VL<V>::sval(d);
        V *dd = (V *)VL<V>::d(d);
        V *di = (V *)VL<V>::dinv(d);
        for (int k = threadIdx.x; k < slots; k += blockDim.x) {
            sv[k] = VL<V>::sval(g)[k];
            ((int32_t *)d.scol)[k] = g.scol[k];
        }
        for (int k = threadIdx.x; k <= nsl; k += blockDim.x) ((int32_t *)d.sptr)[k] = g.sptr[k];
        for (int k = threadIdx.x; k < n; k += blockDim.x) {
            dd[k] = VL<V>::d(g)[k];
            di[k] = VL<V>::dinv(g)[k];
            if (l < a.L) ((int32_t *)d.agg)[k] = g.agg[k];
        }
        if (l > a.G) {
            for (int k = threadIdx.x; k <= n; k += blockDim.x) ((int32_t *)d.mptr)[k] = g.mptr[k];
            for (int k = threadIdx.x; k < g.mptr[n]; k += blockDim.x)
                ((int32_t *)d.memb)[k] = g.memb[k];
        }
    }
    __syncthreads();
}

template <class V>
__device__ void shadow_in(const AmgArgs &a, const AmgLevelDev *sl)
{
    const AmgLevelDev &g = a.lev[a.G], &d = sl[a.G];
    for (int k = threadIdx.x; k < g.n; k += blockDim.x) {
        VL<V>::b(d)[k] = VL<V>::b(g)[k];
        VL<V>::x(d)[k] = VL<V>::x(g)[k];
    }
    __syncthreads();
}

template <class V>
__device__ void shadow_out(const AmgArgs &a, const AmgLevelDev *sl)
{
    const AmgLevelDev &g = a.lev[a.G], &d = sl[a.G];
    for (int k = threadIdx.x; k < g.n; k += blockDim.x) VL<V>::xa(g)[k] = VL<V>::xa(d)[k];
}

// Level 0's right-hand side is the CG residual r; the first pre-smoothing
// sweep from zero is x = omega r / d.  In FP32 the residual is rounded into
// the cycle's own right-hand side.
template <class V>
__device__ __forceinline__ void seed0(const AmgLevelDev &L0, int i, double ri);
template <>
__device__ __forceinline__ void seed0<double>(const AmgLevelDev &L0, int i, double ri)
{
    L0.x[i] = kAmgOmega * ri * L0.dinv[i];
}
template <>
__device__ __forceinline__ void seed0<float>(const AmgLevelDev &L0, int i, double ri)
{
    const float b = (float)ri;
    L0.b32[i] = b;
    L0.x32[i] = (float)kAmgOmega * b * L0.dinv32[i];
}

template <class V>
__global__ void __launch_bounds__(kAmgBlock) k_pcg_amg(AmgArgs a)
{
    __shared__ double buf[2][kAmgBlock];
    __shared__ double tot[2];
    __shared__ AmgScal sc;
    __shared__ int s_coarse_ok;
    // dynamic shared memory, used by block 0 only (every block holds it, so
    // it is sized to the hierarchy: shared memory a block holds is L1 cache
    // its SM does not have): the coarsest factor, the triangular solves'
    // vector, and with the level copy the level table and the levels' data
    extern __shared__ __align__(16) unsigned char s_dyn[];
    const int nc16 = (a.nc * a.nc * 8 + 15) & ~15, nv16 = (a.nc * 8 + 15) & ~15;
    double *const s_chol = reinterpret_cast<double *>(s_dyn);
    double *const s_cy = reinterpret_cast<double *>(s_dyn + nc16);
    AmgLevelDev *const s_lev = reinterpret_cast<AmgLevelDev *>(s_dyn + nc16 + nv16);
    unsigned char *const s_levdata = s_dyn + nc16 + nv16 + a.lev_table_bytes;
    const int t0 = threadIdx.x, step = blockDim.x;
    const AmgLevelDev &L0 = a.lev[0];
    const int N = L0.n;
    const Span s0 = grid_rows(N);
    unsigned gen = 0;
    bool ok = true;
    int it = 0;

    // ---- setup: diagonal and row coefficients on level 0, Galerkin
    // matrices, coarsest factor
    phase_rows0(a, s0, t0, step);
    for (int l = 1; l < a.G && l <= a.L && ok; ++l) {
        ok = grid_sync(a.bar, gen, a.spin);
        if (!ok) break;
        phase_galerkin(a, l, grid_rows(a.lev[l].n), t0, step);
        phase_galerkin_edges(a, l, grid_rows(a.lev[l].ne), t0, step);
    }
    if (ok) ok = grid_sync(a.bar, gen, a.spin);
    if (blockIdx.x == 0) {
        for (int l = a.G; l <= a.L; ++l) {
            if (l == 0) continue;
            phase_galerkin(a, l, Span{0, a.lev[l].n}, t0, step);
            phase_galerkin_edges(a, l, Span{0, a.lev[l].ne}, t0, step);
            __syncthreads();
        }
        if (threadIdx.x < 32) {
            const bool cok = coarse_factor(a, s_chol);
            if (threadIdx.x == 0) s_coarse_ok = cok ? 1 : 0;
        }
        __syncthreads();
        if (threadIdx.x == 0) *(volatile int *)a.coarse_ok = s_coarse_ok;
        if (a.shadow && a.L > 0) shadow_setup<V>(a, s_lev, s_levdata);
    }
    const AmgLevelDev *blev = (a.shadow && a.L > 0) ? s_lev : a.lev;

    // ---- r = b - A x, norms
    if (ok) {
        double v[2] = {0.0, 0.0};
        for (int i = s0.lo + t0; i < s0.hi; i += step) {
            const double bi = a.b[i];
            const double ri = bi - row_ax(a, L0, 0, i, a.x);
            a.r[i] = ri;
            seed0<V>(L0, i, ri);                         // first pre-smoothing sweep
            v[0] += bi * bi;
            v[1] += ri * ri;
        }
        ok = cg_grid_sum<2, kAmgBlock>(v, a.partB, a.bar, gen, a.spin, buf, tot);
    }
    if (threadIdx.x == 0) {
        sc.nb = sqrt(tot[0]);
        sc.nr0 = sqrt(tot[1]);
        sc.nr = sc.nr0;
        sc.thresh = fmax(a.tol * sc.nb, a.reltol * sc.nr0);
        sc.alpha = sc.beta = sc.rho = 0.0;
        sc.phase = sc.nb == 0.0 ? 4 : (sc.nr0 <= sc.thresh ? 1 : (a.maxit <= 0 ? 2 : 0));
        if (ok && sc.phase == 0 && *(volatile int *)a.coarse_ok == 0) sc.phase = 5;
    }
    __syncthreads();
    if (ok && sc.phase == 4) {
        for (int i = s0.lo + t0; i < s0.hi; i += step) a.x[i] = 0.0;
    } else if (ok && sc.phase == 0) {
        while (true) {
            // ---- z = V(r): level 0's b is r, its result lands in xa = z
            for (int l = 0; l < a.G && l < a.L; ++l) {
                // (the barrier before the first sweep of level 0 is the one
                // that ended the previous phase)
                if (l > 0 && !(ok = grid_sync(a.bar, gen, a.spin))) break;
                phase_sweep<V>(a.lev, l, VL<V>::x(a.lev[l]), VL<V>::xa(a.lev[l]),
                               grid_rows(a.lev[l].n), t0, step);
                if (!(ok = grid_sync(a.bar, gen, a.spin))) break;
                phase_restrict<V>(a.lev, l, grid_rows(a.lev[l + 1].n), t0, step);
            }
            if (!ok) break;
            if (a.L == 0) {
                // a single level: the exact solve
                if (blockIdx.x == 0 && threadIdx.x < 32) coarse_solve<V>(a, a.lev, s_chol, s_cy);
            } else {
                if (!(ok = grid_sync(a.bar, gen, a.spin))) break;
                if (blockIdx.x == 0) {
                    if (blev != a.lev) shadow_in<V>(a, blev);
                    block_levels_down_up<V>(a, blev, s_chol, s_cy);
                    if (blev != a.lev) shadow_out<V>(a, blev);
                }
            }
            double v1[1] = {0.0};
            for (int l = min(a.G, a.L) - 1; l >= 0; --l) {
                if (!(ok = grid_sync(a.bar, gen, a.spin))) break;
                phase_prolong_sweep<V>(a.lev, l, grid_rows(a.lev[l].n), t0, step);
                if (!(ok = grid_sync(a.bar, gen, a.spin))) break;
                phase_sweep<V>(a.lev, l, VL<V>::x(a.lev[l]), VL<V>::xa(a.lev[l]),
                               grid_rows(a.lev[l].n), t0, step);
            }
            if (!ok) break;
            if (a.L == 0 && !(ok = grid_sync(a.bar, gen, a.spin))) break;
            // rho = r.z (z = level 0's xa, in FP64)
            const V *z = VL<V>::xa(L0);
            for (int i = s0.lo + t0; i < s0.hi; i += step) v1[0] += a.r[i] * (double)z[i];
            if (!(ok = cg_grid_sum<1, kAmgBlock>(v1, a.partA, a.bar, gen, a.spin, buf, tot))) break;
            ++it;
            if (threadIdx.x == 0) {
                const double rho = tot[0];
                sc.beta = it == 1 ? 0.0 : rho / sc.rho;
                sc.rho = rho;
                if (!(rho > 0.0) || !isfinite(rho)) sc.phase = 3;
            }
            __syncthreads();
            if (sc.phase == 3) break;
            // ---- p = z + beta p
            const double beta = sc.beta;
            for (int i = s0.lo + t0; i < s0.hi; i += step)
                a.p[i] = it == 1 ? (double)z[i] : (double)z[i] + beta * a.p[i];
            if (!(ok = grid_sync(a.bar, gen, a.spin))) break;
            // ---- q = A p, p.q
            double v2[1] = {0.0};
            for (int i = s0.lo + t0; i < s0.hi; i += step) {
                const double qi = row_ax(a, L0, 0, i, a.p);
                a.q[i] = qi;
                v2[0] += a.p[i] * qi;
            }
            if (!(ok = cg_grid_sum<1, kAmgBlock>(v2, a.partB, a.bar, gen, a.spin, buf, tot))) break;
            if (threadIdx.x == 0) {
                const double pq = tot[0];
                if (!(pq > 0.0) || !isfinite(pq)) { sc.phase = 3; sc.alpha = 0.0; }
                else sc.alpha = sc.rho / pq;
            }
            __syncthreads();
            if (sc.phase == 3) break;
            // ---- x += alpha p, r -= alpha q, ||r||; next cycle's first sweep
            const double alpha = sc.alpha;
            double v3[1] = {0.0};
            for (int i = s0.lo + t0; i < s0.hi; i += step) {
                // all loads before the stores
                const double xi = a.x[i], pi = a.p[i], rio = a.r[i], qi = a.q[i];
                a.x[i] = xi + alpha * pi;
                const double ri = rio - alpha * qi;
                a.r[i] = ri;
                seed0<V>(L0, i, ri);
                v3[0] += ri * ri;
            }
            if (!(ok = cg_grid_sum<1, kAmgBlock>(v3, a.partA, a.bar, gen, a.spin, buf, tot))) break;
            if (threadIdx.x == 0) {
                sc.nr = sqrt(tot[0]);
                if (!isfinite(sc.nr)) sc.phase = 3;
                else if (sc.nr <= sc.thresh) sc.phase = 1;
                else if (it >= a.maxit) sc.phase = 2;
            }
            __syncthreads();
            if (sc.phase != 0) break;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const int ph = sc.phase;
        a.stats->iters = it;
        a.stats->status = !ok ? FV_E_TIMEOUT
                        : (ph == 3 || ph == 5) ? FV_E_DIVERGED
                        : ph == 2 ? FV_E_NOT_CONVERGED : FV_OK;
        const bool zero = ph == 4;
        a.stats->res0 = zero ? 0.0 : sc.nr0 / sc.nb;
        a.stats->res = zero ? 0.0 : sc.nr / sc.nb;
        a.stats->outer = 1;
    }
}

// ------------------------------------------------------------ building --

template <class T>
fv_status upload(DeviceArena &ar, const T **d, const std::vector<T> &h)
{
    T *p = nullptr;
    fv_status st = ar.alloc_n(&p, h.empty() ? 1 : h.size());
    if (st != FV_OK) return st;
    if (!h.empty() && cudaMemcpy(p, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice) != cudaSuccess)
        return FV_E_CUDA;
    *d = p;
    return FV_OK;
}

// Rows of a graph in SELL-32 slices: the off-diagonal entries of each row in
// ascending column (= ascending edge), slot k of row i at
// sptr[i / 32] + 32 k + i % 32; a slice is as wide as its longest row and
// the padding slots hold column i and edge -1.
void graph_sell(const Graph &g, std::vector<int32_t> &sptr, std::vector<int32_t> &scol,
                std::vector<int32_t> &sedge)
{
    const size_t ne = g.a.size();
    std::vector<int32_t> rptr(g.n + 1, 0);
    for (size_t e = 0; e < ne; ++e) { ++rptr[g.a[e] + 1]; ++rptr[g.b[e] + 1]; }
    for (int i = 0; i < g.n; ++i) rptr[i + 1] += rptr[i];
    std::vector<int32_t> rcol(2 * ne), redge(2 * ne), cur(rptr.begin(), rptr.end() - 1);
    // edges are ordered by (a, b): for row i the edges with b == i (columns
    // a < i) come in ascending a, then those with a == i in ascending b
    for (size_t e = 0; e < ne; ++e) {
        const int i = g.b[e];
        rcol[cur[i]] = g.a[e]; redge[cur[i]++] = (int32_t)e;
    }
    for (size_t e = 0; e < ne; ++e) {
        const int i = g.a[e];
        rcol[cur[i]] = g.b[e]; redge[cur[i]++] = (int32_t)e;
    }
    const int nsl = (g.n + 31) / 32;
    sptr.assign(nsl + 1, 0);
    for (int sl = 0; sl < nsl; ++sl) {
        int K = 0;
        for (int i = 32 * sl; i < std::min(g.n, 32 * sl + 32); ++i) K = std::max(K, rptr[i + 1] - rptr[i]);
        sptr[sl + 1] = sptr[sl] + 32 * K;
    }
    scol.assign(sptr[nsl], 0);
    sedge.assign(sptr[nsl], -1);
    for (int sl = 0; sl < nsl; ++sl) {
        const int K = (sptr[sl + 1] - sptr[sl]) / 32;
        for (int lane = 0; lane < 32; ++lane) {
            const int i = 32 * sl + lane;
            for (int k = 0; k < K; ++k) {
                const int e = sptr[sl] + 32 * k + lane;
                const bool real = i < g.n && k < rptr[i + 1] - rptr[i];
                scol[e] = real ? rcol[rptr[i] + k] : (i < g.n ? i : 0);
                sedge[e] = real ? redge[rptr[i] + k] : -1;
            }
        }
    }
}

// CSR of the items k (ascending) grouped by key[k] in [0, n); items with key < 0 skipped
void group(int n, const std::vector<int32_t> &key, std::vector<int32_t> &ptr,
           std::vector<int32_t> &list)
{
    ptr.assign(n + 1, 0);
    for (int32_t k : key) if (k >= 0) ++ptr[k + 1];
    for (int i = 0; i < n; ++i) ptr[i + 1] += ptr[i];
    list.resize(ptr[n]);
    std::vector<int32_t> cur(ptr.begin(), ptr.end() - 1);
    for (size_t t = 0; t < key.size(); ++t)
        if (key[t] >= 0) list[cur[key[t]]++] = (int32_t)t;
}

fv_status amg_build(fv_mesh *m, AmgData **out)
{
    const int N = m->N, F = m->F;
    // level-0 weights |S_f| Delta_f from the device geometry
    std::vector<double> mag(F), del(F);
    if (F > 0) {
        FV_CUDA(cudaStreamSynchronize(m->stream));
        FV_CUDA(cudaMemcpy(mag.data(), m->magSf, sizeof(double) * F, cudaMemcpyDeviceToHost));
        FV_CUDA(cudaMemcpy(del.data(), m->delta, sizeof(double) * F, cudaMemcpyDeviceToHost));
    }
    std::vector<Graph> g(1);
    g[0].n = N;
    g[0].a.assign(m->plan.own.begin(), m->plan.own.begin() + F);
    g[0].b.assign(m->plan.nei.begin(), m->plan.nei.begin() + F);
    g[0].w.resize(F);
    for (int f = 0; f < F; ++f) g[0].w[f] = mag[f] * del[f];
    std::vector<std::vector<int32_t>> agg, emap;
    while (g.back().n > kAmgNmin && (int)g.size() < kAmgMaxLev) {
        std::vector<int32_t> ag, em;
        Graph c = coarsen(g.back(), ag, em);
        if ((double)c.n > 0.9 * g.back().n) break;
        agg.push_back(std::move(ag));
        emap.push_back(std::move(em));
        g.push_back(std::move(c));
    }
    const int L = (int)g.size() - 1;
    FV_CHECK(g[L].n <= kAmgCoarseMax, FV_E_UNSUPPORTED,
             "multigrid coarsening stalled at %d nodes (the mesh graph is too weakly connected)",
             g[L].n);
    AmgData *h = new (std::nothrow) AmgData();
    FV_CHECK(h != nullptr, FV_E_NOMEM, "host allocation failed");
    h->L = L;
    // levels above this size run over the whole grid (FVGB_AMG_BLOCK_ROWS
    // overrides the default for tuning)
    long block_rows = kAmgBlockRows;
    if (const char *env = std::getenv("FVGB_AMG_BLOCK_ROWS")) block_rows = std::atol(env);
    int G = 1;
    while (G < L && g[G].n > block_rows) ++G;
    h->G = G;
    std::vector<AmgLevelDev> lv(L + 1);
    DeviceArena &ar = h->arena;
    fv_status st = FV_OK;
    auto fail = [&](fv_status s) { amg_release(h); return s; };
    for (int l = 0; l <= L; ++l) {
        AmgLevelDev &d = lv[l];
        std::memset(&d, 0, sizeof(d));
        d.n = g[l].n;
        d.ne = (int)g[l].a.size();
        h->n[l] = d.n;
        h->ne[l] = d.ne;
        std::vector<int32_t> sptr, scol, sedge;
        graph_sell(g[l], sptr, scol, sedge);
        if ((st = upload(ar, &d.sptr, sptr)) != FV_OK) return fail(st);
        if ((st = upload(ar, &d.scol, scol)) != FV_OK) return fail(st);
        if ((st = upload(ar, &d.sedge, sedge)) != FV_OK) return fail(st);
        if ((st = ar.alloc_n(&d.sval, scol.empty() ? 1 : scol.size())) != FV_OK) return fail(st);
        if (l < L && (st = upload(ar, &d.agg, agg[l])) != FV_OK) return fail(st);
        if (l > 0) {
            std::vector<int32_t> ptr, list, inner_key(g[l - 1].a.size(), -1);
            group(d.n, agg[l - 1], ptr, list);
            if ((st = upload(ar, &d.mptr, ptr)) != FV_OK) return fail(st);
            if ((st = upload(ar, &d.memb, list)) != FV_OK) return fail(st);
            for (size_t e = 0; e < inner_key.size(); ++e)
                if (emap[l - 1][e] < 0) inner_key[e] = agg[l - 1][g[l - 1].a[e]];
            group(d.n, inner_key, ptr, list);
            if ((st = upload(ar, &d.iptr, ptr)) != FV_OK) return fail(st);
            if ((st = upload(ar, &d.inner, list)) != FV_OK) return fail(st);
            group(d.ne, emap[l - 1], ptr, list);
            if ((st = upload(ar, &d.eptr, ptr)) != FV_OK) return fail(st);
            if ((st = upload(ar, &d.elist, list)) != FV_OK) return fail(st);
            if ((st = ar.alloc_n(&d.o, d.ne ? d.ne : 1)) != FV_OK) return fail(st);
        }
        if ((st = ar.alloc_n(&d.d, d.n)) != FV_OK) return fail(st);
        if ((st = ar.alloc_n(&d.dinv, d.n)) != FV_OK) return fail(st);
        // FP32 copies for the mixed-precision cycle
        if ((st = ar.alloc_n(&d.sval32, scol.empty() ? 1 : scol.size())) != FV_OK) return fail(st);
        if ((st = ar.alloc_n(&d.d32, d.n)) != FV_OK) return fail(st);
        if ((st = ar.alloc_n(&d.dinv32, d.n)) != FV_OK) return fail(st);
        if ((st = ar.alloc_n(&d.b32, d.n)) != FV_OK) return fail(st);
        if ((st = ar.alloc_n(&d.x32, d.n)) != FV_OK) return fail(st);
        if ((st = ar.alloc_n(&d.xa32, d.n)) != FV_OK) return fail(st);
        if (l > 0 && (st = ar.alloc_n(&d.b, d.n)) != FV_OK) return fail(st);
        if ((st = ar.alloc_n(&d.x, d.n)) != FV_OK) return fail(st);
        if ((st = ar.alloc_n(&d.xa, d.n)) != FV_OK) return fail(st);
    }
    if ((st = ar.alloc_n(&h->r, N)) != FV_OK) return fail(st);
    if ((st = ar.alloc_n(&h->p, N)) != FV_OK) return fail(st);
    if ((st = ar.alloc_n(&h->q, N)) != FV_OK) return fail(st);
    lv[0].b = h->r;            // level 0 smooths the CG residual
    h->z = lv[0].xa;
    if ((st = ar.alloc_n(&h->coarse_ok, 1)) != FV_OK) return fail(st);
    if ((st = ar.alloc_n(&h->lev, L + 1)) != FV_OK) return fail(st);
    FV_CUDA(cudaMemcpy(h->lev, lv.data(), sizeof(AmgLevelDev) * (L + 1), cudaMemcpyHostToDevice));
    int per_sm = 0;
    int per_sm32 = 0;
    FV_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pcg_amg<double>, kAmgBlock, 0));
    FV_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm32, k_pcg_amg<float>, kAmgBlock, 0));
    per_sm = std::min(per_sm, per_sm32);
    FV_CHECK(per_sm >= 1, FV_E_CUDA, "multigrid CG kernel cannot be resident");
    h->grid = m->sm_count * std::min(per_sm, 2);
    // dynamic shared memory: the coarsest factor and vector, and block 0's
    // copy of the levels it runs (the layout of shadow_setup, FP64 sizes) if
    // that keeps two blocks per SM; FVGB_AMG_SHADOW=0 keeps those levels in
    // global memory
    {
        auto a16 = [](size_t b) { return (b + 15) & ~(size_t)15; };
        const size_t nc = g[L].n;
        const size_t base = a16(8 * nc * nc) + a16(8 * nc);
        const size_t table = a16(sizeof(AmgLevelDev) * (L + 1));
        size_t bytes = 0;
        for (int l = G; l <= L && L > 0; ++l) {
            const size_t n = g[l].n, nsl = (n + 31) / 32;
            std::vector<int32_t> sptr, scol, sedge;
            graph_sell(g[l], sptr, scol, sedge);
            const size_t slots = scol.size();
            bytes += a16(8 * slots) + 5 * a16(8 * n) + a16(4 * (nsl + 1)) + a16(4 * slots);
            if (l < L) bytes += a16(4 * n);
            if (l > G) bytes += a16(4 * (n + 1)) + a16(4 * (size_t)g[l - 1].n);
        }
        const char *env = std::getenv("FVGB_AMG_SHADOW");
        const bool want = !(env && std::atoi(env) == 0);
        auto fits = [&](size_t dyn) {
            int p64 = 0, p32 = 0;
            const int sb = (int)dyn;
            bool ok = cudaFuncSetAttribute(k_pcg_amg<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, sb) == cudaSuccess &&
                      cudaFuncSetAttribute(k_pcg_amg<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, sb) == cudaSuccess &&
                      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p64, k_pcg_amg<double>, kAmgBlock, sb) == cudaSuccess &&
                      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p32, k_pcg_amg<float>, kAmgBlock, sb) == cudaSuccess;
            (void)cudaGetLastError();
            return ok ? std::min(p64, p32) : 0;
        };
        h->lev_table_bytes = (int)table;
        if (want && L > 0 && bytes <= (size_t)kAmgShadowMax && fits(base + table + bytes) >= std::min(per_sm, 2)) {
            h->shadow = 1;
            h->dyn_bytes = (int)(base + table + bytes);
        } else {
            h->dyn_bytes = (int)(base + table);
            const int p = fits(h->dyn_bytes);
            FV_CHECK(p >= 1, FV_E_CUDA, "multigrid CG kernel cannot be resident");
            h->grid = m->sm_count * std::min(p, 2);
        }
    }
    *out = h;
    return FV_OK;
}

}  // namespace

fv_status amg_prepare(fv_mesh *m)
{
    if (m->amg) return FV_OK;
    AmgData *h = nullptr;
    fv_status st = amg_build(m, &h);
    if (st != FV_OK) return st;
    m->amg = h;
    return FV_OK;
}

fv_status launch_pcg_amg(const fv_mesh *m, const AmgProblem &pb)
{
    fv_status st = amg_prepare(const_cast<fv_mesh *>(m));
    if (st != FV_OK) return st;
    const AmgData *h = m->amg;
    const KrylovWork &w = m->kw;
    AmgArgs a;
    a.L = h->L;
    a.G = h->G;
    a.nc = h->n[h->L];
    a.lev = h->lev;
    a.d0 = pb.diag;
    a.o0 = pb.off;
    a.o0_sign = pb.off_sign;
    a.fp32 = pb.fp32;
    a.shadow = h->shadow;
    a.lev_table_bytes = h->lev_table_bytes;
    a.b = pb.b;
    a.x = pb.x;
    a.r = h->r;
    a.z = h->z;
    a.p = h->p;
    a.q = h->q;
    const int gp = w.G > w.Gcg ? w.G : w.Gcg;
    a.partA = w.partials;
    a.partB = w.partials + (size_t)gp * kParts;
    a.coarse_ok = h->coarse_ok;
    a.bar = w.bar;
    a.spin = g_spin_limit;
    a.tol = pb.tol;
    a.reltol = pb.reltol;
    a.maxit = pb.maxit;
    a.stats = pb.stats;
    FV_CUDA(cudaMemsetAsync(w.bar, 0, sizeof(GridBar), m->stream));
    // about 4 rows per thread before another block is worth a grid barrier
    int G = (m->N + 4 * kAmgBlock - 1) / (4 * kAmgBlock);
    G = std::max(1, std::min(std::min(G, h->grid), gp));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(G);
    cfg.blockDim = dim3(kAmgBlock);
    cfg.dynamicSmemBytes = (size_t)h->dyn_bytes;
    cfg.stream = m->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    void *args[] = {&a};
    const void *fn = pb.fp32 ? (const void *)k_pcg_amg<float> : (const void *)k_pcg_amg<double>;
    FV_CUDA(cudaLaunchKernelExC(&cfg, fn, args));
    return FV_OK;
}

}  // namespace fvgb

using namespace fvgb;

extern "C" fv_status fv_amg_coarsen_host(int32_t n, int32_t ne, const int32_t *ea,
                                         const int32_t *eb, const double *ew, int32_t *agg,
                                         int32_t *emap, int32_t *n_coarse, int32_t *ne_coarse,
                                         int32_t *cea, int32_t *ceb, double *cew)
{
    FV_CHECK(n >= 0 && ne >= 0 && agg && n_coarse && ne_coarse, FV_E_INVALID, "bad arguments");
    FV_CHECK(ne == 0 || (ea && eb && ew && emap && cea && ceb && cew), FV_E_INVALID,
             "edge arrays missing");
    Graph g;
    g.n = n;
    g.a.assign(ea, ea + ne);
    g.b.assign(eb, eb + ne);
    g.w.assign(ew, ew + ne);
    for (int e = 0; e < ne; ++e) {
        FV_CHECK(g.a[e] >= 0 && g.a[e] < g.b[e] && g.b[e] < n, FV_E_INVALID,
                 "edge %d is not (lower, higher) within range", e);
        FV_CHECK(e == 0 || g.a[e - 1] < g.a[e] || (g.a[e - 1] == g.a[e] && g.b[e - 1] < g.b[e]),
                 FV_E_INVALID, "edges are not ordered by (lower, higher)");
        FV_CHECK(g.w[e] > 0.0, FV_E_INVALID, "edge %d has a non-positive weight", e);
    }
    std::vector<int32_t> ag, em;
    Graph c = coarsen(g, ag, em);
    std::copy(ag.begin(), ag.end(), agg);
    std::copy(em.begin(), em.end(), emap);
    *n_coarse = c.n;
    *ne_coarse = (int32_t)c.a.size();
    std::copy(c.a.begin(), c.a.end(), cea);
    std::copy(c.b.begin(), c.b.end(), ceb);
    std::copy(c.w.begin(), c.w.end(), cew);
    return FV_OK;
}

extern "C" fv_status fv_amg_info(const fv_mesh *mc, int32_t *n_levels, int32_t *sizes)
{
    FV_CHECK(mc && n_levels, FV_E_INVALID, "NULL argument");
    fv_mesh *m = const_cast<fv_mesh *>(mc);
    fv_status st = amg_prepare(m);
    if (st != FV_OK) return st;
    *n_levels = m->amg->L + 1;
    if (sizes)
        for (int l = 0; l <= m->amg->L; ++l) sizes[l] = m->amg->n[l];
    return FV_OK;
}
