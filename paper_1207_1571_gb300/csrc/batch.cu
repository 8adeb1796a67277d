// batch.cu -- many independent cases advanced together (not in the paper,
// which runs one case per GPU).
//
// The cases are joined into one block-diagonal "union" mesh: no face joins
// two cases, so the cell-gather assembly and correction kernels of the
// single-case path cover every case in one launch each (per-cell viscosity
// and per-cell reference-pressure flags carry what differs between cases).
// The linear solves are per case: one block owns one case at a time,
// taking cases from a work queue ordered by decreasing size, and
// synchronises with __syncthreads only, so cases of different sizes and
// iteration counts never wait for each other.  A PISO step is therefore a
// fixed sequence of ten launches, captured once into a CUDA graph.
//
// Schedule knobs (autotuned per batch): threads per block, rows per thread
// per loop trip, and the block reduction (shuffle tree in every warp, or
// shared-memory staging summed by a few warps).  All variants add in a
// fixed order, so every schedule is deterministic.
#include <algorithm>
#include <cstring>
#include <new>
#include <numeric>
#include <vector>

#include <cooperative_groups.h>

#include "fvgb_internal.h"

struct fv_batch {
    int ncase = 0;
    int precision = FV_PREC_FP64;
    fv_mesh *mesh = nullptr;
    fv_case *cs = nullptr;
    std::vector<int> start, count, cell_base, nface_int, nface_bnd, fbase_int, fbase_bnd;
    int32_t *d_start = nullptr, *d_count = nullptr, *d_order = nullptr, *d_next = nullptr;
    fvgb::DevSolveStats *d_stats = nullptr;     // [ncase][3 + FV_MAX_CORR]
    fvgb::DevSolveStats *h_stats = nullptr;
    double *save = nullptr;                     // state copy for the autotuner
    int cfg = 0;                                // schedule index
    cudaGraphExec_t graph = nullptr;
    fv_piso_params graph_prm{};
    fvgb::DeviceArena arena;
};

namespace fvgb {
namespace {

constexpr int kStatStride = 3 + FV_MAX_CORR;

// ------------------------------------------------------------ schedules --

// block = threads per block, unroll = rows per thread per loop trip,
// red = block reduction (0 shuffle tree, 1 shared-memory staging),
// cl = blocks per case for the pressure and momentum solves (a thread-block
// cluster sharing one case through distributed shared memory; the momentum
// solve uses blocks of at most 512 threads).
struct Sched {
    int block, unroll, red, cl;
};
constexpr Sched kScheds[] = {{256, 2, 0, 1},  {256, 2, 1, 1},  {512, 1, 1, 1},  {512, 2, 1, 1},
                             {1024, 2, 1, 1}, {512, 2, 1, 2},  {1024, 2, 1, 2}, {512, 2, 1, 4},
                             {1024, 2, 1, 4}, {1024, 2, 1, 8}};
constexpr int kNSched = sizeof(kScheds) / sizeof(kScheds[0]);
// residual-norm rule of the CG (see krylov.cu): evaluate ||D^1/2 r^|| only
// once min(D) r^.r^ is within kNearStop of thresh^2
constexpr double kNearStop = 16.0;
constexpr double kBoundMargin = 1.0 + 1e-8;

// Block sum; result in tot[] (shared), visible to all threads on return.
template <int BLOCK, int RED, int NV>
__device__ __forceinline__ void bsum(double (&v)[NV], double *tot)
{
    constexpr int W = BLOCK / 32;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (RED == 0) {
        __shared__ double red[NV][W];
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double x = v[k];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
            if (lane == 0) red[k][w] = x;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
#pragma unroll
            for (int k = 0; k < NV; ++k) {
                double x = 0.0;
#pragma unroll
                for (int q = 0; q < W; ++q) x += red[k][q];
                tot[k] = x;
            }
        }
    } else {
        // stage in shared memory; lane l of warp w < NR adds the values
        // w*BLOCK/NR + l + 32 j in a pairwise tree, warp 0 adds the NR
        // results of each lane and shuffles (the cost of a sum on this
        // FP64-bound kernel is its count of FP64 warp instructions: 3 + 8
        // for 512 threads, against 4 + 5 per warp and 4 on thread 0)
        constexpr int NR = W < 4 ? W : 4;
        constexpr int per = BLOCK / (32 * NR);
        __shared__ double stg[NV][BLOCK];
        __shared__ double lanes[NV][NR][32];
#pragma unroll
        for (int k = 0; k < NV; ++k) stg[k][threadIdx.x] = v[k];
        __syncthreads();
        if (w < NR) {
#pragma unroll
            for (int k = 0; k < NV; ++k) {
                double t[per];
#pragma unroll
                for (int j = 0; j < per; ++j) t[j] = stg[k][w * (BLOCK / NR) + lane + 32 * j];
#pragma unroll
                for (int st = 1; st < per; st <<= 1)
#pragma unroll
                    for (int j = 0; j + st < per; j += 2 * st) t[j] += t[j + st];
                lanes[k][w][lane] = t[0];
            }
        }
        __syncthreads();
        if (w == 0) {
#pragma unroll
            for (int k = 0; k < NV; ++k) {
                double x;
                if (NR == 4) {
                    x = (lanes[k][0][lane] + lanes[k][1][lane]) + (lanes[k][2][lane] + lanes[k][3][lane]);
                } else {
                    x = lanes[k][0][lane];
#pragma unroll
                    for (int q = 1; q < NR; ++q) x += lanes[k][q][lane];
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
                if (lane == 0) tot[k] = x;
            }
        }
    }
    __syncthreads();
}

struct RowS {
    int e0, K;
};
__device__ __forceinline__ RowS rowspan(const int32_t *__restrict__ sp, int i)
{
    const int s = i >> 5;
    const int p0 = sp[s], p1 = sp[s + 1];
    return {p0 + (i & 31), (p1 - p0) >> 5};
}

// queue: every block takes the next case until none is left
__device__ __forceinline__ int next_case(int32_t *counter, int *slot)
{
    if (threadIdx.x == 0) *slot = atomicAdd(counter, 1);
    __syncthreads();
    const int q = *slot;
    __syncthreads();
    return q;
}

// ---------------------------------------------------- cluster helpers ----
// A case of a solve is owned by a cluster of CL blocks (CL = 1:
// one block).  Phases are separated by a cluster barrier (release/acquire at
// cluster scope, so rows written by one block are visible to the others);
// reductions add the CL block totals, read through distributed shared
// memory in rank order, so every block holds the same bits.

template <int CL>
__device__ __forceinline__ void csync()
{
    if (CL == 1) __syncthreads();
    else cooperative_groups::this_cluster().sync();
}

template <int BLOCK, int RED, int CL, int NV>
__device__ __forceinline__ void csum(double (&v)[NV], double *tot, double *cpart, int &par)
{
    bsum<BLOCK, RED, NV>(v, tot);
    if (CL == 1) return;
    cooperative_groups::cluster_group cl = cooperative_groups::this_cluster();
    if (threadIdx.x < NV) cpart[par * 8 + threadIdx.x] = tot[threadIdx.x];
    cl.sync();
    if (threadIdx.x < NV) {
        double x = cl.map_shared_rank(cpart, 0)[par * 8 + threadIdx.x];
        for (int r = 1; r < CL; ++r) x += cl.map_shared_rank(cpart, r)[par * 8 + threadIdx.x];
        tot[threadIdx.x] = x;
    }
    par ^= 1;    // the next reduction uses the other half (see the barrier argument above)
    __syncthreads();
}

// Minimum over the cluster's blocks (every thread receives it).
template <int BLOCK, int CL>
__device__ __forceinline__ double cmin(double v)
{
    __shared__ double wmin[BLOCK / 32];
    __shared__ double bmin;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) wmin[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = wmin[0];
        for (int w = 1; w < BLOCK / 32; ++w) m = fmin(m, wmin[w]);
        bmin = m;
    }
    if (CL > 1) {
        cooperative_groups::cluster_group cl = cooperative_groups::this_cluster();
        cl.sync();
        double m = bmin;
        for (int r = 0; r < CL; ++r) m = fmin(m, *cl.map_shared_rank(&bmin, r));
        cl.sync();                 // every block has read every block's bmin
        __syncthreads();
        if (threadIdx.x == 0) bmin = m;
    }
    __syncthreads();
    const double r = bmin;
    __syncthreads();
    return r;
}

// next case for the cluster: rank 0 takes it from the queue
template <int CL>
__device__ __forceinline__ int cluster_next_case(int32_t *counter, int *slot)
{
    if (CL == 1) return next_case(counter, slot);
    cooperative_groups::cluster_group cl = cooperative_groups::this_cluster();
    if (cl.block_rank() == 0 && threadIdx.x == 0) *slot = atomicAdd(counter, 1);
    cl.sync();
    const int q = *cl.map_shared_rank(slot, 0);
    cl.sync();
    return q;
}

// --------------------------------------------------------------- CG ----

struct BCg {
    int ncase;
    const int32_t *start, *count, *order;
    int32_t *next;
    const int32_t *slice_ptr, *col;
    double *val;
    const double *diag, *b;
    double *x, *s, *r, *p, *q, *y;
    double tol, reltol;
    int maxit;
    DevSolveStats *stats;     // + case * kStatStride
};

template <int BLOCK, int U, int RED, int CL>
__global__ void __launch_bounds__(BLOCK) k_pcg_batch(BCg a)
{
    __shared__ int slot;
    __shared__ double tot[3], cpart[16];
    __shared__ double sc_alpha, sc_beta, sc_rho, sc_thr, sc_nb, sc_nr0, sc_nr, sc_dmin;
    __shared__ int sc_phase, sc_exact;
    const int rank = CL == 1 ? 0 : (int)cooperative_groups::this_cluster().block_rank();
    int par = 0;
    for (;;) {
        const int q = cluster_next_case<CL>(a.next, &slot);
        if (q >= a.ncase) break;
        const int cid = a.order[q];
        const int n = a.count[cid], chunk = (n + CL - 1) / CL;
        const int r0 = a.start[cid] + min(n, rank * chunk);
        const int r1 = a.start[cid] + min(n, (rank + 1) * chunk);
        const int i0 = r0 + threadIdx.x;
        int it = 0;
        double dmin = INFINITY;
        for (int i = i0; i < r1; i += BLOCK) {
            const double d = a.diag[i], sq = sqrt(d);
            a.s[i] = 1.0 / sq;
            a.y[i] = a.x[i] * sq;
            dmin = d > 0.0 ? fmin(dmin, d) : 0.0;
        }
        dmin = cmin<BLOCK, CL>(dmin);     // (its cluster barriers also order s and y)
        csync<CL>();
        {
            double v3[3] = {0.0, 0.0, 0.0};
            for (int i = i0; i < r1; i += BLOCK) {
                const RowS rs = rowspan(a.slice_ptr, i);
                const double si = a.s[i], d = a.diag[i];
                double ax = d * a.x[i];
                for (int k = 0; k < rs.K; ++k) {
                    const int e = rs.e0 + 32 * k;
                    const int c = a.col[e];
                    const double v = a.val[e];
                    ax += v * a.x[c];
                    a.val[e] = v * si * a.s[c];
                }
                const double bi = a.b[i];
                const double rh = si * (bi - ax);
                a.r[i] = rh;
                v3[0] += bi * bi;
                v3[1] += d * rh * rh;
                v3[2] += rh * rh;
            }
            csum<BLOCK, RED, CL, 3>(v3, tot, cpart, par);
        }
        if (threadIdx.x == 0) {
            sc_nb = sqrt(tot[0]);
            sc_nr0 = sc_nr = sqrt(tot[1]);
            sc_rho = tot[2];
            sc_thr = fmax(a.tol * sc_nb, a.reltol * sc_nr0);
            sc_alpha = sc_beta = 0.0;
            sc_phase = sc_nb == 0.0 ? 4 : (sc_nr0 <= sc_thr ? 1 : 0);
            sc_dmin = dmin;
            sc_exact = 1;
        }
        __syncthreads();
        if (sc_phase == 4) {
            for (int i = i0; i < r1; i += BLOCK) a.x[i] = 0.0;
        } else if (sc_phase == 0) {
            for (;;) {
                ++it;
                const double al = sc_alpha, be = sc_beta;
                if (it == 1) {
                    for (int i = i0; i < r1; i += BLOCK) a.p[i] = a.r[i];
                } else {
#pragma unroll U
                    for (int i = i0; i < r1; i += BLOCK) {
                        // all loads before the stores
                        const double po = a.p[i], ri = a.r[i], yi = a.y[i];
                        a.p[i] = ri + be * po;
                        a.y[i] = yi + al * po;
                    }
                }
                csync<CL>();
                double v1[1] = {0.0};
#pragma unroll U
                for (int i = i0; i < r1; i += BLOCK) {
                    const RowS rs = rowspan(a.slice_ptr, i);
                    const double pi = a.p[i];
                    double acc = pi;
                    for (int k = 0; k < rs.K; ++k) {
                        const int e = rs.e0 + 32 * k;
                        acc += a.val[e] * a.p[a.col[e]];
                    }
                    a.q[i] = acc;
                    v1[0] += pi * acc;
                }
                csum<BLOCK, RED, CL, 1>(v1, tot, cpart, par);
                if (threadIdx.x == 0) {
                    const double pq = tot[0];
                    if (!(pq > 0.0) || !isfinite(pq)) { sc_phase = 3; sc_alpha = 0.0; }
                    else sc_alpha = sc_rho / pq;
                }
                __syncthreads();
                if (sc_phase == 3) break;
                // r^ -= alpha q and r^.r^; ||D^1/2 r^||^2 only once min(D) r^.r^
                // allows the stop (the rule of the single-case CG: identical
                // iterates and counts, two FP64 operations per row saved)
                const double alpha = sc_alpha;
                const bool exact = sc_exact || it >= a.maxit;
                double v2[2] = {0.0, 0.0};
                if (exact) {
                    for (int i = i0; i < r1; i += BLOCK) {
                        const double ri = a.r[i] - alpha * a.q[i];
                        a.r[i] = ri;
                        v2[0] += ri * ri;
                        v2[1] += (a.diag[i] * ri) * ri;
                    }
                } else {
                    double acc = 0.0;
#pragma unroll U
                    for (int i = i0; i < r1; i += BLOCK) {
                        const double qi = a.q[i], rio = a.r[i];
                        const double ri = rio - alpha * qi;
                        a.r[i] = ri;
                        acc += ri * ri;
                    }
                    v2[0] = acc;
                }
                csum<BLOCK, RED, CL, 2>(v2, tot, cpart, par);
                if (threadIdx.x == 0)
                    sc_exact = exact ? 1 : (sc_dmin * tot[0] > sc_thr * sc_thr * kBoundMargin ? 0 : 2);
                __syncthreads();
                if (sc_exact == 2) {
                    double v4[1] = {0.0};
                    for (int i = i0; i < r1; i += BLOCK) {
                        const double ri = a.r[i];
                        v4[0] += (a.diag[i] * ri) * ri;
                    }
                    csum<BLOCK, RED, CL, 1>(v4, tot + 1, cpart, par);
                }
                if (threadIdx.x == 0) {
                    const double rho = tot[0];
                    const bool have = sc_exact != 0;
                    sc_nr = have ? sqrt(tot[1]) : sqrt(sc_dmin * rho);
                    if (!isfinite(sc_nr) || !isfinite(rho)) sc_phase = 3;
                    else if (have && sc_nr <= sc_thr) sc_phase = 1;
                    else if (it >= a.maxit) sc_phase = 2;
                    else {
                        sc_beta = rho / sc_rho;
                        sc_rho = rho;
                        sc_exact = sc_dmin * rho <= kNearStop * sc_thr * sc_thr ? 1 : 0;
                    }
                }
                __syncthreads();
                if (sc_phase != 0) break;
            }
            const double af = sc_phase == 3 ? 0.0 : sc_alpha;
            for (int i = i0; i < r1; i += BLOCK) a.x[i] = a.s[i] * (a.y[i] + af * a.p[i]);
        }
        if (threadIdx.x == 0 && rank == 0) {
            DevSolveStats *st = a.stats + (size_t)cid * kStatStride;
            const int ph = sc_phase;
            st->iters = it;
            st->status = ph == 3 ? FV_E_DIVERGED : ph == 2 ? FV_E_NOT_CONVERGED : FV_OK;
            st->res0 = ph == 4 ? 0.0 : sc_nr0 / sc_nb;
            st->res = ph == 4 ? 0.0 : sc_nr / sc_nb;
            st->outer = 1;
        }
        __syncthreads();
    }
}

// ------------------------------------------------- mixed-precision CG ----
// Per-case version of the single-case mixed-precision solve: FP32
// reliable-update CG deflated by the constant mode, FP64 true residual,
// stopping test, solution and reductions.

constexpr double kBReliable = 0.1;

struct BMix {
    int ncase;
    const int32_t *start, *count, *order;
    int32_t *next;
    const int32_t *slice_ptr, *col;
    const double *val;
    float *val32;
    const double *diag, *b;
    double *x, *s, *r64, *a1;
    float *r, *p, *q, *e, *w, *v;
    double tol, reltol;
    int maxit;
    DevSolveStats *stats;
};

template <int BLOCK, int U, int RED, int CL>
__global__ void __launch_bounds__(BLOCK) k_pcg_mixed_batch(BMix a)
{
    __shared__ int slot;
    __shared__ double tot[3], cpart[16];
    __shared__ double s_nb, s_nr0, s_nr, s_thr, s_rho, s_ref, s_ratio, s_alpha, s_beta, s_mu,
        s_delta, s_shift;
    __shared__ int s_phase, s_refresh, s_restart, s_bad, s_defl;
    const int rank = CL == 1 ? 0 : (int)cooperative_groups::this_cluster().block_rank();
    int par = 0;
    for (;;) {
        const int qq = cluster_next_case<CL>(a.next, &slot);
        if (qq >= a.ncase) break;
        const int cid = a.order[qq];
        const int n = a.count[cid], chunk = (n + CL - 1) / CL;
        const int r0 = a.start[cid] + min(n, rank * chunk);
        const int r1 = a.start[cid] + min(n, (rank + 1) * chunk);
        const int i0 = r0 + threadIdx.x;
        int it = 0, outer = 0;
        for (int i = i0; i < r1; i += BLOCK) a.s[i] = 1.0 / sqrt(a.diag[i]);
        csync<CL>();
        {
            double v1[1] = {0.0};
            for (int i = i0; i < r1; i += BLOCK) {
                const RowS rs = rowspan(a.slice_ptr, i);
                const double si = a.s[i];
                double row = a.diag[i];
                for (int k = 0; k < rs.K; ++k) {
                    const int e = rs.e0 + 32 * k;
                    const double v = a.val[e];
                    row += v;
                    a.val32[e] = (float)(v * si * a.s[a.col[e]]);
                }
                a.a1[i] = row;
                a.w[i] = (float)(1.0 / si);
                a.v[i] = (float)(si * row);
                v1[0] += row;
            }
            csum<BLOCK, RED, CL, 1>(v1, tot, cpart, par);
        }
        if (threadIdx.x == 0) {
            s_phase = 0; s_alpha = s_beta = s_delta = 0.0; s_restart = 1; s_bad = 0;
            s_refresh = 0; s_nr = 0.0; s_mu = tot[0];
            s_defl = (tot[0] > 0.0 && isfinite(tot[0])) ? 1 : 0;
        }
        __syncthreads();
        for (;;) {
            {
                double v2[2] = {0.0, 0.0};
                for (int i = i0; i < r1; i += BLOCK) {
                    const RowS rs = rowspan(a.slice_ptr, i);
                    double ax = a.diag[i] * a.x[i];
                    for (int k = 0; k < rs.K; ++k) {
                        const int e = rs.e0 + 32 * k;
                        ax += a.val[e] * a.x[a.col[e]];
                    }
                    const double bi = a.b[i], ri = bi - ax;
                    a.r64[i] = ri;
                    v2[0] += bi * bi;
                    v2[1] += ri;
                }
                csum<BLOCK, RED, CL, 2>(v2, tot, cpart, par);
            }
            if (threadIdx.x == 0) {
                if (outer == 0) s_nb = sqrt(tot[0]);
                s_shift = s_defl ? tot[1] / s_mu : 0.0;
            }
            __syncthreads();
            {
                const double sh = s_shift;
                double v3[3] = {0.0, 0.0, 0.0};
                for (int i = i0; i < r1; i += BLOCK) {
                    const double ri = a.r64[i] - sh * a.a1[i];
                    a.x[i] += sh;
                    const float rh = (float)(a.s[i] * ri);
                    a.r[i] = rh;
                    a.e[i] = 0.0f;
                    v3[0] += ri * ri;
                    v3[1] += (double)rh * (double)rh;
                    v3[2] += (double)a.v[i] * (double)rh;
                }
                csum<BLOCK, RED, CL, 3>(v3, tot, cpart, par);
            }
            if (threadIdx.x == 0) {
                const double prev = s_nr;
                s_nr = sqrt(tot[0]);
                if (outer == 0) {
                    s_nr0 = s_nr;
                    s_thr = fmax(a.tol * s_nb, a.reltol * s_nr0);
                    if (s_nb == 0.0) s_phase = 4;
                } else if (s_refresh == 2) {
                    s_bad = s_nr >= prev ? s_bad + 1 : 0;
                    if (s_bad >= 2) s_phase = 3;
                }
                if (s_phase == 0) {
                    if (!isfinite(s_nr)) s_phase = 3;
                    else if (s_nr <= s_thr) s_phase = 1;
                    else if (it >= a.maxit) s_phase = 2;
                }
                s_beta = (outer > 0 && !s_restart && s_rho > 0.0) ? tot[1] / s_rho : 0.0;
                s_rho = s_ref = tot[1];
                s_ratio = tot[1] > 0.0 ? s_nr / sqrt(tot[1]) : 0.0;
                s_delta = s_defl ? tot[2] / s_mu : 0.0;
                s_alpha = 0.0;
                s_refresh = 0;
            }
            __syncthreads();
            ++outer;
            if (s_phase != 0) break;
            for (;;) {
                ++it;
                const float al = (float)s_alpha, be = (float)s_beta, de = (float)s_delta;
                if (s_restart) {
                    for (int i = i0; i < r1; i += BLOCK) a.p[i] = fmaf(-de, a.w[i], a.r[i]);
                } else {
#pragma unroll U
                    for (int i = i0; i < r1; i += BLOCK) {
                        const float po = a.p[i];
                        a.e[i] = fmaf(al, po, a.e[i]);
                        a.p[i] = fmaf(-de, a.w[i], fmaf(be, po, a.r[i]));
                    }
                }
                csync<CL>();
                float pq32 = 0.0f;
#pragma unroll U
                for (int i = i0; i < r1; i += BLOCK) {
                    const RowS rs = rowspan(a.slice_ptr, i);
                    const float pi = a.p[i];
                    float acc = pi;
                    for (int k = 0; k < rs.K; ++k) {
                        const int e = rs.e0 + 32 * k;
                        acc = fmaf(a.val32[e], a.p[a.col[e]], acc);
                    }
                    a.q[i] = acc;
                    pq32 = fmaf(pi, acc, pq32);
                }
                double v1[1] = {(double)pq32};
                csum<BLOCK, RED, CL, 1>(v1, tot, cpart, par);
                if (threadIdx.x == 0) {
                    s_restart = 0;
                    const double pq = tot[0];
                    if (!(pq > 0.0) || !isfinite(pq)) { s_refresh = 2; s_alpha = 0.0; }
                    else s_alpha = s_rho / pq;
                }
                __syncthreads();
                if (s_refresh == 2) break;
                const float a32 = (float)s_alpha;
                float rr32 = 0.0f, vr32 = 0.0f;
#pragma unroll U
                for (int i = i0; i < r1; i += BLOCK) {
                    const float ri = fmaf(-a32, a.q[i], a.r[i]);
                    a.r[i] = ri;
                    rr32 = fmaf(ri, ri, rr32);
                    vr32 = fmaf(a.v[i], ri, vr32);
                }
                double v2[2] = {(double)rr32, (double)vr32};
                csum<BLOCK, RED, CL, 2>(v2, tot, cpart, par);
                if (threadIdx.x == 0) {
                    const double rn = tot[0];
                    if (!isfinite(rn)) s_refresh = 2;
                    else if (rn <= kBReliable * kBReliable * s_ref || s_ratio * sqrt(rn) <= s_thr ||
                             it >= a.maxit)
                        s_refresh = 1;
                    else {
                        s_beta = rn / s_rho;
                        s_rho = rn;
                        s_delta = s_defl ? tot[1] / s_mu : 0.0;
                    }
                }
                __syncthreads();
                if (s_refresh) break;
            }
            const float a32 = (float)s_alpha;
            for (int i = i0; i < r1; i += BLOCK) a.x[i] += a.s[i] * (double)fmaf(a32, a.p[i], a.e[i]);
            if (threadIdx.x == 0 && s_refresh == 2) s_restart = 1;
            csync<CL>();
        }
        if (s_phase == 4)
            for (int i = i0; i < r1; i += BLOCK) a.x[i] = 0.0;
        if (threadIdx.x == 0 && rank == 0) {
            DevSolveStats *st = a.stats + (size_t)cid * kStatStride;
            const int ph = s_phase;
            st->iters = it;
            st->status = ph == 3 ? FV_E_DIVERGED : ph == 2 ? FV_E_NOT_CONVERGED : FV_OK;
            st->res0 = ph == 4 ? 0.0 : s_nr0 / s_nb;
            st->res = ph == 4 ? 0.0 : s_nr / s_nb;
            st->outer = outer;
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------- BiCGStab ----

struct BBi {
    int ncase, N;
    const int32_t *start, *count, *order;
    int32_t *next;
    const int32_t *slice_ptr, *col;
    const double *val, *diag, *src, *gradp, *V;
    double *x, *dinv;
    double *r, *rh, *p, *v, *y, *s, *z, *t;   // [3][N]
    double tol, reltol;
    int maxit;
    DevSolveStats *stats;
};

// A vec on row i for the components flagged in act, the row's coefficients
// read once for all three; each component's sum runs diagonal first, then
// the row's entries in slot order
__device__ __forceinline__ void bspmv3(const BBi &a, int i, double d, const double *vec,
                                       const int (&act)[3], double (&out)[3])
{
    const RowS rs = rowspan(a.slice_ptr, i);
    const size_t NN = a.N;
#pragma unroll
    for (int c = 0; c < 3; ++c) out[c] = act[c] ? d * vec[c * NN + i] : 0.0;
    for (int k = 0; k < rs.K; ++k) {
        const int e = rs.e0 + 32 * k;
        const double v = a.val[e];
        const size_t j = (size_t)a.col[e];
#pragma unroll
        for (int c = 0; c < 3; ++c)
            if (act[c]) out[c] += v * vec[c * NN + j];
    }
}

// A case is owned by a cluster of CL blocks (rows split evenly between them),
// with the cluster barriers and sums of the pressure solve; CL = 1: one block.
// Registers are capped so that 1024 threads per SM stay resident (without the
// cap the compiler took up to 128 per thread: one 512-thread block per SM).
template <int BLOCK, int U, int RED, int CL>
__global__ void __launch_bounds__(BLOCK, 1024 / BLOCK) k_bicgstab_batch(BBi a)
{
    __shared__ int slot;
    __shared__ double tot[6], cpart[16];
    __shared__ double s_nb[3], s_nr0[3], s_nr[3], s_thr[3], s_rho[3], s_rho_old[3], s_alpha[3],
        s_omega[3];
    __shared__ int s_active[3], s_iters[3], s_status[3], s_zero[3], s_nact;
    const size_t NN = a.N;
    const int rank = CL == 1 ? 0 : (int)cooperative_groups::this_cluster().block_rank();
    int par = 0;
    for (;;) {
        const int q = cluster_next_case<CL>(a.next, &slot);
        if (q >= a.ncase) break;
        const int cid = a.order[q];
        const int n = a.count[cid], chunk = (n + CL - 1) / CL;
        const int r0 = a.start[cid] + min(n, rank * chunk);
        const int r1 = a.start[cid] + min(n, (rank + 1) * chunk);
        const int i0 = r0 + threadIdx.x;
        double v6[6] = {0, 0, 0, 0, 0, 0};
        const int all[3] = {1, 1, 1};
        for (int i = i0; i < r1; i += BLOCK) {
            const double d = a.diag[i];
            a.dinv[i] = 1.0 / d;
            double ax[3];
            bspmv3(a, i, d, a.x, all, ax);
            for (int c = 0; c < 3; ++c) {
                const double bi = a.src[c * NN + i] - a.V[i] * a.gradp[c * NN + i];
                const double ri = bi - ax[c];
                a.r[c * NN + i] = ri;
                a.rh[c * NN + i] = ri;
                v6[2 * c] += bi * bi;
                v6[2 * c + 1] += ri * ri;
            }
        }
        csum<BLOCK, RED, CL, 6>(v6, tot, cpart, par);
        if (threadIdx.x == 0) {
            s_nact = 0;
            for (int c = 0; c < 3; ++c) {
                s_nb[c] = sqrt(tot[2 * c]);
                s_nr0[c] = s_nr[c] = sqrt(tot[2 * c + 1]);
                s_thr[c] = fmax(a.tol * s_nb[c], a.reltol * s_nr0[c]);
                s_rho[c] = tot[2 * c + 1];
                s_rho_old[c] = s_alpha[c] = s_omega[c] = 1.0;
                s_iters[c] = 0;
                s_status[c] = FV_OK;
                s_zero[c] = s_nb[c] == 0.0;
                s_active[c] = !s_zero[c] && s_nr0[c] > s_thr[c];
                s_nact += s_active[c];
                if (s_zero[c]) s_nr0[c] = s_nr[c] = 0.0;
            }
        }
        __syncthreads();
        for (int c = 0; c < 3; ++c)
            if (s_zero[c])
                for (int i = i0; i < r1; i += BLOCK) a.x[c * NN + i] = 0.0;
        int it = 0;
        while (s_nact > 0) {
            ++it;
            double beta[3], omega[3];
            int act[3];
            for (int c = 0; c < 3; ++c) {
                act[c] = s_active[c];
                omega[c] = s_omega[c];
                beta[c] = (s_rho[c] / s_rho_old[c]) * (s_alpha[c] / s_omega[c]);
            }
#pragma unroll U
            for (int i = i0; i < r1; i += BLOCK) {
                // every component's loads are issued before the first store
                const double di = a.dinv[i];
                double rr[3], pp[3], vv[3];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    rr[c] = pp[c] = vv[c] = 0.0;
                    if (!act[c]) continue;
                    const size_t j = c * NN + i;
                    rr[c] = a.r[j];
                    if (it > 1) { pp[c] = a.p[j]; vv[c] = a.v[j]; }
                }
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    if (!act[c]) continue;
                    const size_t j = c * NN + i;
                    const double pn = it == 1 ? rr[c] : rr[c] + beta[c] * (pp[c] - omega[c] * vv[c]);
                    a.p[j] = pn;
                    a.y[j] = pn * di;
                }
            }
            csync<CL>();      // the product gathers other rows' y
            double v3[3] = {0, 0, 0};
#pragma unroll U
            for (int i = i0; i < r1; i += BLOCK) {
                const double d = a.diag[i];
                double rh[3], ay[3];
#pragma unroll
                for (int c = 0; c < 3; ++c) rh[c] = act[c] ? a.rh[c * NN + i] : 0.0;
                bspmv3(a, i, d, a.y, act, ay);
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    if (!act[c]) continue;
                    a.v[c * NN + i] = ay[c];
                    v3[c] += rh[c] * ay[c];
                }
            }
            csum<BLOCK, RED, CL, 3>(v3, tot, cpart, par);
            if (threadIdx.x == 0)
                for (int c = 0; c < 3; ++c) {
                    if (!s_active[c]) continue;
                    if (tot[c] == 0.0 || !isfinite(tot[c])) {
                        s_status[c] = FV_E_DIVERGED; s_iters[c] = it; s_active[c] = 0; --s_nact;
                    } else {
                        s_alpha[c] = s_rho[c] / tot[c];
                    }
                }
            __syncthreads();
            double alpha[3];
            for (int c = 0; c < 3; ++c) { act[c] = s_active[c]; alpha[c] = s_alpha[c]; }
#pragma unroll U
            for (int i = i0; i < r1; i += BLOCK) {
                const double di = a.dinv[i];
                double rr[3], vv[3];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    rr[c] = act[c] ? a.r[c * NN + i] : 0.0;
                    vv[c] = act[c] ? a.v[c * NN + i] : 0.0;
                }
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    if (!act[c]) continue;
                    const size_t j = c * NN + i;
                    const double si = rr[c] - alpha[c] * vv[c];
                    a.s[j] = si;
                    a.z[j] = si * di;
                }
            }
            csync<CL>();      // the product gathers other rows' z
            double w6[6] = {0, 0, 0, 0, 0, 0};
#pragma unroll U
            for (int i = i0; i < r1; i += BLOCK) {
                const double d = a.diag[i];
                double ss[3], az[3];
#pragma unroll
                for (int c = 0; c < 3; ++c) ss[c] = act[c] ? a.s[c * NN + i] : 0.0;
                bspmv3(a, i, d, a.z, act, az);
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    if (!act[c]) continue;
                    const double ti = az[c];
                    a.t[c * NN + i] = ti;
                    w6[2 * c] += ti * ss[c];
                    w6[2 * c + 1] += ti * ti;
                }
            }
            csum<BLOCK, RED, CL, 6>(w6, tot, cpart, par);
            if (threadIdx.x == 0)
                for (int c = 0; c < 3; ++c)
                    if (s_active[c]) s_omega[c] = tot[2 * c + 1] > 0.0 ? tot[2 * c] / tot[2 * c + 1] : 0.0;
            __syncthreads();
            for (int c = 0; c < 3; ++c) omega[c] = s_omega[c];
            double u6[6] = {0, 0, 0, 0, 0, 0};
#pragma unroll U
            for (int i = i0; i < r1; i += BLOCK) {
                double xn[3], rn[3], rh[3];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    xn[c] = rn[c] = rh[c] = 0.0;
                    if (!act[c]) continue;
                    const size_t j = c * NN + i;
                    xn[c] = a.x[j] + (alpha[c] * a.y[j] + omega[c] * a.z[j]);
                    rn[c] = a.s[j] - omega[c] * a.t[j];
                    rh[c] = a.rh[j];
                }
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    if (!act[c]) continue;
                    const size_t j = c * NN + i;
                    a.x[j] = xn[c];
                    a.r[j] = rn[c];
                    u6[2 * c] += rh[c] * rn[c];
                    u6[2 * c + 1] += rn[c] * rn[c];
                }
            }
            csum<BLOCK, RED, CL, 6>(u6, tot, cpart, par);
            if (threadIdx.x == 0)
                for (int c = 0; c < 3; ++c) {
                    if (!s_active[c]) continue;
                    s_nr[c] = sqrt(tot[2 * c + 1]);
                    int stop = 0;
                    if (!isfinite(s_nr[c])) { s_status[c] = FV_E_DIVERGED; stop = 1; }
                    else if (s_nr[c] <= s_thr[c]) stop = 1;
                    else if (it >= a.maxit) { s_status[c] = FV_E_NOT_CONVERGED; stop = 1; }
                    else if (s_omega[c] == 0.0) { s_status[c] = FV_E_DIVERGED; stop = 1; }
                    if (stop) { s_iters[c] = it; s_active[c] = 0; --s_nact; }
                    s_rho_old[c] = s_rho[c];
                    s_rho[c] = tot[2 * c];
                }
            __syncthreads();
        }
        if (threadIdx.x == 0 && rank == 0)
            for (int c = 0; c < 3; ++c) {
                DevSolveStats *st = a.stats + (size_t)cid * kStatStride + c;
                st->iters = s_iters[c];
                st->status = s_status[c];
                st->res0 = s_nb[c] > 0.0 ? s_nr0[c] / s_nb[c] : 0.0;
                st->res = s_nb[c] > 0.0 ? s_nr[c] / s_nb[c] : 0.0;
                st->outer = 1;
            }
        __syncthreads();
    }
}

// ------------------------------------------------------------ launches --

template <int BLOCK, int U, int RED, int CL>
fv_status launch_batch_solvers(fv_batch *bt, int which, const void *argp)
{
    const fv_mesh *m = bt->mesh;
    constexpr int BB = BLOCK < 512 ? BLOCK : 512;      // momentum solve: blocks of <= 512
    const void *fn = which == 0 ? (const void *)k_bicgstab_batch<BB, U, RED, CL>
                   : which == 1 ? (const void *)k_pcg_batch<BLOCK, U, RED, CL>
                                : (const void *)k_pcg_mixed_batch<BLOCK, U, RED, CL>;
    const int block = which == 0 ? BB : BLOCK;
    const int cl = CL;
    int per_sm = 0;
    FV_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, block, 0));
    if (per_sm < 1) per_sm = 1;
    int groups = m->sm_count * per_sm / cl;
    if (groups > bt->ncase) groups = bt->ncase;
    if (groups < 1) groups = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(groups * cl);
    cfg.blockDim = dim3(block);
    cfg.stream = m->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cl;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    void *args[] = {const_cast<void *>(argp)};
    FV_CUDA(cudaLaunchKernelExC(&cfg, fn, args));
    return FV_OK;
}

fv_status dispatch(fv_batch *bt, int which, const void *argp)
{
    switch (bt->cfg) {
    case 0: return launch_batch_solvers<256, 2, 0, 1>(bt, which, argp);
    case 1: return launch_batch_solvers<256, 2, 1, 1>(bt, which, argp);
    case 2: return launch_batch_solvers<512, 1, 1, 1>(bt, which, argp);
    case 3: return launch_batch_solvers<512, 2, 1, 1>(bt, which, argp);
    case 4: return launch_batch_solvers<1024, 2, 1, 1>(bt, which, argp);
    case 5: return launch_batch_solvers<512, 2, 1, 2>(bt, which, argp);
    case 6: return launch_batch_solvers<1024, 2, 1, 2>(bt, which, argp);
    case 7: return launch_batch_solvers<512, 2, 1, 4>(bt, which, argp);
    case 8: return launch_batch_solvers<1024, 2, 1, 4>(bt, which, argp);
    default: return launch_batch_solvers<1024, 2, 1, 8>(bt, which, argp);
    }
}

fv_status batch_bicgstab(fv_batch *bt, const fv_piso_params *prm)
{
    fv_case *c = bt->cs;
    const fv_mesh *m = bt->mesh;
    const KrylovWork &w = m->kw;
    BBi a;
    a.ncase = bt->ncase;
    a.N = m->N;
    a.start = bt->d_start;
    a.count = bt->d_count;
    a.order = bt->d_order;
    a.next = bt->d_next;
    a.slice_ptr = m->slice_ptr;
    a.col = m->col;
    a.val = c->Mo;
    a.diag = c->Md;
    a.src = c->src;
    a.gradp = c->gradp;
    a.V = m->V;
    a.x = c->u;
    a.dinv = w.dinv;
    a.r = w.bv[0]; a.rh = w.bv[1]; a.p = w.bv[2]; a.v = w.bv[3];
    a.y = w.bv[4]; a.s = w.bv[5]; a.z = w.bv[6]; a.t = w.bv[7];
    a.tol = prm->u_tol;
    a.reltol = 0.0;
    a.maxit = prm->u_maxit;
    a.stats = bt->d_stats;
    FV_CUDA(cudaMemsetAsync(bt->d_next, 0, sizeof(int32_t), m->stream));
    return dispatch(bt, 0, &a);
}

fv_status batch_pcg(fv_batch *bt, const fv_piso_params *prm, int k)
{
    fv_case *c = bt->cs;
    const fv_mesh *m = bt->mesh;
    const KrylovWork &w = m->kw;
    if (bt->precision == FV_PREC_MIXED) {
        BMix a;
        a.ncase = bt->ncase;
        a.start = bt->d_start;
        a.count = bt->d_count;
        a.order = bt->d_order;
        a.next = bt->d_next + 1;
        a.slice_ptr = m->slice_ptr;
        a.col = m->col;
        a.val = c->Po;
        a.val32 = w.val32;
        a.diag = c->Pd;
        a.b = c->pbv;
        a.x = c->p;
        a.s = w.dinv;
        a.r64 = w.r;
        a.a1 = w.y;
        a.r = w.f32[0]; a.p = w.f32[1]; a.q = w.f32[2]; a.e = w.f32[3];
        a.w = w.f32[4]; a.v = w.f32[5];
        a.tol = prm->p_tol;
        a.reltol = 0.0;
        a.maxit = prm->p_maxit;
        a.stats = bt->d_stats + 3 + k;
        FV_CUDA(cudaMemsetAsync(bt->d_next + 1, 0, sizeof(int32_t), m->stream));
        return dispatch(bt, 2, &a);
    }
    BCg a;
    a.ncase = bt->ncase;
    a.start = bt->d_start;
    a.count = bt->d_count;
    a.order = bt->d_order;
    a.next = bt->d_next + 1;
    a.slice_ptr = m->slice_ptr;
    a.col = m->col;
    a.val = c->Po;
    a.diag = c->Pd;
    a.b = c->pbv;
    a.x = c->p;
    a.s = w.dinv;
    a.r = w.r; a.p = w.p; a.q = w.q; a.y = w.y;
    a.tol = prm->p_tol;
    a.reltol = 0.0;
    a.maxit = prm->p_maxit;
    a.stats = bt->d_stats + 3 + k;
    FV_CUDA(cudaMemsetAsync(bt->d_next + 1, 0, sizeof(int32_t), m->stream));
    return dispatch(bt, 1, &a);
}

fv_status batch_enqueue(fv_batch *bt, const fv_piso_params *prm)
{
    fv_case *c = bt->cs;
    const fv_mesh *m = bt->mesh;
    StepArgs sa{1.0 / prm->dt, 1.0, -1, prm->p_ref_value};
    fv_status st;
#define BSTAGE(stg, nl, call)                                   \
    do {                                                        \
        const int id__ = prof_begin((stg), m->stream);          \
        st = (call);                                            \
        prof_end(id__, m->stream);                              \
        prof_count((stg), (nl));                                \
        if (st != FV_OK) return st;                             \
    } while (0)
    if (m->nonorth) BSTAGE(FV_PROF_MOMENTUM, 1, launch_grad_u(c));
    BSTAGE(FV_PROF_MOMENTUM, 1, launch_momentum(c, sa));
    BSTAGE(FV_PROF_BICGSTAB, 1, batch_bicgstab(bt, prm));
    const int nl = 1 + prm->n_nonorth;
    for (int k = 0; k < prm->n_corr; ++k) {
        BSTAGE(FV_PROF_HBYA, 1, launch_hbya(c));
        for (int j = 0; j < nl; ++j) {
            if (j > 0) BSTAGE(FV_PROF_PRESSURE, 1, launch_grad_p(c));
            BSTAGE(FV_PROF_PRESSURE, 1, launch_pressure(c, sa));
            BSTAGE(FV_PROF_PCG, 1, batch_pcg(bt, prm, k * nl + j));
        }
        BSTAGE(FV_PROF_CORRECT, 1, launch_correct_piso(c));
    }
#undef BSTAGE
    return FV_OK;
}

int worse_status(int a, int b)
{
    auto rank = [](int s) {
        return s == FV_E_TIMEOUT ? 3 : s == FV_E_DIVERGED ? 2 : s == FV_E_NOT_CONVERGED ? 1 : 0;
    };
    return rank(b) > rank(a) ? b : a;
}

fv_status batch_stats(fv_batch *bt, int n_corr, fv_step_stats *out)
{
    const fv_mesh *m = bt->mesh;
    const size_t n = (size_t)bt->ncase * kStatStride;
    FV_CUDA(cudaMemcpyAsync(bt->h_stats, bt->d_stats, sizeof(DevSolveStats) * n,
                            cudaMemcpyDeviceToHost, m->stream));
    FV_CUDA(cudaStreamSynchronize(m->stream));
    int worst = FV_OK;
    for (int c = 0; c < bt->ncase; ++c) {
        const DevSolveStats *d = bt->h_stats + (size_t)c * kStatStride;
        int st = FV_OK;
        fv_step_stats *o = out ? out + c : nullptr;
        if (o) std::memset(o, 0, sizeof(*o));
        for (int k = 0; k < 3 + n_corr; ++k) {
            st = worse_status(st, d[k].status);
            if (!o) continue;
            fv_solve_stats *t = k < 3 ? &o->u[k] : &o->p[k - 3];
            t->iters = d[k].iters;
            t->status = d[k].status;
            t->res0 = d[k].res0;
            t->res = d[k].res;
            t->outer = d[k].outer;
        }
        if (o) {
            o->n_p = n_corr;
            o->status = st;
        }
        worst = worse_status(worst, st);
    }
    return (fv_status)worst;
}

fv_status check_prm(const fv_piso_params *prm)
{
    FV_CHECK(prm != nullptr, FV_E_INVALID, "params are NULL");
    FV_CHECK(prm->dt > 0.0, FV_E_INVALID, "dt must be positive");
    FV_CHECK(prm->n_corr >= 1 && prm->n_corr <= FV_MAX_CORR, FV_E_INVALID, "bad n_corr");
    FV_CHECK(prm->n_nonorth >= 0 && prm->n_corr * (1 + prm->n_nonorth) <= FV_MAX_CORR,
             FV_E_INVALID, "n_corr * (1 + n_nonorth) must be at most %d", FV_MAX_CORR);
    FV_CHECK(prm->p_maxit >= 0 && prm->u_maxit >= 0, FV_E_INVALID, "negative iteration limit");
    return FV_OK;
}

}  // namespace
}  // namespace fvgb

using namespace fvgb;

extern "C" fv_status fv_batch_destroy(fv_batch *bt)
{
    if (!bt) return FV_OK;
    if (bt->mesh) cudaStreamSynchronize(bt->mesh->stream);
    if (bt->graph) cudaGraphExecDestroy(bt->graph);
    if (bt->h_stats) cudaFreeHost(bt->h_stats);
    bt->arena.release();
    if (bt->cs) fv_case_destroy(bt->cs);
    if (bt->mesh) fv_mesh_destroy(bt->mesh);
    delete bt;
    return FV_OK;
}

extern "C" fv_status fv_batch_create(const fv_mesh_desc *descs, int32_t n, const double *nu,
                                     const int32_t *p_ref_cells, int32_t precision, void *stream,
                                     fv_batch **out)
{
    FV_CHECK(descs && nu && out && n > 0, FV_E_INVALID, "bad batch arguments");
    FV_CHECK(precision == FV_PREC_FP64 || precision == FV_PREC_MIXED, FV_E_INVALID,
             "unknown precision %d", precision);
    *out = nullptr;
    fv_batch *bt = new (std::nothrow) fv_batch();
    FV_CHECK(bt != nullptr, FV_E_NOMEM, "host allocation failed");
    bt->ncase = n;
    bt->precision = precision;
    fv_status st = FV_OK;
    try {
        // the union mesh: cells, internal faces and boundary faces of case c
        // follow those of case c-1
        long long N = 0, F = 0, B = 0, NP = 0;
        bt->cell_base.resize(n);
        bt->fbase_int.resize(n);
        bt->fbase_bnd.resize(n);
        bt->nface_int.resize(n);
        bt->nface_bnd.resize(n);
        for (int c = 0; c < n; ++c) {
            const fv_mesh_desc &d = descs[c];
            FV_CHECK(d.n_cells > 0 && d.n_internal_faces >= 0 && d.n_boundary_faces >= 0 &&
                         d.owner && d.Sf && d.Cf && d.C && d.V && (d.n_patches == 0 || d.patches),
                     FV_E_INVALID, "case %d: bad mesh description", c);
            FV_CHECK(nu[c] >= 0.0, FV_E_INVALID, "case %d: negative viscosity", c);
            bt->cell_base[c] = (int)N;
            bt->fbase_int[c] = (int)F;
            bt->fbase_bnd[c] = (int)B;
            bt->nface_int[c] = d.n_internal_faces;
            bt->nface_bnd[c] = d.n_boundary_faces;
            N += d.n_cells;
            F += d.n_internal_faces;
            B += d.n_boundary_faces;
            NP += d.n_patches;
        }
        FV_CHECK(N + F + B < (1LL << 31), FV_E_INVALID, "batch too large");
        const long long M = F + B;
        std::vector<int32_t> own(M), nei(F);
        std::vector<double> Sf(3 * M), Cf(3 * M), C(3 * N), V(N);
        std::vector<fv_patch> pt;
        pt.reserve(NP);
        for (int c = 0; c < n; ++c) {
            const fv_mesh_desc &d = descs[c];
            const int nb = bt->cell_base[c], fi = bt->fbase_int[c], fb = bt->fbase_bnd[c];
            const long long Mc = (long long)d.n_internal_faces + d.n_boundary_faces;
            for (int f = 0; f < d.n_internal_faces; ++f) {
                own[fi + f] = d.owner[f] + nb;
                nei[fi + f] = d.neighbour[f] + nb;
                for (int k = 0; k < 3; ++k) {
                    Sf[k * M + fi + f] = d.Sf[k * Mc + f];
                    Cf[k * M + fi + f] = d.Cf[k * Mc + f];
                }
            }
            for (int j = 0; j < d.n_boundary_faces; ++j) {
                const long long g = F + fb + j, f = d.n_internal_faces + j;
                own[g] = d.owner[f] + nb;
                for (int k = 0; k < 3; ++k) {
                    Sf[k * M + g] = d.Sf[k * Mc + f];
                    Cf[k * M + g] = d.Cf[k * Mc + f];
                }
            }
            for (int i = 0; i < d.n_cells; ++i) {
                for (int k = 0; k < 3; ++k) C[k * N + nb + i] = d.C[(long long)k * d.n_cells + i];
                V[nb + i] = d.V[i];
            }
            for (int q = 0; q < d.n_patches; ++q) {
                fv_patch p = d.patches[q];
                p.start += fb;
                pt.push_back(p);
            }
        }
        fv_mesh_desc u{};
        u.n_cells = (int)N;
        u.n_internal_faces = (int)F;
        u.n_boundary_faces = (int)B;
        u.n_patches = (int)pt.size();
        u.owner = own.data();
        u.neighbour = nei.data();
        u.Sf = Sf.data();
        u.Cf = Cf.data();
        u.C = C.data();
        u.V = V.data();
        u.patches = pt.data();
        u.renumber = 1;
        if ((st = fv_mesh_create(&u, stream, &bt->mesh)) != FV_OK) { fv_batch_destroy(bt); return st; }
        fv_mesh *m = bt->mesh;
        // every case is one connected block of the renumbered order
        bt->start.resize(n);
        bt->count.resize(n);
        for (int c = 0; c < n; ++c) {
            int lo = INT32_MAX, hi = -1;
            for (int i = 0; i < descs[c].n_cells; ++i) {
                const int j = m->plan.cell_new_of_old[bt->cell_base[c] + i];
                lo = std::min(lo, j);
                hi = std::max(hi, j);
            }
            if (hi - lo + 1 != descs[c].n_cells) {
                set_error("case %d is not connected (its cells are not one block after renumbering)", c);
                fv_batch_destroy(bt);
                return FV_E_INVALID;
            }
            bt->start[c] = lo;
            bt->count[c] = descs[c].n_cells;
        }
        if ((st = fv_case_create(m, 0.0, precision, &bt->cs)) != FV_OK) { fv_batch_destroy(bt); return st; }
        fv_case *cs = bt->cs;
        std::vector<double> nuc(N);
        std::vector<int8_t> pin(N, 0);
        for (int c = 0; c < n; ++c) {
            for (int i = 0; i < bt->count[c]; ++i) nuc[bt->start[c] + i] = nu[c];
            const int ref = p_ref_cells ? p_ref_cells[c] : -1;
            if (ref >= 0) {
                FV_CHECK(ref < descs[c].n_cells, FV_E_INVALID, "case %d: reference cell out of range", c);
                pin[m->plan.cell_new_of_old[bt->cell_base[c] + ref]] = 1;
            }
        }
        std::vector<int32_t> order(n);
        std::iota(order.begin(), order.end(), 0);
        std::stable_sort(order.begin(), order.end(),
                         [&](int x, int y) { return bt->count[x] > bt->count[y]; });
        DeviceArena &ar = bt->arena;
        cudaStream_t s = m->stream;
        if ((st = cs->arena.alloc_n(&cs->nu_cell, N)) != FV_OK ||
            (st = cs->arena.alloc_n(&cs->pin, N)) != FV_OK ||
            (st = ar.alloc_n(&bt->d_start, n)) != FV_OK || (st = ar.alloc_n(&bt->d_count, n)) != FV_OK ||
            (st = ar.alloc_n(&bt->d_order, n)) != FV_OK || (st = ar.alloc_n(&bt->d_next, 2)) != FV_OK ||
            (st = ar.alloc_n(&bt->d_stats, (size_t)n * kStatStride)) != FV_OK ||
            (st = ar.alloc_n(&bt->save, (size_t)4 * N + M)) != FV_OK) {
            fv_batch_destroy(bt);
            return st;
        }
        if (precision == FV_PREC_MIXED && !m->kw.val32) {
            // FP32 work space of the mixed-precision pressure solves
            if ((st = m->arena.alloc_n(&m->kw.val32, (size_t)m->nnz)) != FV_OK) { fv_batch_destroy(bt); return st; }
            for (int k = 0; k < 6; ++k)
                if ((st = m->arena.alloc_n(&m->kw.f32[k], (size_t)N)) != FV_OK) { fv_batch_destroy(bt); return st; }
        }
        cudaError_t e = cudaMallocHost(&bt->h_stats, sizeof(DevSolveStats) * n * kStatStride);
        if (e != cudaSuccess) { bt->h_stats = nullptr; fv_batch_destroy(bt); return cuda_status(e, "cudaMallocHost"); }
        e = cudaMemcpyAsync(cs->nu_cell, nuc.data(), sizeof(double) * N, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(cs->pin, pin.data(), N, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(bt->d_start, bt->start.data(), 4 * n, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(bt->d_count, bt->count.data(), 4 * n, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(bt->d_order, order.data(), 4 * n, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(bt->d_stats, 0, sizeof(DevSolveStats) * n * kStatStride, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) { fv_batch_destroy(bt); return cuda_status(e, "batch upload"); }
        bt->cfg = 3;   // 512 threads, two rows per trip, staged reduction until tuned
    } catch (const std::bad_alloc &) {
        fv_batch_destroy(bt);
        set_error("host allocation failed in fv_batch_create");
        return FV_E_NOMEM;
    }
    *out = bt;
    return FV_OK;
}

extern "C" fv_status fv_batch_piso_step(fv_batch *bt, const fv_piso_params *prm,
                                        fv_step_stats *per_case)
{
    FV_CHECK(bt, FV_E_INVALID, "NULL batch");
    fv_status st = check_prm(prm);
    if (st != FV_OK) return st;
    if ((st = batch_enqueue(bt, prm)) != FV_OK) return st;
    if (!per_case) return FV_OK;
    return batch_stats(bt, prm->n_corr * (1 + prm->n_nonorth), per_case);
}

extern "C" fv_status fv_batch_run_graph(fv_batch *bt, const fv_piso_params *prm, int32_t n_steps,
                                        fv_step_stats *per_case)
{
    FV_CHECK(bt && n_steps >= 0, FV_E_INVALID, "bad arguments");
    fv_status st = check_prm(prm);
    if (st != FV_OK) return st;
    cudaStream_t s = bt->mesh->stream;
    FV_CHECK(s != nullptr, FV_E_UNSUPPORTED, "graph replay needs a non-default stream");
    if (bt->graph && std::memcmp(&bt->graph_prm, prm, sizeof(*prm)) != 0) {
        cudaGraphExecDestroy(bt->graph);
        bt->graph = nullptr;
    }
    if (!bt->graph) {
        cudaGraph_t g = nullptr;
        FV_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        st = batch_enqueue(bt, prm);
        const cudaError_t e = cudaStreamEndCapture(s, &g);
        if (st != FV_OK) { if (g) cudaGraphDestroy(g); return st; }
        if (e != cudaSuccess) return cuda_status(e, "cudaStreamEndCapture");
        const cudaError_t e2 = cudaGraphInstantiate(&bt->graph, g, 0);
        cudaGraphDestroy(g);
        if (e2 != cudaSuccess) { bt->graph = nullptr; return cuda_status(e2, "cudaGraphInstantiate"); }
        bt->graph_prm = *prm;
    }
    for (int k = 0; k < n_steps; ++k) FV_CUDA(cudaGraphLaunch(bt->graph, s));
    if (!per_case) return FV_OK;
    return batch_stats(bt, prm->n_corr * (1 + prm->n_nonorth), per_case);
}

extern "C" fv_status fv_batch_get_fields(const fv_batch *bt, int32_t c, double *u, double *p,
                                         double *phi)
{
    FV_CHECK(bt && c >= 0 && c < bt->ncase, FV_E_INVALID, "bad case index");
    const fv_mesh *m = bt->mesh;
    const int N = m->N, M = m->M;
    std::vector<double> U((size_t)3 * N), Pp(N), Ph(M);
    fv_status st = fv_case_get_fields_host(bt->cs, U.data(), Pp.data(), Ph.data(), 1);
    if (st != FV_OK) return st;
    const int nb = bt->cell_base[c], n = bt->count[c];
    for (int i = 0; i < n; ++i) {
        if (u)
            for (int k = 0; k < 3; ++k) u[(size_t)k * n + i] = U[(size_t)k * N + nb + i];
        if (p) p[i] = Pp[nb + i];
    }
    if (phi) {
        const int Fi = bt->nface_int[c], Bc = bt->nface_bnd[c];
        for (int f = 0; f < Fi; ++f) phi[f] = Ph[bt->fbase_int[c] + f];
        for (int j = 0; j < Bc; ++j) phi[Fi + j] = Ph[m->F + bt->fbase_bnd[c] + j];
    }
    return FV_OK;
}

extern "C" fv_status fv_batch_set_schedule(fv_batch *bt, int32_t schedule)
{
    FV_CHECK(bt && schedule >= 0 && schedule < kNSched, FV_E_INVALID, "schedule out of range 0..%d",
             kNSched - 1);
    bt->cfg = schedule;
    if (bt->graph) { cudaGraphExecDestroy(bt->graph); bt->graph = nullptr; }
    return FV_OK;
}

extern "C" fv_status fv_batch_schedule_info(int32_t schedule, int32_t *info)
{
    FV_CHECK(info && schedule >= 0 && schedule < kNSched, FV_E_INVALID, "schedule out of range");
    info[0] = kScheds[schedule].block;
    info[1] = kScheds[schedule].unroll;
    info[2] = kScheds[schedule].red;
    info[3] = kNSched;
    info[4] = kScheds[schedule].cl;
    return FV_OK;
}

// Time one PISO step per schedule from the same state (saved and restored
// around each trial) and keep the fastest.
extern "C" fv_status fv_batch_autotune(fv_batch *bt, const fv_piso_params *prm, int32_t *best,
                                       double *ms)
{
    FV_CHECK(bt, FV_E_INVALID, "NULL batch");
    fv_status st = check_prm(prm);
    if (st != FV_OK) return st;
    fv_case *c = bt->cs;
    const fv_mesh *m = bt->mesh;
    cudaStream_t s = m->stream;
    const size_t N = m->N, M = m->M;
    double *su = bt->save, *sp = bt->save + 3 * N, *sf = bt->save + 4 * N;
    FV_CUDA(cudaMemcpyAsync(su, c->u, sizeof(double) * 3 * N, cudaMemcpyDeviceToDevice, s));
    FV_CUDA(cudaMemcpyAsync(sp, c->p, sizeof(double) * N, cudaMemcpyDeviceToDevice, s));
    FV_CUDA(cudaMemcpyAsync(sf, c->phi, sizeof(double) * M, cudaMemcpyDeviceToDevice, s));
    cudaEvent_t e0, e1;
    FV_CUDA(cudaEventCreate(&e0));
    FV_CUDA(cudaEventCreate(&e1));
    float bestms = 1e30f;
    int bestcfg = bt->cfg;
    for (int k = 0; k < kNSched && st == FV_OK; ++k) {
        bt->cfg = k;
        float t = 0.0f;
        for (int rep = 0; rep < 2 && st == FV_OK; ++rep) {   // first run warms up
            cudaMemcpyAsync(c->u, su, sizeof(double) * 3 * N, cudaMemcpyDeviceToDevice, s);
            cudaMemcpyAsync(c->p, sp, sizeof(double) * N, cudaMemcpyDeviceToDevice, s);
            cudaMemcpyAsync(c->phi, sf, sizeof(double) * M, cudaMemcpyDeviceToDevice, s);
            cudaEventRecord(e0, s);
            st = batch_enqueue(bt, prm);
            cudaEventRecord(e1, s);
            if (cudaEventSynchronize(e1) != cudaSuccess) st = FV_E_CUDA;
            cudaEventElapsedTime(&t, e0, e1);
        }
        if (ms) ms[k] = t;
        if (t < bestms) { bestms = t; bestcfg = k; }
    }
    cudaMemcpyAsync(c->u, su, sizeof(double) * 3 * N, cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(c->p, sp, sizeof(double) * N, cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(c->phi, sf, sizeof(double) * M, cudaMemcpyDeviceToDevice, s);
    cudaStreamSynchronize(s);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != FV_OK) return st;
    bt->cfg = bestcfg;
    if (bt->graph) { cudaGraphExecDestroy(bt->graph); bt->graph = nullptr; }
    if (best) *best = bestcfg;
    return FV_OK;
}
